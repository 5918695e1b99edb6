"""The key switch that allocates nothing (he_keyswitch_noalloc), checked
against the regular key switch through the C ABI, twice in a row.

It is for callers that cannot allocate device memory on demand (allocation
synchronises the device and can fail under fragmentation, or another
allocator owns all of the GPU's memory); its scratch is a static device array
shared by every call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_08383_gb300 import build, he       # noqa: E402

build.build_library()


def test_keyswitch_noalloc_matches_regular_twice():
    log_n, level = 11, 9
    g = he.Context(log_n, [60] + [40] * 12, [60, 60], dnum=4, seed=17)
    g.gen_relin_key()
    rng = np.random.default_rng(3)
    n = g.n
    d_first = None
    ref_first = None
    for call in range(2):
        d = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in g.primes[: level + 1]])
        ref0, ref1 = g.keyswitch(d, level, 0)                    # coefficient form in and out
        if call == 0:
            d_first, ref_first = d, (ref0, ref1)
        dt = torch.from_numpy(d.view(np.int64).copy()).cuda()
        g.ntt_device(dt, 0)                                      # to NTT form
        out = torch.empty((2, level + 1, n), dtype=torch.int64, device="cuda")
        mem_before = g.memory()
        g.keyswitch_noalloc(dt, level, 0, out)
        torch.cuda.synchronize()
        # the library's device arena is neither drawn on nor grown by the call
        assert g.memory() == mem_before, f"call {call}"
        g.ntt_device(out[0], 0, inverse=True)
        g.ntt_device(out[1], 0, inverse=True)
        got = out.cpu().numpy().view(np.uint64)
        assert (got[0] == ref0).all() and (got[1] == ref1).all(), f"call {call}"
    # the context's own key switch still works after the calls
    again = g.keyswitch(d_first, level, 0)
    assert (again[0] == ref_first[0]).all() and (again[1] == ref_first[1]).all()


def test_keyswitch_noalloc_rejects_oversized():
    g = he.Context(14, [60] + [40] * 21, [60, 60], dnum=11, seed=1)
    g.gen_relin_key()
    level = 21
    dt = torch.zeros((level + 1, g.n), dtype=torch.int64, device="cuda")
    out = torch.empty((2, level + 1, g.n), dtype=torch.int64, device="cuda")
    with pytest.raises(he.HeError) as ei:
        g.keyswitch_noalloc(dt, level, 0, out)
    assert ei.value.code == he.HE_EINVAL
