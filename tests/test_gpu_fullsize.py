"""Bootstrapped CutMax at the full size of the benchmark: N = 2^16, the
31 + 10 prime chain with dnum = 3 and h = 192, 32,000 heavy-tailed logits and
the paper's HE setting T = 4, p = [16, 4, 4, 6], c = [5, 3, 3, 3], in the
launch configuration bench.py times.  The decrypted output is compared with
the FP64 mirror of the same circuit (max-abs 1e-3) and its argmax with the
plaintext's; a batch of two 128,256-logit streams (four ciphertexts each) with
shared scalar chains is checked the same way."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench                                        # noqa: E402
from oracle import cutmax_fp64 as F                 # noqa: E402
from paper_2509_08383_gb300 import build, he        # noqa: E402
from paper_2509_08383_gb300 import plan as P        # noqa: E402
from paper_2509_08383_gb300 import synth            # noqa: E402

build.build_library()
SLOTS = 1 << 15


@pytest.fixture(scope="module")
def full():
    log_n, qb, pb, dnum, pl, gen, _, boot = bench.workload("cfg2")
    g = he.Context(log_n, qb, pb, dnum, h=boot[0], seed=1, arena_bytes=48 << 30)
    g.bootstrap_prepare(*boot[1:])
    g.cutmax_prepare(pl)
    return g, pl, gen


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_cutmax_32k_logits_n65536(full, seed):
    g, pl, gen = full
    x = gen(seed)
    z = g.cutmax(g.encrypt(P.pack(x, SLOTS, pl.packing), g.delta, 100 + seed), pl)
    dec = g.decrypt(z, pl.n)
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3
    assert int(np.argmax(dec)) == int(np.argmax(x))


def test_shared_batch_128k_logits_n65536(full):
    g, _, _ = full
    n = 128256
    gen = (lambda s: synth.logits_gaussian(s, n=n, sd=2.0, gap=0.5))
    pl = P.calibrate(lambda i: gen(100000 + i), 60, n, SLOTS, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                     tol_k=bench.INVSQRT_TOL, k_max=20, d_max=14, tol_d=bench.INVSQRT_TOL, bootstrap=True)
    pl.shared = True
    assert pl.cts == 4
    g.cutmax_prepare(pl)
    xs = [gen(s) for s in range(2)]
    cts = [g.encrypt(v, g.delta, 200 + 4 * s + c) for s, x in enumerate(xs) for c, v in enumerate(P.pack_cts(x, SLOTS))]
    Z = g.cutmax(g.batch_pack(cts), pl)
    for s, x in enumerate(xs):
        dec = np.concatenate([g.decrypt(g.batch_member(Z, 4 * s + c)) for c in range(4)])[:n]
        assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3, s
        assert int(np.argmax(dec)) == int(np.argmax(x))
