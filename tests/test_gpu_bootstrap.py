"""GPU bootstrapping vs the oracle's bootstrapping, through the C ABI.

The two sides encode their transform constants with different float64
algorithms (factored FFT stages vs the dense matrix), so ciphertexts differ in
their low bits; both must decrypt to the input message within the
bootstrapping error, and to each other.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import ckks as ock                      # noqa: E402
from oracle import encoding as oenc                 # noqa: E402
from oracle.bootstrap import Bootstrapper           # noqa: E402
from paper_2509_08383_gb300 import build, he        # noqa: E402

build.build_library()

LOG_N = 11
QB = [55] + [40] * 3 + [60] * 3 + [60] * 10 + [58] * 3
PB = [61] * 7
H, K, R, D = 64, 14, 4, 31


@pytest.fixture(scope="module")
def boot_pair():
    g = he.Context(LOG_N, QB, PB, dnum=3, h=H, seed=12)
    g.bootstrap_prepare(K, R, D)
    o = ock.Context(LOG_N, QB, PB, dnum=3, h=H, seed=12)
    ob = Bootstrapper(o, K=K, r=R, d=D)
    ob.gen_keys()
    return g, o, ob


def test_bootstrap_matches_message_and_oracle(boot_pair):
    g, o, ob = boot_pair
    rng = np.random.default_rng(0)
    z = rng.uniform(-1, 1, g.slots)
    delta = 2.0 ** 40
    pt = oenc.encode(z, LOG_N, delta)
    cg = g.encrypt_poly(pt, delta, 5, level=0)
    co = o.encrypt(pt, delta, 5, level=0)
    assert (cg.export() == co.export()).all()
    bg = g.bootstrap(cg)
    bo = ob.bootstrap(co)
    assert bg.level == bo.level == len(QB) - 1 - 16   # d = 31: both evaluations take 6 + r levels
    dg = g.decrypt(bg, complex_out=True)
    do = oenc.decode(o.decrypt(bo), LOG_N, bo.scale)
    assert np.abs(dg - z).max() < 1e-6
    assert np.abs(do - z).max() < 1e-6
    assert np.abs(dg - do).max() < 1e-6


def test_bootstrap_twice_and_from_higher_level(boot_pair):
    g, _, _ = boot_pair
    rng = np.random.default_rng(1)
    z = rng.uniform(-2, 2, g.slots)
    ct = g.encrypt(z, g.delta, 9, level=2)
    b1 = g.bootstrap(ct)
    sq = g.rescale(g.mul(b1, b1))            # use a level, then refresh again
    b2 = g.bootstrap(sq)
    assert np.abs(g.decrypt(b2) - z * z).max() < 1e-5
