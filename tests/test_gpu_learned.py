"""Learned inverse-square-root stand-in: GPU training kernels and the
encrypted circuit with the learned quadratic.

The trainer is pinned to the closed form of its optimum: the network is a
quadratic in x, so the best it can reach is the least-squares quadratic
minimising sum (f(x) sqrt(x) - 1)^2, computed here with numpy.  The circuit
with a learned iteration is bit-exact to the oracle's circuit (leveled) and
within 1e-3 of its FP64 mirror (bootstrapped)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import ckks as ock                      # noqa: E402
from oracle import cutmax_fp64 as F                 # noqa: E402
from oracle import encoding as oenc                 # noqa: E402
from oracle.circuit import HE, cutmax_he, required_rotations  # noqa: E402
from paper_2509_08383_gb300 import build, he        # noqa: E402
from paper_2509_08383_gb300 import learned          # noqa: E402
from paper_2509_08383_gb300 import plan as P        # noqa: E402
from paper_2509_08383_gb300 import synth            # noqa: E402

build.build_library()
LOG_N = 11
SLOTS = 1 << (LOG_N - 1)
DELTA = 2.0 ** 40


def lstsq_quad(xs):
    r = np.sqrt(xs)
    M = np.stack([xs * xs * r, xs * r, r], axis=1)
    abc, *_ = np.linalg.lstsq(M, np.ones_like(xs), rcond=None)
    return abc


def loss(abc, xs):
    return float(np.mean(((abc[0] * xs * xs + abc[1] * xs + abc[2]) * np.sqrt(xs) - 1.0) ** 2))


@pytest.mark.parametrize("lo,hi", [(0.9, 1.1), (0.25, 2.5), (0.05, 12.0)])
def test_training_reaches_least_squares_optimum(lo, hi):
    g = he.Context(LOG_N, [60] + [40] * 3, [60], dnum=2, seed=1, arena_bytes=256 << 20)
    rng = np.random.default_rng(3)
    xs = np.exp(rng.uniform(np.log(lo), np.log(hi), 20000))
    abc, l_gpu = g.learn_invsqrt(xs, steps=4000, lr=2e-2, seed=5)
    best = loss(lstsq_quad(xs), xs)
    assert abs(l_gpu - loss(np.array(abc), xs)) <= 1e-3 + 0.05 * loss(np.array(abc), xs)
    assert loss(np.array(abc), xs) <= best * 1.05 + 1e-7, (loss(np.array(abc), xs), best)
    with pytest.raises(he.HeError):
        g.learn_invsqrt(np.array([1.0, -2.0, 3.0]))


def test_leveled_learned_iteration_bit_exact():
    """T = 2, p = 3, c = 5 at N = 2^11 with the first iteration's inverse square
    root the least-squares quadratic of its calibrated range."""
    q, pbits = [60] + [40] * 21, [60, 60]
    n = 1024

    def learn(t, kap, xs, ab):
        if t:
            return None
        grid = np.geomspace(*ab, 2001)
        return list(lstsq_quad(grid))

    pl = P.calibrate(lambda i: synth.logits_gaussian(6000 + i, n=n), 40, n, SLOTS, 2, 3, 5.0, k_fixed=2,
                     d_fixed=1, learn=learn)
    assert pl.k[0] == 0 and pl.k[1] == 2 and pl.lq is not None
    g = he.Context(LOG_N, q, pbits, dnum=11, seed=13)
    o = ock.Context(LOG_N, q, pbits, dnum=11, seed=13)
    g.cutmax_prepare(pl)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    x = synth.logits_gaussian(55, n=n)
    pt = oenc.encode(P.pack(x, SLOTS, pl.packing), LOG_N, DELTA)
    zg = g.cutmax(g.encrypt_poly(pt, DELTA, 3), pl)
    zo = cutmax_he(HE(o, DELTA), o.encrypt(pt, DELTA, 3), pl)
    assert (zg.export() == zo.export()).all()
    dec = g.decrypt(zg, n)
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3
    assert int(np.argmax(dec)) == int(np.argmax(x))


def test_bootstrapped_learned_plan():
    """Heavy-tailed logits, T = 4, p = [16, 4, 4, 6], c = [5, 3, 3, 3],
    bootstrapping: variances logged from the plain plan, the network trained on
    the GPU, the plan keeps the quadratic where it is within 8% over the
    calibrated range (iteration 0 at least); decrypted within 1e-3 of the
    mirror, argmax exact, fewer levels than the plain plan."""
    qb = [47] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
    pb = [61] * 10
    nv = 1000
    kw = dict(sample=lambda i: synth.logits_heavy_tail(8000 + i, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][i % 3]),
              n_cal=150, n=nv, slots=SLOTS, T=4, p=[16, 4, 4, 6], c=[5.0, 3.0, 3.0, 3.0], margin=2.0, tol_k=2.0 ** -10,
              k_max=20, d_max=14, tol_d=2.0 ** -10, bootstrap=True)
    plain = P.calibrate(**kw)
    logged = learned.log_variances(plain, synth.HeavyTail(nv, heavy=5), range(20000, 22000), workers=4)
    g = he.Context(LOG_N, qb, pb, dnum=3, h=64, seed=31, arena_bytes=2 << 30)
    g.bootstrap_prepare(14, 4, 31)
    lpl, report = learned.learned_plan(g, plain, kw, logged)
    assert report[0]["kept"] and lpl.k[0] == 0
    assert lpl.depth() < plain.depth()
    g.cutmax_prepare(lpl)
    for s in range(3):
        x = synth.logits_heavy_tail(s, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][s % 3])
        z = g.cutmax(g.encrypt(P.pack(x, SLOTS, lpl.packing), DELTA, 90 + s), lpl)
        dec = g.decrypt(z, nv)
        assert np.abs(dec - F.cutmax_circuit(x, lpl)).max() < 1e-3, s
        assert int(np.argmax(dec)) == int(np.argmax(x))


@pytest.mark.parametrize("alpha", [21.85, 58.4])
def test_beta_noise_from_encrypted_uniforms(alpha):
    """G = U^(1/alpha) (Lemma 2 / Observation 1) from encrypted uniforms: the
    GPU evaluates the degree-31 Chebyshev interpolant at Chebyshev nodes; its
    values match the same series in FP64 (CKKS noise) and U^(1/alpha) within
    the interpolation error for U >= 1e-2."""
    g = he.Context(LOG_N, [60] + [40] * 12, [60, 60], dnum=13, seed=17)
    g.gen_relin_key()
    d = 31
    u = synth.uniforms(4, SLOTS)
    G = g.decrypt(g.beta_noise(g.encrypt(u, DELTA, 7), alpha, d))
    th = np.pi * (np.arange(d + 1) + 0.5) / (d + 1)
    f = ((np.cos(th) + 1) / 2) ** (1 / alpha)
    c = np.array([2 / (d + 1) * np.sum(f * np.cos(k * th)) for k in range(d + 1)])
    c[0] /= 2
    series = np.polynomial.chebyshev.chebval(2 * u - 1, c)
    assert np.abs(G - series).max() < 1e-4
    big = u >= 1e-2
    bound = float(np.abs(np.polynomial.chebyshev.chebval(2 * np.linspace(1e-2, 1, 100001) - 1, c)
                         - np.linspace(1e-2, 1, 100001) ** (1 / alpha)).max())
    assert np.abs(G[big] - u[big] ** (1 / alpha)).max() < bound + 1e-4
    with pytest.raises(he.HeError):
        g.beta_noise(g.encrypt(u, DELTA, 8), -1.0)
