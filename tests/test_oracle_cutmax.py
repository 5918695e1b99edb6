"""Pins of the FP64 CutMax oracle and of the encrypted circuit on the oracle.

Closed forms, the lemmas of App. E, the T_min table printed in App. E, the
Goldschmidt identities of App. B.1, the Beta / Gumbel sampling lemmas of
Sect. 3.3 and the depth of the encrypted circuit.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import cutmax_fp64 as F
from paper_2509_08383_gb300 import plan as P
from paper_2509_08383_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_tmin_table_reproduced():
    """App. E table: T_min for n=32768, p=13, c=5 (all twelve entries)."""
    for delta, k10, k100 in _rows("tmin_table.txt"):
        d = float(delta)
        assert F.t_min(10, d, 5.0, 32768, 13) == int(k10)
        assert F.t_min(100, d, 5.0, 32768, 13) == int(k100)


def test_paper_speedup_arithmetic():
    v = {k: float(x) for k, x in _rows("paper_latency.txt")}
    lo = v["nexus_bert_30522"] / v["cutmax_mistral_32768"]
    hi = v["nexus_llama3_128256"] / v["cutmax_qwen_151936"]
    assert round(lo) == v["speedup_low"] and round(hi) == v["speedup_high"]


def test_n2_closed_form():
    """n = 2: r = (+1, -1) for any distinct pair, so z = (1 + 1/c, 1 - 1/c)."""
    for x in ([3.0, -7.5], [0.1, 0.2], [1e6, -1e6]):
        z = F.semi_standardize(x, 4.0)
        hi, lo = (0, 1) if x[0] > x[1] else (1, 0)
        assert z[hi] == pytest.approx(1.25) and z[lo] == pytest.approx(0.75)


def test_scaled_one_hot_closed_form():
    n, c = 17, 3.0
    x = np.zeros(n)
    x[5] = 2.7
    z = F.semi_standardize(x, c)
    assert z[5] == pytest.approx(1 + math.sqrt(n - 1) / c)
    assert np.allclose(np.delete(z, 5), 1 - 1 / (c * math.sqrt(n - 1)))


def test_scale_and_shift_invariance():
    rng = np.random.default_rng(0)
    x = rng.normal(size=500)
    assert np.allclose(F.semi_standardize(x, 5.0), F.semi_standardize(7.3 * x - 2.0, 5.0))
    assert np.allclose(F.cutmax_exact(x, 3, 5, 5.0), F.cutmax_exact(4.0 * x + 9.0, 3, 5, 5.0))


def test_lemma_ordering_and_gap():
    """Lemma 1 (S_c strictly increasing) and Lemma 2 (delta-gap -> delta/c gap)."""
    rng = np.random.default_rng(1)
    for s in range(20):
        x = rng.normal(size=300)
        c = 1.0 + 9.0 * rng.random()
        z = F.semi_standardize(x, c)
        assert (np.argsort(z, kind="stable") == np.argsort(x, kind="stable")).all()
        srt = np.sort(x)
        delta = (srt[-1] - srt[-2]) / x.std()
        zs = np.sort(z)
        assert zs[-1] - zs[-2] >= delta / c - 1e-12


def test_lemma_gap_ratio_growth():
    """Lemma 4/5: Gamma(y') >= Gamma(y) (1 + delta/(c + sqrt n))^p when all z > 0."""
    rng = np.random.default_rng(2)
    checked = 0
    for s in range(40):
        n = 200
        y = rng.random(n) + 0.5        # positive entries so Gamma is a ratio of positives
        c = 5.0
        z = F.semi_standardize(y, c)
        if z.min() <= 0:
            continue
        srt = np.sort(y)
        delta = (srt[-1] - srt[-2]) / y.std()
        for p in (1, 3, 7):
            y2 = z ** p
            assert F.gap_ratio(y2) >= F.gap_ratio(y) ** 0 * F.gap_growth_bound(delta, c, n, p) * (1 - 1e-12)
            assert F.gap_ratio(z ** p) == pytest.approx(F.gap_ratio(z) ** p)
        checked += 1
    assert checked > 20


def test_cutmax_converges_to_one_hot():
    """Sect. 3.1 convergence, with the paper's best T=4 setting (p, c) = (13, 15)
    of Table "Convergence of CutMax": Z is one-hot at argmax X."""
    for s in range(5):
        x = synth.logits_heavy_tail(s, n=4096, gap=1.0)
        Z = F.cutmax_exact(x, 4, 13, 15.0)
        assert np.argmax(Z) == np.argmax(x) and Z.max() > 0.9999


def test_cutmax_fixed_point_closed_form():
    """A one-hot state maps to z_k = 1 + sqrt(n-1)/c, z_j = 1 - 1/(c sqrt(n-1)),
    so the limit of max Z is z_k^p / (z_k^p + (n-1) z_j^p)."""
    n, p, c = 4096, 5, 5.0
    x = synth.logits_heavy_tail(0, n=n, gap=1.0)
    Z = F.cutmax_exact(x, 12, p, c)
    zk, zj = 1 + math.sqrt(n - 1) / c, 1 - 1 / (c * math.sqrt(n - 1))
    assert Z.max() == pytest.approx(zk ** p / (zk ** p + (n - 1) * zj ** p), rel=1e-9)


def test_goldschmidt_inverse_telescopes():
    """prod_{i<=d}(1 + a^(2^i)) = (1 - a^(2^(d+1)))/(1 - a), a = 1 - x (App. B.1)."""
    x = np.linspace(0.05, 1.95, 101)
    for d in range(0, 7):
        a = 1.0 - x
        assert np.allclose(F.goldschmidt_inv(x, d), (1 - a ** (2 ** (d + 1))) / x, rtol=1e-12, atol=1e-12)
    assert np.abs(F.goldschmidt_inv(x, 12) * x - 1).max() < 1e-9


def test_goldschmidt_invsqrt_converges_monotonically():
    x = np.geomspace(0.05, 2.5, 50)
    errs = [np.abs(F.goldschmidt_invsqrt(x, k, 1.0) * np.sqrt(x) - 1).max() for k in range(1, 9)]
    assert all(b <= a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    # one iteration from y0 is exactly one Newton step for 1/sqrt(x)
    y0 = 0.9
    assert np.allclose(F.goldschmidt_invsqrt(x, 1, y0), y0 * (3 - x * y0 * y0) / 2)


def test_beta_cut_lemma():
    """Lemma 2: G ~ Beta(alpha,1) with alpha = ln(1-p)/ln p has P(G > p) = p;
    Observation 1 generalises to P(G > p) = q with alpha = ln(1-q)/ln p."""
    for p in (0.5, 0.9, 0.95):
        a = F.beta_alpha(p)
        assert 1 - p ** a == pytest.approx(p)
        u = synth.uniforms(int(p * 100), 200000)
        g = F.beta_noise(u, a)
        assert abs((g > p).mean() - p) < 0.005
        assert stats.kstest(g[:20000], stats.beta(a, 1).cdf).pvalue > 1e-4
    a = F.beta_alpha(0.9, 0.95)
    assert a == pytest.approx(math.log(0.05) / math.log(0.9)) and a == pytest.approx(28.433, abs=1e-3)


def test_gumbel_max_is_softmax():
    """Lemma 3.2 (Gumbel-max trick): argmax(X + G) ~ softmax(X)."""
    x = np.array([0.3, -1.0, 1.2, 0.0, 0.7])
    rng = np.random.default_rng(9)
    draws = 200000
    u = rng.random((draws, len(x)))
    idx = np.argmax(x[None, :] + F.gumbel_noise(u), axis=1)
    cnt = np.bincount(idx, minlength=len(x))
    pr = np.exp(x) / np.exp(x).sum()
    assert stats.chisquare(cnt, pr * draws).pvalue > 1e-4


def test_power_by_squaring_depth_and_value():
    for p in range(1, 20):
        assert F.power_by_squaring(1.01, p) == pytest.approx(1.01 ** p)
        assert P.power_depth(p) == math.ceil(math.log2(p)) if p > 1 else P.power_depth(p) == 0


def _cfg1_plan(slots=1024):
    return P.calibrate(lambda i: synth.logits_gaussian(1000 + i), 60, 1024, slots, 2, 3, 5.0,
                       k_fixed=2, d_fixed=2)


def test_circuit_mirror_close_to_alg1():
    pl = _cfg1_plan(8192)
    assert pl.depth() == 21
    for s in range(10):
        x = synth.logits_gaussian(s)
        assert np.abs(F.cutmax_circuit(x, pl) - F.cutmax_exact(x, 2, 3, 5.0)).max() < 1e-6
        assert np.argmax(F.cutmax_circuit(x, pl)) == np.argmax(x)


@pytest.mark.parametrize("packing_slots", [1024, 2048])
def test_encrypted_circuit_on_oracle(packing_slots):
    """Alg. 2 on oracle CKKS: consumes exactly plan.depth() levels, decrypts to
    the FP64 mirror within 1e-3 (max-abs) and keeps the argmax."""
    from oracle import ckks
    from oracle import encoding as enc
    from oracle.circuit import HE, cutmax_he, required_rotations
    log_n = 11
    slots = 1 << (log_n - 1)
    pl = _cfg1_plan(slots)
    if packing_slots != slots:
        # padded packing: 1000 real entries in 1024 slots
        pl = P.calibrate(lambda i: synth.logits_gaussian(1000 + i, n=1000), 60, 1000, slots, 2, 3, 5.0,
                         k_fixed=2, d_fixed=2)
    ctx = ckks.Context(log_n, [60] + [40] * 21, [60, 60], dnum=11, seed=3)
    ctx.gen_relin_key()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    x = synth.logits_gaussian(5, n=pl.n)
    delta = 2.0 ** 40
    ct = ctx.encrypt(enc.encode(P.pack(x, slots, pl.packing), log_n, delta), delta, 1)
    z = cutmax_he(HE(ctx, delta), ct, pl)
    assert ctx.top_level - z.level == pl.depth()
    dec = enc.decode(ctx.decrypt(z), log_n, z.scale).real[: pl.n]
    ref = F.cutmax_circuit(x, pl)
    assert np.abs(dec - ref).max() < 1e-3
    assert np.argmax(dec) == np.argmax(x)


def test_chebyshev_interpolant_definition():
    """The interpolant passes through f at the d + 1 Chebyshev nodes, and a
    polynomial of degree <= d is reproduced exactly (T_3 -> e_3); numpy's
    Chebyshev fit at the same nodes gives the same coefficients."""
    from oracle.circuit import chebyshev_interpolant
    d = 15
    f = lambda t: np.exp(0.7 * t) / (2.0 + t)
    c = chebyshev_interpolant(f, d)
    nodes = np.cos(np.pi * (np.arange(d + 1) + 0.5) / (d + 1))
    assert np.abs(np.polynomial.chebyshev.chebval(nodes, c) - f(nodes)).max() < 1e-13
    assert np.abs(c - np.polynomial.chebyshev.chebfit(nodes, f(nodes), d)).max() < 1e-12
    e3 = chebyshev_interpolant(lambda t: 4 * t ** 3 - 3 * t, d)
    assert np.abs(e3 - np.eye(d + 1)[3]).max() < 1e-14


@pytest.mark.slow
def test_beta_noise_on_oracle_ciphertexts():
    """Alg. 3's cut noise G = U^(1/alpha) evaluated on oracle ciphertexts of
    uniforms (Lemma 2 / Observation 1): its decryption equals the degree-31
    Chebyshev series evaluated in float64 (up to CKKS noise) and U^(1/alpha)
    within the interpolation error for U >= 1e-2; 7 levels are spent."""
    from oracle import ckks
    from oracle import encoding as enc
    from oracle.circuit import HE, beta_noise_he, chebyshev_interpolant, nucleus_alpha
    log_n, delta, d = 10, 2.0 ** 40, 31
    ctx = ckks.Context(log_n, [60] + [40] * 8, [60, 60], dnum=3, seed=5)
    ctx.gen_relin_key()
    he = HE(ctx, delta)
    alpha = nucleus_alpha(0.9)
    assert alpha == pytest.approx(math.log(0.1) / math.log(0.9))
    assert nucleus_alpha(0.9, 0.95) == pytest.approx(math.log(0.05) / math.log(0.9))
    u = synth.uniforms(11, 1 << (log_n - 1))
    ct = ctx.encrypt(enc.encode(u, log_n, delta), delta, 3)
    G = beta_noise_he(he, ct, alpha, d)
    assert G.level == ctx.top_level - 7
    got = enc.decode(ctx.decrypt(G), log_n, G.scale).real
    c = chebyshev_interpolant(lambda t: ((t + 1) / 2) ** (1 / alpha), d)
    assert np.abs(got - np.polynomial.chebyshev.chebval(2 * u - 1, c)).max() < 1e-5
    big = u >= 1e-2
    grid = np.linspace(1e-2, 1, 20001)
    bound = np.abs(np.polynomial.chebyshev.chebval(2 * grid - 1, c) - grid ** (1 / alpha)).max()
    assert np.abs(got[big] - u[big] ** (1 / alpha)).max() < bound + 1e-5


# ------------------------------------------------ relaxed Goldschmidt steps (App. B)
def test_relaxed_goldschmidt_is_the_relaxed_newton_recursion():
    """With per-step constants alpha_i the coupled pair (g = x y, h = y/2) runs
    y <- y (alpha_i - x y^2 / 2): the recursion on y alone, written here without
    the pair, gives the same values; alpha_i = 3/2 is the plain iteration."""
    rng = np.random.default_rng(3)
    x = np.geomspace(1e-3, 2.0, 200)
    for k in (1, 2, 5, 9):
        al = list(rng.uniform(1.5, 2.2, size=k))
        y0 = 0.6
        y = np.full_like(x, y0)
        for a in al:
            y = y * (a - x * y * y / 2.0)
        assert np.allclose(F.goldschmidt_invsqrt(x, k, y0, al), y, rtol=1e-12, atol=0)
        assert (F.goldschmidt_invsqrt(x, k, y0, [1.5] * k) == F.goldschmidt_invsqrt(x, k, y0)).all()


def test_relaxed_plan_mirror_equals_plain_at_newton_constants():
    """The FP64 mirror with relaxation constants all 3/2 is the plain circuit, bit for bit."""
    pl = _cfg1_plan(8192)
    x = synth.logits_gaussian(4)
    rel = P.CutMaxPlan(**{**pl.to_dict(), "relax": [[1.5] * k for k in pl.k]})
    assert (F.cutmax_circuit(x, rel) == F.cutmax_circuit(x, pl)).all()


def test_relaxed_calibration_reaches_tolerance_in_fewer_steps():
    """calibrate(relax=True) on heavy-tailed logits (the config-2 shape, 2,000
    entries): every Goldschmidt iteration reaches the tolerance over the whole
    calibrated margin range (checked here against 1/sqrt(x) itself), in fewer
    steps in total than Newton's constant, with the argmax of the plan's FP64
    circuit correct on held-out vectors."""
    n, tol = 2000, 2.0 ** -10

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    kw = dict(margin=2.0, tol_k=tol, k_max=20, d_max=14, tol_d=tol, bootstrap=True)
    plain = P.calibrate(lambda i: gen(100 + i), 60, n, 2048, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], **kw)
    rel = P.calibrate(lambda i: gen(100 + i), 60, n, 2048, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], relax=True, **kw)
    assert sum(rel.k) < sum(plain.k)
    for t in range(4):
        a, b = rel.extra["V_range"][t]
        xs = np.geomspace(a * rel.kappa[t] / 2.0, b * rel.kappa[t] * 2.0, 3001)
        y = F.goldschmidt_invsqrt(xs, rel.k[t], rel.y0[t], rel.relax[t])
        assert np.abs(y * np.sqrt(xs) - 1.0).max() < tol
        assert len(rel.relax[t]) == rel.k[t] and all(1.5 <= v <= 3.5 for v in rel.relax[t])
    for s in range(30):
        x = gen(5000 + s)
        assert np.argmax(F.cutmax_circuit(x, rel)) == np.argmax(x)


def test_encrypted_relaxed_circuit_on_oracle():
    """Alg. 2 on oracle CKKS with relaxed Goldschmidt steps: the same levels
    as the plain plan, decrypted within 1e-3 of the relaxed FP64 mirror."""
    from oracle import ckks
    from oracle import encoding as enc
    from oracle.circuit import HE, cutmax_he, required_rotations
    log_n = 11
    slots = 1 << (log_n - 1)
    pl = P.CutMaxPlan(**{**_cfg1_plan(slots).to_dict(), "relax": [[1.8, 1.5], [1.7, 1.55]]})
    ctx = ckks.Context(log_n, [60] + [40] * 21, [60, 60], dnum=11, seed=3)
    ctx.gen_relin_key()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    x = synth.logits_gaussian(6, n=pl.n)
    delta = 2.0 ** 40
    ct = ctx.encrypt(enc.encode(P.pack(x, slots, pl.packing), log_n, delta), delta, 1)
    z = cutmax_he(HE(ctx, delta), ct, pl)
    assert ctx.top_level - z.level == pl.depth()
    dec = enc.decode(ctx.decrypt(z), log_n, z.scale).real[: pl.n]
    ref = F.cutmax_circuit(x, pl)
    assert np.abs(dec - ref).max() < 1e-3
    assert np.abs(ref - F.cutmax_circuit(x, _cfg1_plan(slots))).max() > 1e-6   # the constants take effect
