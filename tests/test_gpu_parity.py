"""CUDA path vs the CPU oracle, through the C ABI.

Integer work (NTT, keys, encryption, key switching, rescale, rotations, the
whole leveled circuit) must match bit for bit given the same integer
plaintexts and seeds.  Float64 encoding may differ in the last bit of a
coefficient before rounding, so encodings are compared within +-1.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import ckks as ock                     # noqa: E402
from oracle import cutmax_fp64 as F                # noqa: E402
from oracle import encoding as oenc                # noqa: E402
from oracle.circuit import HE, cutmax_he, nucleus_he, required_rotations  # noqa: E402
from paper_2509_08383_gb300 import build, he       # noqa: E402
from paper_2509_08383_gb300 import plan as P       # noqa: E402
from paper_2509_08383_gb300 import synth           # noqa: E402

build.build_library()

CFG1_Q = [60] + [40] * 21
CFG1_P = [60, 60]


def pair(log_n, qbits, pbits, dnum, h=0, seed=5):
    g = he.Context(log_n, qbits, pbits, dnum, h=h, seed=seed)
    o = ock.Context(log_n, qbits, pbits, dnum, h=h, seed=seed)
    return g, o


@pytest.fixture(scope="module")
def small():
    g, o = pair(11, CFG1_Q, CFG1_P, dnum=11)
    for c in (g, o):
        c.gen_relin_key()
    return g, o


# ------------------------------------------------------------------ NTT
@pytest.mark.parametrize("log_n", [10, 11, 12, 13, 14, 15, 16])
def test_ntt_bit_exact(log_n):
    qbits = [60, 40, 61, 36]
    g = he.Context(log_n, qbits, [60], dnum=2, arena_bytes=256 << 20)
    primes = g.primes
    rng = np.random.default_rng(log_n)
    data = np.stack([rng.integers(0, q, 1 << log_n, dtype=np.uint64) for q in primes[:4]])
    t = torch.from_numpy(data.view(np.int64)).cuda()
    g.ntt_device(t, 0)
    got = t.cpu().numpy().view(np.uint64)
    for i in range(4):
        assert (got[i] == ock.ntt(data[i], log_n, primes[i])).all()
    g.ntt_device(t, 0, inverse=True)
    assert (t.cpu().numpy().view(np.uint64) == data).all()
    # edge values: all zeros and all q-1
    for fill in ("zero", "max"):
        d2 = np.stack([np.full(1 << log_n, 0 if fill == "zero" else q - 1, dtype=np.uint64) for q in primes[:4]])
        t2 = torch.from_numpy(d2.view(np.int64).copy()).cuda()
        g.ntt_device(t2, 0)
        got2 = t2.cpu().numpy().view(np.uint64)
        for i in range(4):
            assert (got2[i] == ock.ntt(d2[i], log_n, primes[i])).all()


# ------------------------------------------------------------------ context, keys, encryption
def test_primes_secret_keys_match(small):
    g, o = small
    assert g.primes == o.primes
    assert (g.secret() == o.secret()).all()
    for digit in (0, o.beta - 1):
        for which in (0, 1):
            assert (g.key_export(0, digit, which) == o.key_export(0, digit, which)).all()
    gr = ock.rot_galois(11, 5)
    g.gen_galois_key(gr)
    o.gen_galois_key(gr)
    assert (g.key_export(gr, 3, 0) == o.key_export(gr, 3, 0)).all()


def test_sparse_secret_matches():
    g, o = pair(12, [60, 40, 40], [60], dnum=3, h=64, seed=9)
    s = g.secret()
    assert (s == o.secret()).all() and np.abs(s).sum() == 64


def test_encrypt_decrypt_bit_exact(small):
    g, o = small
    rng = np.random.default_rng(1)
    m = np.rint(rng.normal(size=g.n) * 2.0 ** 40)
    for level in (-1, 0, 5):
        cg = g.encrypt_poly(m, 2.0 ** 40, 77, level)
        co = o.encrypt(m, 2.0 ** 40, 77, None if level < 0 else level)
        assert (cg.export() == co.export()).all()
        assert (g.decrypt_poly(cg) == o.decrypt(co)).all()


def test_encode_within_one(small):
    g, o = small
    rng = np.random.default_rng(2)
    z = rng.normal(size=g.slots) + 1j * rng.normal(size=g.slots)
    mg = g.encode(z, 2.0 ** 40)
    mo = oenc.encode(z, g.log_n, 2.0 ** 40)
    assert np.abs(mg - mo).max() <= 1
    assert (mg != mo).mean() < 0.05
    ct = g.encrypt(z, 2.0 ** 40, 3)
    assert np.abs(g.decrypt(ct, complex_out=True) - z).max() < 1e-6


# ------------------------------------------------------------------ operations
def _same_ct(g, o, rng, level=None, scale=2.0 ** 40, ctr=11):
    m = np.rint(rng.normal(size=g.n) * scale)
    return g.encrypt_poly(m, scale, ctr, -1 if level is None else level), o.encrypt(m, scale, ctr, level)


def test_ops_bit_exact(small):
    g, o = small
    rng = np.random.default_rng(3)
    a_g, a_o = _same_ct(g, o, rng, ctr=1)
    b_g, b_o = _same_ct(g, o, rng, ctr=2)
    eq = lambda x, y: (x.export() == y.export()).all() and x.level == y.level
    assert eq(g.add(a_g, b_g), o.add(a_o, b_o))
    assert eq(g.sub(a_g, b_g), o.sub(a_o, b_o))
    assert eq(g.mul_int(a_g, -12345), o.mul_int(a_o, -12345))
    assert eq(g.add_const(a_g, 0.75), o.add_intd(a_o, float(np.rint(0.75 * a_o.scale))))
    prod_g, prod_o = g.mul(a_g, b_g), o.mul(a_o, b_o)
    assert eq(prod_g, prod_o)
    rs_g, rs_o = g.rescale(prod_g), o.rescale(prod_o)
    assert eq(rs_g, rs_o) and rs_g.scale == rs_o.scale
    # product and rescale in one rounded division by q_l P
    mr_g, mr_o = g.mul_rescale(a_g, b_g), o.mul_rescale(a_o, b_o)
    assert eq(mr_g, mr_o) and mr_g.scale == mr_o.scale == rs_o.scale
    # constant multiplication with the scale rule
    c, target = -0.3125, 2.0 ** 40
    E = (target * float(o.primes[a_o.level])) / a_o.scale
    ref = o.rescale(o.mul_intd(a_o, float(np.rint(c * E)), a_o.scale * E))
    got = g.mul_const(a_g, c, target)
    assert eq(got, ref) and got.scale == ref.scale
    # mixed levels: product at the lower level
    low_g, low_o = g.drop(a_g, 7), o.drop(a_o, 7)
    assert eq(g.mul(low_g, b_g), o.mul(low_o, o.drop(b_o, 7)))


@pytest.mark.parametrize("r", [1, 2, 64, 511, -3])
def test_rotation_bit_exact(small, r):
    g, o = small
    rng = np.random.default_rng(4)
    a_g, a_o = _same_ct(g, o, rng, ctr=5)
    g.gen_rot_keys([r])
    o.gen_rot_key(r)
    assert (g.rotate(a_g, r).export() == o.rotate(a_o, r).export()).all()


def test_conjugation_and_low_level_rotation(small):
    g, o = small
    rng = np.random.default_rng(5)
    a_g, a_o = _same_ct(g, o, rng, level=3, ctr=6)
    cj = 2 * g.n - 1
    g.gen_galois_key(cj)
    o.gen_galois_key(cj)
    assert (g.conj(a_g).export() == o.conj(a_o).export()).all()
    g.gen_rot_keys([1])
    o.gen_rot_key(1)
    a0_g, a0_o = _same_ct(g, o, rng, level=0, ctr=7)
    assert (g.rotate(a0_g, 1).export() == o.rotate(a0_o, 1).export()).all()


@pytest.mark.parametrize("rots", [[3], [1, 2, 3, 4, 5, 6, 7], [8, 16, 24, 32, 40, 48, 56], [-2, 5, 511]])
def test_rotsum_stage_bit_exact(small, rots):
    """A hoisted stage a + sum_r rot(a, r) (one shared ModUp, the key products
    of every rotation summed by the fused inner-product kernel, one ModDown):
    bit-exact to the oracle's, written from the definition."""
    g, o = small
    rng = np.random.default_rng(len(rots) + sum(rots))
    a_g, a_o = _same_ct(g, o, rng, ctr=41)
    g.gen_rot_keys(rots)
    for r in rots:
        o.gen_rot_key(r)
    s_g, s_o = g.rotsum_stage(a_g, rots), o.rotsum_stage(a_o, rots)
    assert s_g.level == s_o.level and s_g.scale == s_o.scale
    assert (s_g.export() == s_o.export()).all()


@pytest.mark.parametrize("log_radix", [1, 2, 3, 4])
def test_rotsum_radix_bit_exact(log_radix):
    """he_rotsum over 10 doublings in hoisted stages of radix 2, 4, 8 and 16:
    bit-exact to the oracle's stages, and every slot holds the total."""
    from oracle.circuit import rotsum_stages
    g, o = pair(11, CFG1_Q, CFG1_P, dnum=11, seed=19)
    g.set_rotsum_radix(log_radix)
    rots = sorted({r for st in rotsum_stages(10, log_radix) for r in st})
    g.gen_rot_keys(rots)
    for r in rots:
        o.gen_rot_key(r)
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, g.slots)
    pt = oenc.encode(z, g.log_n, 2.0 ** 40)
    s_g = g.rotsum(g.encrypt_poly(pt, 2.0 ** 40, 3), 10)
    s_o = HE(o, 2.0 ** 40, log_radix).rotsum(o.encrypt(pt, 2.0 ** 40, 3), 10)
    assert (s_g.export() == s_o.export()).all()
    assert np.abs(g.decrypt(s_g) - z.sum()).max() < 1e-5
    with pytest.raises(he.HeError):
        g.set_rotsum_radix(5)


@pytest.mark.parametrize("level", [0, 1, 9, 21])
def test_keyswitch_raw_bit_exact(small, level):
    g, o = small
    rng = np.random.default_rng(level)
    d = np.stack([rng.integers(0, q, g.n, dtype=np.uint64) for q in g.primes[: level + 1]])
    og = g.keyswitch(d, level, 0)
    oo = o.keyswitch(d, level, 0)
    assert (og[0] == oo[0]).all() and (og[1] == oo[1]).all()


def _moddown_inputs(ctx, l, seed):
    """Accumulators over q_0..q_l, p_0..p_(K-1) holding random x in
    (-Q_l P/2, Q_l P/2) and, in polynomial 0, every x whose x / P lies closest
    to a rounding boundary (x mod P = (P -+ 1)/2, near several multiples of P)."""
    import math
    import random
    qs, ps = ctx.primes[: l + 1], ctx.primes[ctx.nq:]
    P, M = math.prod(ps), math.prod(qs) * math.prod(ps)
    rng = random.Random(seed)
    edge = [0, 1, -1, (P - 1) // 2, (P + 1) // 2, -(P - 1) // 2, -(P + 1) // 2]
    for _ in range(60):
        k = rng.randrange(-math.prod(qs) // 2 + 1, math.prod(qs) // 2 - 1)
        edge += [k * P + (P - 1) // 2, k * P + (P + 1) // 2, k * P - (P - 1) // 2, k * P - (P + 1) // 2]
    xs0 = edge + [rng.randrange(-M // 2 + 1, M // 2) for _ in range(ctx.n - len(edge))]
    xs1 = [rng.randrange(-M // 2 + 1, M // 2) for _ in range(ctx.n)]
    rows = list(qs) + list(ps)
    acc0 = np.array([[x % p for x in xs0] for p in rows], dtype=np.uint64)
    acc1 = np.array([[x % p for x in xs1] for p in rows], dtype=np.uint64)
    want = []
    for xs in (xs0, xs1):
        r = [(2 * x + P) // (2 * P) for x in xs]          # round(x / P); P odd: no ties
        want.append(np.array([[v % q for v in r] for q in qs], dtype=np.uint64))
    return acc0, acc1, want


@pytest.mark.parametrize("pbits", [[60, 60, 61], [61] * 10])
def test_moddown_exact_at_rounding_boundaries(pbits):
    """ModDown is the rounded division by P on the GPU too, including the x
    nearest to +-P/2, where the float64 estimate of the rounding cannot decide
    and the exact mixed-radix comparison takes over; bit-exact to the oracle."""
    qb = [60, 40, 40, 40]
    g = he.Context(10, qb, pbits, dnum=2, seed=3, arena_bytes=256 << 20)
    o = ock.Context(10, qb, pbits, dnum=2, seed=3)
    for l in (0, 2, 3):
        acc0, acc1, want = _moddown_inputs(o, l, 7 + l)
        g0, g1 = g.moddown(acc0, acc1, l)
        o0, o1 = o.moddown(acc0, acc1, l)
        assert (g0 == want[0]).all() and (g1 == want[1]).all()
        assert (o0 == g0).all() and (o1 == g1).all()


def test_rescale_chain_to_zero(small):
    g, o = small
    rng = np.random.default_rng(6)
    a_g, a_o = _same_ct(g, o, rng, ctr=8)
    for _ in range(a_g.level):
        a_g, a_o = g.rescale(a_g), o.rescale(a_o)
        assert (a_g.export() == a_o.export()).all()
    assert a_g.level == 0
    with pytest.raises(he.HeError) as ei:
        g.rescale(a_g)
    assert ei.value.code == he.HE_ELEVEL


def test_missing_key_is_an_error(small):
    g, _ = small
    rng = np.random.default_rng(7)
    a = g.encrypt_poly(np.rint(rng.normal(size=g.n) * 2 ** 30), 2.0 ** 30, 9)
    with pytest.raises(he.HeError) as ei:
        g.automorphism(a, 2 * 777 + 1)
    assert ei.value.code == he.HE_ENOKEY


# ------------------------------------------------------------------ CutMax circuit
def _cfg1_plan(slots, n=1024):
    return P.calibrate(lambda i: synth.logits_gaussian(1000 + i, n=n), 60, n, slots, 2, 3, 5.0, k_fixed=2, d_fixed=2)


def _circuit_pair(log_n, seed=3):
    g, o = pair(log_n, CFG1_Q, CFG1_P, dnum=11, seed=seed)
    return g, o


def _run_cutmax_pair(g, o, pl, x, ctr=1):
    delta = 2.0 ** 40
    pt = oenc.encode(P.pack(x, g.slots, pl.packing), g.log_n, delta)
    g.cutmax_prepare(pl)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    zg = g.cutmax(g.encrypt_poly(pt, delta, ctr), pl)
    zo = cutmax_he(HE(o, delta), o.encrypt(pt, delta, ctr), pl)
    return zg, zo


@pytest.mark.parametrize("seed", [0, 5])
def test_cutmax_bit_exact_small(seed):
    """Whole leveled CutMax (Alg. 2), N = 2^11, 21 levels: bit-exact ciphertexts."""
    g, o = _circuit_pair(11)
    pl = _cfg1_plan(g.slots)
    x = synth.logits_gaussian(seed)
    zg, zo = _run_cutmax_pair(g, o, pl, x)
    assert zg.level == zo.level == 0 and zg.scale == zo.scale
    assert (zg.export() == zo.export()).all()
    dec = g.decrypt(zg, pl.n)
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3
    assert np.argmax(dec) == np.argmax(x)


def test_cutmax_relaxed_bit_exact():
    """Leveled CutMax with relaxed Goldschmidt steps (per-step constants in
    place of 3/2), N = 2^11: bit-exact ciphertexts, the FP64 mirror within 1e-3."""
    g, o = _circuit_pair(11)
    pl = P.CutMaxPlan(**{**_cfg1_plan(g.slots).to_dict(), "relax": [[1.8, 1.5], [1.7, 1.55]]})
    x = synth.logits_gaussian(8)
    zg, zo = _run_cutmax_pair(g, o, pl, x)
    assert zg.level == zo.level == 0 and zg.scale == zo.scale
    assert (zg.export() == zo.export()).all()
    assert np.abs(g.decrypt(zg, pl.n) - F.cutmax_circuit(x, pl)).max() < 1e-3


def test_relax_constant_out_of_range_is_an_error():
    g = he.Context(11, CFG1_Q, CFG1_P, dnum=11, seed=4)
    pl = P.CutMaxPlan(**{**_cfg1_plan(g.slots).to_dict(), "relax": [[0.5, 1.5], [1.5, 1.5]]})
    with pytest.raises(he.HeError) as ei:
        g.cutmax_prepare(pl)
    assert ei.value.code == he.HE_ERANGE


def test_cutmax_cfg1_full_size():
    """Config 1: N = 2^14, 1024 logits replicated 8x, T = 2, p = 3: bit-exact."""
    g, o = _circuit_pair(14)
    pl = _cfg1_plan(g.slots)
    x = synth.logits_gaussian(11)
    zg, zo = _run_cutmax_pair(g, o, pl, x)
    assert (zg.export() == zo.export()).all()
    dec = g.decrypt(zg, pl.n)
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3
    assert np.abs(dec - F.cutmax_exact(x, 2, 3, 5.0)).max() < 1e-3
    assert np.argmax(dec) == np.argmax(x)


def test_cutmax_padded_packing():
    """n = 1000 real logits zero-padded into 1024 slots (mask + variance correction)."""
    g = he.Context(11, CFG1_Q, CFG1_P, dnum=11, seed=4)
    pl = _cfg1_plan(g.slots, n=1000)
    assert pl.packing == "pad"
    x = synth.logits_gaussian(2, n=1000)
    g.cutmax_prepare(pl)
    z = g.cutmax(g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 1), pl)
    dec = g.decrypt(z)
    assert np.abs(dec[:1000] - F.cutmax_circuit(x, pl)).max() < 1e-3
    assert np.abs(dec[1000:]).max() < 1e-3
    assert np.argmax(dec[:1000]) == np.argmax(x)


def test_nucleus_bit_exact():
    """Alg. 3 with client-encrypted Beta(alpha,1) cut noise (HE_RAND_BETA):
    bit-exact to the oracle."""
    g, o = _circuit_pair(11, seed=8)
    pl = _cfg1_plan(g.slots)
    x = synth.logits_gaussian(3)
    alpha = F.beta_alpha(0.9)
    G = F.beta_noise(synth.uniforms(3, pl.n), alpha)
    delta = 2.0 ** 40
    ptx = oenc.encode(P.pack(x, g.slots, pl.packing), g.log_n, delta)
    ptg = oenc.encode(P.pack(G, g.slots, pl.packing), g.log_n, delta)
    g.cutmax_prepare(pl)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    zg = g.nucleus_sample(g.encrypt_poly(ptx, delta, 1), g.encrypt_poly(ptg, delta, 2), pl, 0.9)
    zo = nucleus_he(HE(o, delta), o.encrypt(ptx, delta, 1), o.encrypt(ptg, delta, 2), pl)
    assert (zg.export() == zo.export()).all()
    assert np.argmax(g.decrypt(zg, pl.n)) == np.argmax(x + G)


@pytest.mark.parametrize("top_p,q", [(0.9, 0.0), (0.95, 0.9)])
def test_nucleus_uniform_noise_matches_oracle(top_p, q):
    """Alg. 3 with the cut noise drawn by the server (HE_RAND_UNIFORM): the
    library takes alpha = ln(1-q)/ln(p) (Lemma 2 / Observation 1) and evaluates
    G = U^(1/alpha) on the encrypted uniforms, then CutMax(X + G).  The oracle
    runs the same steps with its own Chebyshev evaluation (each T_k by
    recurrence), so the ciphertexts differ in rounding: the noise agrees within
    1e-5, the sample within 1e-3, and the argmax is the one of x + the noise
    polynomial in float64."""
    from oracle.circuit import beta_noise_he, chebyshev_interpolant, nucleus_alpha
    qb, pb = [60] + [40] * 28, [60, 60, 60]
    g, o = pair(11, qb, pb, dnum=10, seed=12)
    pl = _cfg1_plan(g.slots)
    x = synth.logits_gaussian(21)
    u = synth.uniforms(21, pl.n)
    delta = 2.0 ** 40
    ptx = oenc.encode(P.pack(x, g.slots, pl.packing), g.log_n, delta)
    ptu = oenc.encode(P.pack(u, g.slots, pl.packing), g.log_n, delta)
    g.cutmax_prepare(pl)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    xg, ug = g.encrypt_poly(ptx, delta, 1), g.encrypt_poly(ptu, delta, 2)
    xo, uo = o.encrypt(ptx, delta, 1), o.encrypt(ptu, delta, 2)
    alpha = nucleus_alpha(top_p, q)
    Gg = g.decrypt(g.beta_noise(ug, alpha, he.HE_NUCLEUS_DEGREE), pl.n)
    Go_ct = beta_noise_he(HE(o, delta), uo, alpha, he.HE_NUCLEUS_DEGREE)
    Go = oenc.decode(o.decrypt(Go_ct), g.log_n, Go_ct.scale).real[: pl.n]
    assert np.abs(Gg - Go).max() < 1e-5
    zg = g.nucleus_sample(xg, ug, pl, top_p, q, kind="uniform")
    zo = nucleus_he(HE(o, delta), xo, uo, pl, top_p, q, kind="uniform", degree=he.HE_NUCLEUS_DEGREE)
    assert zg.level == zo.level and zg.scale == pytest.approx(zo.scale, rel=1e-12)
    dg = g.decrypt(zg, pl.n)
    do = oenc.decode(o.decrypt(zo), g.log_n, zo.scale).real[: pl.n]
    assert np.abs(dg - do).max() < 1e-3
    c = chebyshev_interpolant(lambda t: ((t + 1) / 2) ** (1 / alpha), he.HE_NUCLEUS_DEGREE)
    want = int(np.argmax(x + np.polynomial.chebyshev.chebval(2 * u - 1, c)))
    assert int(np.argmax(dg)) == int(np.argmax(do)) == want


def test_beta_noise_at_the_uniforms_scale_on_60bit_levels():
    """The cut noise from uniforms encrypted at scale 2^60 seven levels above
    the 40-bit levels (on the 60-bit primes of the bootstrapping chain, where
    a product keeps a 2^60 scale): the series works at U's scale and lands on
    the 40-bit levels at Delta, seven levels lower; GPU and oracle agree
    within 1e-5 and follow the interpolant of U^(1/alpha) in float64."""
    from oracle.circuit import beta_noise_he, chebyshev_interpolant, nucleus_alpha
    qb, pb = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3, [61] * 10
    g, o = pair(11, qb, pb, dnum=3, h=64, seed=14)
    g.gen_relin_key()
    o.gen_relin_key()
    u = synth.uniforms(33, g.slots)
    su, lu = 2.0 ** 60, 20
    ptu = oenc.encode(u, g.log_n, su)
    ug, uo = g.encrypt_poly(ptu, su, 5, level=lu), o.encrypt(ptu, su, 5, level=lu)
    alpha = nucleus_alpha(0.9)
    Gg_ct = g.beta_noise(ug, alpha, he.HE_NUCLEUS_DEGREE)
    Go_ct = beta_noise_he(HE(o, 2.0 ** 40), uo, alpha, he.HE_NUCLEUS_DEGREE)
    assert Gg_ct.level == Go_ct.level == lu - 7
    assert Gg_ct.scale == pytest.approx(2.0 ** 40, rel=1e-9) and Go_ct.scale == pytest.approx(2.0 ** 40, rel=1e-9)
    Gg = g.decrypt(Gg_ct)
    Go = oenc.decode(o.decrypt(Go_ct), g.log_n, Go_ct.scale).real
    assert np.abs(Gg - Go).max() < 1e-5
    c = chebyshev_interpolant(lambda t: ((t + 1) / 2) ** (1 / alpha), he.HE_NUCLEUS_DEGREE)
    assert np.abs(Gg - np.polynomial.chebyshev.chebval(2 * u - 1, c)).max() < 1e-5


def test_nucleus_groups_equal_per_group_calls():
    """nucleus_sample_groups: two streams at top-p 0.9 and 0.95 in one batch
    (server-drawn noise, per-stream scalar chains) give each stream the bits
    of nucleus_sample on it alone; bad groupings are HE_EINVAL."""
    qb, pb = [60] + [40] * 28, [60, 60, 60]
    g = he.Context(11, qb, pb, dnum=10, seed=12)
    pl = _cfg1_plan(g.slots)
    g.cutmax_prepare(pl)
    xs = [synth.logits_gaussian(30 + s) for s in range(2)]
    us = [synth.uniforms(30 + s, pl.n) for s in range(2)]
    X = [g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 40 + s) for s, x in enumerate(xs)]
    U = [g.encrypt(P.pack(u, g.slots, pl.packing), g.delta, 50 + s) for s, u in enumerate(us)]
    ps = [0.9, 0.95]
    Z = g.nucleus_sample_groups(g.batch_pack(X), g.batch_pack(U), pl, ps, kind="uniform")
    for s in range(2):
        z1 = g.nucleus_sample(X[s], U[s], pl, ps[s], kind="uniform")
        zs = g.batch_member(Z, s)
        assert zs.level == z1.level and zs.scale == z1.scale and (zs.export() == z1.export()).all()
    for bad in ([0.9, 0.95, 0.9], [0.9, 1.5]):
        with pytest.raises(he.HeError) as e:
            g.nucleus_sample_groups(g.batch_pack(X), g.batch_pack(U), pl, bad, kind="uniform")
        assert e.value.code == he.HE_EINVAL


def test_nucleus_and_add_reject_bad_arguments(small):
    """Top-p mass outside (0, 1), an unknown noise kind and operands of
    different scales are HE_EINVAL (an addition of mismatched scales would
    silently change the message)."""
    g, _ = small
    rng = np.random.default_rng(9)
    a = g.encrypt(rng.normal(size=g.slots), 2.0 ** 40, 31)
    b = g.encrypt(rng.normal(size=g.slots), 2.0 ** 40 * (1 + 1e-6), 32)
    with pytest.raises(he.HeError) as ei:
        g.add(a, b)
    assert ei.value.code == he.HE_EINVAL
    pl = _cfg1_plan(g.slots)
    for top_p, q in ((1.0, 0.0), (0.0, 0.0), (0.9, 1.0)):
        with pytest.raises(he.HeError) as ei:
            g.nucleus_sample(a, a, pl, top_p, q)
        assert ei.value.code == he.HE_EINVAL
    with pytest.raises(he.HeError) as ei:
        g.nucleus_sample(a, b, pl, 0.9)
    assert ei.value.code == he.HE_EINVAL


def test_circuit_too_deep_is_an_error():
    g = he.Context(11, [60] + [40] * 8, CFG1_P, dnum=3, seed=1)
    pl = _cfg1_plan(g.slots)
    g.cutmax_prepare(pl)
    ct = g.encrypt(np.zeros(g.slots), g.delta, 1)
    with pytest.raises(he.HeError) as ei:
        g.cutmax(ct, pl)
    assert ei.value.code == he.HE_ELEVEL


def test_ledger_model_matches_leveled_circuit():
    from paper_2509_08383_gb300 import ledger
    g = he.Context(11, CFG1_Q, CFG1_P, dnum=11, seed=6)
    pl = _cfg1_plan(g.slots)
    g.cutmax_prepare(pl)
    ct = g.encrypt(P.pack(synth.logits_gaussian(4), g.slots, pl.packing), g.delta, 1)
    g.ledger(reset=True)
    g.cutmax(ct, pl)
    ks, nb = g.ledger(reset=True)
    model, nb_model = ledger.cutmax_ledger(pl, len(CFG1_Q), 11)
    assert nb == nb_model == 0
    assert {i: int(v) for i, v in enumerate(ks) if v} == model
