"""Pins of the CKKS oracle against things other than itself.

Each test checks the oracle against a textbook definition computed another
way (Python big integers, sympy, schoolbook products, brute-force sums) or
against an identity the mathematics fixes, chosen so that a dropped term, a
wrong sign, a wrong index or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest
import sympy

from oracle import ckks
from oracle import encoding as enc


# ------------------------------------------------------------- primes / psi
@pytest.mark.parametrize("log_n,bits", [(4, [30, 30, 31]), (11, [60, 40, 40, 60]), (14, [60] + [40] * 5 + [60, 60])])
def test_prime_chain_rule(log_n, bits):
    ps = [int(p) for p in ckks.gen_primes(log_n, bits)]
    two_n = 2 << log_n
    assert len(set(ps)) == len(ps)
    for b in sorted(set(bits)):
        chosen = [p for p, bb in zip(ps, bits) if bb == b]
        # every candidate k*2N+1 in (min chosen, 2^b) that is prime must be chosen
        k_hi = ((1 << b) - 1) // two_n
        k_lo = (min(chosen) - 1) // two_n
        expect = [k * two_n + 1 for k in range(k_hi, k_lo - 1, -1) if sympy.isprime(k * two_n + 1)]
        assert chosen == expect
        for p in chosen:
            assert p % two_n == 1 and p.bit_length() == b


@pytest.mark.parametrize("log_n", [3, 10, 16])
def test_psi_is_canonical_primitive_root(log_n):
    q = int(ckks.gen_primes(log_n, [50])[0])
    psi = int(ckks.lib().or_find_psi(q, log_n))
    n = 1 << log_n
    assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1
    # first x = 2,3,... whose (q-1)/2N power has order 2N
    for x in range(2, 200):
        c = pow(x, (q - 1) // (2 * n), q)
        if pow(c, n, q) == q - 1:
            assert c == psi
            break


# ------------------------------------------------------------- NTT
@pytest.mark.parametrize("log_n", [3, 4, 6])
def test_ntt_matches_evaluation_definition_bigint(log_n):
    n = 1 << log_n
    q = int(ckks.gen_primes(log_n, [40])[0])
    psi = int(ckks.lib().or_find_psi(q, log_n))
    rng = np.random.default_rng(log_n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    A = ckks.ntt(a, log_n, q)
    for i in range(n):
        e = 2 * int(format(i, f"0{log_n}b")[::-1], 2) + 1
        x = pow(psi, e, q)
        assert int(A[i]) == sum(int(a[k]) * pow(x, k, q) for k in range(n)) % q
    assert (ckks.ntt_def(a, log_n, q, psi) == A).all()


@pytest.mark.parametrize("log_n", [3, 4, 6])
def test_ntt_product_is_negacyclic_convolution(log_n):
    n = 1 << log_n
    q = int(ckks.gen_primes(log_n, [59])[0])
    rng = np.random.default_rng(7 + log_n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    A, B = ckks.ntt(a, log_n, q), ckks.ntt(b, log_n, q)
    prod = ckks.intt(np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64), log_n, q)
    # Python big-int negacyclic convolution
    ref = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                ref[k] += int(a[i]) * int(b[j])
            else:
                ref[k - n] -= int(a[i]) * int(b[j])
    assert [int(v) for v in prod] == [v % q for v in ref]
    assert (ckks.schoolbook(a, b, log_n, q) == prod).all()


@pytest.mark.parametrize("log_n", [10, 14, 16])
def test_ntt_inverse_roundtrip(log_n):
    q = int(ckks.gen_primes(log_n, [61])[0])
    rng = np.random.default_rng(log_n)
    a = rng.integers(0, q, 1 << log_n, dtype=np.uint64)
    assert (ckks.intt(ckks.ntt(a, log_n, q), log_n, q) == a).all()


# ------------------------------------------------------------- randomness
def test_philox_bijective_and_uniform():
    key = [0x1234, 0xABCD]
    outs = np.array([ckks.philox([i, 0, 0, 0], key) for i in range(4096)])
    assert len({tuple(o) for o in outs}) == 4096
    bits = np.unpackbits(outs.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01
    # changing one counter word or key word changes ~half the output bits
    a = ckks.philox([5, 6, 7, 8], key)
    for ctr, k in [([5, 6, 7, 9], key), ([5, 6, 7, 8], [0x1235, 0xABCD])]:
        b = ckks.philox(ctr, k)
        flips = np.unpackbits((a ^ b).view(np.uint8)).sum()
        assert 30 < flips < 98


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for ln in f:
            ln = ln.split("#")[0].split()
            if ln:
                rows.append(ln)
    return rows


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the published known-answer vectors of Salmon et
    al. (SC'11, Random123): a wrong multiplier, Weyl constant, round count or
    word order fails at least one of them."""
    rows = _golden("philox_kat.txt")
    assert len(rows) == 3
    for r in rows:
        w = [int(v, 16) for v in r]
        ctr, key, want = w[0:4], w[4:6], w[6:10]
        assert [int(v) for v in ckks.philox(ctr, key)] == want


def _discrete_gauss_cdf(sigma, bound=19):
    """P(|e| <= k), k = 0..bound-1, of the discrete Gaussian
    rho(x) = exp(-x^2 / (2 sigma^2)) on the integers |x| <= bound, 60 digits."""
    import mpmath
    mpmath.mp.dps = 60
    rho = [mpmath.exp(-mpmath.mpf(k) ** 2 / (2 * mpmath.mpf(sigma) ** 2)) for k in range(bound + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    out, acc = [], mpmath.mpf(0)
    for k in range(bound):
        acc += rho[k] if k == 0 else 2 * rho[k]
        out.append(acc / z)
    return out


def test_gaussian_cdt_is_the_discrete_gaussian():
    """The error sampler's thresholds are floor(2^64 P(|e| <= k)) of the
    discrete Gaussian of width 3.2 truncated to |e| <= 19, up to float64
    accumulation (a relative 7e-15).  A rounded continuous Gaussian differs by
    ~6e-4 in P(e = 0), a dropped factor 2 or a wrong width by far more."""
    import mpmath
    cdt = ckks.gauss_cdt(3.2)
    cdf = _discrete_gauss_cdf(3.2)
    for k in range(19):
        exact = int(mpmath.floor(cdf[k] * mpmath.mpf(2) ** 64))
        assert abs(int(cdt[k]) - exact) <= 1 << 17, k
    # the continuous Gaussian rounded to the nearest integer is a different table
    cont0 = mpmath.erf(mpmath.mpf(0.5) / (mpmath.mpf(3.2) * mpmath.sqrt(2)))
    assert abs(float(cdf[0]) - float(cont0)) > 5e-4


def test_gaussian_sampler_maps_philox_words_through_the_table():
    """Each error e_k takes one Philox block with counter (k, 0, object,
    domain) under the seed's key: |e_k| = #{j : cdt_j <= word1:word0} and the
    sign is bit 0 of word 2; recomputed here from the pinned Philox and the
    exact mpmath thresholds."""
    import mpmath
    seed, obj, dom, log_n = 0x0123456789ABCDEF, 7, 2, 12
    e = ckks.sample_gauss(seed, obj, dom, 3.2, log_n)
    cdf = _discrete_gauss_cdf(3.2)
    thr = [int(mpmath.floor(c * mpmath.mpf(2) ** 64)) for c in cdf]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in range(1 << log_n):
        w = [int(v) for v in ckks.philox([k, 0, obj, dom], key)]
        u = (w[1] << 32) | w[0]
        mag = sum(1 for t in thr if t <= u)
        assert int(e[k]) == (-mag if w[2] & 1 else mag)


def test_secret_distributions():
    s = ckks.sample_secret(11, 14, 0)
    counts = np.bincount(s.astype(np.int64) + 1, minlength=3) / len(s)
    assert np.allclose(counts, 1 / 3, atol=0.02)
    sp = ckks.sample_secret(11, 14, 192)
    assert (np.abs(sp) == 1).sum() == 192 and set(np.unique(sp)) <= {-1, 0, 1}


def test_gaussian_moments():
    e = ckks.sample_gauss(5, 3, 2, 3.2, 16)
    assert abs(e.mean()) < 0.06
    assert abs(e.std() - 3.2) < 0.05
    assert np.abs(e).max() <= 19


# ------------------------------------------------------------- encoding
@pytest.mark.parametrize("log_n", [4, 8, 10])
def test_encode_decode_match_defining_sums(log_n):
    rng = np.random.default_rng(log_n)
    h = (1 << log_n) // 2
    z = rng.normal(size=h) + 1j * rng.normal(size=h)
    m_fft = enc.encode_real_values(z, log_n, 2.0 ** 30)
    m_bf = enc.encode_bruteforce(z, log_n, 2.0 ** 30)
    assert np.abs(m_fft - m_bf).max() < 1e-3
    m = np.rint(m_fft)
    assert np.abs(enc.decode(m, log_n, 2.0 ** 30) - enc.decode_bruteforce(m, log_n, 2.0 ** 30)).max() < 1e-9
    # decoding the real-coefficient polynomial returns the slots
    assert np.abs(enc.decode(m, log_n, 2.0 ** 30) - z).max() < 1e-6


def test_slot_rotation_is_automorphism():
    """m(X) -> m(X^(5^r)) rotates the slots left by r (plaintext identity)."""
    log_n, n = 8, 256
    rng = np.random.default_rng(3)
    z = rng.normal(size=n // 2)
    m = enc.encode(z, log_n, 2.0 ** 30)
    for r in [1, 5, 64]:
        g = ckks.rot_galois(log_n, r)
        assert g == pow(5, r, 2 * n)
        out = np.zeros(n)
        for k in range(n):
            e = (k * g) % (2 * n)
            if e < n:
                out[e] = m[k]
            else:
                out[e - n] = -m[k]
        assert np.abs(enc.decode(out, log_n, 2.0 ** 30).real - np.roll(z, -r)).max() < 1e-6


# ------------------------------------------------------------- encryption / ops
@pytest.fixture(scope="module")
def small_ctx():
    ctx = ckks.Context(10, [60, 40, 40, 40], [60, 60], dnum=2, seed=21)
    ctx.gen_relin_key()
    for r in [1, 2, 3]:
        ctx.gen_rot_key(r)
    ctx.gen_galois_key(ctx.conj_galois())
    return ctx


def _enc_vec(ctx, z, ctr, scale=2.0 ** 40):
    return ctx.encrypt(enc.encode(z, ctx.log_n, scale), scale, ctr)


def test_decrypt_is_message_plus_small_error(small_ctx):
    """Dec(Enc(m)) = m + e with |e| bounded by the Gaussian tail (Sect. 2.1)."""
    ctx = small_ctx
    rng = np.random.default_rng(1)
    m = np.rint(rng.normal(size=ctx.n) * 2.0 ** 35)
    ct = ctx.encrypt(m, 2.0 ** 35, 9)
    e = ctx.decrypt(ct) - m
    assert np.abs(e).max() <= 19 and np.abs(e).std() > 1.0
    # c0 + c1*s with the exported secret, in big integers, limb 0
    s = ctx.secret().astype(np.int64)
    c = ct.export()
    q0 = ctx.primes[0]
    c0 = [int(v) for v in c[0, 0]]
    c1 = [int(v) for v in c[1, 0]]
    n = ctx.n
    acc = list(c0)
    for i in range(n):
        if c1[i] == 0:
            continue
        for j in np.nonzero(s)[0]:
            k = i + int(j)
            v = c1[i] * int(s[j])
            if k < n:
                acc[k] += v
            else:
                acc[k - n] -= v
    acc = [((v % q0) + q0 // 2) % q0 - q0 // 2 for v in acc[:64]]
    assert np.array_equal(np.array(acc, dtype=np.float64), ctx.decrypt(ct)[:64])


def test_homomorphic_add_mul_rotate_conj(small_ctx):
    ctx = small_ctx
    rng = np.random.default_rng(2)
    h = ctx.slots
    a = rng.normal(size=h)
    b = rng.normal(size=h) + 1j * rng.normal(size=h)
    ca, cb = _enc_vec(ctx, a, 1), _enc_vec(ctx, b, 2)
    dec = lambda ct: enc.decode(ctx.decrypt(ct), ctx.log_n, ct.scale)
    assert np.abs(dec(ctx.add(ca, cb)) - (a + b)).max() < 1e-8
    assert np.abs(dec(ctx.sub(ca, cb)) - (a - b)).max() < 1e-8
    prod = ctx.rescale(ctx.mul(ca, cb))
    assert prod.level == ctx.top_level - 1
    assert abs(prod.scale - 2.0 ** 80 / ctx.primes[ctx.top_level]) < 1e-6 * prod.scale
    assert np.abs(dec(prod) - a * b).max() < 1e-7
    assert np.abs(dec(ctx.rotate(cb, 3)) - np.roll(b, -3)).max() < 1e-7
    assert np.abs(dec(ctx.conj(cb)) - np.conj(b)).max() < 1e-7
    assert np.abs(dec(ctx.mul_int(ca, -7)) - (-7 * a)).max() < 1e-7
    # multiplying by the monomial X^(N/2) multiplies every slot by i
    assert np.abs(dec(ctx.mul_monomial(cb, ctx.n // 2)) - 1j * b).max() < 1e-8


def test_keyswitch_relation(small_ctx):
    """(o0, o1) = KS(d) satisfies o0 + o1*s = d*s^2 + small (mod q_i), every limb."""
    ctx = small_ctx
    l, n = ctx.top_level, ctx.n
    rng = np.random.default_rng(4)
    d = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.primes[: l + 1]])
    o0, o1 = ctx.keyswitch(d, l, 0)
    s = ctx.secret().astype(np.int64)
    for i in range(l + 1):
        q = ctx.primes[i]
        sq = ckks.ntt(np.mod(s, q).astype(np.uint64), ctx.log_n, q)
        s2 = np.array([(int(x) * int(x)) % q for x in sq], dtype=np.uint64)
        mul = lambda x, y: ckks.intt(np.array([(int(u) * int(v)) % q for u, v in
                                               zip(ckks.ntt(x, ctx.log_n, q), y)], dtype=np.uint64), ctx.log_n, q)
        lhs = (o0[i].astype(object) + mul(o1[i], sq).astype(object)) % q
        rhs = mul(d[i], s2).astype(object)
        diff = np.array([((int(x) - int(y)) % q + q // 2) % q - q // 2 for x, y in zip(lhs, rhs)])
        # key-switching noise: far below q_i
        assert np.abs(diff).max() < 2 ** 20


def test_moddown_is_rounded_division():
    """ModDown of hybrid key switching is the rounded division round(x / P) by
    the special modulus P, checked with Python integers on random x in
    (-Q_l P / 2, Q_l P / 2) and on the x whose x / P lies closest to a rounding
    boundary from either side (x mod P = (P - 1)/2 or (P + 1)/2), and 0, +-1.
    An approximate conversion from P to Q_l (off by up to one P per special
    prime) fails this."""
    import random
    ctx = ckks.Context(10, [60, 40, 40, 40], [60, 60, 61], dnum=2, seed=3)
    n, l, K = ctx.n, 2, 3
    qs, ps = ctx.primes[: l + 1], ctx.primes[ctx.nq:]
    P, M = math.prod(ps), math.prod(qs) * math.prod(ps)
    rng = random.Random(7)
    edge = [0, 1, -1, (P - 1) // 2, (P + 1) // 2, -(P - 1) // 2, -(P + 1) // 2]
    for _ in range(24):
        k = rng.randrange(-math.prod(qs) // 2 + 1, math.prod(qs) // 2 - 1)
        edge += [k * P + (P - 1) // 2, k * P + (P + 1) // 2]
    xs0 = edge + [rng.randrange(-M // 2 + 1, M // 2) for _ in range(n - len(edge))]
    xs1 = [rng.randrange(-M // 2 + 1, M // 2) for _ in range(n)]
    rows = list(qs) + list(ps)
    acc0 = np.array([[x % p for x in xs0] for p in rows], dtype=np.uint64)
    acc1 = np.array([[x % p for x in xs1] for p in rows], dtype=np.uint64)
    o0, o1 = ctx.moddown(acc0, acc1, l)
    for xs, o in ((xs0, o0), (xs1, o1)):
        r = [(2 * x + P) // (2 * P) for x in xs]          # round(x / P); P odd: no ties
        want = np.array([[v % q for v in r] for q in qs], dtype=np.uint64)
        assert (o == want).all()


def test_rescale_divides_by_last_prime(small_ctx):
    ctx = small_ctx
    rng = np.random.default_rng(5)
    m = np.rint(rng.normal(size=ctx.n) * 2.0 ** 50)
    ct = ctx.encrypt(m, 2.0 ** 50, 3)
    r = ctx.rescale(ct)
    ql = ctx.primes[ctx.top_level]
    # each rounded coefficient errs by <= 1/2, so Dec errs by <= (1 + |s|_1)/2
    bound = 0.5 * (1 + np.abs(ctx.secret()).sum()) + 20.0 / ql
    err = np.abs(ctx.decrypt(r) - m / ql)
    assert err.max() <= bound and r.scale == 2.0 ** 50 / ql


def test_mod_raise_adds_multiple_of_q0():
    """ModRaise of a level-0 ciphertext decrypts, over Q, to m + e + q0*I with
    |I| <= (|s|_1 + 1)/2 (centred lift), checked exactly in big integers."""
    h = 16
    ctx = ckks.Context(10, [60, 40, 40], [60], dnum=3, h=h, seed=8)
    rng = np.random.default_rng(6)
    m = np.rint(rng.normal(size=ctx.n) * 2.0 ** 30)
    ct0 = ctx.encrypt(m, 2.0 ** 30, 4, level=0)
    up = ctx.mod_raise(ct0, 2)
    s = ctx.secret().astype(np.int64)
    assert np.abs(s).sum() == h
    n, q = ctx.n, ctx.primes
    c = up.export()
    lo = ctx.decrypt(ct0)                     # m + e, exact (fits a double)
    assert np.abs(lo - m).max() <= 19
    Q = q[0] * q[1] * q[2]
    # CRT of each lifted coefficient, then c0 + c1*s over the integers mod Q
    def crt(limbs):
        out = []
        for k in range(n):
            v = 0
            for i in range(3):
                Mi = Q // q[i]
                v += int(limbs[i][k]) * Mi * pow(Mi, -1, q[i])
            v %= Q
            out.append(v - Q if v > Q // 2 else v)
        return out
    c0, c1 = crt(c[0]), crt(c[1])
    t = list(c0)
    for j in np.nonzero(s)[0]:
        for k in range(n):
            idx = k + int(j)
            if idx < n:
                t[idx] += c1[k] * int(s[j])
            else:
                t[idx - n] -= c1[k] * int(s[j])
    t = [((v % Q) + Q // 2) % Q - Q // 2 for v in t]
    for k in range(n):
        I, r = divmod(t[k] - int(lo[k]), q[0])
        assert r == 0 and abs(I) <= (h + 1) // 2 + 1


def test_hoisted_rotsum_stage():
    """A hoisted stage a + sum_r rot(a, r) (one ModUp of c1 whose digits are
    read through each automorphism, the key products summed, one ModDown) is
    a valid key switch: with one rotation its decryption equals that of
    add(a, rot(a, r)) up to key-switching noise (exact integers; the two
    differ only in where the approximate basis conversion meets the
    automorphism's sign flips); with seven it decrypts to the sum of the
    rotated slot vectors (App. D), and a full rotate-and-sum in stages of 8
    puts the total in every slot."""
    from oracle.circuit import HE, rotsum_stages
    ctx = ckks.Context(10, [60, 40, 40, 40], [60, 60], dnum=2, seed=13)
    rots = sorted({r for st in rotsum_stages(9, 3) for r in st} | {5})
    for r in rots:
        ctx.gen_rot_key(r)
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, ctx.slots)
    scale = 2.0 ** 40
    a = ctx.encrypt(enc.encode(z, 10, scale), scale, 7)
    one = ctx.rotsum_stage(a, [5])
    ref = ctx.add(a, ctx.rotate(a, 5))
    assert one.level == ref.level and one.scale == ref.scale
    assert np.abs(ctx.decrypt(one) - ctx.decrypt(ref)).max() < 2 ** 20
    assert not (one.export() == ref.export()).all()    # a different, equally valid key switch
    seven = ctx.rotsum_stage(a, list(range(1, 8)))
    want = sum(np.roll(z, -r) for r in range(8))
    assert np.abs(enc.decode(ctx.decrypt(seven), 10, seven.scale).real - want).max() < 1e-6
    full = HE(ctx, scale).rotsum(a, 9)
    assert np.abs(enc.decode(ctx.decrypt(full), 10, full.scale).real - z.sum()).max() < 1e-5
    with pytest.raises(RuntimeError):
        ctx.rotsum_stage(a, [11])                    # no key for 11


def test_mul_rescale_one_rounding():
    """The product with its rescale in one rounded division by q_l P decrypts
    like rescale(mul(a, b)) (they differ by the rounding of one division
    instead of two: a few units per coefficient), at the same level and scale,
    and to the slot-wise product of the messages."""
    ctx = ckks.Context(10, [60, 40, 40, 40], [60, 60, 61], dnum=2, seed=23)
    ctx.gen_relin_key()
    rng = np.random.default_rng(8)
    za, zb = rng.uniform(-1, 1, ctx.slots), rng.uniform(-1, 1, ctx.slots)
    scale = 2.0 ** 40
    a = ctx.encrypt(enc.encode(za, 10, scale), scale, 1)
    b = ctx.encrypt(enc.encode(zb, 10, scale), scale, 2)
    fused, ref = ctx.mul_rescale(a, b), ctx.rescale(ctx.mul(a, b))
    assert fused.level == ref.level == ctx.top_level - 1 and fused.scale == ref.scale
    d = np.abs(ctx.decrypt(fused) - ctx.decrypt(ref))
    assert d.max() <= 0.5 * (1 + np.abs(ctx.secret()).sum()) + 1
    got = enc.decode(ctx.decrypt(fused), 10, fused.scale).real
    assert np.abs(got - za * zb).max() < 1e-6
    low = ctx.drop(a, 0)
    with pytest.raises(RuntimeError):
        ctx.mul_rescale(low, low)                    # level 0 cannot be rescaled
