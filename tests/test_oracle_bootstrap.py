"""Pins of the bootstrapping oracle: the slot-root matrix against the
encoding's defining sums, its unitarity, the Chebyshev approximation of the
scaled cosine, and an end-to-end refresh of a level-0 ciphertext."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as Ch

from oracle import ckks
from oracle import encoding as enc
from oracle.bootstrap import Bootstrapper, chebyshev_coeffs, evalmod_function, slot_roots_matrix, trace


@pytest.mark.parametrize("log_n", [4, 8])
def test_slot_roots_matrix_is_decoding(log_n):
    n = 1 << log_n
    h = n // 2
    rng = np.random.default_rng(log_n)
    m = rng.normal(size=n)
    V = slot_roots_matrix(log_n)
    w = m[:h] + 1j * m[h:]
    assert np.allclose(V @ w, enc.decode_bruteforce(m, log_n, 1.0))
    assert np.allclose(V @ V.conj().T, h * np.eye(h))


@pytest.mark.parametrize("K,d", [(14, 40), (24, 48)])
def test_chebyshev_scaled_cosine(K, d):
    f = evalmod_function(K, 3)
    c = chebyshev_coeffs(f, d)
    x = np.linspace(-1, 1, 5001)
    assert np.abs(Ch.chebval(x, c) - f(x)).max() < 1e-12
    # r = 3 double angles of cos(theta/8) give cos(theta) = sin(2 pi (K+1) x)
    y = f(x)
    for _ in range(3):
        y = 2 * y * y - 1
    assert np.allclose(y, np.sin(2 * np.pi * (K + 1) * x), atol=1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("scale_ratio", [1.0, 1.03])
def test_oracle_bootstrap_refreshes(scale_ratio):
    """Refresh of a level-0 ciphertext back to its own message, at the
    bootstrapping's reference scale and at a scale 3 % off it (a circuit's
    scales drift away from Delta)."""
    log_n = 11
    qb = [55] + [40] * 3 + [60] * 3 + [60] * 10 + [58] * 3
    ctx = ckks.Context(log_n, qb, [61] * 7, dnum=3, h=64, seed=2)
    bs = Bootstrapper(ctx, K=14, r=3, d=40)
    bs.gen_keys()
    rng = np.random.default_rng(0)
    z = rng.uniform(-1, 1, ctx.slots)
    scale = 2.0 ** 40 * scale_ratio
    ct = ctx.encrypt(enc.encode(z, log_n, scale), scale, 1, level=0)
    out = bs.bootstrap(ct)
    assert out.level == len(qb) - 1 - 16
    dec = enc.decode(ctx.decrypt(out), log_n, out.scale)
    assert np.abs(dec - z).max() < 1e-6


def _decrypt_exact(ctx, ct):
    """c0 + c1 s over the integers mod Q_level (centred), by CRT of the exported limbs."""
    n, q, lv = ctx.n, ctx.primes, ct.level
    Q = 1
    for i in range(lv + 1):
        Q *= q[i]
    c = ct.export()

    def crt(limbs):
        out = []
        for k in range(n):
            v = 0
            for i in range(lv + 1):
                Mi = Q // q[i]
                v += int(limbs[i][k]) * Mi * pow(Mi, -1, q[i])
            out.append(v % Q)
        return out
    c0, c1 = crt(c[0]), crt(c[1])
    s = ctx.secret().astype(np.int64)
    t = list(c0)
    for j in np.nonzero(s)[0]:
        for k in range(n):
            idx = k + int(j)
            if idx < n:
                t[idx] += c1[k] * int(s[j])
            else:
                t[idx - n] -= c1[k] * int(s[j])
    return [((v % Q) + Q // 2) % Q - Q // 2 for v in t]


def test_trace_keeps_coefficients_0_and_half():
    """The trace of a ModRaised ciphertext decrypts, over Q, to
    (N/2) (t_0 + t_(N/2) X^(N/2)) with t the raised plaintext, up to the
    key-switching noise of its rotations: exact big-integer check."""
    ctx = ckks.Context(8, [60, 40, 40], [60, 60], dnum=3, h=16, seed=5)
    for i in range(7):                               # rotations 1, 2, ..., N/4
        ctx.gen_rot_key(1 << i)
    rng = np.random.default_rng(8)
    m = np.rint(rng.normal(size=ctx.n) * 2.0 ** 30)
    up = ctx.mod_raise(ctx.encrypt(m, 2.0 ** 30, 3, level=0), 2)
    t = _decrypt_exact(ctx, up)
    tr = _decrypt_exact(ctx, trace(ctx, up))
    n, h = ctx.n, ctx.n // 2
    noise = 2 ** 24
    assert abs(t[0]) > 2 ** 50                       # t_0 = m_0 + q0 I_0 is far above the noise
    assert abs(tr[0] - h * t[0]) < noise and abs(tr[h] - h * t[h]) < noise
    assert max(abs(tr[k]) for k in range(n) if k not in (0, h)) < noise


@pytest.mark.slow
def test_oracle_constant_bootstrap():
    """One complex value in every slot comes back at the input's scale (3 %
    off the reference scale); a vector that is not constant comes back as its
    slot average (the trace is the projection onto the constants)."""
    log_n = 11
    qb = [55] + [40] * 3 + [60] * 3 + [60] * 10 + [58] * 3
    ctx = ckks.Context(log_n, qb, [61] * 7, dnum=3, h=64, seed=2)
    bs = Bootstrapper(ctx, K=14, r=4, d=31)
    bs.gen_keys()
    bs.gen_const_keys()
    scale = 2.0 ** 40 * 1.03
    val = 0.3 - 0.7j
    ct = ctx.encrypt(enc.encode(np.full(ctx.slots, val), log_n, scale), scale, 1, level=0)
    out = bs.bootstrap_const(ct)
    assert out.level == bs.out_level() and abs(out.scale / scale - 1) < 1e-9
    assert np.abs(enc.decode(ctx.decrypt(out), log_n, out.scale) - val).max() < 1e-6
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, ctx.slots) + 1j * rng.uniform(-1, 1, ctx.slots)
    out = bs.bootstrap_const(ctx.encrypt(enc.encode(z, log_n, 2.0 ** 40), 2.0 ** 40, 2, level=0))
    assert np.abs(enc.decode(ctx.decrypt(out), log_n, out.scale) - z.mean()).max() < 1e-6
