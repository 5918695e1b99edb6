"""Pins of the bootstrapping oracle: the slot-root matrix against the
encoding's defining sums, its unitarity, the Chebyshev approximation of the
scaled cosine, and an end-to-end refresh of a level-0 ciphertext."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as Ch

from oracle import ckks
from oracle import encoding as enc
from oracle.bootstrap import Bootstrapper, chebyshev_coeffs, evalmod_function, slot_roots_matrix


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
