"""Bit-exact GPU vs oracle at the full-vocabulary parameter set: N = 2^16, the
30-prime chain of the benchmark (47-bit base, 13 x 40, 3 x 60, 10 x 60, 3 x 58
bits: logQ 1521), 10 special 61-bit primes, dnum = 3 (10-prime digits, a
10-prime P), ternary secret of Hamming weight 192.

These are the shapes a config-2 decode runs on: 10-prime digits through the
128-bit basis conversion, 40-row key inner products, a 10-prime ModDown.  Each
operation is compared with the oracle ciphertext for ciphertext (coefficient
form) at the top level (29) and at level 13, where computation happens between
bootstraps.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import ckks as ock                     # noqa: E402
from paper_2509_08383_gb300 import build, he       # noqa: E402

build.build_library()

CFG2_Q = [47] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
CFG2_P = [61] * 10
LOG_N = 16
SCALE = 2.0 ** 40


@pytest.fixture(scope="module")
def cfg2():
    g = he.Context(LOG_N, CFG2_Q, CFG2_P, dnum=3, h=192, seed=41, arena_bytes=6 << 30)
    o = ock.Context(LOG_N, CFG2_Q, CFG2_P, dnum=3, h=192, seed=41)
    assert g.primes == o.primes
    assert (g.secret() == o.secret()).all() and np.abs(g.secret()).sum() == 192
    for c in (g, o):
        c.gen_relin_key()
    g.gen_rot_keys([1])
    o.gen_rot_key(1)
    return g, o


def _pair_ct(g, o, level, ctr, seed):
    rng = np.random.default_rng(seed)
    m = np.rint(rng.normal(size=g.n) * SCALE)
    return g.encrypt_poly(m, SCALE, ctr, level), o.encrypt(m, SCALE, ctr, level)


def _same(a, b):
    return a.level == b.level and (a.export() == b.export()).all()


def test_cfg2_keys_match(cfg2):
    g, o = cfg2
    for digit in (0, 2):
        for which in (0, 1):
            assert (g.key_export(0, digit, which) == o.key_export(0, digit, which)).all()
    gr = ock.rot_galois(LOG_N, 1)
    assert (g.key_export(gr, 1, 0) == o.key_export(gr, 1, 0)).all()


@pytest.mark.parametrize("level", [29, 13])
def test_cfg2_keyswitch_bit_exact(cfg2, level):
    g, o = cfg2
    rng = np.random.default_rng(100 + level)
    d = np.stack([rng.integers(0, q, g.n, dtype=np.uint64) for q in g.primes[: level + 1]])
    og, oo = g.keyswitch(d, level, 0), o.keyswitch(d, level, 0)
    assert (og[0] == oo[0]).all() and (og[1] == oo[1]).all()


@pytest.mark.parametrize("level", [29, 13])
def test_cfg2_rotation_bit_exact(cfg2, level):
    g, o = cfg2
    a_g, a_o = _pair_ct(g, o, level, 5 + level, level)
    assert _same(g.rotate(a_g, 1), o.rotate(a_o, 1))


@pytest.mark.parametrize("level", [29, 13])
def test_cfg2_rescale_bit_exact(cfg2, level):
    g, o = cfg2
    a_g, a_o = _pair_ct(g, o, level, 40 + level, 1000 + level)
    r_g, r_o = g.rescale(a_g), o.rescale(a_o)
    assert _same(r_g, r_o) and r_g.scale == r_o.scale


@pytest.mark.parametrize("level", [29, 13])
def test_cfg2_product_relin_rescale_bit_exact(cfg2, level):
    """Tensor product, relinearisation (hybrid key switch) and rescale."""
    g, o = cfg2
    a_g, a_o = _pair_ct(g, o, level, 60 + level, 2000 + level)
    b_g, b_o = _pair_ct(g, o, level, 61 + level, 3000 + level)
    p_g, p_o = g.mul(a_g, b_g), o.mul(a_o, b_o)
    assert _same(p_g, p_o)
    r_g, r_o = g.rescale(p_g), o.rescale(p_o)
    assert _same(r_g, r_o) and r_g.scale == r_o.scale
    # the same product with its rescale in one rounded division by q_l P (11 divisor primes)
    f_g, f_o = g.mul_rescale(a_g, b_g), o.mul_rescale(a_o, b_o)
    assert _same(f_g, f_o) and f_g.scale == f_o.scale == r_o.scale


def test_cfg2_rotsum_stage_bit_exact(cfg2):
    """One hoisted stage of seven rotations (radix 8) at level 13: the fused
    seven-key inner product over 24 + 10 rows, one ModDown."""
    g, o = cfg2
    rots = list(range(1, 8))
    g.gen_rot_keys(rots)
    for r in rots[1:]:
        o.gen_rot_key(r)
    a_g, a_o = _pair_ct(g, o, 13, 90, 5000)
    s_g, s_o = g.rotsum_stage(a_g, rots), o.rotsum_stage(a_o, rots)
    assert _same(s_g, s_o) and s_g.scale == s_o.scale


def test_cfg2_decrypt_bit_exact(cfg2):
    g, o = cfg2
    a_g, a_o = _pair_ct(g, o, 13, 77, 4000)
    assert (g.decrypt_poly(a_g) == o.decrypt(a_o)).all()
