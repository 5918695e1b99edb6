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


def _bitrev(n):
    b = n.bit_length() - 1
    return np.array([int(format(i, f"0{b}b")[::-1], 2) for i in range(n)])


def test_bootstrap_stages(boot_pair):
    """Each stage of the GPU bootstrapping against its closed form.

    ModRaise gives t = m + q0 I; CoeffToSlot puts (t_j + i t_(j+h)) / (q0 (K+1))
    in bit-reversed slot order; EvalMod gives sin(2 pi (K+1) x) of its input
    slots (the Chebyshev series must not add more than ~1e-11, since the
    read-out multiplies its error by q0 / (2 pi s_fix)); the recombined
    ciphertext holds the message coefficients m / s_fix.
    """
    g, _, _ = boot_pair
    h = g.slots
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, h)
    delta = 2.0 ** 40
    pt = oenc.encode(z, LOG_N, delta)
    ct = g.encrypt_poly(pt, delta, 11, level=0)
    br = _bitrev(h)
    s0 = g.bootstrap_stage(ct, 0)
    t = g.decrypt_poly(s0)
    I = np.round((t - pt) / g.primes[0])
    assert np.abs(t - pt - I * g.primes[0]).max() < 2 ** 12     # t = m + q0 I (+ encryption noise)
    assert np.abs(I).max() <= K
    cvec = ((t[:h] + 1j * t[h:]) / s0.scale)[br]
    d3 = g.decrypt(g.bootstrap_stage(ct, 3), complex_out=True)
    assert np.abs(d3 - cvec).max() < 1e-12
    d4 = g.decrypt(g.bootstrap_stage(ct, 4), complex_out=True)
    d5 = g.decrypt(g.bootstrap_stage(ct, 5), complex_out=True)
    assert np.abs(d4 - cvec.real).max() < 1e-12
    assert np.abs(d5 - cvec.imag).max() < 1e-12
    d6 = g.decrypt(g.bootstrap_stage(ct, 6), complex_out=True)
    d7 = g.decrypt(g.bootstrap_stage(ct, 7), complex_out=True)
    assert np.abs(d6 - np.sin(2 * np.pi * (K + 1) * d4.real)).max() < 1e-11
    assert np.abs(d7 - np.sin(2 * np.pi * (K + 1) * d5.real)).max() < 1e-11
    d8 = g.decrypt(g.bootstrap_stage(ct, 8), complex_out=True)
    mvec = ((pt[:h] + 1j * pt[h:]) / delta)[br]
    assert np.abs(d8 - mvec).max() < 1e-7


def test_constant_bootstrap(boot_pair):
    """Bootstrapping of one complex value in every slot by the trace over
    X -> X^(5^k): the value comes back within the bootstrapping error at the
    general bootstrap's output level; for a slot vector that is not constant
    the trace is the projection onto the constants, so the result is the slot
    average (coefficient 0 of the plaintext is the mean real part, coefficient
    N/2 the mean imaginary part); a batch gives each member's own result."""
    g, _, _ = boot_pair
    h = g.slots
    g.gen_rot_keys([1 << i for i in range(LOG_N - 1)])
    delta = 2.0 ** 40
    val = 0.3 - 0.7j
    pt = oenc.encode(np.full(h, val), LOG_N, delta)
    others = np.delete(np.arange(2 * h), [0, h])
    assert np.abs(pt[others]).max() == 0 and pt[0] == round(0.3 * delta) and pt[h] == round(-0.7 * delta)
    c1 = g.encrypt_poly(pt, delta, 21, level=0)
    b1 = g.bootstrap_const(c1)
    assert b1.level == len(QB) - 1 - 16
    assert abs(b1.scale / delta - 1) < 1e-9          # lands on the input's scale, as he_bootstrap does
    assert np.abs(g.decrypt(b1, complex_out=True) - val).max() < 1e-6
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, h) + 1j * rng.uniform(-1, 1, h)
    c2 = g.encrypt_poly(oenc.encode(z, LOG_N, delta), delta, 22, level=3)
    b2 = g.bootstrap_const(c2)
    assert np.abs(g.decrypt(b2, complex_out=True) - z.mean()).max() < 1e-6
    bb = g.bootstrap_const(g.batch_pack([c1, g.drop(c2, 0)]))
    for i, b in enumerate((b1, b2)):
        assert (g.batch_member(bb, i).export() == b.export()).all()


@pytest.mark.parametrize("scale_ratio", [1.03, 0.97])
def test_bootstrap_reads_message_at_any_input_scale(boot_pair, scale_ratio):
    """A circuit's scales drift away from Delta; both bootstraps must hand back
    the input's message (not the message times the squared scale ratio)."""
    g, _, _ = boot_pair
    g.gen_rot_keys([1 << i for i in range(LOG_N - 1)])
    scale = 2.0 ** 40 * scale_ratio
    rng = np.random.default_rng(6)
    z = rng.uniform(-1, 1, g.slots)
    b = g.bootstrap(g.encrypt(z, scale, 31, level=0))
    assert np.abs(g.decrypt(b) - z).max() < 1e-6
    val = 0.4 + 0.1j
    bc = g.bootstrap_const(g.encrypt(np.full(g.slots, val), scale, 32, level=0))
    assert np.abs(g.decrypt(bc, complex_out=True) - val).max() < 1e-6


def test_constant_bootstrap_matches_oracle(boot_pair):
    """GPU and oracle constant bootstraps of the same ciphertext (bit-identical
    inputs) both return the value, to each other's precision."""
    g, o, ob = boot_pair
    g.gen_rot_keys([1 << i for i in range(LOG_N - 1)])
    ob.gen_const_keys()
    delta = 2.0 ** 40
    val = 0.45 + 0.2j
    pt = oenc.encode(np.full(g.slots, val), LOG_N, delta)
    cg = g.encrypt_poly(pt, delta, 41, level=0)
    co = o.encrypt(pt, delta, 41, level=0)
    assert (cg.export() == co.export()).all()
    bg = g.bootstrap_const(cg)
    bo = ob.bootstrap_const(co)
    assert bg.level == bo.level
    dg = g.decrypt(bg, complex_out=True)
    do = oenc.decode(o.decrypt(bo), LOG_N, bo.scale)
    assert np.abs(dg - val).max() < 1e-6 and np.abs(do - val).max() < 1e-6
    assert np.abs(dg - do).max() < 1e-6
