"""Batches of ciphertexts and vocabularies spread over several ciphertexts.

A batch (he_batch_pack) holds several ciphertexts back to back; every
operation on it runs once for all members.  Each member's result must be bit
for bit the result of the same operation on that ciphertext alone.  A
vocabulary longer than the slot count spreads over several zero-padded
ciphertexts (Sect. 3.2 assumes n = a * slots; the sums over the vocabulary
add the ciphertexts before the rotate-and-sum), checked bit for bit against
the oracle's circuit on the same ciphertext list and against the FP64 mirror.
"""
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
from paper_2509_08383_gb300 import plan as P        # noqa: E402
from paper_2509_08383_gb300 import synth            # noqa: E402

build.build_library()

LOG_N = 11
SLOTS = 1 << (LOG_N - 1)
CFG1_Q = [60] + [40] * 21
CFG1_P = [60, 60]
DELTA = 2.0 ** 40


@pytest.fixture(scope="module")
def small():
    g = he.Context(LOG_N, CFG1_Q, CFG1_P, dnum=11, seed=7)
    g.gen_relin_key()
    g.gen_rot_keys([1, 3, -2, 2, 4, 5, 6, 7])
    g.gen_galois_key(2 * g.n - 1)
    return g


def _members(g, b):
    return [g.batch_member(b, i).export() for i in range(b.batch)]


def test_batch_pack_and_member(small):
    g = small
    rng = np.random.default_rng(1)
    cts = [g.encrypt(rng.uniform(-1, 1, SLOTS), DELTA, i) for i in range(3)]
    b = g.batch_pack(cts)
    assert b.batch == 3 and b.level == cts[0].level
    for i, e in enumerate(_members(g, b)):
        assert (e == cts[i].export()).all()
    b2 = g.batch_pack([b, cts[1]])                 # batches concatenate
    assert b2.batch == 4
    assert (g.batch_member(b2, 3).export() == cts[1].export()).all()
    low = g.drop(cts[2], 5)                          # packed at the lowest level
    b3 = g.batch_pack([cts[0], low])
    assert b3.level == 5
    assert (g.batch_member(b3, 0).export() == g.drop(cts[0], 5).export()).all()
    with pytest.raises(he.HeError):                  # one ciphertext's data only
        b.export()


OPS = {
    "add": lambda g, x, y: g.add(x, y),
    "sub": lambda g, x, y: g.sub(x, y),
    "mul_relin": lambda g, x, y: g.mul(x, y),
    "mul_rescale": lambda g, x, y: g.rescale(g.mul(x, y)),
    "mul_rescale_fused": lambda g, x, y: g.mul_rescale(x, y),
    "rotate_1": lambda g, x, y: g.rotate(x, 1),
    "rotate_-2": lambda g, x, y: g.rotate(x, -2),
    "conjugate": lambda g, x, y: g.conj(x),
    "mul_const": lambda g, x, y: g.mul_const(x, 0.7, DELTA),
    "add_const": lambda g, x, y: g.add_const(x, 0.3),
    "mul_int": lambda g, x, y: g.mul_int(x, -5),
    "rotsum_3": lambda g, x, y: g.rotsum(x, 3),
    "rotsum_stage_3": lambda g, x, y: g.rotsum_stage(x, [1, 3, 4]),
    "drop_5": lambda g, x, y: g.drop(x, 5),
}


@pytest.mark.parametrize("name", sorted(OPS))
def test_batch_ops_bit_identical(small, name):
    g = small
    rng = np.random.default_rng(2)
    xs = [g.encrypt(rng.uniform(-1, 1, SLOTS), DELTA, 10 + i) for i in range(3)]
    ys = [g.encrypt(rng.uniform(-1, 1, SLOTS), DELTA, 20 + i) for i in range(3)]
    op = OPS[name]
    got = _members(g, op(g, g.batch_pack(xs), g.batch_pack(ys)))
    for i in range(3):
        assert (got[i] == op(g, xs[i], ys[i]).export()).all(), (name, i)


def _leveled_plan(n, seed0):
    return P.calibrate(lambda i: synth.logits_gaussian(seed0 + i, n=n), 40, n, SLOTS, 2, 3, 5.0,
                       k_fixed=2, d_fixed=2)


def test_batched_cutmax_equals_single_streams(small):
    g = small
    pl = _leveled_plan(1024, 3000)
    g.cutmax_prepare(pl)
    xs = [synth.logits_gaussian(40 + i) for i in range(3)]
    cts = [g.encrypt(P.pack(x, SLOTS, pl.packing), DELTA, 30 + i) for i, x in enumerate(xs)]
    Z = g.cutmax(g.batch_pack(cts), pl)
    assert Z.batch == 3
    got = _members(g, Z)
    for i in range(3):
        assert (got[i] == g.cutmax(cts[i], pl).export()).all()


def test_multict_stream_bit_exact_vs_oracle():
    n = 2500                                          # three ciphertexts, the last zero-padded
    pl = _leveled_plan(n, 5000)
    assert pl.cts == 3 and pl.packing == "pad" and pl.pad == 3 * SLOTS - n
    g = he.Context(LOG_N, CFG1_Q, CFG1_P, dnum=11, seed=9)
    o = ock.Context(LOG_N, CFG1_Q, CFG1_P, dnum=11, seed=9)
    g.cutmax_prepare(pl)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    x = synth.logits_gaussian(77, n=n)
    pts = [oenc.encode(v, LOG_N, DELTA) for v in P.pack_cts(x, SLOTS)]
    cg = [g.encrypt_poly(pt, DELTA, 40 + c) for c, pt in enumerate(pts)]
    co = [o.encrypt(pt, DELTA, 40 + c) for c, pt in enumerate(pts)]
    Zg = g.cutmax(g.batch_pack(cg), pl)
    Zo = cutmax_he(HE(o, DELTA), co, pl)
    for c in range(3):
        assert (g.batch_member(Zg, c).export() == Zo[c].export()).all(), c
    dec = np.concatenate([g.decrypt(g.batch_member(Zg, c)) for c in range(3)])[:n]
    ref = F.cutmax_circuit(x, pl)
    assert np.abs(dec - ref).max() < 1e-3
    assert int(np.argmax(dec)) == int(np.argmax(x))


# ------------------------------------------------------------------ bootstrapped batches
BQ = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
BP = [61] * 10
BH, BK, BR, BD = 64, 14, 4, 31


@pytest.fixture(scope="module")
def boot():
    g = he.Context(LOG_N, BQ, BP, dnum=3, h=BH, seed=23, arena_bytes=3 << 30)
    g.bootstrap_prepare(BK, BR, BD)
    return g


def test_batched_bootstrap_bit_identical(boot):
    g = boot
    rng = np.random.default_rng(5)
    cts = [g.encrypt(rng.uniform(-1, 1, SLOTS), DELTA, 50 + i, level=0) for i in range(2)]
    got = _members(g, g.bootstrap(g.batch_pack(cts)))
    for i in range(2):
        assert (got[i] == g.bootstrap(cts[i]).export()).all()


def test_batched_multict_bootstrapped_cutmax(boot):
    """Two streams of 2,300 logits (three ciphertexts each) in one batch, the
    paper's HE setting T = 4, p = [16, 4, 4, 6], c = [5, 3, 3, 3]."""
    g = boot
    n = 2300

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    pl = P.calibrate(lambda i: gen(7000 + i), 120, n, SLOTS, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                     tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True)
    assert pl.cts == 3
    g.cutmax_prepare(pl)
    xs = [gen(i) for i in range(2)]
    streams = [[g.encrypt(v, DELTA, 60 + 3 * s + c) for c, v in enumerate(P.pack_cts(x, SLOTS))]
               for s, x in enumerate(xs)]
    Z = g.cutmax(g.batch_pack([ct for st in streams for ct in st]), pl)
    assert Z.batch == 6
    for s, x in enumerate(xs):
        dec = np.concatenate([g.decrypt(g.batch_member(Z, 3 * s + c)) for c in range(3)])[:n]
        ref = F.cutmax_circuit(x, pl)
        assert np.abs(dec - ref).max() < 1e-3, s
        assert int(np.argmax(dec)) == int(np.argmax(x)) == int(np.argmax(F.cutmax_exact(x, 4, pl.p, pl.c)))
    # one stream alone gives the same ciphertexts
    Z1 = g.cutmax(g.batch_pack(streams[1]), pl)
    for c in range(3):
        assert (g.batch_member(Z1, c).export() == g.batch_member(Z, 3 + c).export()).all()


def test_shared_scalar_chains(boot):
    """Four streams of 1,000 logits in one batch with the scalar chains shared
    (one packed inverse-square-root and inverse chain for the batch): within
    1e-3 of each stream's FP64 mirror, argmax exact, and fewer bootstraps than
    four separate runs."""
    g = boot
    n = 1000

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    pl = P.calibrate(lambda i: gen(9000 + i), 120, n, SLOTS, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                     tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True)
    pl.shared = True
    g.cutmax_prepare(pl)
    xs = [gen(i) for i in range(4)]
    cts = [g.encrypt(P.pack(x, SLOTS, pl.packing), DELTA, 80 + i) for i, x in enumerate(xs)]
    g.ledger(reset=True)
    Z = g.cutmax(g.batch_pack(cts), pl)
    _, nb_shared = g.ledger(reset=True)
    g.cutmax(cts[0], pl)
    _, nb_one = g.ledger(reset=True)
    for s, x in enumerate(xs):
        dec = g.decrypt(g.batch_member(Z, s), n)
        assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-3, s
        assert int(np.argmax(dec)) == int(np.argmax(x))
    assert nb_shared < 4 * nb_one
