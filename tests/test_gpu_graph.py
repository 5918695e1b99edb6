"""cutmax through a CUDA graph (he_cutmax_graph) against direct calls.

The graph replays the kernels of a direct call on the same data, so every
output must be bit-identical to cutmax on the same input: on the first call
(which runs directly and captures), on replays, on replays with another input,
with batches, after a plan change (a second graph) and after a change of the
rotate-and-sum radix (the graph retires and is captured again).  The ledger
must advance on a replay exactly as on a direct call, and clearing the graphs
must give their memory back.  The direct calls are themselves bit-exact to
the oracle (test_gpu_parity.py); the bootstrapped circuit is checked here
against the FP64 mirror as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import cutmax_fp64 as F                 # noqa: E402
from paper_2509_08383_gb300 import build, he        # noqa: E402
from paper_2509_08383_gb300 import plan as P        # noqa: E402
from paper_2509_08383_gb300 import synth            # noqa: E402

build.build_library()

CFG1_Q, CFG1_P = [60] + [40] * 21, [60, 60]
QB = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
PB = [61] * 10
NV = 1000


def _same(a, b):
    return a.level == b.level and a.scale == b.scale and a.batch == b.batch and (a.export() == b.export()).all()


def _export_batch(g, z):
    return np.concatenate([g.batch_member(z, i).export().ravel() for i in range(z.batch)])


@pytest.fixture(scope="module")
def leveled():
    g = he.Context(11, CFG1_Q, CFG1_P, dnum=11, seed=3)
    pl = P.calibrate(lambda i: synth.logits_gaussian(1000 + i, n=1024), 60, 1024, g.slots, 2, 3, 5.0, k_fixed=2,
                     d_fixed=2)
    g.cutmax_prepare(pl)
    return g, pl


def test_graph_leveled_bit_identical_and_replayed(leveled):
    g, pl = leveled
    xs = [synth.logits_gaussian(s) for s in range(3)]
    cts = [g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 10 + s) for s, x in enumerate(xs)]
    c0 = g.graph_stats()
    direct = [g.cutmax(ct, pl) for ct in cts]
    outs = [g.cutmax_graph(cts[0], pl), g.cutmax_graph(cts[0], pl), g.cutmax_graph(cts[1], pl),
            g.cutmax_graph(cts[2], pl)]
    c1 = g.graph_stats()
    assert (c1[0] - c0[0], c1[1] - c0[1], c1[2] - c0[2]) == (1, 3, 0)
    for z, d in zip(outs, [direct[0], direct[0], direct[1], direct[2]]):
        assert _same(z, d)
    for s, x in enumerate(xs):
        assert int(np.argmax(g.decrypt(outs[s + 1], pl.n))) == int(np.argmax(x))


def test_graph_ledger_and_launches_advance_as_direct(leveled):
    g, pl = leveled
    ct = g.encrypt(P.pack(synth.logits_gaussian(7), g.slots, pl.packing), g.delta, 77)
    g.cutmax_graph(ct, pl)                      # captured (or already)
    g.ledger(reset=True)
    l0 = he.launch_count()
    g.cutmax(ct, pl)
    l_direct = he.launch_count() - l0
    ops_d = g.ledger_ops()                      # read before the reset
    ks_d, nb_d = g.ledger(reset=True)
    l0 = he.launch_count()
    g.cutmax_graph(ct, pl)
    l_graph = he.launch_count() - l0
    ops_g = g.ledger_ops()
    ks_g, nb_g = g.ledger(reset=True)
    assert list(ks_g) == list(ks_d) and nb_g == nb_d
    for k in ops_d:
        assert list(ops_g[k]) == list(ops_d[k])
    assert l_graph == l_direct


def test_graph_batch_and_plan_change(leveled):
    g, pl = leveled
    xs = [synth.logits_gaussian(20 + s) for s in range(2)]
    cts = [g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 30 + s) for s, x in enumerate(xs)]
    batch = g.batch_pack(cts)
    c0 = g.graph_stats()
    d = g.cutmax(batch, pl)
    z1, z2 = g.cutmax_graph(batch, pl), g.cutmax_graph(batch, pl)
    assert (_export_batch(g, z1) == _export_batch(g, d)).all() and (_export_batch(g, z2) == _export_batch(g, d)).all()
    # another plan (c = 4): a second graph, bit-identical to its own direct call
    pl2 = P.CutMaxPlan(**{**pl.to_dict(), "c": [4.0, 4.0]})
    g.cutmax_prepare(pl2)
    d2 = g.cutmax(cts[0], pl2)
    y1, y2 = g.cutmax_graph(cts[0], pl2), g.cutmax_graph(cts[0], pl2)
    assert _same(y1, d2) and _same(y2, d2)
    c1 = g.graph_stats()
    assert c1[0] - c0[0] == 2 and c1[1] - c0[1] == 2


def test_graph_radix_change_recaptures_and_clear_frees(leveled):
    g, pl = leveled
    ct = g.encrypt(P.pack(synth.logits_gaussian(40), g.slots, pl.packing), g.delta, 40)
    g.cutmax_graph(ct, pl)
    g.set_rotsum_radix(2)
    g.cutmax_prepare(pl)
    d = g.cutmax(ct, pl)
    c0 = g.graph_stats()
    z1, z2 = g.cutmax_graph(ct, pl), g.cutmax_graph(ct, pl)
    c1 = g.graph_stats()
    assert _same(z1, d) and _same(z2, d)
    assert (c1[0] - c0[0], c1[1] - c0[1]) == (1, 1)
    g.set_rotsum_radix(3)
    del z1, z2, d
    before = g.memory()[0]
    g.graph_clear()
    assert g.memory()[0] < before
    z = g.cutmax_graph(ct, pl)                  # captured again after the clear
    assert _same(z, g.cutmax(ct, pl))


def test_graph_under_profiling_runs_directly(leveled):
    g, pl = leveled
    ct = g.encrypt(P.pack(synth.logits_gaussian(50), g.slots, pl.packing), g.delta, 50)
    c0 = g.graph_stats()
    he.profile_enable(0)
    try:
        z = g.cutmax_graph(ct, pl)
    finally:
        he.profile_enable(-1)
    c1 = g.graph_stats()
    assert c1[2] - c0[2] == 1
    assert _same(z, g.cutmax(ct, pl))


def test_graph_bootstrapped_bit_identical():
    """Bootstrapped CutMax (T = 4, p = [16, 4, 4, 6], refreshes, constant
    bootstraps), N = 2^11: the graph's outputs equal the direct call's bits and
    match the FP64 mirror."""
    pl = P.calibrate(lambda i: synth.logits_heavy_tail(1000 + i, n=NV, heavy=5, gap=0.2), 200, NV, 1 << 10, 4,
                     [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0, tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6,
                     bootstrap=True)
    g = he.Context(11, QB, PB, dnum=3, h=64, seed=21)
    g.bootstrap_prepare(14, 4, 31)
    g.cutmax_prepare(pl)
    xs = [synth.logits_heavy_tail(s, n=NV, heavy=5, gap=[0.05, 0.2, 1.0][s]) for s in range(3)]
    cts = [g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 1 + s) for s, x in enumerate(xs)]
    outs = [g.cutmax_graph(ct, pl) for ct in cts]
    assert g.graph_stats()[:2] == (1, 2)
    for x, ct, z in zip(xs, cts, outs):
        assert _same(z, g.cutmax(ct, pl))
        dec = g.decrypt(z)
        assert np.abs(dec[:NV] - F.cutmax_circuit(x, pl)).max() < 1e-3
        assert int(np.argmax(dec[:NV])) == int(np.argmax(x))


def test_context_switch_routes_cutmax_and_nucleus_through_graphs(leveled):
    """he_ctx_set_graphs: cutmax and nucleus_sample (client-drawn noise) give
    the direct calls' bits, through replayed graphs."""
    g, pl = leveled
    x = synth.logits_gaussian(60)
    G = F.beta_noise(synth.uniforms(60, pl.n), F.beta_alpha(0.9))
    ct = g.encrypt(P.pack(x, g.slots, pl.packing), g.delta, 60)
    gb = g.encrypt(P.pack(G, g.slots, pl.packing), g.delta, 62)
    d = [g.cutmax(ct, pl), g.nucleus_sample(ct, gb, pl, 0.9)]
    c0 = g.graph_stats()
    g.set_graphs(True)
    try:
        for _ in range(2):
            r = [g.cutmax(ct, pl), g.nucleus_sample(ct, gb, pl, 0.9)]
            for a, b in zip(r, d):
                assert _same(a, b)
    finally:
        g.set_graphs(False)
    c1 = g.graph_stats()
    assert c1[1] - c0[1] >= 2      # the second round replays
    assert int(np.argmax(g.decrypt(d[1], pl.n))) == int(np.argmax(x + G))


def test_graph_count_is_bounded_least_recently_used_first(leveled):
    """A context keeps at most 16 graphs: after 17 plans the first one's graph
    is gone (using it again captures anew), the most recent ones replay, and
    every output still equals the direct call's bits."""
    g, pl = leveled
    g.graph_clear()
    ct = g.encrypt(P.pack(synth.logits_gaussian(70), g.slots, pl.packing), g.delta, 70)
    plans = [P.CutMaxPlan(**{**pl.to_dict(), "c": [5.0 + 0.25 * i, 5.0]}) for i in range(17)]
    for p in plans:
        g.cutmax_prepare(p)
    c0 = g.graph_stats()
    for p in plans:                                   # 17 captures; the 17th evicts plans[0]
        g.cutmax_graph(ct, p)
    c1 = g.graph_stats()
    assert c1[0] - c0[0] == 17
    z = g.cutmax_graph(ct, plans[16])                 # still held: a replay
    assert g.graph_stats()[1] - c1[1] == 1 and _same(z, g.cutmax(ct, plans[16]))
    z = g.cutmax_graph(ct, plans[0])                  # evicted: captured again
    assert g.graph_stats()[0] - c1[0] == 1 and _same(z, g.cutmax(ct, plans[0]))
    g.graph_clear()
