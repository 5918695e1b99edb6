"""Host logic of the autotuner: the coordinate search, the rejection of a
candidate that loses an argmax, and the JSON round trip keyed by parameter
set.  A fake context and timer stand in for the GPU."""
import json

from paper_2509_08383_gb300 import autotune
from paper_2509_08383_gb300 import plan as P

Q, PB = [47] + [40] * 13 + [60] * 16, [61] * 10


class FakeCtx:
    def __init__(self, dnum):
        self.dnum, self.radix, self.prepared = dnum, 3, []

    def set_rotsum_radix(self, r):
        self.radix = r

    def cutmax_prepare(self, plan):
        self.prepared.append((self.radix, plan.shared))


def test_search_picks_fastest_candidate_that_keeps_every_argmax():
    # ms by (dnum, log2 radix); radix 16 is fastest but loses an argmax
    ms = {(3, 1): 300.0, (3, 2): 240.0, (3, 3): 220.0, (3, 4): 200.0, (4, 3): 230.0, (5, 3): 210.0}
    bad = {(3, 4)}
    made = []

    def make_ctx(d):
        made.append(d)
        return FakeCtx(d)

    def timer(g, cts, plan, check, reps, warm):
        return ms[(g.dnum, g.radix)], (g.dnum, g.radix) not in bad

    pl = P.CutMaxPlan(n=8, slots=8, packing="replicate", T=1, p=[3], c=[5.0], k=[2], kappa=[1.0], y0=[1.0], d=2,
                      kappa_f=1.0, bootstrap=True)
    choice, table = autotune.tune_decode(make_ctx, pl, lambda g: [0], lambda g, i, z: True, dnums=(3, 4, 5),
                                         log=lambda m: None, timer=timer)
    assert choice == {"rotsum_log_radix": 3, "dnum": 5}
    assert made == [3, 4, 5]
    assert table["radix"]["16"]["argmax_ok"] is False and table["radix"]["8"]["ms"] == 220.0
    assert table["dnum"]["4"]["ms"] == 230.0


def test_chain_mode_per_batch():
    g = FakeCtx(3)
    ms = {("a", True): 100.0, ("a", False): 120.0, ("b", True): 90.0, ("b", False): 80.0}

    def timer(gg, cts, plan, check, reps, warm):
        return ms[(cts[0], plan.shared)], check(0, None)

    pl = P.CutMaxPlan(n=8, slots=8, packing="replicate", T=1, p=[3], c=[5.0], k=[2], kappa=[1.0], y0=[1.0], d=2,
                      kappa_f=1.0, bootstrap=True)
    batches = {"a": (pl, "a", lambda z: True), "b": (pl, "b", lambda z: True)}
    choice, table = autotune.tune_chains(g, batches, log=lambda m: None, timer=timer)
    assert choice == {"a": "shared", "b": "stream"}
    assert table["b"]["stream"]["ms"] == 80.0
    assert [s for _, s in g.prepared] == [True, False, True, False]


def test_save_and_load_keyed_by_parameter_set(tmp_path):
    path = str(tmp_path / "t.json")
    choice = {"rotsum_log_radix": 3, "dnum": 3, "chains": {"8192": "shared"}}
    rec = autotune.save(path, 16, Q, PB, 192, choice, {"radix": {}}, "w")
    assert json.load(open(path))["choice"] == choice
    if rec["device"] is None:  # no GPU here: the device is not compared
        assert autotune.load(16, Q, PB, 192, path) == choice
    assert autotune.load(16, Q, PB, 64, path) is None
    assert autotune.load(16, Q[:-1], PB, 192, path) is None
    assert autotune.load(16, Q, PB, 192, str(tmp_path / "missing.json")) is None
