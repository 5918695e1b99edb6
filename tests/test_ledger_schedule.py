"""The refresh schedule of the bootstrapped circuit (host logic, CPU).

The library and the operation-count model pick, per iteration, whether to
refresh h by a constant bootstrap and whether to bootstrap Y early, by
playing every combination on the level bookkeeping.  Whatever they pick must
cost no more (general bootstrap 7, constant 3) than making no optional
refresh at all, and must leave every level non-negative.
"""
import pytest

from paper_2509_08383_gb300 import ledger
from paper_2509_08383_gb300 import plan as P
from paper_2509_08383_gb300 import synth

QB = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
BOOT = (14, 4, 31)


@pytest.fixture(scope="module")
def plan_boot():
    n = 1000

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    return P.calibrate(lambda i: gen(1000 + i), 200, n, 1024, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                       tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True)


def _cost(pl):
    ks, nb, nc = ledger.cutmax_ledger(pl, len(QB), 11, boot=BOOT, qbits=QB, detail=True)
    assert all(level >= 0 for level in ks)
    return 7 * (nb - nc) + 3 * nc, nb, nc


def test_schedule_costs_no_more_than_no_optional_refresh(plan_boot, monkeypatch):
    chosen = _cost(plan_boot)
    monkeypatch.setattr(ledger, "refresh_schedule",
                        lambda plan, qb, y, out, padded: ([False] * plan.T, [False] * plan.T))
    plain = _cost(plan_boot)
    assert chosen[0] <= plain[0]
    assert chosen[2] >= 1                                  # scalars do take the constant bootstrap


def test_schedule_is_deterministic_and_sized(plan_boot):
    out = ledger.Sim(len(QB), 11, BOOT).bootstrap(0)
    a = ledger.refresh_schedule(plan_boot, QB, out, out, plan_boot.pad != 0)
    b = ledger.refresh_schedule(plan_boot, QB, out, out, plan_boot.pad != 0)
    assert a == b and len(a[0]) == len(a[1]) == plan_boot.T


@pytest.mark.parametrize("relax", [False, True])
def test_ledger_agrees_with_the_oracle_circuit_on_levels(relax):
    """Two independent level bookkeepings of the bootstrapped circuit: the
    operation-count model (ledger.py, the library's rules) and the oracle's
    circuit played on LevelSim with its own refresh schedule.  For a plan with
    Newton's constant and a relaxed one (their Goldschmidt steps differ in
    count, not in levels per step) they bootstrap the same number of
    ciphertexts of each kind."""
    from oracle import ckks as ock
    from oracle.circuit import HE, LevelSim, _DryBoot, _SimCt, _boot_circuit, refresh_schedule
    n = 1000

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    pl = P.calibrate(lambda i: gen(1000 + i), 200, n, 1024, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                     tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True, relax=relax)
    ctx = ock.Context(11, QB, [61] * 10, dnum=3, h=64, seed=21)
    out = ledger.Sim(len(QB), 11, BOOT).bootstrap(0)
    delta = 2.0 ** 40
    ct = _SimCt(len(QB) - 1, delta)
    hr, yb = refresh_schedule(HE(ctx, delta), ct, pl, out)
    dry = _DryBoot(out)
    _boot_circuit(HE(LevelSim(ctx.primes, ctx.nq, ctx.log_n), delta), _SimCt(out, delta), pl, dry, hr, yb, {})
    ks, nb, nc = ledger.cutmax_ledger(pl, len(QB), 11, boot=BOOT, qbits=QB, detail=True)
    assert (dry.general, dry.const) == (nb - nc, nc)


@pytest.mark.parametrize("relax", [False, True])
def test_shared_schedule_agrees_with_the_oracle_circuit(relax):
    """Shared scalar chains: the library's schedule rule (ledger.py, written
    after the circuit's level rules) and the oracle's shared circuit played on
    LevelSim with its own schedule bootstrap the same number of ciphertexts,
    for batches of 2, 4 and 16 streams of one ciphertext and of 2 and 4
    streams of two."""
    from oracle import ckks as ock
    from oracle.circuit import HE, LevelSim, _DryBoot, _shared_circuit, _SimCt, refresh_schedule_shared
    n = 1000

    def gen(i):
        return synth.logits_heavy_tail(i, n=n, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])

    pl = P.calibrate(lambda i: gen(1000 + i), 200, n, 1024, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                     tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True, relax=relax)
    ctx = ock.Context(11, QB, [61] * 10, dnum=3, h=64, seed=21)
    out = ledger.Sim(len(QB), 11, BOOT).bootstrap(0)
    delta = 2.0 ** 40
    for S in (2, 4, 16):
        hr, yb = refresh_schedule_shared(HE(ctx, delta), [_SimCt(len(QB) - 1, delta)] * S, pl, out)
        dry = _DryBoot(out)
        _shared_circuit(HE(LevelSim(ctx.primes, ctx.nq, ctx.log_n), delta), [_SimCt(out, delta)] * S, pl, dry,
                        hr, yb)
        lhr, lyb, cost = ledger.refresh_schedule_shared(pl, QB, out, out, pl.pad != 0, S, S)
        assert dry.general == cost, (S, dry.general, cost)
    # streams of two zero-padded ciphertexts (1,500 logits in 1,024 slots each)
    n2 = 1500
    pl2 = P.calibrate(lambda i: synth.logits_heavy_tail(2000 + i, n=n2, heavy=5, gap=[0.05, 0.2, 1.0][i % 3]), 100,
                      n2, 1024, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0, tol_k=1e-6, k_max=20, d_max=14,
                      tol_d=1e-6, bootstrap=True, relax=relax)
    assert pl2.cts == 2
    for S in (2, 4):
        streams = [[_SimCt(len(QB) - 1, delta)] * 2 for _ in range(S)]
        hr, yb = refresh_schedule_shared(HE(ctx, delta), streams, pl2, out)
        dry = _DryBoot(out)
        _shared_circuit(HE(LevelSim(ctx.primes, ctx.nq, ctx.log_n), delta), [[_SimCt(out, delta)] * 2] * S, pl2,
                        dry, hr, yb)
        lhr, lyb, cost = ledger.refresh_schedule_shared(pl2, QB, out, out, True, 2 * S, S)
        assert dry.general == cost, (S, dry.general, cost)
