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


@pytest.mark.slow
def test_oracle_bootstrapped_circuit_replays_on_levels():
    """The oracle's bootstrapped CutMax (Alg. 2 with refreshes) at N = 2^11:
    the level-only replay that picks its refresh schedule predicts the real
    run exactly (output level, scale, general and constant refreshes, and the
    circuit's key switches at every level), the schedule is no costlier than
    making no optional refresh, and the decrypted output is the FP64 mirror of
    the same circuit within 1e-6, with the argmax of the logits."""
    from oracle import cutmax_fp64 as F
    from oracle.circuit import (HE, LevelSim, _boot_circuit, _DryBoot, _SimCt, cutmax_he_boot,
                                refresh_schedule, required_rotations)
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    log_n, nv, delta = 11, 1000, 2.0 ** 40
    qb = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
    gen = lambda i: synth.logits_heavy_tail(i, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])
    pl = P.calibrate(lambda i: gen(1000 + i), 200, nv, 1 << (log_n - 1), 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0],
                     margin=2.0, tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True)
    ctx = ckks.Context(log_n, qb, [61] * 10, dnum=3, h=64, seed=21)
    bs = Bootstrapper(ctx, K=14, r=4, d=31)
    bs.gen_keys()
    bs.gen_const_keys()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    x = gen(7)
    ct = ctx.encrypt(enc.encode(P.pack(x, 1 << (log_n - 1), pl.packing), log_n, delta), delta, 3)
    he = HE(ctx, delta)
    st = {}
    out = cutmax_he_boot(he, ct, pl, bs, stats=st)
    # the replay of the chosen schedule
    sim = LevelSim(ctx.primes, ctx.nq, log_n)
    dry = _DryBoot(bs.out_level())
    start = _SimCt(min(ct.level, bs.out_level()), ct.scale)
    rep = _boot_circuit(HE(sim, delta), start, pl, dry, st["h_refresh"], st["y_boot"], {})
    assert rep.level == out.level and rep.scale == pytest.approx(out.scale, rel=1e-9)
    assert (dry.general, dry.const) == (st["general"], st["const"]) and st["x_refresh"] == 0
    assert sim.ks == st["ks"]
    # no optional refresh at all costs at least as much
    sim0, dry0 = LevelSim(ctx.primes, ctx.nq, log_n), _DryBoot(bs.out_level())
    _boot_circuit(HE(sim0, delta), start, pl, dry0, [0] * pl.T, [0] * pl.T, {})
    assert 7 * dry.general + 3 * dry.const <= 7 * dry0.general + 3 * dry0.const
    assert refresh_schedule(he, ct, pl, bs.out_level()) == (st["h_refresh"], st["y_boot"])
    dec = enc.decode(ctx.decrypt(out), log_n, out.scale).real[:nv]
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-6
    assert int(np.argmax(dec)) == int(np.argmax(x))


@pytest.mark.slow
def test_oracle_shared_chains_circuit():
    """The oracle's bootstrapped CutMax for a batch of streams with the scalar
    chains shared (packed into slot classes, one chain for the batch, handed
    back per stream), N = 2^11, two streams of 1,000 heavy-tailed logits with
    relaxed Goldschmidt steps: each stream's output is its own FP64 mirror
    within 1e-5 with the argmax of its logits; the level-only replay of the
    chosen schedule predicts the real run's levels, scales and bootstrapped
    ciphertexts; and the batch bootstraps fewer ciphertexts than two runs of
    the one-stream circuit would."""
    from oracle import cutmax_fp64 as F
    from oracle.circuit import (HE, LevelSim, _DryBoot, _shared_circuit, _SimCt, cutmax_he_boot_shared,
                                refresh_schedule, required_rotations, _boot_circuit)
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    log_n, nv, delta = 11, 1000, 2.0 ** 40
    qb = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
    gen = lambda i: synth.logits_heavy_tail(i, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])
    pl = P.calibrate(lambda i: gen(1000 + i), 200, nv, 1 << (log_n - 1), 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0],
                     margin=2.0, tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True, relax=True)
    pl.shared = True
    ctx = ckks.Context(log_n, qb, [61] * 10, dnum=3, h=64, seed=22)
    bs = Bootstrapper(ctx, K=14, r=4, d=31)
    bs.gen_keys()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    xs = [gen(11), gen(12)]
    cts = [ctx.encrypt(enc.encode(P.pack(x, 1 << (log_n - 1), pl.packing), log_n, delta), delta, 40 + s)
           for s, x in enumerate(xs)]
    he = HE(ctx, delta)
    st = {}
    outs = cutmax_he_boot_shared(he, cts, pl, bs, stats=st)
    dry = _DryBoot(bs.out_level())
    start = [_SimCt(min(c.level, bs.out_level()), c.scale) for c in cts]
    rep = _shared_circuit(HE(LevelSim(ctx.primes, ctx.nq, log_n), delta), start, pl, dry, st["h_refresh"],
                          st["y_boot"])
    for r, o in zip(rep, outs):
        assert r.level == o.level and r.scale == pytest.approx(o.scale, rel=1e-9)
    assert dry.general == st["bootstrapped"]
    one = _DryBoot(bs.out_level())
    hr1, yb1 = refresh_schedule(he, cts[0], pl, bs.out_level())
    _boot_circuit(HE(LevelSim(ctx.primes, ctx.nq, log_n), delta), start[0], pl, one, hr1, yb1, {})
    assert st["bootstrapped"] < 2 * (one.general + one.const)
    for x, o in zip(xs, outs):
        dec = enc.decode(ctx.decrypt(o), log_n, o.scale).real[:nv]
        assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-5
        assert int(np.argmax(dec)) == int(np.argmax(x))


@pytest.mark.slow
def test_oracle_bootstrapped_circuit_multi_ciphertext_stream():
    """A vocabulary longer than the slot count (2,500 logits in three
    zero-padded ciphertexts of 1,024 slots, N = 2^11) through the oracle's
    bootstrapped circuit with relaxed steps: the sums add the three
    ciphertexts before the rotate-and-sum and the scalars serve all three;
    the outputs are the FP64 mirror within 1e-5 with the argmax of the
    logits, and the level-only replay of the schedule predicts the run."""
    from oracle import cutmax_fp64 as F
    from oracle.circuit import HE, LevelSim, _boot_circuit, _DryBoot, _SimCt, cutmax_he_boot, required_rotations
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    log_n, nv, delta = 11, 2500, 2.0 ** 40
    slots = 1 << (log_n - 1)
    qb = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
    gen = lambda i: synth.logits_heavy_tail(i, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])
    pl = P.calibrate(lambda i: gen(1000 + i), 120, nv, slots, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0],
                     margin=2.0, tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True, relax=True)
    assert pl.cts == 3
    ctx = ckks.Context(log_n, qb, [61] * 10, dnum=3, h=64, seed=23)
    bs = Bootstrapper(ctx, K=14, r=4, d=31)
    bs.gen_keys()
    bs.gen_const_keys()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    x = gen(8)
    cts = [ctx.encrypt(enc.encode(v, log_n, delta), delta, 60 + c) for c, v in enumerate(P.pack_cts(x, slots))]
    st = {}
    outs = cutmax_he_boot(HE(ctx, delta), cts, pl, bs, stats=st)
    dry = _DryBoot(bs.out_level())
    start = [_SimCt(min(c.level, bs.out_level()), c.scale) for c in cts]
    rep = _boot_circuit(HE(LevelSim(ctx.primes, ctx.nq, log_n), delta), start, pl, dry, st["h_refresh"],
                        st["y_boot"], {})
    assert [r.level for r in rep] == [o.level for o in outs]
    assert (dry.general, dry.const) == (st["general"], st["const"])
    assert st["general"] == 3 * st["vector_refreshes"]
    dec = np.concatenate([enc.decode(ctx.decrypt(o), log_n, o.scale).real for o in outs])[:nv]
    assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-5
    assert int(np.argmax(dec)) == int(np.argmax(x))


@pytest.mark.slow
def test_oracle_shared_chains_multi_ciphertext_streams():
    """Shared scalar chains over two streams of 1,500 logits, each in two
    zero-padded ciphertexts (N = 2^11, relaxed steps): every stream's output
    is its FP64 mirror within 1e-5 with the argmax of its logits."""
    from oracle import cutmax_fp64 as F
    from oracle.circuit import HE, cutmax_he_boot_shared, required_rotations
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    log_n, nv, delta = 11, 1500, 2.0 ** 40
    slots = 1 << (log_n - 1)
    qb = [55] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
    gen = lambda i: synth.logits_heavy_tail(i, n=nv, heavy=5, gap=[0.05, 0.2, 1.0][i % 3])
    pl = P.calibrate(lambda i: gen(1000 + i), 100, nv, slots, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0],
                     margin=2.0, tol_k=1e-6, k_max=20, d_max=14, tol_d=1e-6, bootstrap=True, relax=True)
    pl.shared = True
    assert pl.cts == 2
    ctx = ckks.Context(log_n, qb, [61] * 10, dnum=3, h=64, seed=24)
    bs = Bootstrapper(ctx, K=14, r=4, d=31)
    bs.gen_keys()
    for r in required_rotations(pl):
        ctx.gen_rot_key(r)
    xs = [gen(13), gen(14)]
    streams = [[ctx.encrypt(enc.encode(v, log_n, delta), delta, 70 + 4 * s + c)
                for c, v in enumerate(P.pack_cts(x, slots))] for s, x in enumerate(xs)]
    st = {}
    outs = cutmax_he_boot_shared(HE(ctx, delta), streams, pl, bs, stats=st)
    for x, o in zip(xs, outs):
        dec = np.concatenate([enc.decode(ctx.decrypt(c), log_n, c.scale).real for c in o])[:nv]
        assert np.abs(dec - F.cutmax_circuit(x, pl)).max() < 1e-5
        assert int(np.argmax(dec)) == int(np.argmax(x))
