"""Learned inverse-square-root stand-in for the CutMax circuit.

The inverse square root of Sect. 3.2 is a generic approximation (App. B: the
Goldschmidt iteration here, 2 levels per step).  This module learns a cheaper
stand-in from the inputs the circuit actually meets:

1. log the range-scaled variances x_t = kappa_t V_t of the plan's own FP64
   circuit over seeded logit vectors (the client-side calibration run of the
   plan, never encrypted data);
2. train, on the GPU with the library's FP32 kernels (he_learn_invsqrt), a
   1 -> 16 -> 1 network with square activations per iteration t; it is a
   quadratic A x^2 + B x + C, evaluated homomorphically in 2 levels;
3. recalibrate the plan with the quadratic offered at every iteration and
   keep it where its relative error over the calibrated margin range stays
   within `accept`; elsewhere the Goldschmidt iteration remains (the plain
   approximation is the fallback).
"""
import math
import multiprocessing as mp

import numpy as np

from . import plan as P


def _trace_chunk(args):
    """x_t = kappa_t V_t of every iteration for the vectors of one chunk."""
    gen, seeds, pl = args
    out = np.zeros((len(seeds), pl.T))
    n = pl.n
    for r, s in enumerate(seeds):
        y = np.asarray(gen(s), dtype=np.float64).copy()
        for t in range(pl.T):
            S = y.sum()
            D = n * y - S
            V = float((D * D).sum())
            x = pl.kappa[t] * V
            out[r, t] = x
            h = P.invsqrt_half_at(pl.k, pl.y0, pl.lq, t, x, pl.relax)
            rn = pl.norm[t] ** (1.0 / pl.p[t]) if pl.bootstrap else 1.0
            u = D * (2.0 * math.sqrt(pl.kappa[t] * n) / pl.c[t] * rn) * h + rn
            y = P._power(u, pl.p[t])
    return out


def log_variances(pl, gen, seeds, workers=None):
    """[len(seeds), T] range-scaled variances of the plan's circuit (FP64),
    over a spawn pool (safe after CUDA initialisation); `gen` must pickle.
    Rows come in chunk order, not seed order."""
    seeds = list(seeds)
    workers = workers or max(1, min(16, mp.cpu_count()))
    chunks = [c for c in (seeds[i::workers] for i in range(workers)) if c]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_trace_chunk, [(gen, c, pl) for c in chunks])
    return np.concatenate(parts, axis=0)


def _acc_chunk(args):
    gen, seeds, pl = args
    ok, mz = 0, []
    n = pl.n
    for s in seeds:
        x = np.asarray(gen(s), dtype=np.float64)
        y = x.copy()
        for t in range(pl.T):
            S = y.sum()
            D = n * y - S
            V = float((D * D).sum())
            h = P.invsqrt_half_at(pl.k, pl.y0, pl.lq, t, pl.kappa[t] * V, pl.relax)
            rn = pl.norm[t] ** (1.0 / pl.p[t]) if pl.bootstrap else 1.0
            u = D * (2.0 * math.sqrt(pl.kappa[t] * n) / pl.c[t] * rn) * h + rn
            y = P._power(u, pl.p[t])
        a = 1.0 - pl.kappa_f * y.sum()
        f, sq = 1.0 + a, a
        for _ in range(pl.d):
            sq = sq * sq
            f = f * (1.0 + sq)
        z = y * pl.kappa_f * f
        ok += int(np.argmax(z)) == int(np.argmax(x))
        mz.append(float(z.max()))
    return ok, mz


def fp64_accuracy(pl, gen, seeds, workers=None):
    """Argmax accuracy and max Z of the plan's circuit in FP64 over seeded vectors
    (spawn pool): (correct, count, mean max Z, min max Z)."""
    seeds = list(seeds)
    workers = workers or max(1, min(16, mp.cpu_count()))
    chunks = [c for c in (seeds[i::workers] for i in range(workers)) if c]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        parts = pool.map(_acc_chunk, [(gen, c, pl) for c in chunks])
    mz = [v for _, m in parts for v in m]
    return sum(o for o, _ in parts), len(seeds), float(np.mean(mz)), float(np.min(mz))


def quad_rel_err(abc, a, b, n=4001):
    """max |2 h sqrt(x) - 1| of h = quadratic / 2 over a geometric grid of [a, b],
    and whether the quadratic stays positive there."""
    x = np.geomspace(a, b, n)
    f = abc[0] * x * x + abc[1] * x + abc[2]
    return float(np.abs(f * np.sqrt(x) - 1.0).max()), bool((f > 0).all())


def learned_plan(ctx, plain, calib_kw, logged, accept=0.08, steps=3000, lr=1e-2, seed=0):
    """Recalibrate with a learned quadratic offered at each iteration.

    plain: the plain plan the variances were logged with; calib_kw: the
    arguments of plan.calibrate for it; logged: [vectors, T] from
    log_variances.  Returns (plan, report) with report[t] = training loss,
    relative error over the margin range and whether it was kept."""
    report = {}

    def learn(t, kap, xs_cal, ab):
        data = logged[:, t] * (kap / plain.kappa[t])
        # the logged inputs, plus as many spread log-uniformly over the
        # calibrated margin range, which the plan guarantees for any input
        xs = np.concatenate([data, np.geomspace(ab[0], ab[1], len(data))])
        abc, loss = ctx.learn_invsqrt(xs, steps=steps, lr=lr, seed=seed + t)
        err, pos = quad_rel_err(abc, *ab)
        keep = pos and err <= accept
        report[t] = {"logged": int(len(data)), "samples": int(len(xs)), "train_loss": loss, "range_rel_err": err,
                     "kept": keep,
                     "abc": abc}
        return abc if keep else None

    pl = P.calibrate(**calib_kw, learn=learn)
    return pl, report
