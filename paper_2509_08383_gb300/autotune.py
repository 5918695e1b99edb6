"""Autotuner for the runtime choices of the encrypted CutMax path, measured on
the GPU at hand and persisted as JSON.

Choices (none changes what the circuit computes; they change the order of
rounding steps, so outputs move only at the noise level):

- ``rotsum_log_radix`` (1..4): hoisting radix of the rotate-and-sum
  reductions (App. D; the mean and variance sums of Alg. 2 and the trace of
  the constant bootstrap).  A stage of radix r shares one ModUp and one
  ModDown among r - 1 rotations; a larger radix means fewer stages but more
  evaluation keys (r - 1 per stage) streamed by each stage.
- ``dnum``: the number of digits of the hybrid key switch at a fixed special
  modulus P.  Fewer digits mean fewer extension rows to basis-convert, NTT and
  multiply with the key; more digits mean smaller digits (less key-switch
  noise) at the same security (log QP is unchanged).
- ``chains`` (batched streams, per vocabulary size): the scalar chains of a
  batch packed across its streams in one ciphertext (one set of general
  bootstraps for every stream) or kept per stream (constant bootstraps of
  every member, one launch for the batch).

Every candidate runs the full decode it is meant for: whole CutMax calls timed
with CUDA events on the library's stream, L2 flushed before each, the argmax
of every decode checked; a candidate that loses an argmax is rejected.  The
search is coordinate-wise: the radix at the first dnum candidate, then dnum
at the best radix, then the batch chain mode.  The file records every
timing next to the choices, the device and the parameter set it was measured
on; ``load`` returns the choices only for a matching device and parameter
set.
"""
import gc
import hashlib
import json
import os
import time

import numpy as np

TUNED_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned")
RADICES = (1, 2, 3, 4)


def chain_key(log_n, qbits, pbits, h):
    """Identifier of a parameter set: ring degree, prime bit sizes, secret weight."""
    s = json.dumps([log_n, list(qbits), list(pbits), h])
    return hashlib.sha1(s.encode()).hexdigest()[:12]


def default_path(log_n):
    return os.path.join(TUNED_DIR, f"gb300_n{1 << log_n}.json")


def device_name():
    import torch
    return torch.cuda.get_device_name(0) if torch.cuda.is_available() else None


def load(log_n, qbits, pbits, h, path=None):
    """The tuned choices for this parameter set on this device, or None."""
    path = path or default_path(log_n)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    if t.get("chain") != chain_key(log_n, qbits, pbits, h):
        return None
    dev = device_name()
    if dev is not None and t.get("device") != dev:
        return None
    return t["choice"]


def time_decodes(g, cts, plan, check, reps, warm):
    """Mean ms of `reps` CutMax calls after `warm` untimed ones (CUDA events
    on the current stream, 256 MiB written between calls to flush L2), and
    whether every decode passed `check(i, z)`."""
    import torch
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ts, ok = [], True
    for i in range(warm + reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        z = g.cutmax(cts[i % len(cts)], plan)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warm:
            ts.append(e0.elapsed_time(e1))
        ok = ok and check(i % len(cts), z)
        del z
    return float(np.mean(ts)), ok


def tune_decode(make_ctx, plan, inputs, check, dnums=(3, 4, 5), radices=RADICES, reps=4, warm=2, log=print,
                timer=time_decodes):
    """Radix then dnum for one decode workload.

    make_ctx(dnum) -> a bootstrap-ready context; inputs(g) -> ciphertexts to
    decode; check(g, i, z) -> argmax of decode i correct; timer as
    time_decodes."""
    table = {"radix": {}, "dnum": {}}
    d0 = dnums[0]
    g = make_ctx(d0)
    cts = inputs(g)
    best_r, best_ms = None, None
    for r in radices:
        t0 = time.perf_counter()
        g.set_rotsum_radix(r)
        g.cutmax_prepare(plan)  # the rotation keys this radix needs
        ms, ok = timer(g, cts, plan, lambda i, z: check(g, i, z), reps, warm)
        table["radix"][str(1 << r)] = {"ms": ms, "argmax_ok": ok, "setup_s": time.perf_counter() - t0}
        log(f"radix {1 << r}: {ms:.2f} ms per decode, argmax {'ok' if ok else 'LOST'}")
        if ok and (best_ms is None or ms < best_ms):
            best_r, best_ms = r, ms
    if best_r is None:
        raise RuntimeError("no rotate-and-sum radix kept every argmax")
    table["dnum"][str(d0)] = {"ms": best_ms, "argmax_ok": True}
    del cts, g
    gc.collect()  # the context's device memory goes back before the next one
    best_d = d0
    for d in dnums[1:]:
        t0 = time.perf_counter()
        g = make_ctx(d)
        g.set_rotsum_radix(best_r)
        g.cutmax_prepare(plan)
        cts = inputs(g)
        ms, ok = timer(g, cts, plan, lambda i, z: check(g, i, z), reps, warm)
        table["dnum"][str(d)] = {"ms": ms, "argmax_ok": ok, "setup_s": time.perf_counter() - t0}
        log(f"dnum {d}: {ms:.2f} ms per decode, argmax {'ok' if ok else 'LOST'}")
        if ok and ms < best_ms:
            best_d, best_ms = d, ms
        del cts, g
        gc.collect()
    return {"rotsum_log_radix": best_r, "dnum": best_d}, table


def tune_chains(g, batches, reps=2, warm=1, log=print, timer=time_decodes):
    """Scalar-chain mode per batch.  batches: {name: (plan, batch ciphertext,
    check(z) -> all argmaxes correct)}; the plan's `shared` flag is switched."""
    from . import plan as P
    choice, table = {}, {}
    for name, (pl, batch, check) in batches.items():
        row = {}
        for mode in ("shared", "stream"):
            p = P.CutMaxPlan(**{**pl.to_dict(), "shared": mode == "shared"})
            g.cutmax_prepare(p)
            ms, ok = timer(g, [batch], p, lambda i, z: check(z), reps, warm)
            row[mode] = {"ms": ms, "argmax_ok": ok}
            log(f"batch {name}, chains {mode}: {ms:.1f} ms, argmax {'ok' if ok else 'LOST'}")
        if hasattr(g, "graph_clear"):
            g.graph_clear()  # the batch's CUDA graphs give their memory back
        good = [m for m in row if row[m]["argmax_ok"]] or list(row)
        choice[name] = min(good, key=lambda m: row[m]["ms"])
        table[name] = row
    return choice, table


def save(path, log_n, qbits, pbits, h, choice, table, workload):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    rec = {"device": device_name(), "chain": chain_key(log_n, qbits, pbits, h), "log_n": log_n,
           "qbits": list(qbits), "pbits": list(pbits), "h": h, "workload": workload, "choice": choice,
           "measured": table, "how": "full CutMax decodes timed with CUDA events, L2 flushed before each; "
                                     "coordinate search radix -> dnum -> batch chain mode; a candidate that "
                                     "loses an argmax is rejected"}
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    return rec
