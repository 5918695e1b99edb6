"""Benchmark: encrypted CutMax decodes/s on synthetic LLM-shaped logits.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload cfg1|cfg2|cfg3|cfg4|cfg5|tune|mul16|rot16|ntt16|boot16|bootc16]
                [--newton] [--no-graph] [--chains tuned|shared|stream] [--tokens T] [--no-cpu-baseline]

One step = one encrypted CutMax (Alg. 2) over one freshly encrypted logit
vector.  `value` times the device work with CUDA events on the library's
stream (inputs already encrypted and resident in HBM, L2 flushed between
steps); `e2e` times the public C-ABI path from pinned host logits to host
results (encode + encrypt + CutMax + decrypt + decode, copies included).
Multi-GPU: independent replicas per rank (no data-path collective).
--impl reference times the CPU oracle on the machine's host cores.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted CutMax decodes/sec (vocab 32k, N=2^16), 1 GB300"
# ncu dram__bytes_read.sum + dram__bytes_write.sum of both NTT passes per limb at
# N=2^16 (40-limb forward and inverse of `--workload ntt16`; ncu starts each
# pass with cold caches, so the data is counted once per pass), from one
# capture of the NTT source whose hash is `src`; once the source changes
# (ntt_source_hash() differs) the bench reports traffic null
NTT_DRAM = {"src": "06cea59ef67fbd85",
            "per_limb": {0: (21175040 + 0 + 62799872 + 23296) / 40, 1: (62797056 + 3840 + 21181696 + 0) / 40}}
# integer-pipe ceiling of the NTT: a Shoup butterfly on 64-bit words takes 1.04
# warp instructions (33 thread instructions: ncu sm__inst_executed of a 90-limb
# forward transform / its 90 x 2^19 butterflies), and an SM issues at most 4
# warp instructions per clock: 152 SMs x 4 x 2.07 GHz / 1.04
NTT_WARP_INSTR_PER_BUTTERFLY = 1.04
ALU_ISSUE_PEAK = 152 * 4 * 2.07e9
PROF_NAMES = {0: "ntt_forward (k_ntt_cols+k_ntt_rows)", 1: "ntt_inverse (k_ntt_rows+k_ntt_cols)",
              2: "keyswitch_inner (k_keyswitch_inner)", 3: "bconv (k_bconv)"}


def ntt_source_hash():
    """Hash of the NTT kernels' source (their section of kernels.cu and the
    shared arithmetic header) that the DRAM traffic figures were taken on."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2509_08383_gb300", "csrc")
    k = open(os.path.join(csrc, "kernels.cu")).read()
    a, b = k.find("// ------------------------------------------------------------------ NTT"), \
        k.find("// ------------------------------------------------------------------ elementwise")
    body = k[a:b] + open(os.path.join(csrc, "common.cuh")).read()
    return hashlib.sha256(body.encode()).hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# base prime 47 bits: a bootstrap refreshes with error ~(q0 / Delta) x the EvalMod
# approximation error, so q0 = 2^47 against Delta = 2^40 keeps it near 1e-7 for
# messages up to 2 (about 1.5e-5 with a 55-bit q0)
CFG2_Q = [47] + [40] * 13 + [60] * 3 + [60] * 10 + [58] * 3
# relative error of the invsqrt and inverse approximations: 10 bits, inside
# the 7..13-bit range of the invsqrt benchmarks the paper reprints (App. B)
INVSQRT_TOL = 2.0 ** -10
CFG2_P = [61] * 10


# Goldschmidt's inverse square root with calibrated per-step relaxation
# constants (App. B); --newton keeps Newton's 3/2 in every step
RELAX = True


def workload(name):
    """(log_n, q bits, p bits, dnum, plan, logits generator, description, bootstrap (h, K, r, d) or None)."""
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    if name == "cfg2":
        log_n, n = 16, 32000
        gen = synth.HeavyTail(n, (0.05, 0.2, 1.0))
        pl = P.calibrate(lambda i: gen(100000 + i), 200, n, 1 << (log_n - 1), 4, [16, 4, 4, 6],
                         [5.0, 3.0, 3.0, 3.0], margin=2.0, tol_k=INVSQRT_TOL, k_max=20, d_max=14,
                         tol_d=INVSQRT_TOL, bootstrap=True, relax=RELAX)
        desc = {"workload": "CutMax T=4 p=[16,4,4,6] c=[5,3,3,3], 32000 logits N(0,9) + 50 heavy-tail "
                            "Exp(1.5), top-1 gap in {0.05,0.2,1.0}, zero-padded in N=2^16 slots, CKKS "
                            "bootstrapping when levels run out (logQ<=1521, dnum=3, h=192)",
                "log_n": log_n, "n": n, "T": 4, "k": pl.k, "d": pl.d,
                "goldschmidt": "relaxed" if pl.relax is not None else "newton"}
        return log_n, CFG2_Q, CFG2_P, 3, pl, gen, desc, (192, 24, 4, 31)
    if name == "cfg1":
        log_n, qb, pb, dnum = 14, [60] + [40] * 21, [60, 60], 11
        n = 1024
        pl = P.calibrate(lambda i: synth.logits_gaussian(1000 + i, n=n), 100, n, 1 << (log_n - 1), 2, 3, 5.0,
                         k_fixed=2, d_fixed=2)
        gen = lambda s: synth.logits_gaussian(s, n=n)
        desc = {"workload": "CutMax T=2 p=3 c=5, 1024 logits N(0,4) replicated in N=2^14 slots, leveled "
                            "(L=21, 40-bit scale, dnum=11)", "log_n": log_n, "n": n, "T": 2}
        return log_n, qb, pb, dnum, pl, gen, desc, None
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws
    return None, rank, ws


OP_CLASSES = ("rot", "mul", "rescale", "plain_mul", "add")


class OracleOps:
    """The oracle's operations at the bench parameter set, timed one by one
    (a bounded sample: one of each class per level).  Each class stands for a
    row of the library's ledger: rot = automorphism + key switch (every key
    switch that is not a relinearisation), mul = tensor product + key switch,
    rescale, plain_mul = product with an encoded plaintext, add."""

    def __init__(self, log_n, qb, pb, dnum, h):
        from oracle import ckks as ock
        self.ock = ock
        self.log_n = log_n
        self.o = ock.Context(log_n, qb, pb, dnum, h=h, seed=1)
        self.o.gen_relin_key()
        self.o.gen_rot_key(1)
        self.nq = len(qb)

    def time_level(self, level, threads=0):
        """{class: seconds} of one operation of each class at `level` on
        `threads` threads (0: every core of this process)."""
        ock, o = self.ock, self.o
        old = ock.get_threads()
        ock.set_threads(threads)
        try:
            rng = np.random.default_rng(level)
            n = 1 << self.log_n
            m = np.rint(rng.normal(size=n) * 2.0 ** 40)
            a, b = o.encrypt(m, 2.0 ** 40, 1, level), o.encrypt(m, 2.0 ** 40, 2, level)
            pt = np.rint(rng.normal(size=n) * 2.0 ** 20)
            ops = {"rot": lambda: o.rotate(a, 1), "mul": lambda: o.mul(a, b), "rescale": lambda: o.rescale(a),
                   "plain_mul": lambda: o.mul_plain(a, pt, 2.0 ** 60), "add": lambda: o.add(a, b)}
            out = {}
            for cls in OP_CLASSES:
                t0 = time.perf_counter()
                ops[cls]()
                out[cls] = time.perf_counter() - t0
            return out
        finally:
            ock.set_threads(old)


def census_seconds(census, times):
    """Seconds of one decode: sum over levels and classes of count x the time
    per operation at that level, linear between the timed levels.  census:
    {"ks", "tensor", "rescale", "plain_mul", "add"} -> {level: count}."""
    lv = sorted(times)

    def t(cls, l):
        return float(np.interp(l, lv, [times[x][cls] for x in lv]))

    tot = 0.0
    for l, c in census["ks"].items():
        tot += (c - census["tensor"].get(l, 0)) * t("rot", l)
    for cls, key in (("mul", "tensor"), ("rescale", "rescale"), ("plain_mul", "plain_mul"), ("add", "add")):
        for l, c in census[key].items():
            tot += c * t(cls, l)
    return tot


def census_levels(census, nq):
    """Three timing levels spanning the census: the lowest level with a
    rescale's worth of limbs (>= 1), the middle, the top."""
    used = [l for k in census.values() for l, c in k.items() if c]
    lo = max(1, min(used))
    return [lo, (lo + nq - 1) // 2, nq - 1]


def cfg2_census():
    """Key switches and bootstraps of one config-2 decode from the circuit's
    level model (ledger.py), for the reference arm, which runs no GPU code;
    the other op classes are not in that model and count zero there."""
    from paper_2509_08383_gb300 import ledger
    log_n, qb, pb, dnum, pl, gen, desc, boot = workload("cfg2")
    ks, nb = ledger.cutmax_ledger(pl, len(qb), log_n, boot=boot[1:], qbits=qb)
    return {"ks": ks, "tensor": {}, "rescale": {}, "plain_mul": {}, "add": {}}, nb


def run_reference(args):
    """The CPU oracle as it stands, on this machine's host cores."""
    dist, rank, ws = dist_setup(args)
    if rank != 0:
        return
    from oracle import ckks as ock
    from oracle import encoding as oenc
    from oracle.circuit import HE, cutmax_he, required_rotations
    from paper_2509_08383_gb300 import plan as P
    log_n, qb, pb, dnum, pl, gen, desc, boot = workload(args.workload)
    times, cpu_s = [], 0.0
    if boot is None:
        o = ock.Context(log_n, qb, pb, dnum, seed=1)
        o.gen_relin_key()
        for r in required_rotations(pl):
            o.gen_rot_key(r)
        delta = 2.0 ** 40
        for step in range(args.warmup + args.steps):
            x = gen(50000 + step)
            t0 = time.perf_counter()
            ct = o.encrypt(oenc.encode(P.pack(x, 1 << (log_n - 1), pl.packing), log_n, delta), delta, step)
            z = cutmax_he(HE(o, delta), ct, pl)
            oenc.decode(o.decrypt(z), log_n, z.scale)
            dt = time.perf_counter() - t0
            cpu_s += dt
            if step >= args.warmup:
                times.append(dt)
        sample = f"{args.steps} full CutMax decodes (encrypt + CutMax + decrypt) on the oracle"
        extrapolated = False
    else:
        census, nb = cfg2_census()
        levels = census_levels(census, len(qb))
        ops = OracleOps(log_n, qb, pb, dnum, boot[0])
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            tl = {l: ops.time_level(l) for l in levels}
            cpu_s += time.perf_counter() - t0
            if step >= args.warmup:
                times.append(census_seconds(census, tl))
        sample = (f"each step times one oracle rotation and one product (each with its key switch), a rescale, a "
                  f"plaintext product and an addition at levels {levels} ({cpu_s / (args.warmup + args.steps):.1f} s "
                  f"per step), and scales them by one decode's {sum(census['ks'].values())} key switches by level "
                  f"({nb} bootstraps) from the circuit's level model; extrapolated: a full decode on the oracle is "
                  "hours, its dense bootstrap does not fit at N=2^16")
        extrapolated = True
    T = sum(times)
    val = args.steps / T
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "decodes/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": desc, "extrapolated": extrapolated, "cpu_seconds_run": cpu_s,
           "cpu_baseline": {"value": val, "unit": "decodes/s", "cores": ock.get_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "decodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def cpu_baseline(args, census=None):
    """Bounded oracle sample of the bench workload, in decodes/s."""
    from oracle import ckks as ock
    from oracle import encoding as oenc
    from oracle.circuit import HE, cutmax_he, required_rotations
    from paper_2509_08383_gb300 import plan as P
    log_n, qb, pb, dnum, pl, gen, _, boot = workload(args.workload)
    if boot is not None:
        levels = census_levels(census, len(qb))
        ops = OracleOps(log_n, qb, pb, dnum, boot[0])
        t0 = time.perf_counter()
        tl = {l: ops.time_level(l) for l in levels}
        t_all = census_seconds(census, tl)
        mid = levels[1]
        one = ops.time_level(mid, threads=1)
        # single thread: the middle level timed on one core, the other levels
        # scaled by the all-core level profile of each class
        t1 = {l: {c: one[c] * tl[l][c] / tl[mid][c] for c in OP_CLASSES} for l in levels}
        t_one = census_seconds(census, t1)
        per = {c: sum(census[k].values()) for c, k in (("ks", "ks"), ("tensor", "tensor"), ("rescale", "rescale"),
                                                        ("plain_mul", "plain_mul"), ("add", "add"))}
        return {"value": 1.0 / t_all, "unit": "decodes/s", "cores": ock.get_threads(), "kind": "oracle",
                "sample": f"one oracle rotation and one product (each with its key switch), a rescale, a plaintext "
                          f"product and an addition timed at levels {levels} ({time.perf_counter() - t0:.1f} s of "
                          "CPU work), scaled by the per-level counts of every op class of one decode in the library's "
                          f"ledger ({per}); extrapolated",
                "single_thread": {"value": 1.0 / t_one, "unit": "decodes/s", "cores": 1,
                                  "sample": f"the level-{mid} operations on one core, other levels scaled by the "
                                            "all-core profile"},
                "per_op_seconds_all_cores": {str(l): tl[l] for l in levels},
                "per_op_seconds_one_core": {str(mid): one}}
    o = ock.Context(log_n, qb, pb, dnum, seed=1)
    o.gen_relin_key()
    for r in required_rotations(pl):
        o.gen_rot_key(r)
    delta = 2.0 ** 40
    x = gen(777)
    ct = o.encrypt(oenc.encode(P.pack(x, 1 << (log_n - 1), pl.packing), log_n, delta), delta, 1)
    t0 = time.perf_counter()
    cutmax_he(HE(o, delta), ct, pl)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "decodes/s", "cores": ock.get_threads(), "kind": "oracle",
            "sample": "1 full CutMax decode of the bench workload on the oracle (ciphertext already encrypted)"}


CFG3_VOCABS = [8192, 32000, 50257, 128256]


def run_cfg3(args):
    """64 concurrent decode streams, 16 per vocabulary size in CFG3_VOCABS
    (1/1/2/4 ciphertexts each at N=2^16), logits N(0, 2^2) with the top
    entry 0.5 above the second, the paper's HE circuit (T=4, p=[16,4,4,6],
    c=[5,3,3,3]) with bootstrapping.  Batched: one batch per vocabulary size,
    every homomorphic step one launch for all its streams; the scalar chains
    shared across the batch's streams or kept per stream, the rotate-and-sum
    radix and dnum as the autotuner picked them (`--workload tune`; without
    its file: shared chains, radix 8, dnum 3).  Sequential: one stream at a
    time; every stream of a vocabulary costs the same, so one stream per
    vocabulary is timed and counted 16 times."""
    import torch
    from paper_2509_08383_gb300 import autotune, build, he
    from paper_2509_08383_gb300 import plan as P
    build.build_library()
    torch.cuda.set_device(0)
    per = 16
    tuned = autotune.load(16, CFG2_Q, CFG2_P, 192)
    dnum = tuned["dnum"] if tuned else 3
    chains = dict(tuned["chains"]) if tuned else {}
    if args.chains != "tuned":
        chains = {str(v): args.chains for v in CFG3_VOCABS}
    g = he.Context(16, CFG2_Q, CFG2_P, dnum, h=192, seed=1, arena_bytes=200 << 30)
    g.bootstrap_prepare(24, 4, 31)
    if tuned:
        g.set_rotsum_radix(tuned["rotsum_log_radix"])
    groups = cfg3_batches(g, per, CFG3_VOCABS, chains)
    stream = torch.cuda.current_stream()
    run = g.cutmax_graph if args.graph else g.cutmax  # the first call of each shape captures its graph

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {}
    with ClockSampler(0) as clk:
        t_batch, t_seq, acc = 0.0, 0.0, []
        for v, pl, xs, batch, one in groups:
            for it in range(args.warmup + args.steps):
                flush.zero_()
                g.ledger(reset=True)
                ms, Z = timed(lambda: run(batch, pl))
                _, nb = g.ledger(reset=True)
                if it >= args.warmup:
                    t_batch += ms / args.steps
            # argmax of every stream of the batch
            ok = batch_argmax_ok(g, Z, xs, pl)
            acc.append(ok)
            pl1 = P.CutMaxPlan(**{**pl.to_dict(), "shared": False})
            b1 = g.batch_pack(one)
            for it in range(args.warmup + args.steps):
                flush.zero_()
                g.ledger(reset=True)
                ms1, _ = timed(lambda: run(b1, pl1))
                _, nb1 = g.ledger(reset=True)
                if it >= args.warmup:
                    t_seq += per * ms1 / args.steps
            g.graph_clear()  # this vocabulary's graphs give their memory back
            res[str(v)] = {"cts_per_stream": pl.cts, "chains": "shared" if pl.shared else "stream",
                           "batched_ms": ms, "batched_bootstraps": nb,
                           "single_stream_ms": ms1, "single_stream_bootstraps": nb1, "argmax_ok": ok, "k": pl.k,
                           "d": pl.d}
            del Z
    n_streams = per * len(CFG3_VOCABS)
    out = {"metric": "batched encrypted CutMax decodes/sec, 64 streams of vocabularies 8192/32000/50257/128256 "
                     "(N=2^16), 1 GB300", "value": 1000.0 * n_streams / t_batch, "unit": "decodes/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": "64 decode streams, 16 per vocabulary 8192/32000/50257/128256 (1/1/2/4 "
                                  "ciphertexts), N(0,4) logits with top gap 0.5, T=4 p=[16,4,4,6] c=[5,3,3,3], "
                                  "bootstrapping, one batch per vocabulary (scalar chain mode per vocabulary "
                                  "in per_vocabulary)",
                      "dnum": dnum, "rotsum_radix": 1 << (tuned["rotsum_log_radix"] if tuned else 3),
                      "tuned": bool(tuned), "cuda_graph": bool(args.graph),
                      "graph_stats": dict(zip(("captured", "replayed", "direct"), g.graph_stats())),
                      "l2": "flushed between steps (256 MiB write)"},
           "sequential": {"value": 1000.0 * n_streams / t_seq, "unit": "decodes/s", "ms_per_step": t_seq,
                          "how": "one stream per vocabulary timed alone, times 16"},
           "speedup_vs_sequential": t_seq / t_batch, "argmax_correct": sum(acc), "streams": n_streams,
           "per_vocabulary": res, "clocks": clk.summary()}
    print(json.dumps(out))


def cfg3_batches(g, per, vocabs, chains=None):
    """Per vocabulary size: its calibrated plan, the batch of `per` encrypted
    streams, the plaintext logits and the member count per stream."""
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    slots = g.n // 2
    groups = []
    for v in vocabs:
        gen = (lambda s, v=v: synth.logits_gaussian(s, n=v, sd=2.0, gap=0.5))
        pl = P.calibrate(lambda i: gen(100000 + i), 60, v, slots, 4, [16, 4, 4, 6], [5.0, 3.0, 3.0, 3.0], margin=2.0,
                         tol_k=INVSQRT_TOL, k_max=20, d_max=14, tol_d=INVSQRT_TOL, bootstrap=True, relax=RELAX)
        pl.shared = (chains or {}).get(str(v), "shared") == "shared"
        g.cutmax_prepare(pl)
        xs = [gen(s) for s in range(per)]
        cts = []
        for s, x in enumerate(xs):
            vecs = P.pack_cts(x, slots) if pl.cts > 1 else [P.pack(x, slots, pl.packing)]
            cts += [g.encrypt(vv, g.delta, 1000 * v + 10 * s + c) for c, vv in enumerate(vecs)]
        groups.append((v, pl, xs, g.batch_pack(cts), cts[:pl.cts]))
    return groups


def batch_argmax_ok(g, Z, xs, pl):
    ok = 0
    for s, x in enumerate(xs):
        dec = np.concatenate([g.decrypt(g.batch_member(Z, s * pl.cts + c)) for c in range(pl.cts)])[:len(x)]
        ok += int(np.argmax(dec)) == int(np.argmax(x))
    return ok


def run_tune(args):
    """Autotune the runtime choices (rotate-and-sum radix, dnum, batch chain
    mode) on full decodes of the benchmark's workloads and write the JSON the
    other workloads read: the radix and dnum on the 32,000-logit decode, the
    chain mode per vocabulary on 16-stream batches of the four vocabulary
    sizes."""
    import torch
    from paper_2509_08383_gb300 import autotune, build, he
    from paper_2509_08383_gb300 import plan as P
    build.build_library()
    torch.cuda.set_device(0)
    log_n, qb, pb, dnum, pl, gen, desc, boot = workload("cfg2")
    slots = 1 << (log_n - 1)
    xs = [gen(30000 + s) for s in range(4)]

    def make_ctx(d):
        g = he.Context(log_n, qb, pb, d, h=boot[0], seed=1, arena_bytes=64 << 30)
        g.bootstrap_prepare(*boot[1:])
        g.set_graphs(args.graph)  # candidates are timed as the benches run them
        return g

    inputs = lambda g: [g.encrypt(P.pack(x, slots, pl.packing), g.delta, 7 + s) for s, x in enumerate(xs)]
    check = lambda g, i, z: int(np.argmax(g.decrypt(z, pl.n))) == int(np.argmax(xs[i]))
    log = lambda m: print(m, file=sys.stderr, flush=True)
    choice, table = autotune.tune_decode(make_ctx, pl, inputs, check, dnums=(3, 4, 5), log=log)
    free, total = torch.cuda.mem_get_info()
    log(f"device memory free after the decode search: {free / 2**30:.1f} of {total / 2**30:.1f} GiB")
    g = he.Context(log_n, qb, pb, choice["dnum"], h=boot[0], seed=1, arena_bytes=200 << 30)
    g.bootstrap_prepare(*boot[1:])
    g.set_graphs(args.graph)
    g.set_rotsum_radix(choice["rotsum_log_radix"])
    batches = {}
    for v, bpl, bxs, batch, _ in cfg3_batches(g, 16, CFG3_VOCABS):
        batches[str(v)] = (bpl, batch, lambda Z, bxs=bxs, bpl=bpl: batch_argmax_ok(g, Z, bxs, bpl) == len(bxs))
    choice["chains"], table["chains"] = autotune.tune_chains(g, batches, log=log)
    rec = autotune.save(autotune.default_path(log_n), log_n, qb, pb, boot[0], choice, table,
                        {"decode": desc["workload"], "batches": "16 streams per vocabulary "
                         + "/".join(map(str, CFG3_VOCABS)) + ", N(0,4) logits, top gap 0.5"})
    print(json.dumps(rec))


def run_cfg4(args):
    """Learned inverse square root vs the plain approximation on the full
    workload (32,000 logits, N=2^16, bootstrapping).  About 100k variances
    (25,000 vectors x T=4) are logged from the plain plan's FP64 circuit; the
    network is trained on the GPU; the plan keeps the learned quadratic where
    its error over the calibrated range is within 8%.  Reported: levels,
    bootstraps, key switches and latency per decode (CUDA events), and argmax
    accuracy over 10,000 seeded vectors (FP64 circuit) and over the encrypted
    decodes, for both plans."""
    from paper_2509_08383_gb300 import learned
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    log_n, qb, pb, dnum, plain, gen, desc, boot = workload("cfg2")
    calib_kw = dict(sample=lambda i: gen(100000 + i), n_cal=200, n=plain.n, slots=plain.slots, T=4,
                    p=[16, 4, 4, 6], c=[5.0, 3.0, 3.0, 3.0], margin=2.0, tol_k=INVSQRT_TOL, k_max=20, d_max=14,
                    tol_d=INVSQRT_TOL, bootstrap=True, relax=RELAX)
    t0 = time.perf_counter()
    logged = learned.log_variances(plain, gen, range(600000, 625000))  # spawn pool, before CUDA
    t_log = time.perf_counter() - t0
    acc_plain = learned.fp64_accuracy(plain, gen, range(800000, 810000))
    import torch
    from paper_2509_08383_gb300 import build, he
    build.build_library()
    torch.cuda.set_device(0)
    g = he.Context(log_n, qb, pb, dnum, h=boot[0], seed=1, arena_bytes=48 << 30)
    g.bootstrap_prepare(*boot[1:])
    g.set_graphs(args.graph)
    t0 = time.perf_counter()
    lpl, report = learned.learned_plan(g, plain, calib_kw, logged)
    t_train = time.perf_counter() - t0
    acc_learned = learned.fp64_accuracy(lpl, gen, range(800000, 810000))
    slots = 1 << (log_n - 1)
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(0) as clk:
        for name, pl in (("plain", plain), ("learned", lpl)):
            g.cutmax_prepare(pl)
            ms, ok = [], 0
            for s in range(args.warmup + args.steps):
                x = gen(900000 + s)
                ct = g.encrypt(P.pack(x, slots, pl.packing), g.delta, 50 + s)
                g.ledger(reset=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                z = g.cutmax(ct, pl)
                e1.record(stream)
                torch.cuda.synchronize()
                ks, nb = g.ledger(reset=True)
                ok += int(np.argmax(g.decrypt(z, pl.n))) == int(np.argmax(x))
                if s >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            res[name] = {"ms_per_decode": float(np.mean(ms)), "decodes_per_s": 1000.0 / float(np.mean(ms)),
                         "levels": pl.depth(), "k": list(pl.k), "bootstraps_per_decode": nb,
                         "keyswitches_per_decode": int(ks.sum()), "encrypted_argmax": [ok, args.warmup + args.steps]}
    res["plain"]["fp64_argmax"] = {"correct": acc_plain[0], "of": acc_plain[1], "mean_max_z": acc_plain[2],
                                   "min_max_z": acc_plain[3]}
    res["learned"]["fp64_argmax"] = {"correct": acc_learned[0], "of": acc_learned[1], "mean_max_z": acc_learned[2],
                                     "min_max_z": acc_learned[3]}
    out = {"metric": "encrypted CutMax decodes/sec with the learned inverse square root (vocab 32k, N=2^16), 1 GB300",
           "value": res["learned"]["decodes_per_s"], "unit": "decodes/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["learned"]["ms_per_decode"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": desc["workload"] + "; learned 1-16-1 square-activation inverse square root",
                      "variances_logged": int(logged.size), "log_seconds": t_log, "train_seconds": t_train,
                      "cuda_graph": bool(args.graph)},
           "training": {str(t): v for t, v in report.items()}, "plain": res["plain"], "learned": res["learned"],
           "speedup_vs_plain": res["plain"]["ms_per_decode"] / res["learned"]["ms_per_decode"],
           "clocks": clk.summary()}
    print(json.dumps(out))


def _nucleus_set(x, p):
    """Smallest top-probability token set with softmax mass >= p."""
    pr = np.exp(x - x.max())
    pr /= pr.sum()
    order = np.argsort(-pr, kind="stable")
    return set(order[:int(np.searchsorted(np.cumsum(pr[order]), p) + 1)].tolist())


def run_cfg5(args):
    """HE nucleus (top-p) sampling decode loop (Alg. 3): 16 streams of 128,256
    logits (4 ciphertexts each) at N=2^16, 8 streams at p = 0.9 and 8 at
    p = 0.95 in one batch (alpha = ln(1-p)/ln(p) per group).  Per token the
    client encrypts each stream's logits (regenerated from the seed: N(0, 2^2),
    top gap 0.5) at the bootstrap output level and its uniforms U seven levels
    higher at scale 2^60, on the 60-bit primes, so that the noise's seven levels
    come on top of the circuit's; the server draws G = U^(1/alpha) from them
    (nucleus_sample_groups with HE_RAND_UNIFORM: alpha per group in the library,
    degree-31 Chebyshev) and samples CutMax(X + G) for all 16 streams at once,
    with bootstrapping and shared scalar chains; the client decrypts and takes
    the argmax as the token.  The
    plain plan and the learned plan (learned inverse square root) run side by
    side.  Reported: tokens/s of the server work (CUDA events) and end to end,
    agreement of the tokens with the FP64 sampler argmax(x + U^(1/alpha)), and
    tokens outside the top-p nucleus of softmax(x)."""
    from paper_2509_08383_gb300 import learned
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import synth
    n, per, slots = 128256, 8, 1 << 15
    deg = 31  # the library's HE_NUCLEUS_DEGREE (checked against he.HE_NUCLEUS_DEGREE below)
    ps = [0.9, 0.95]
    alphas = [math.log(1.0 - p) / math.log(p) for p in ps]

    def logits(stream, step):
        return synth.logits_gaussian(1000003 * (stream + 1) + step, n=n, sd=2.0, gap=0.5)

    gen = synth.Gaussian(n, 2.0, 0.5)
    # plan on logits plus cut noise (the circuit's input is x + G)
    calib_kw = dict(sample=lambda i: gen(300000 + i) + synth.uniforms(300000 + i, n) ** (1.0 / alphas[i % 2]),
                    n_cal=60, n=n, slots=slots, T=4, p=[16, 4, 4, 6], c=[5.0, 3.0, 3.0, 3.0], margin=2.0,
                    tol_k=INVSQRT_TOL, k_max=20, d_max=14, tol_d=INVSQRT_TOL, bootstrap=True, relax=RELAX)
    plain = P.calibrate(**calib_kw)
    plain.shared = True
    logged = learned.log_variances(plain, gen, range(500000, 505000))  # spawn pool, before CUDA
    import torch
    from paper_2509_08383_gb300 import build, he
    build.build_library()
    torch.cuda.set_device(0)
    g = he.Context(16, CFG2_Q, CFG2_P, 3, h=192, seed=1, arena_bytes=200 << 30)
    g.bootstrap_prepare(24, 4, 31)
    g.set_graphs(args.graph)
    assert he.HE_NUCLEUS_DEGREE == deg
    lpl, report = learned.learned_plan(g, plain, calib_kw, logged)
    lpl.shared = True
    stream = torch.cuda.current_stream()
    out_level = None
    res = {}
    with ClockSampler(0) as clk:
        for name, pl in (("plain", plain), ("learned", lpl)):
            g.cutmax_prepare(pl)
            t_dev, t_e2e, agree, agree_poly, outside, total = 0.0, 0.0, 0, 0, 0, 0
            th = np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1)
            for step in range(args.warmup + args.tokens):
                timed = step >= args.warmup
                t0 = time.perf_counter()
                xs, us, cts, uts = [], [], [], []
                for st in range(2 * per):  # streams 0..per-1 at ps[0], per..2per-1 at ps[1]
                    x, u = logits(st, step), synth.uniforms(7000003 * (st + 1) + step, n)
                    xs.append(x)
                    us.append(u)
                    for c, v in enumerate(P.pack_cts(x, slots)):
                        cts.append(g.encrypt(v, g.delta, (st * 64 + step) * 8 + c, level=13))
                    for c, v in enumerate(P.pack_cts(u, slots)):  # seven levels up, on the 60-bit primes
                        uts.append(g.encrypt(v, 2.0 ** 60, (st * 64 + step) * 8 + 4 + c, level=13 + 7))
                X, U = g.batch_pack(cts), g.batch_pack(uts)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                Z = g.nucleus_sample_groups(X, U, pl, ps, kind="uniform")  # one CutMax for all 16 streams
                e1.record(stream)
                torch.cuda.synchronize()
                toks = []
                for st in range(2 * per):
                    dec = np.concatenate([g.decrypt(g.batch_member(Z, st * 4 + c)) for c in range(4)])[:n]
                    toks.append(int(np.argmax(dec)))
                t1 = time.perf_counter()
                if timed:
                    t_dev += e0.elapsed_time(e1) / 1000.0
                    t_e2e += t1 - t0
                    for st, (x, u, tok) in enumerate(zip(xs, us, toks)):
                        p, alpha = ps[st // per], alphas[st // per]
                        f = ((np.cos(th) + 1) / 2) ** (1 / alpha)
                        cc = np.array([2 / (deg + 1) * np.sum(f * np.cos(k * th)) for k in range(deg + 1)])
                        cc[0] /= 2
                        agree += tok == int(np.argmax(x + u ** (1.0 / alpha)))
                        agree_poly += tok == int(np.argmax(x + np.polynomial.chebyshev.chebval(2 * u - 1, cc)))
                        outside += tok not in _nucleus_set(x, p)
                        total += 1
            g.graph_clear()  # this plan's graph gives its memory back
            res[name] = {"tokens_per_s": total / t_dev, "tokens_per_s_e2e": total / t_e2e,
                         "ms_per_token_step": 1000.0 * t_dev / args.tokens, "tokens": total,
                         "agree_fp64_sampler": agree, "agree_fp64_same_noise_polynomial": agree_poly,
                         "outside_top_p_nucleus": outside, "k": list(pl.k), "levels": pl.depth()}
    out = {"metric": "encrypted nucleus-sampling tokens/sec, 16 streams x vocab 128,256 (N=2^16), 1 GB300",
           "value": res["learned"]["tokens_per_s"], "unit": "tokens/s", "n_gpus": 1, "steps": args.tokens,
           "warmup": args.warmup, "ms_per_step": res["learned"]["ms_per_token_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": {"workload": "Alg. 3 decode loop: 16 streams (8 at top-p 0.9, 8 at 0.95) x 128,256 logits "
                                  "N(0,4) top gap 0.5 in 4 ciphertexts, G = U^(1/alpha) from encrypted uniforms "
                                  "(degree-31 Chebyshev), CutMax T=4 p=[16,4,4,6] c=[5,3,3,3], bootstrapping, "
                                  "shared scalar chains, one batch of 16 streams (nucleus_sample_groups)",
                      "tokens": args.tokens, "streams": 2 * per,
                      "cuda_graph": bool(args.graph)},
           "plain": res["plain"], "learned": res["learned"],
           "training": {str(t): {k: v for k, v in r.items() if k != "abc"} for t, r in report.items()},
           "clocks": clk.summary()}
    print(json.dumps(out))


def run_micro(args):
    """Micro workloads for kernel profiles at the N=2^16 parameter set (the
    same kernels as a CutMax step at full size): mul16 = one homomorphic
    multiplication (tensor product, hybrid key switch and rescale in one
    rounded division by q_l P) at the top level; rot16 = one rotation (automorphism + hybrid key switch) at the top
    level; ntt16 = a forward and an inverse NTT of one 40-limb block (every
    prime of the chain, 21 MB); boot16 = one bootstrapping of a level-0
    ciphertext; bootc16 = one constant bootstrapping (trace form) of a level-0
    ciphertext holding one complex value in every slot."""
    import torch
    from paper_2509_08383_gb300 import build, he
    build.build_library()
    torch.cuda.set_device(0)
    boot = args.workload in ("boot16", "bootc16")
    g = he.Context(16, CFG2_Q, CFG2_P, 3, h=192, seed=1, arena_bytes=(24 << 30) if boot else (4 << 30))
    rng = np.random.default_rng(0)
    slots = 1 << 15
    roof = None
    if args.workload == "bootc16":
        g.bootstrap_prepare(24, 4, 31)
        g.gen_rot_keys([1 << i for i in range(15)])
        cts = [g.encrypt(np.full(slots, 0.9 + 0.2j), g.delta, 0, level=0)]
        op = lambda: g.bootstrap_const(cts[0])
        metric, unit = "constant bootstraps/s (N=2^16, K=24, r=4, d=31, dnum=3)", "boot/s"
        wl = ("CKKS bootstrapping of a level-0 ciphertext holding one complex value in every slot "
              "(trace form), N=2^16, 30 primes + 10 special primes, h=192")
    elif boot:
        g.bootstrap_prepare(24, 4, 31)
        cts = [g.encrypt(rng.uniform(-1, 1, slots), g.delta, 0, level=0)]
        op = lambda: g.bootstrap(cts[0])
        metric, unit = "bootstraps/s (N=2^16, K=24, r=4, d=31, dnum=3)", "boot/s"
        wl = "CKKS bootstrapping of a level-0 ciphertext, N=2^16, 30 primes + 10 special primes, h=192"
    elif args.workload == "ntt16":
        limbs = len(CFG2_Q) + len(CFG2_P)
        blk = torch.randint(0, 1 << 39, (limbs, 1 << 16), dtype=torch.int64, device="cuda")
        op = lambda: (g.ntt_device(blk, 0), g.ntt_device(blk, 0, inverse=True))
        metric, unit = "NTT forward + inverse, 40 limbs (N=2^16)", "pairs/s"
        wl = "negacyclic NTT then INTT of a 40-limb block (every prime of the N=2^16 chain), in place"
        roof = 2 * 16.0 * limbs * (1 << 16)  # algorithmic bytes per step: read + write each limb, twice
    elif args.workload == "rot16":
        g.gen_rot_keys([1])
        cts = [g.encrypt(rng.uniform(-1, 1, slots), g.delta, 0)]
        op = lambda: g.rotate(cts[0], 1)
        metric, unit = "homomorphic rotations/s (N=2^16, level 29, dnum=3)", "rot/s"
        wl = "slot rotation by 1 (automorphism + hybrid key switch), N=2^16, 30 primes + 10 special primes"
        l1, K, beta = len(CFG2_Q), len(CFG2_P), 3
        # automorphism (read + write both polynomials) + key switch: d in, beta key digits
        # (b and a over l+1+K primes), two output polynomials
        roof = 8.0 * (1 << 16) * (4 * l1 + l1 + 2 * beta * (l1 + K) + 2 * l1)
    else:
        g.gen_relin_key()
        cts = [g.encrypt(rng.uniform(-1, 1, slots), g.delta, s) for s in range(2)]
        op = lambda: g.mul_rescale(cts[0], cts[1])
        metric, unit = "homomorphic multiplications/s (N=2^16, level 29, dnum=3)", "mul/s"
        wl = ("ciphertext product + relinearisation + rescale (one rounded division by q_l P), N=2^16, "
              "30 primes + 10 special primes")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    nsteps = args.warmup + args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    with ClockSampler(0) as clk:
        for s in range(nsteps):
            flush.zero_()
            if s >= args.warmup:
                torch.cuda.nvtx.range_push("timed_step")
            ev[s][0].record(stream)
            z = op()
            ev[s][1].record(stream)
            if s >= args.warmup:
                torch.cuda.nvtx.range_pop()
            del z
        torch.cuda.synchronize()
    ms = sum(ev[s][0].elapsed_time(ev[s][1]) for s in range(args.warmup, nsteps)) / args.steps
    out = {"metric": metric, "value": 1000.0 / ms, "unit": unit, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "dtype": "u64", "data": "synthetic", "clocks": clk.summary(),
           "config": {"workload": wl, "l2": "flushed between steps"}}
    if roof:
        peak, kind = measured_peaks()
        out["roofline"] = {"bound": "hbm", "achieved": roof / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": roof / (ms * 1e-3) / 1e9 / peak, "traffic": None, "peak_source": kind}
    print(json.dumps(out))


def keyswitch_block(g, ks_by_level, log_n, qb, pb, dnum, stream, flush, peak, reps=10, warm=3):
    """Whole rotations (automorphism + hybrid key switch) timed with CUDA events
    at the top level and at the median level of the decode's key switches, L2
    flushed before each.  Algorithmic bytes per the key switch's definition:
    the input polynomial (l+1) N words, the beta key digits (b and a over
    l+1+K primes), the two outputs; plus the automorphism's read and write of
    both polynomials."""
    import torch
    n, K = 1 << log_n, len(pb)
    alpha = -(-len(qb) // dnum)
    lv = sorted(ks_by_level)
    acc, tot, med = 0, sum(ks_by_level.values()), lv[0]
    for l in lv:
        acc += ks_by_level[l]
        if 2 * acc >= tot:
            med = l
            break
    out = []
    for l in (len(qb) - 1, med):
        ct = g.encrypt(np.linspace(-1, 1, n // 2), g.delta, 4242, level=l)
        ts = []
        for i in range(warm + reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z = g.rotate(ct, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            del z
            if i >= warm:
                ts.append(e0.elapsed_time(e1))
        ms = float(np.mean(ts))
        beta = -(-(l + 1) // alpha)
        ks_bytes = 8.0 * n * ((l + 1) + 2 * beta * (l + 1 + K) + 2 * (l + 1))
        rot_bytes = ks_bytes + 8.0 * n * 4 * (l + 1)
        gbs = rot_bytes / (ms * 1e-3) / 1e9
        out.append({"level": l, "op": "rotation (automorphism + hybrid key switch)", "ms": ms,
                    "keyswitch_bytes": ks_bytes, "algorithmic_bytes": rot_bytes, "achieved_gbs": gbs,
                    "peak_gbs": peak, "frac": gbs / peak, "what": "top level" if l == len(qb) - 1 else
                    "median level of the decode's key switches"})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2", choices=["cfg1", "cfg2", "cfg3", "cfg4", "cfg5", "tune", "mul16",
                                                           "rot16", "ntt16", "boot16", "bootc16"])
    ap.add_argument("--tokens", type=int, default=32, help="cfg5: tokens decoded per stream")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--newton", action="store_true",
                    help="Goldschmidt steps with Newton's constant 3/2 only (no calibrated relaxation)")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="call cutmax / nucleus_sample directly instead of replaying their CUDA graphs")
    ap.add_argument("--chains", default="tuned", choices=["tuned", "shared", "stream"],
                    help="cfg3: scalar chains packed across a batch's streams (general bootstraps), kept per "
                         "stream (constant bootstraps, one launch for the batch), or as the autotuner chose")
    args = ap.parse_args()
    global RELAX
    RELAX = not args.newton
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("mul16", "rot16", "ntt16", "boot16", "bootc16"):
        return run_micro(args)
    if args.workload == "cfg3":
        return run_cfg3(args)
    if args.workload == "tune":
        return run_tune(args)
    if args.workload == "cfg4":
        return run_cfg4(args)
    if args.workload == "cfg5":
        return run_cfg5(args)

    import torch
    dist, rank, ws = dist_setup(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2509_08383_gb300 import build, he
    from paper_2509_08383_gb300 import plan as P
    from paper_2509_08383_gb300 import replicas
    build.build_library()
    log_n, qb, pb, dnum, pl, gen, desc, boot = workload(args.workload)
    if boot is not None:
        g = he.Context(log_n, qb, pb, dnum, h=boot[0], seed=1 + rank, arena_bytes=64 << 30)
        g.bootstrap_prepare(*boot[1:])
    else:
        g = he.Context(log_n, qb, pb, dnum, seed=1 + rank)
    g.cutmax_prepare(pl)
    slots = 1 << (log_n - 1)
    stream = torch.cuda.current_stream()
    nsteps = args.warmup + args.steps
    cts = [g.encrypt(P.pack(gen(10000 * rank + s), slots, pl.packing), g.delta, s) for s in range(nsteps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
    # dominant kernel class: one instrumented CutMax per class (untimed)
    share = {}
    for cls in PROF_NAMES:
        he.profile_enable(cls)
        z = g.cutmax(cts[0], pl)
        torch.cuda.synchronize()
        share[cls] = he.profile_read(cls)[1]
        del z
    he.profile_enable(-1)
    dom = max(share, key=share.get)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # timed region: no instrumentation; CUDA events on the library's stream.
    # With CUDA graphs (the default) the first warm-up decode runs directly and
    # captures the graph; the others replay it.
    run = g.cutmax_graph if args.graph else g.cutmax
    g.ledger(reset=True)
    l0 = he.launch_count()
    with ClockSampler(local) as clk:
        for s in range(nsteps):
            flush.zero_()
            if s >= args.warmup:
                torch.cuda.nvtx.range_push("timed_step")
            ev[s][0].record(stream)
            z = run(cts[s], pl)
            ev[s][1].record(stream)
            if s >= args.warmup:
                torch.cuda.nvtx.range_pop()
            if s == args.warmup - 1:
                torch.cuda.synchronize()
                l0 = he.launch_count()
                g.ledger(reset=True)
            del z
        torch.cuda.synchronize()
    launches = he.launch_count() - l0
    ops = g.ledger_ops()
    ks_led, nboot = g.ledger(reset=True)
    census = {"ks": {i: int(v) // args.steps for i, v in enumerate(ks_led) if v}}
    for k, v in ops.items():
        census[k] = {i: int(c) // args.steps for i, c in enumerate(v) if c}
    ks_by_level = census["ks"]
    ms = sum(ev[s][0].elapsed_time(ev[s][1]) for s in range(args.warmup, nsteps)) / args.steps
    ms = replicas.max_over_ranks(ms, dist, device="cuda")
    if dist:
        dist.barrier()
    # roofline of the dominant class: the same timed steps again with CUDA
    # events around every launch of that class (on the launch stream); these
    # instrumented steps are not part of `value`
    he.profile_enable(dom)
    t_ins = []
    for s in range(args.warmup, nsteps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        z = g.cutmax(cts[s], pl)
        e1.record(stream)
        del z
        torch.cuda.synchronize()
        t_ins.append(e0.elapsed_time(e1))
    n_dom, ms_dom, bytes_dom = he.profile_read(dom)
    he.profile_enable(-1)
    peak, peak_kind = measured_peaks()
    achieved = (bytes_dom / n_dom) / (ms_dom / n_dom * 1e-3) / 1e9 if n_dom else 0.0
    # DRAM bytes per launch of the dominant class from the ncu capture of the
    # current NTT source (null once that source has changed), scaled by the
    # limbs a launch moves
    traffic = None
    if (dom in (0, 1) and log_n == 16 and n_dom and NTT_DRAM["src"] == ntt_source_hash()
            and NTT_DRAM["per_limb"][dom]):
        traffic = NTT_DRAM["per_limb"][dom] * (bytes_dom / n_dom) / (16.0 * (1 << log_n))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": PROF_NAMES[dom], "launches": n_dom,
                "avg_launch_us": 1000.0 * ms_dom / max(n_dom, 1),
                "algorithmic_bytes_per_launch": bytes_dom / max(n_dom, 1),
                "share_of_step": (ms_dom / args.steps) / ms if ms else None, "peak_source": peak_kind,
                "measured_over": f"{args.steps} instrumented repeats of the timed steps (CUDA events around every "
                                 f"launch of the class, {float(np.mean(t_ins)):.1f} ms per step with them); `value` "
                                 "comes from the uninstrumented steps",
                "class_ms_per_step": {PROF_NAMES[c]: v for c, v in share.items()}}
    if dom in (0, 1) and n_dom:
        # the NTT binds on integer issue, not on HBM: butterflies per second
        # against the issue ceiling
        fly = (bytes_dom / n_dom) / (16.0 * (1 << log_n)) * (1 << (log_n - 1)) * log_n
        fly_s = fly / (ms_dom / n_dom * 1e-3)
        ceil = ALU_ISSUE_PEAK / NTT_WARP_INSTR_PER_BUTTERFLY
        roofline["alu"] = {"achieved": fly_s, "peak": ceil, "unit": "butterflies/s", "frac": fly_s / ceil,
                           "peak_source": "152 SMs x 4 warp instructions per clock x 2.07 GHz / "
                                          f"{NTT_WARP_INSTR_PER_BUTTERFLY} warp instructions per butterfly (ncu)"}
    ks_block = keyswitch_block(g, ks_by_level, log_n, qb, pb, dnum, stream, flush, peak) if log_n == 16 else None
    value = ws * 1000.0 / ms

    # end to end through the C ABI: pinned host logits -> host outputs
    pin = torch.empty(slots, dtype=torch.float64).pin_memory()
    out = np.zeros(pl.n)
    e2e_times = []
    argmax_ok, top_z = 0, []
    for s in range(nsteps):
        x_s = gen(20000 + s)
        pin.numpy()[:] = P.pack(x_s, slots, pl.packing)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ct = g.encrypt(pin.numpy(), g.delta, 100000 + s)
        z = run(ct, pl)
        out[:] = g.decrypt(z, pl.n)
        t1 = time.perf_counter()
        argmax_ok += int(np.argmax(out)) == int(np.argmax(x_s))
        top_z.append(float(out.max()))
        if s >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e = ws * args.steps / replicas.max_over_ranks(sum(e2e_times), dist, device="cuda")

    res = {"metric": METRIC, "value": value, "unit": "decodes/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": dict(desc, l2="flushed between steps (256 MiB write)", parallelism=f"replicas x{ws}",
                          cuda_graph=bool(args.graph), graph_stats=dict(zip(("captured", "replayed", "direct"),
                                                                            g.graph_stats()))),
           "clocks": clk.summary(),
           "e2e": {"value": e2e, "unit": "decodes/s", "h2d_bytes_per_step": slots * 8,
                   "d2h_bytes_per_step": pl.n * 8},
           "gpu_launches": int(launches), "roofline": roofline,
           "check": {"argmax_correct": argmax_ok, "decodes": nsteps, "mean_max_z": float(np.mean(top_z)),
                     "what": "decrypted end-to-end outputs: argmax vs the plaintext logits, mean of max Z"},
           "ledger": {"keyswitches_per_decode": int(sum(ks_by_level.values())),
                      "bootstraps_per_decode": nboot / args.steps,
                      "ops_per_decode": {k: int(sum(v.values())) for k, v in census.items() if k != "ks"}}}
    if ks_block:
        res["keyswitch"] = ks_block
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            res["cpu_baseline"] = cpu_baseline(args, census)
        print(json.dumps(res))


if __name__ == "__main__":
    main()
