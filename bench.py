#!/usr/bin/env python3
"""Seeding-stage benchmark: reads/s seeded + located on one GB300 (or N replicas).

One step = SMEM finding + max-occ flag + locate (mb_seed_batch then mb_locate) over one
batch of reads.  Default workload: 1 Gbp repeat-rich synthetic reference (45% repeats,
0.5% N runs) and 10M 2x150 bp pairs (20M reads), min_len 19, max_occ 500, SA rate 32.
The index build is timed separately and is not part of the step.

Prints one JSON line.  `--impl reference` times the CPU oracle (the plain reference
implementation of the same stage) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    3: "1 Gbp repeat-rich reference (45% repeats: tandem/segdup/satellite 5:2:1, 0.5% N runs), "
       "10M 2x150 bp pairs, insert N(400,50), subst 0.1%->1% along the read, 0.01% indels",
    2: "100 Mbp repeat-rich reference (8% repeats, 0.5% N runs), 1M 2x150 bp pairs",
    1: "1 Mbp uniform reference, 10,000 single-end 150 bp reads, 0.5% substitutions",
}


BLOCK_BYTES = 32   # one occurrence block (64 BWT rows) per 32-byte sector


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, pg) -> float:
    """The largest value of x over all ranks (timing is the slowest rank's); identity at N=1."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, units_per_rank_step: int, ms: float) -> float:
    """Weak scaling: every rank processes its own batch of the same size each step."""
    return world * steps * units_per_rank_step / (ms / 1000.0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def gather_ceiling(gib: float = 4, modes=((0, "indep", 2048), (1, "chain", 512), (2, "chain_l2only", 512))):
    """Random 64-/32-byte block reads over a buffer of `gib` GiB (probe library): independent
    reads (bandwidth ceiling) and dependent chains (LF-walk pattern), GB/s of bytes requested."""
    import ctypes
    from paper_2606_15357_gb300.nvcc_build import build_probe
    L = ctypes.CDLL(build_probe())
    L.mb_probe_gather.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                  ctypes.POINTER(ctypes.c_float)]
    L.mb_probe_gather.restype = ctypes.c_double
    out = {}
    ms = ctypes.c_float()
    for mode, name, iters in modes:
        for bb in (64, 32):
            out[f"random{bb}_{name}_GBps"] = L.mb_probe_gather(int(gib * (1 << 30)), mode, bb, iters,
                                                                ctypes.byref(ms))
    out["buffer_GiB"] = gib
    return out


def locate_sweep(mb, torch, idx, out, m, hits, nh, opts, reps: int = 3):
    """The locate forms on one step's records (plain mb_locate calls, device buffers): plain walks,
    walks that join and walks to the rate-4 samples at several walks per lane, each timed with CUDA
    events (kernel time from the library's own events, and the whole call), output compared with
    the first form; one JSON line per point, then the work counts of each form."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    want = None
    forms = (("plain", 0, (16, 8, 4, 2)), ("join", mb.MB_LOCATE_JOIN, (4, 2, 1)), ("aux", mb.MB_LOCATE_AUX, (16, 4, 2)))
    for name, fl, depths in forms:
        for depth in depths:
            o = dict(opts, prefetch_depth=depth, flags=(opts.get("flags", 0) & ~(mb.MB_LOCATE_JOIN | mb.MB_LOCATE_AUX)) | fl)
            mb.mb_locate(idx, out, m, opts=o, hits=hits, cap=nh)
            torch.cuda.synchronize()
            mb.profile_reset()
            mb.profile_enable(True)
            e0.record(st)
            for _ in range(reps):
                mb.mb_locate(idx, out, m, opts=o, hits=hits, cap=nh)
            e1.record(st)
            torch.cuda.synchronize()
            mb.profile_enable(False)
            kms, kn = mb.profile_get("locate")
            same = None
            if want is None:
                want = hits[:nh].clone()
            else:
                same = bool(torch.equal(hits[:nh], want))
                if not same:
                    raise SystemExit(f"bench: locate form {name} at {depth} walks per lane disagrees")
            print(json.dumps({"locate_form": name, "walks_per_lane": depth, "kernel_ms": kms / max(kn, 1),
                              "call_ms": e0.elapsed_time(e1) / reps, "identical_output": same}), flush=True)
    for name, fl, _ in forms:
        mb.profile_reset()
        mb.mb_locate(idx, out, m, opts=dict(opts, flags=mb.MB_COUNT | fl), hits=hits, cap=nh)
        print(json.dumps({"locate_form": name, "work": mb.work_counters()}), flush=True)
    return 0


def probe_sweep():
    """Random-read rate against buffer size (L2-resident to far above L2): one JSON line per size,
    with the 32-byte rate also in reads/s."""
    import torch
    torch.cuda.init()
    for gib in (1 / 32, 3 / 32, 1 / 4, 1, 4, 8):
        gc = gather_ceiling(gib, modes=((0, "indep", 2048), (1, "chain", 512)))
        gc["random32_indep_Greads_per_s"] = gc["random32_indep_GBps"] / 32
        print(json.dumps(gc), flush=True)
    return 0


def strip_comments(src: str) -> str:
    """C/C++ source without its // and /* */ comments and blank lines (string and character
    literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).split("\n") if line.strip())


def kernel_source_hash() -> str:
    """Hash of the seeding kernels' code (seed.cu and common.cuh without comments): ties the
    committed DRAM traffic to the code it was measured on."""
    h = hashlib.sha256()
    for f in ("seed.cu", "common.cuh"):
        src = open(os.path.join(ROOT, "paper_2606_15357_gb300", "csrc", f), encoding="utf-8").read()
        h.update(strip_comments(src).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    kernel source (profiles/<kernel>_<workload>.txt lines 'source_hash:' and
    'dram_bytes_per_launch:')."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    mh = re.search(r"source_hash:\s*(\w+)", txt)
    mb = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not mh or not mb or mh.group(1) != kernel_source_hash():
        return None
    return float(mb.group(1))


def ncu_hit_rates(kernel: str, workload: str):
    """(L2 hit %, L1 hit %) of the --set full capture in the same committed summary, if it was
    taken on the current kernel source."""
    if ncu_traffic(kernel, workload) is None:
        return None
    txt = open(os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")).read()
    l2 = re.search(r"- L2 hit rate %:\s*([0-9.]+)", txt)
    l1 = re.search(r"- L1 hit rate %:\s*([0-9.]+)", txt)
    return (float(l2.group(1)), float(l1.group(1))) if l2 and l1 else None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(workload: int, scale: float, rank: int, reads: int = 0):
    t = time.time()
    ref, rd, params = synth.workload(workload, scale)
    if reads and reads < rd.n:   # a subset of the batch (profiling captures only)
        rd = rd.subset(np.arange(reads))
    if rank:
        # weak scaling: every rank seeds its own batch of the same size
        o = rd.n
        kw = dict(mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01, indel=0.0001)
        if workload == 1:
            kw = dict(mode=0, read_len=150, sub_lo=0.005)
        rd = synth.reads(ref, o, synth.SEED[workload] + 1000 * rank, **kw)
    log(f"inputs: |R|={len(ref)} reads={rd.n} bases={len(rd.seq)} ({time.time() - t:.1f}s)")
    return ref, rd, params


# --------------------------------------------------------------------------------- oracle side
def oracle_rate(ref, rd, params, target_s: float, threads: int, min_reads: int = 2048):
    """Time the CPU oracle (index built first, untimed) on a bounded sample of the reads."""
    import oracle
    t = time.time()
    X = oracle.Index(ref, n_seed=0, threads=threads)
    build_s = time.time() - t
    rng = np.random.default_rng(12345)
    n_probe = min(rd.n, min_reads)
    sample = rd.subset(np.sort(rng.choice(rd.n, n_probe, replace=False)))
    t = time.time()
    X.seed(sample.seq, sample.off, params["min_len"], params["min_occ"], params["max_occ"], threads=threads)
    dt = max(time.time() - t, 1e-3)
    n = int(min(rd.n, max(n_probe, n_probe * target_s / dt)))
    sample = rd.subset(np.sort(rng.choice(rd.n, n, replace=False)))
    return X, build_s, sample


def cpu_batched_rate(src, sample, params, threads: int) -> dict:
    """The paper's CPU design (Algorithm 3 with one queue per batch and prefetching, 64-byte
    blocks, 10-mer table, BatchLocate) on the host cores, on the oracle's sample: context for the
    GPU numbers, built from the GPU index's BWT and sampled suffix array."""
    import cpu_batched
    bwt, primary, ssa = src
    t = time.time()
    Y = cpu_batched.Index(bwt, primary, ssa, threads=threads)
    build_s = time.time() - t
    Y.seed(sample.seq[:int(sample.off[min(sample.n, 256)])], sample.off[:min(sample.n, 256) + 1],
           params["min_len"], params["min_occ"], params["max_occ"], threads=threads)   # warm-up
    t = time.time()
    sm, hits = Y.seed(sample.seq, sample.off, params["min_len"], params["min_occ"], params["max_occ"],
                      threads=threads)
    dt = time.time() - t
    return {"value": sample.n / dt, "unit": "reads/s", "cores": threads, "kind": "paper's CPU design",
            "sample": f"the oracle's {sample.n} reads; index from the BWT ({build_s:.0f}s) untimed",
            "seconds": dt, "smems": int(len(sm)), "hits": int(len(hits))}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    ref, rd, params = make_inputs(args.workload, args.scale, 0)
    X, build_s, sample = oracle_rate(ref, rd, params, args.ref_step_s, threads)
    times = []
    for it in range(args.warmup + args.steps):
        t = time.time()
        X.seed(sample.seq, sample.off, params["min_len"], params["min_occ"], params["max_occ"], threads=threads)
        dt = time.time() - t
        if it >= args.warmup:
            times.append(dt)
    T = float(np.sum(times))
    value = args.steps * sample.n / T
    desc = f"{sample.n} reads drawn (seed 12345) from the {rd.n}-read batch, oracle index built first " \
           f"({build_s:.0f}s, untimed)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "reads/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "scale": args.scale, "min_len": params["min_len"],
                   "max_occ": params["max_occ"], "sa_rate": params["sa_rate"], "kmer_k": args.kmer_k},
        "cpu_baseline": {"value": value, "unit": "reads/s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "reads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------- batched / served
def bench_batched(mb, torch, dev, reps: int = 3):
    """Mixed-length workload (100 Mbp repeat-rich reference, 200,000 reads of 100 bp-10 kb):
    one plain launch per length bucket (a preallocated plan per bucket in the default launch
    shape, run one after another), against the batched form (one autotuned plan over the whole
    batch, device work queue, replayed CUDA graph).  Output compared for identity; the autotuner's
    whole grid is reported."""
    ref, rd, params = synth.workload(4)
    G = mb.mb_index_build(torch.from_numpy(ref).to(dev))
    G.drop_sa()
    lens = np.diff(rd.off.astype(np.int64))
    edges = [100 * 2 ** i for i in range(8)] + [10001]
    buckets = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        ids = np.nonzero((lens >= lo) & (lens < hi))[0]
        if len(ids):
            sub = rd.subset(ids)
            s_, o_ = torch.from_numpy(sub.seq).to(dev), torch.from_numpy(sub.off.view(np.int64)).to(dev)
            _, m, nh = mb.mb_seed_batch(G, s_, o_, cap=64 * len(ids))
            P = mb.Plan(G, len(ids), len(sub.seq), m + 64, nh + 64)
            buckets.append((ids, s_, o_, P, m, nh))

    def plain():
        for ids, s_, o_, P, m, nh in buckets:
            P.run(s_, o_)

    plain()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        plain()
    e1.record(st)
    torch.cuda.synchronize()
    plain_s = e0.elapsed_time(e1) / 1000 / reps
    seq, off = torch.from_numpy(rd.seq).to(dev), torch.from_numpy(rd.off.view(np.int64)).to(dev)
    best, tune_ms, grid = mb.autotune(G, seq, off, points=True)
    n_smem = sum(b[4] for b in buckets)
    n_hits = sum(b[5] for b in buckets)
    BP = mb.Plan(G, rd.n, len(rd.seq), n_smem + 64, n_hits + 64, opts=best)
    BP.capture(seq, off)
    BP.replay()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        BP.replay()
    e1.record(st)
    torch.cuda.synchronize()
    batched_s = e0.elapsed_time(e1) / 1000 / reps
    bsm, bhits = BP.result()
    BP.free()
    # the fastest shape with the device work queue (reads handed out in read order), as its own
    # replayed graph: reported beside the autotuner's choice, output compared
    qo, _ = min(((o, t) for o, t in grid if o.flags & mb.MB_BATCHED), key=lambda p: p[1])
    QP = mb.Plan(G, rd.n, len(rd.seq), n_smem + 64, n_hits + 64, opts=qo)
    QP.capture(seq, off)
    QP.replay()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(reps):
        QP.replay()
    e1.record(st)
    torch.cuda.synchronize()
    queue_s = e0.elapsed_time(e1) / 1000 / reps
    qsm, qhits = QP.result()
    QP.free()
    queue_same = qsm.tobytes() == bsm.tobytes() and np.array_equal(qhits, bhits)
    if not queue_same:
        raise SystemExit("bench: the work-queue form disagrees with the autotuned form")
    # identity with the per-bucket launches, put back in read order
    rec, hl = [], []
    for ids, s_, o_, P, m, nh in buckets:
        x, h = P.result()
        for r in x:
            c = 0 if r["flags"] & 1 else int(r["s"])
            rec.append((int(ids[r["read"]]), int(r["qbeg"]), int(r["qend"]), int(r["k"]), int(r["kr"]), int(r["s"])))
            hl.append(h[int(r["hit_off"]):int(r["hit_off"]) + c])
        P.free()
    order = sorted(range(len(rec)), key=lambda i: (rec[i][0], rec[i][1]))
    same = [rec[i] for i in order] == [tuple(int(v) for v in (r["read"], r["qbeg"], r["qend"], r["k"], r["kr"],
                                                                 r["s"])) for r in bsm]
    same = same and np.array_equal(np.concatenate([hl[i] for i in order]), bhits)
    if not same:
        raise SystemExit("bench: batched form disagrees with the per-bucket launches")
    return {"workload": "100 Mbp repeat-rich reference, 200,000 SE reads log-uniform 100 bp-10 kb",
            "reads": rd.n, "bases": int(len(rd.seq)), "smems": n_smem, "hits": n_hits,
            "plain_per_bucket": "one preallocated plan per length bucket (default shape), run in turn",
            "plain_per_bucket_reads_per_s": rd.n / plain_s, "batched_graph_reads_per_s": rd.n / batched_s,
            "plain_per_bucket_bases_per_s": len(rd.seq) / plain_s, "batched_graph_bases_per_s": len(rd.seq) / batched_s,
            "speedup": plain_s / batched_s, "identical_output": bool(same),
            "autotuned": mb.shape_of(best), "autotuned_ms": tune_ms,
            "autotune_grid": [dict(mb.shape_of(o), ms=round(ms, 3)) for o, ms in grid],
            "plain_ms": plain_s * 1000, "batched_ms": batched_s * 1000,
            "work_queue_best": dict(mb.shape_of(qo), graph_reads_per_s=rd.n / queue_s, ms=queue_s * 1000,
                                    identical_output=bool(queue_same))}


def serve_requests(ref, n, seed):
    """Request stream: 80% short (log-uniform 1-4,096 pairs of 2x150), 20% long (log-uniform
    1-4,096 single reads of log-uniform 1-10 kb)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n):
        k = int(np.exp(rng.uniform(0, np.log(4096))))
        if rng.random() < 0.8:
            rd = synth.reads(ref, 2 * k, seed * 7919 + q, mode=1, read_len=150, sub_lo=0.001, sub_hi=0.01,
                             indel=0.0001)
        else:
            rd = synth.reads(ref, k, seed * 7919 + q, mode=2, len_lo=1000, len_hi=10000, sub_lo=0.001,
                             indel=0.0002)
        reqs.append(rd)
    return reqs


# Integer lanes of the GB300 (152 SMs x 4 sub-partitions x 32 lanes) at the 2,070 MHz SM clock: the
# roofline of the mate-rescue prefilter, which counts one compare and one add per q-mer pair.
INT_LANE_OPS_PER_S = 152 * 128 * 2.07e9

# the headline metric: reads seeded and located per second (2x150 bp reads, 1 Gbp index); the line
# also carries the plain-launch form and the served form's p50/p99 latency
METRIC = "reads/s seeded+located (2x150bp, 1 Gbp index) vs plain launch; served p50/p99 ms"


def bench_rescue(mb, torch, dev, ref, n_pairs: int, reps: int = 5):
    """Mate-rescue prefilter (Section 2.7): max_t M_t of 7-mer matches for n_pairs (150 bp read,
    600 bp window) pairs drawn from the reference, device buffers, kernel timed by CUDA events."""
    r, ro, w, wo = synth.rescue_pairs(ref, n_pairs, 0x6D620006)
    dr, dro = torch.from_numpy(r).to(dev), torch.from_numpy(ro.view(np.int64)).to(dev)
    dw, dwo = torch.from_numpy(w).to(dev), torch.from_numpy(wo.view(np.int64)).to(dev)
    best = torch.empty(n_pairs, dtype=torch.int32, device=dev)
    mb.mb_rescue_prefilter(dr, dro, dw, dwo, best=best)   # warm-up
    mb.profile_reset()
    mb.profile_enable(True)
    torch.cuda.synchronize()
    t = time.time()
    for _ in range(reps):
        mb.mb_rescue_prefilter(dr, dro, dw, dwo, best=best)
    torch.cuda.synchronize()
    call_s = (time.time() - t) / reps
    mb.profile_enable(False)
    kms, kn = mb.profile_get("rescue")
    kms /= max(kn, 1)
    q = 7
    compares = float(np.sum((np.diff(ro.astype(np.int64)) - q + 1).clip(0) *
                            (np.diff(wo.astype(np.int64)) - q + 1).clip(0)))
    got = best.cpu().numpy().view(np.uint32)
    achieved = 2 * compares / (kms / 1000.0)
    return {"workload": f"{n_pairs:,} pairs of a 150 bp read and a 600 bp window of the 1 Gbp reference, "
                        "half of them true (read inside the window, 1% substitutions)",
            "q": q, "pairs_per_s": n_pairs / (kms / 1000.0), "call_pairs_per_s": n_pairs / call_s,
            "kernel_ms": kms, "pass_frac": float((got >= 10).mean()),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": INT_LANE_OPS_PER_S / 1e12,
                         "unit": "T int ops/s", "frac": achieved / INT_LANE_OPS_PER_S,
                         "ops": "2 per q-mer pair compared (compare, add)", "compares_per_launch": compares}}


def bench_served(mb, G, ref, n_requests: int, pool: int = 2000, load: float = 0.7,
                 sweep=(0.3, 0.5, 0.9, 0.95), window: int = 4096, seq_prefix: int = 2000,
                 budget_gib: float = 8, opts=None, clients: int = 8):
    """Served form on the resident index: capacity (the whole stream submitted with at most
    `window` requests outstanding), then Poisson arrivals at `load` x capacity; latency per request
    from submit to results on the host.  The stream's requests are drawn (seeded) from `pool`
    generated requests, so host memory stays bounded; every request is copied at submit and
    seeded in full.  The first `seq_prefix` arrivals are also served by sequential plain launches
    (one request at a time through one preallocated plan: copy in, run, copy the results out; no
    allocation per request) for comparison, and the served form's latencies at the other offered
    loads of `sweep` are reported.  Requests are submitted by `clients` threads (a server takes
    submissions from many callers at once; one Python thread alone cannot stage the bases fast
    enough), each with an equal share of the stream and of the window."""
    import collections
    import threading as th
    import torch
    base = serve_requests(ref, min(pool, n_requests), 4242)
    pick = (np.arange(n_requests) if n_requests <= len(base) else
            np.random.default_rng(4243).integers(0, len(base), n_requests))
    reqs = [base[i] for i in pick]
    total_reads = sum(r.n for r in reqs)
    total_bases = sum(int(r.off[-1] - r.off[0]) for r in reqs)
    srv = mb.Server(G, hbm_budget=int(budget_gib * (1 << 30)), opts=opts)

    def submit(r, before=None):
        """Submit; when the staging ring is full (MB_ERR_BUSY), make room first."""
        while True:
            try:
                return srv.submit(r.seq, r.off)
            except mb.MbError as e:
                if e.code != -9:
                    raise
                if before:
                    before()
                else:
                    time.sleep(0.0005)

    counts = {}

    def client(ids, win):
        """One client thread: submits its requests in order with at most `win` outstanding,
        collecting the oldest when the window or the staging ring is full."""
        out = collections.deque()

        def collect_one():
            q, tk = out.popleft()
            sm, hits, _ = srv.wait(tk)
            counts[int(pick[q])] = (len(sm), len(hits))

        for q in ids:
            if len(out) >= win:
                collect_one()
            out.append((q, submit(reqs[q], collect_one if out else None)))
        while out:
            collect_one()

    t = time.time()
    cl = [th.Thread(target=client, args=(range(c, n_requests, clients), max(1, window // clients)))
          for c in range(clients)]
    for c in cl:
        c.start()
    for c in cl:
        c.join()
    cap_s = time.time() - t
    cap_rps = n_requests / cap_s
    cap_counters = srv.counters()
    pct = lambda a, p: float(np.percentile(np.asarray(a), p))

    def poisson(rate, seed):
        """Submit the requests at Poisson arrival times; (latencies in ms, wall seconds)."""
        arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, n_requests))
        lat = [0.0] * n_requests
        tk = [0] * n_requests

        def collect():
            for i in range(n_requests):
                while tk[i] == 0:
                    time.sleep(0.0002)
                _, _, lat[i] = srv.wait(tk[i])

        def submitter(ids):
            for i in ids:
                d = t0 + arrivals[i] - time.time()
                if d > 0:
                    time.sleep(d)
                tk[i] = submit(reqs[i])

        col = th.Thread(target=collect)
        col.start()
        t0 = time.time()
        subs = [th.Thread(target=submitter, args=(range(c, n_requests, clients),)) for c in range(clients)]
        for x in subs:
            x.start()
        for x in subs:
            x.join()
        col.join()
        return lat, time.time() - t0, arrivals

    rate = load * cap_rps
    lat, wall, arrivals = poisson(rate, 17)
    points = []
    for k, ld in enumerate(sweep):
        sl, sw, _ = poisson(ld * cap_rps, 18 + k)
        points.append({"offered_load": ld, "arrival_rate_per_s": ld * cap_rps, "served_reads_per_s": total_reads / sw,
                       "p50_ms": pct(sl, 50), "p95_ms": pct(sl, 95), "p99_ms": pct(sl, 99)})
    stats = srv.counters()
    srv.close()
    # sequential plain launches on the same arrival times (the first seq_prefix arrivals): one plan
    # sized for the largest request, inputs copied in and results copied out per request
    ns = min(seq_prefix, n_requests)
    sub = reqs[:ns]
    mr = max(r.n for r in sub)
    mbases = max(int(r.off[-1] - r.off[0]) for r in sub)
    msm = max(counts[int(pick[q])][0] for q in range(ns))
    mh = max(counts[int(pick[q])][1] for q in range(ns))
    P = mb.Plan(G, mr, mbases, msm + 64, mh + 64, opts=dict(flags=mb.MB_BATCHED))
    dseq = torch.empty(mbases + 16, dtype=torch.uint8, device="cuda")
    doff = torch.empty(mr + 1, dtype=torch.int64, device="cuda")
    seq_lat = []
    t0 = time.time()
    for i, r in enumerate(sub):
        d = t0 + arrivals[i] - time.time()
        if d > 0:
            time.sleep(d)
        nb = int(r.off[-1] - r.off[0])
        dseq[:nb].copy_(torch.from_numpy(r.seq[int(r.off[0]):int(r.off[-1])]))
        doff[:r.n + 1].copy_(torch.from_numpy((r.off - r.off[0]).view(np.int64)))
        P.run(dseq[:nb], doff[:r.n + 1])
        P.result()
        seq_lat.append((time.time() - t0 - arrivals[i]) * 1000)
    seq_wall = time.time() - t0
    P.free()
    return {"requests": n_requests, "reads": total_reads, "bases": total_bases, "distinct_requests": len(base),
            "stream": f"{n_requests} requests drawn (seeded) from {len(base)} generated ones",
            "mix": "80% short (1-4,096 pairs of 2x150), 20% long (1-4,096 reads of 1-10 kb), log-uniform sizes",
            "capacity_requests_per_s": cap_rps, "capacity_reads_per_s": total_reads / cap_s,
            "capacity_bases_per_s": total_bases / cap_s, "capacity_window": window, "clients": clients,
            "offered_load": load, "arrival_rate_per_s": rate,
            "served_reads_per_s": total_reads / wall, "served_bases_per_s": total_bases / wall,
            "served_p50_ms": pct(lat, 50), "served_p95_ms": pct(lat, 95), "served_p99_ms": pct(lat, 99),
            "sequential_plain_requests": ns,
            "sequential_plain": "one preallocated plan, one request at a time (copy in, run, copy out)",
            "sequential_plain_reads_per_s": sum(r.n for r in sub) / seq_wall,
            "sequential_plain_bases_per_s": sum(int(r.off[-1] - r.off[0]) for r in sub) / seq_wall,
            "sequential_plain_p50_ms": pct(seq_lat, 50), "sequential_plain_p95_ms": pct(seq_lat, 95),
            "sequential_plain_p99_ms": pct(seq_lat, 99),
            "load_sweep": points,
            "server_counters_after_capacity_run": cap_counters, "server_counters": stats}


def bench_bisulfite(mb, torch, dev, ref, opts, reps: int = 3):
    """Directional bisulfite set of the 1 Gbp workload (Section 2.9): the 3-base index over
    CT(R).GA(R) (n = 4|R| + 1), 1M pairs of converted reads seeded (read 1 C->T, read 2 G->A),
    located, filtered by strand and split at T-to-C mismatches; device buffers, each step timed
    with CUDA events on the stream (the split's host copy of its pieces included)."""
    rd = synth.bisulfite_reads(ref)
    o = dict(opts, flags=(opts.get("flags", 0) | mb.MB_BS3))
    torch.cuda.synchronize()
    t = time.time()
    G = mb.mb_index_build(torch.from_numpy(ref).to(dev), opts=o)
    torch.cuda.synchronize()
    build_s = time.time() - t
    G.drop_sa()
    seq, off, mate = (torch.from_numpy(rd.seq).to(dev), torch.from_numpy(rd.off.view(np.int64)).to(dev),
                      torch.from_numpy(rd.mate).to(dev))
    ref_d = torch.from_numpy(ref).to(dev)
    cap = 8 * rd.n
    out = torch.empty(cap * 48, dtype=torch.uint8, device=dev)
    _, m, nh = mb.mb_seed_batch(G, seq, off, mate=mate, opts=o, out=out, cap=cap)
    hits = torch.empty(max(nh, 1), dtype=torch.int32, device=dev)
    keep = torch.empty(max(nh, 1), dtype=torch.uint8, device=dev)
    # locate form for this batch: plain walks (16 per lane) or walks that join (2 per lane), the
    # faster of the two on one timed call each (the join's per-call setup scales with the index)
    forms = {"plain": dict(o, flags=o["flags"] & ~mb.MB_LOCATE_JOIN, prefetch_depth=16),
             "join": dict(o, flags=o["flags"] | mb.MB_LOCATE_JOIN, prefetch_depth=2)}
    st = torch.cuda.current_stream()
    form_ms = {}
    for name, fo in forms.items():
        mb.mb_locate(G, out, m, opts=fo, hits=hits, cap=nh)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        mb.mb_locate(G, out, m, opts=fo, hits=hits, cap=nh)
        e1.record(st)
        torch.cuda.synchronize()
        form_ms[name] = e0.elapsed_time(e1)
    loc_form = min(form_ms, key=form_ms.get)
    lo = forms[loc_form]
    mb.mb_bs_filter(G, out, m, mate, hits, nh, keep=keep)
    import ctypes
    oo = mb.Opts(**o)

    def split_into(buf):
        """mb_bs_split into a device buffer of pieces (24 B each); returns the count."""
        n = ctypes.c_uint64()
        cap_p = buf.numel() // 24
        rc = mb.lib().mb_bs_split(G.handle, mb._ptr(ref_d), mb._ptr(seq), mb._ptr(off), rd.n, mb._ptr(mate),
                                  mb._ptr(out), m, mb._ptr(hits), mb._ptr(keep), nh, ctypes.byref(oo), None,
                                  mb._ptr(buf), cap_p, ctypes.byref(n))
        if rc not in (0, mb.MB_ERR_CAPACITY):
            raise mb.MbError(rc, "mb_bs_split")
        return n.value

    need = split_into(torch.empty(24, dtype=torch.uint8, device=dev))
    pieces = torch.empty(max(need, 1) * 24, dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    times = {"seed": [], "locate": [], "filter": [], "split": []}
    npieces = 0
    for it in range(reps + 1):
        ev[0].record(st)
        mb.mb_seed_batch(G, seq, off, mate=mate, opts=o, out=out, cap=cap)
        ev[1].record(st)
        mb.mb_locate(G, out, m, opts=lo, hits=hits, cap=nh)
        ev[2].record(st)
        mb.mb_bs_filter(G, out, m, mate, hits, nh, keep=keep)
        ev[3].record(st)
        npieces = split_into(pieces)
        ev[4].record(st)
        torch.cuda.synchronize()
        if it:
            for k, (a, b) in zip(times, zip(ev[:-1], ev[1:])):
                times[k].append(a.elapsed_time(b))
    ms = {k: float(np.min(v)) for k, v in times.items()}
    total = sum(ms.values())
    res = {"workload": "directional bisulfite set: 1M pairs 2x150 (read 1 C->T, read 2 G->A; 98% non-CpG, "
                       "30% CpG conversion) on the 3-base index of the 1 Gbp reference",
           "n": int(G.n), "index_build_s": build_s, "reads": rd.n, "smems": m, "hits": nh,
           "kept_hits": int(keep[:nh].sum().item()), "pieces": npieces, "ms": ms,
           "locate_form": loc_form, "locate_form_ms": form_ms,
           "seed_locate_reads_per_s": rd.n / ((ms["seed"] + ms["locate"]) / 1000.0),
           "whole_bs_path_reads_per_s": rd.n / (total / 1000.0)}
    del out, hits, keep, seq, off, mate, ref_d, pieces
    G.free()
    torch.cuda.empty_cache()
    return res


# --------------------------------------------------------------------------------- GPU side
def run_gpu(args):
    import torch
    import paper_2606_15357_gb300 as mb
    ws, rank, local = dist_env()
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    l2_default = mb.set_l2_fetch_granularity(0)
    l2_fetch = mb.set_l2_fetch_granularity(args.l2_fetch) if args.l2_fetch else l2_default
    log(f"L2 fetch granularity: default {l2_default} B, in use {l2_fetch} B")

    ref, rd, params = make_inputs(args.workload, args.scale, rank, args.reads)
    opts = dict(min_len=params["min_len"], min_occ=params["min_occ"], max_occ=params["max_occ"],
                sa_rate=params["sa_rate"], kmer_k=args.kmer_k)
    torch.cuda.synchronize()
    t = time.time()
    idx = mb.mb_index_build(torch.from_numpy(ref).to(dev), opts=opts, n_seed=0)
    torch.cuda.synchronize()
    build_s = time.time() - t
    # the BWT and the sampled SA for the CPU comparator (needs the full SA, dropped next)
    cpu_index_src = None
    if rank == 0 and not args.no_cpu_baseline:
        e = idx.export(bwt=True, ssa=True)
        cpu_index_src = (e["bwt"], idx.primary, e["ssa"])
    idx.drop_sa()
    log(f"index: n={idx.n} built in {build_s:.1f}s")

    seq = torch.from_numpy(rd.seq).to(dev)
    off = torch.from_numpy(rd.off.view(np.int64)).to(dev)
    n_reads = rd.n

    # first call sizes the outputs
    cap = 4 * n_reads
    out = torch.empty(cap * 48, dtype=torch.uint8, device=dev)
    try:
        _, m, nh = mb.mb_seed_batch(idx, seq, off, opts=opts, out=out, cap=cap)
    except mb.MbError as e:
        if e.code != mb.MB_ERR_CAPACITY:
            raise
        raise
    hits = torch.empty(max(nh, 1), dtype=torch.int32, device=dev)

    def step():
        _, m_, nh_ = mb.mb_seed_batch(idx, seq, off, opts=opts, out=out, cap=cap)
        mb.mb_locate(idx, out, m_, opts=opts, hits=hits, cap=nh_)
        return m_, nh_

    # launch shape: fixed (--block / --locate-walks, the autotuner's choice on this workload), or
    # autotuned on a sample of the batch with --autotune; used for both forms
    ns = min(n_reads, 1_000_000)
    if args.autotune:
        best, tune_ms = mb.autotune(idx, seq[:int(rd.off[ns])], off[:ns + 1], opts=opts)
        log(f"autotuned on {ns} reads: {mb.shape_of(best)}")
    else:
        best = mb.Opts(block_size=args.block, prefetch_depth=args.locate_walks,
                       flags=(mb.MB_BATCHED if args.queue else 0) | (mb.MB_SMEM_ONE_LOOP if args.one_loop else 0) |
                       (mb.MB_LOCATE_JOIN if args.locate_join else 0),
                       smem_burst=args.smem_burst, smem_wait=args.smem_wait, smem_warps=args.smem_warps)
    opts["block_size"] = best.block_size
    opts["prefetch_depth"] = best.prefetch_depth
    opts["flags"] = best.flags
    opts["smem_burst"] = best.smem_burst
    opts["smem_wait"] = best.smem_wait
    opts["smem_warps"] = best.smem_warps

    if args.locate_sweep:
        return locate_sweep(mb, torch, idx, out, m, hits, nh, opts)

    # work counters of the chosen form (untimed pass with counting kernels)
    mb.profile_reset()
    copts = dict(opts, flags=mb.MB_COUNT | (best.flags & mb.MB_LOCATE_JOIN))
    _, m, nh = mb.mb_seed_batch(idx, seq, off, opts=copts, out=out, cap=cap)
    mb.mb_locate(idx, out, m, opts=copts, hits=hits, cap=nh)
    wc = mb.work_counters()
    log(f"work: {m} SMEMs, {nh} hits, {wc}")

    for _ in range(args.warmup):
        step()
    mb.profile_reset()
    mb.profile_enable(True)
    l0 = mb.launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    mb.profile_enable(False)
    plain_ms = e0.elapsed_time(e1)
    plain_launches = mb.launch_count() - l0

    # the same stage as one captured CUDA graph of an autotuned plan (no host sync inside a step)
    popts = dict(opts, flags=best.flags)
    P = mb.Plan(idx, n_reads, len(rd.seq), m + 1024, nh + 1024, opts=popts)
    P.capture(seq, off)
    for _ in range(args.warmup):
        P.replay()
    _, gm, _, gnh = P.result_ptrs()
    assert (gm, gnh) == (m, nh), "graph form disagrees with the plain launches"
    psm, phits = P.result()
    same = psm.tobytes() == out[:m * 48].cpu().numpy().tobytes() and \
        np.array_equal(phits, hits[:nh].cpu().numpy().view(np.uint32))
    l1 = mb.launch_count()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            P.replay()
        e1.record(st)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    graph_ms = e0.elapsed_time(e1)
    graph_launches = mb.launch_count() - l1
    del psm, phits
    P.free()
    use_graph = same and graph_ms < plain_ms
    ms = graph_ms if use_graph else plain_ms
    launches = graph_launches if use_graph else plain_launches
    ms = max_over_ranks(ms, pg)
    value = whole_job_rate(ws, args.steps, n_reads, ms)
    smem_ms, smem_n = mb.profile_get("smem")
    loc_ms, loc_n = mb.profile_get("locate")
    log(f"timed: plain {plain_ms / args.steps:.1f} ms/step, graph {graph_ms / args.steps:.1f} ms/step "
        f"(identical: {same}); smem {smem_ms / max(smem_n, 1):.1f} ms, locate {loc_ms / max(loc_n, 1):.1f} ms per launch")
    n_bases = int(len(rd.seq))
    forms = {"plain_launch": {"reads_per_s": ws * args.steps * n_reads / (plain_ms / 1000.0),
                              "bases_per_s": ws * args.steps * n_bases / (plain_ms / 1000.0),
                              "ms_per_step": plain_ms / args.steps, "gpu_launches": plain_launches},
             "graph_plan": {"reads_per_s": ws * args.steps * n_reads / (graph_ms / 1000.0),
                            "bases_per_s": ws * args.steps * n_bases / (graph_ms / 1000.0),
                            "ms_per_step": graph_ms / args.steps, "identical_output": bool(same),
                            "gpu_launches": graph_launches, "shape": mb.shape_of(best)},
             "reported": "graph_plan" if use_graph else "plain_launch"}

    # the same graph with locate walks that stop at the index's rate-4 SA samples (MB_LOCATE_AUX):
    # reported beside the headline, which locates through the rate-32 samples of Section 2.4
    if not args.no_aux_form:
        aopts = dict(opts, flags=(best.flags & ~mb.MB_LOCATE_JOIN) | mb.MB_LOCATE_AUX, prefetch_depth=16)
        AP = mb.Plan(idx, n_reads, len(rd.seq), m + 1024, nh + 1024, opts=aopts)
        AP.capture(seq, off)
        for _ in range(args.warmup):
            AP.replay()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            AP.replay()
        e1.record(st)
        torch.cuda.synchronize()
        aux_ms = e0.elapsed_time(e1)
        asm_, ah = AP.result()
        aux_same = asm_.tobytes() == out[:m * 48].cpu().numpy().tobytes() and \
            np.array_equal(ah, hits[:nh].cpu().numpy().view(np.uint32))
        AP.free()
        del asm_, ah
        if not aux_same:
            raise SystemExit("bench: the rate-4 locate form disagrees with the plain launches")
        forms["graph_plan_locate_aux"] = {
            "reads_per_s": ws * args.steps * n_reads / (aux_ms / 1000.0), "ms_per_step": aux_ms / args.steps,
            "identical_output": bool(aux_same), "shape": mb.shape_of(mb.Opts(**aopts)),
            "note": "locate walks stop at the rate-4 SA samples the index keeps for text extension "
                    "(MB_LOCATE_AUX); not the headline, which uses the rate-32 samples"}
        log(f"graph form with MB_LOCATE_AUX: {aux_ms / args.steps:.1f} ms/step (identical: {aux_same})")

    # roofline of the dominant kernel: algorithmic bytes / its event-timed duration
    peak, peak_kind = measured_peaks()
    smem_bytes = (BLOCK_BYTES * (wc["ext_blocks"] + wc["u_walk_steps"]) + 12 * wc["kmer_lookups"] +
                  4 * wc["u_samples"] + 8 * wc["u_text_loads"])
    # locate: 32 B per LF step (an occurrence block or a walk block), 4 B per sampled-S read, and
    # for walks that join 8 B per join (the rank word and the joined row's position)
    loc_bytes = BLOCK_BYTES * wc["lf_steps"] + 4 * wc["sa_reads"] + 8 * wc["joins"]
    if loc_ms / max(loc_n, 1) >= smem_ms / max(smem_n, 1):
        kname, kbytes, kms = "locate", loc_bytes, loc_ms / max(loc_n, 1)
    else:
        kname, kbytes, kms = "smem", smem_bytes, smem_ms / max(smem_n, 1)
    achieved = kbytes / (kms / 1000.0) / 1e9
    wl_tag = {3: "1gbp", 2: "100mbp", 1: "1mbp"}[args.workload]
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                "traffic": ncu_traffic(kname, wl_tag),
                "algorithmic_bytes_per_launch": kbytes,
                "kernels": {"smem": {"ms_per_launch": smem_ms / max(smem_n, 1), "bytes": smem_bytes,
                                     "GBps": smem_bytes / max(smem_ms / max(smem_n, 1), 1e-9) / 1e6},
                            "locate": {"ms_per_launch": loc_ms / max(loc_n, 1), "bytes": loc_bytes,
                                       "GBps": loc_bytes / max(loc_ms / max(loc_n, 1), 1e-9) / 1e6}}}

    # second denominator: the rate at which this GPU serves random 32-byte reads from a buffer far
    # above L2 (probe kernel, same process). Every block access of both kernels is such a read, so
    # this, not the copy bandwidth, is the ceiling a DRAM-bound gather can reach.
    if roofline["traffic"]:
        roofline["dram_GBps"] = roofline["traffic"] / (kms / 1000.0) / 1e9
    # per kernel: DRAM bytes of the committed capture, their rate, random 32-byte sectors per
    # second (every block access is one such sector) and the capture's cache hit rates
    for kn, kd in roofline["kernels"].items():
        t = ncu_traffic(kn, wl_tag)
        if t:
            sec = kd["ms_per_launch"] / 1000.0
            kd["dram_bytes"] = t
            kd["dram_GBps"] = t / sec / 1e9
            kd["dram_sectors_per_s"] = t / 32 / sec
        hr = ncu_hit_rates(kn, wl_tag)
        if hr:
            kd["l2_hit_pct"], kd["l1_hit_pct"] = hr
    if not args.no_probe:
        gc = gather_ceiling(args.probe_gib)
        roofline["gather_ceiling"] = gc
        g = gc.get("random32_indep_GBps", 0)
        if g and g > 0:
            roofline["random_read_ceiling_GBps"] = g
            roofline["frac_of_random_read_ceiling"] = roofline.get("dram_GBps", achieved) / g
            roofline["frac_of_random_read_ceiling_basis"] = "dram_GBps" if "dram_GBps" in roofline else "achieved"
        log(f"gather ceiling: {gc}")

    # end to end through the public API with pinned host buffers: the pipelined one-call form
    # (chunks alternate between two streams, copies overlap kernels), and the two calls
    # mb_seed_batch + mb_locate for comparison
    e2e = None
    if not args.no_e2e:
        seq_h = torch.from_numpy(rd.seq).pin_memory()
        off_h = torch.from_numpy(rd.off.view(np.int64)).pin_memory()
        out_h = torch.empty(m * 48, dtype=torch.uint8).pin_memory()
        hits_h = torch.empty(max(nh, 1), dtype=torch.int32).pin_memory()
        k2 = max(1, args.steps)
        eopts = dict(opts, flags=best.flags)   # the same launch shape as the graph form
        mb.seed_locate(idx, seq_h, off_h, opts=eopts, out=out_h, cap=m, hits=hits_h, hits_cap=nh)   # warm-up
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.time()
        for _ in range(k2):
            m2, nh2 = mb.seed_locate(idx, seq_h, off_h, opts=eopts, out=out_h, cap=m, hits=hits_h, hits_cap=nh)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.time() - t0, pg)
        t0 = time.time()
        for _ in range(k2):
            _, m3, nh3 = mb.mb_seed_batch(idx, seq_h, off_h, opts=opts, out=out_h, cap=m)
            mb.mb_locate(idx, out_h, m3, opts=opts, hits=hits_h, cap=nh3)
        torch.cuda.synchronize()
        dt2 = max_over_ranks(time.time() - t0, pg)
        # the end-to-end call must return exactly what the device-timed forms return (the plain
        # launches above, which equal the graph form when `same` holds)
        m2, nh2 = mb.seed_locate(idx, seq_h, off_h, opts=eopts, out=out_h, cap=m, hits=hits_h, hits_cap=nh)
        e2e_same = (m2, nh2) == (m, nh) and out_h.numpy().tobytes() == out[:m * 48].cpu().numpy().tobytes() and \
            np.array_equal(hits_h[:nh].numpy(), hits[:nh].cpu().numpy())
        if not (e2e_same and same):
            raise SystemExit(f"bench: forms disagree (graph == plain: {same}, mb_seed_locate == plain: {e2e_same})")
        e2e = {"value": ws * k2 * n_reads / dt, "unit": "reads/s",
               "h2d_bytes_per_step": int(seq_h.numel() + off_h.numel() * 8),
               "d2h_bytes_per_step": int(m * 48 + nh * 4),
               "call": "mb_seed_locate (pinned host buffers, 4M-read chunks seeded on two streams, the batch located at once)",
               "two_calls_reads_per_s": ws * k2 * n_reads / dt2,
               "note": "two_calls = mb_seed_batch + mb_locate on host buffers (the records are staged back in)",
               "identical_output": bool(e2e_same)}
        log(f"e2e: {e2e}")

    rescue = None
    if rank == 0 and not args.no_rescue:
        rescue = bench_rescue(mb, torch, dev, ref, args.rescue_pairs)
        log(f"rescue prefilter: {rescue}")

    served = None
    if rank == 0 and not args.no_serve:
        served = bench_served(mb, idx, ref, args.serve_requests, pool=args.serve_pool,
                              budget_gib=args.serve_budget_gib, clients=args.serve_clients,
                              opts=dict(min_len=opts["min_len"], min_occ=opts["min_occ"], max_occ=opts["max_occ"],
                                        prefetch_depth=args.serve_walks))
        log(f"served: {served}")
    del out, hits
    torch.cuda.empty_cache()
    batched = None
    if rank == 0 and not args.no_batched:
        batched = bench_batched(mb, torch, dev)
        log(f"batched: {batched}")

    bisulfite = None
    if rank == 0 and not args.no_bisulfite and args.workload == 3:
        bisulfite = bench_bisulfite(mb, torch, dev, ref, dict(opts, flags=best.flags))
        log(f"bisulfite: {bisulfite}")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        X, obuild_s, sample = oracle_rate(ref, rd, params, args.cpu_s, threads)
        t = time.time()
        X.seed(sample.seq, sample.off, params["min_len"], params["min_occ"], params["max_occ"], threads=threads)
        dt = time.time() - t
        # one core, on a smaller sample of the same draw (about a tenth of the time budget)
        n1 = max(64, min(sample.n, int(sample.n / dt * args.cpu_s / 10 / threads)))
        one = sample.subset(np.arange(n1))
        t = time.time()
        X.seed(one.seq, one.off, params["min_len"], params["min_occ"], params["max_occ"], threads=1)
        dt1 = time.time() - t
        cpu = {"value": sample.n / dt, "unit": "reads/s", "cores": threads, "kind": "oracle",
               "sample": f"{sample.n} reads drawn from the {rd.n}-read batch; oracle index build "
                         f"({obuild_s:.0f}s) untimed", "seconds": dt,
               "single_core": {"value": one.n / dt1, "unit": "reads/s", "cores": 1,
                               "sample": f"the first {one.n} reads of that sample", "seconds": dt1}}
        # the survey's definition of the SMEM kernel's algorithmic bytes, from the oracle's own count
        # of Algorithm 3 with the 10-mer cache (Section 2.5) on this sample: 64 B per distinct
        # 128-row block an extension step reads, 12 B per cache lookup; scaled per read to the step
        t = time.time()
        st_, bl_, lk_ = X.count_alg3(sample.seq, sample.off, params["min_len"], params["min_occ"], block_rows=128,
                                     kmer_k=10)
        per_read = (64 * bl_ + 12 * lk_) / sample.n
        survey_bytes = per_read * n_reads
        sm_ms = roofline["kernels"]["smem"]["ms_per_launch"]
        ach = survey_bytes / (sm_ms / 1000.0) / 1e9
        roofline["survey_definition"] = {
            "kernel": "smem", "definition": "64 B x distinct 128-row blocks per Algorithm 3 extension step with the "
                                            "10-mer cache + 12 B per cache lookup (oracle's count on the CPU sample, "
                                            "scaled per read)",
            "bytes_per_read": per_read, "steps_per_read": st_ / sample.n, "lookups_per_read": lk_ / sample.n,
            "bytes_per_launch": survey_bytes, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "sample_reads": sample.n, "count_s": time.time() - t}
        log(f"survey-definition roofline: {roofline['survey_definition']}")
        del X
        cpu["batched_prefetch"] = cpu_batched_rate(cpu_index_src, sample, params, threads)
        cpu_index_src = None
        log(f"cpu baseline: {cpu}")

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "reads/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "scale": args.scale, "reads_per_step": n_reads,
                   "pairs_per_step": n_reads // 2, "min_len": params["min_len"], "max_occ": params["max_occ"],
                   "sa_rate": params["sa_rate"], "kmer_k": args.kmer_k, "parallelism": f"replicas{ws}",
                   "l2": "inputs larger than L2 (reads 3 GB; index blocks 1 GB, 14-mer table 3.2 GB)",
                   "occ_block_bytes": BLOCK_BYTES, "l2_fetch_granularity": l2_fetch,
                   "smem_per_step": m, "hits_per_step": nh, "index_build_s": build_s},
        "smems_per_s": ws * args.steps * m / (ms / 1000.0),
        "hits_per_s": ws * args.steps * nh / (ms / 1000.0),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "forms": forms,
        "batched": batched,
        "rescue_prefilter": rescue,
        "served": served,
        "bisulfite": bisulfite,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", type=int, default=3, choices=[1, 2, 3])
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-s", type=float, default=15.0, help="target seconds of oracle work")
    ap.add_argument("--ref-step-s", type=float, default=8.0, help="reference arm: seconds per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the random-read ceiling probe")
    ap.add_argument("--l2-fetch", type=int, default=32,
                    help="L2 fetch granularity for this process (32/64/128; 0 = leave the default)")
    ap.add_argument("--no-batched", action="store_true", help="skip the mixed-length batched comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-form measurement")
    ap.add_argument("--no-rescue", action="store_true", help="skip the mate-rescue prefilter measurement")
    ap.add_argument("--no-aux-form", action="store_true", help="skip the graph form with MB_LOCATE_AUX")
    ap.add_argument("--locate-sweep", action="store_true",
                    help="only time the locate forms (plain, joined, rate-4) on one step's records, one JSON line each")
    ap.add_argument("--no-bisulfite", action="store_true", help="skip the bisulfite (3-base index) measurement")
    ap.add_argument("--rescue-pairs", type=int, default=1_000_000)
    ap.add_argument("--serve-requests", type=int, default=50_000,
                    help="requests in the served stream (Poisson arrivals)")
    ap.add_argument("--serve-budget-gib", type=float, default=8,
                    help="device memory budget of the served form's slots (GiB)")
    ap.add_argument("--serve-clients", type=int, default=8, help="client threads submitting to the served form")
    ap.add_argument("--serve-walks", type=int, default=16, choices=[1, 2, 4, 8, 16],
                    help="locate walks per lane in the served form's slots")
    ap.add_argument("--serve-pool", type=int, default=2000,
                    help="distinct generated requests the stream draws from")
    ap.add_argument("--probe-gib", type=float, default=1, help="buffer of the random-gather probe (GiB)")
    ap.add_argument("--probe-sweep", action="store_true",
                    help="only the random-read probe over buffer sizes 1/32 .. 8 GiB (one JSON line each)")
    ap.add_argument("--kmer-k", type=int, default=14, choices=range(1, 17),
                    help="k of the k-mer ds-interval table (Section 2.5 uses 10; same SMEMs for any k; "
                         "12 * 4^k bytes, 51.5 GB at 16)")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the launch shape on 1M reads instead of --block / --locate-walks")
    ap.add_argument("--no-autotune", action="store_true", help="(default) fixed launch shape")
    ap.add_argument("--block", type=int, default=512, choices=[128, 256, 512])
    ap.add_argument("--no-queue", dest="queue", action="store_false",
                    help="SMEM kernel walks fixed read ranges per warp instead of a device work queue")
    ap.add_argument("--locate-walks", type=int, default=2, choices=[1, 2, 4, 8, 16])
    ap.add_argument("--one-loop", action="store_true", help="SMEM kernel in its one-loop form")
    ap.add_argument("--locate-join", dest="locate_join", action="store_true", default=True,
                    help="(default) locate with walks that join (MB_LOCATE_JOIN)")
    ap.add_argument("--no-locate-join", dest="locate_join", action="store_false",
                    help="plain locate walks: every walk runs to its sampled row")
    ap.add_argument("--smem-burst", type=int, default=0, help="SMEM kernel block steps between service passes")
    ap.add_argument("--smem-wait", type=int, default=0, help="SMEM kernel lanes out of the loop that call a pass")
    ap.add_argument("--smem-warps", type=int, default=0,
                    help="SMEM kernel register budget: resident warps per SM aimed at (40: block 256 only; 48)")
    ap.add_argument("--reads", type=int, default=0,
                    help="seed only the first N reads of the batch (for ncu captures of the full index)")
    args = ap.parse_args()
    if args.probe_sweep:
        return probe_sweep()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
