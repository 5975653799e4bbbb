"""Benchmark: filtered block-sparse multiply C = A.A on synthetic water.

Default workload: 2048 water molecules (6144 atoms, dimension 47104, O 13x13 /
H 5x5 blocks, 6 A cutoff, entries N(0,1)*exp(-0.5 r), symmetric, +5 on the
diagonal), eps = 1e-10, FP64, one seed. It stands in for the paper's
H2O-DFT-LS matrices (Table 1), which are not available.

A "step" is one whole multiply (block norms, symbolic phase with the filter,
grouping of the products, numeric block products). Inputs stay resident in HBM.
For the default workload A (272 MB) and C (1.6 GB) are larger than the 129 MB
L2 and no flush is done; workloads whose A and C together fit in twice the L2
get 256 MB written between the timed steps.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered GFLOP/s per SpGEMM vs roofline; multiplies/s + p99 latency, rel err≤1e-12"
# FP64 FMA issue rate of one SM of the GB300 per clock (2 DFMA = 4 FLOP): the
# FP64 peak is derived as SMs x 4 FLOP x the SM clock sampled under load.
FP64_FLOP_PER_SM_CLK = 4
WORKLOADS = {
    "water2048": dict(kind="water", n=2048, seed=1, eps=1e-10),
    "water64": dict(kind="water", n=64, seed=0, eps=1e-10),
    "water32": dict(kind="water", n=32, seed=0, eps=1e-10),  # the smallest serving request
    "water512": dict(kind="water", n=512, seed=1, eps=1e-10),
    "amorphous4096": dict(kind="amorphous", n=4096, seed=2, eps=1e-8),
    "amorphous1024": dict(kind="amorphous", n=1024, seed=2, eps=1e-8),  # profiling size
    # Table 1 analogues scaled to one GPU: Dense (block 32, full) and S-E (block 6, 0.05%)
    "dense4096": dict(kind="dense", n=128, bs=32, seed=3, eps=1e-10),
    "se40000": dict(kind="sparse", n=40000, bs=6, occ=5e-4, seed=5, eps=1e-10),
    "se10000": dict(kind="sparse", n=10000, bs=6, occ=5e-4, seed=5, eps=1e-10),  # profiling size
}
L2_BYTES = 128 << 20  # GB300 L2 (129 MB), rounded down
PRECISIONS = {"fp64": 0, "bf16x3": 1, "tf32x2": 2}
SPLIT_KERNELS = {"panel": 0, "blocks": 1, "chunks": 2}  # BSM_SPLIT_*
SPLIT_KERNEL_SYMBOLS = {0: "k_numeric_split_panel", 1: "k_numeric_split_pipe", 2: "k_numeric_split_cat"}
# FP64 numeric kernels (BSM_FP64_*): name -> (number, kernel symbol)
FP64_KERNELS = {"t16b2": (0, "k_numeric_fp64_t16"), "t16b3": (1, "k_numeric_fp64_t16"),
                "t32": (2, "k_numeric_fp64_t32"), "pk12": (3, "k_numeric_fp64_pk"),
                "pk16": (4, "k_numeric_fp64_pk"), "g8": (5, "k_numeric_fp64_g8")}
FP64_BY_NUMBER = {v[0]: k for k, v in FP64_KERNELS.items()}
# DRAM bytes (read + write) per launch of a kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, profiles/): valid only while
# the code that decides it is unchanged -- the kernel's own source section and,
# for the FP64 kernels, the row-order work list (SHA-256 of each section) --
# for that variant (fp64 kernel name or split precision) and workload at its
# default eps.
MEASURED_TRAFFIC = {
    ("pk12", "water2048"): dict(
        sections=[("paper_1705_10218_gb300/csrc/k_numeric_fp64.cu",
                   ("// pk\n", "cudaError_t launch_numeric_fp64("),
                   "7bbcdcfe0e18d9a1b4f6759ea308f217cc9b13f32aaa2edbd5433183548b5194"),
                  ("paper_1705_10218_gb300/csrc/k_classes.cu",
                   ("// Work in a row order.", "}  // namespace bsm"),
                   "b173af39936271e55c6a2623c0b1222afaca8a97ab34ff8f9a0ec78e9ecdf01b"),
                  ("paper_1705_10218_gb300/csrc/bsm_api.cu",
                   ("static void bfs_row_order(", "static uint64_t next_order_id("),
                   "113dd9175f43cb3ea209f7d880be5023dd9fd7acdf547fa5077ea74319814288")],
        bytes=2.983e9 + 1.559e9),
}


def kernel_source_sha(source, section):
    """SHA-256 of the part of a source file between two markers (the kernel's
    own code), or None when the file or a marker is missing."""
    import hashlib

    try:
        with open(os.path.join(ROOT, source)) as f:
            text = f.read()
    except OSError:
        return None
    a = text.find(section[0])
    b = text.find(section[1], a + 1) if a >= 0 else -1
    if a < 0 or b < 0:
        return None
    return hashlib.sha256(text[a:b].encode()).hexdigest()


def measured_traffic(variant, workload):
    """DRAM bytes per launch from the ncu capture, or None when there is none
    for this variant and workload or the code behind it changed since."""
    m = MEASURED_TRAFFIC.get((variant, workload))
    if m is None or any(kernel_source_sha(src, sec) != sha for src, sec, sha in m["sections"]):
        return None
    return m["bytes"]


def measured_peak(key, fallback):
    """(value, source) from MEASURED_PEAKS.json, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), f"measured ({key}, MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def fp64_peak_gflops(n_sm, clocks):
    """FP64 FMA peak derived from the device: SMs x 2 DFMA (4 FLOP) per clock x
    the median SM clock sampled during the timed region (the maximum clock when
    no sample was taken). Returns (GFLOP/s, how it was derived)."""
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    src = "sampled median SM clock under load"
    if not mhz:
        mhz = measured_peak("sm_max_mhz", 2070.0)[0]
        src = "maximum SM clock (no clock samples)"
    peak = n_sm * FP64_FLOP_PER_SM_CLK * float(mhz) / 1e3
    return peak, (f"derived: {n_sm} SMs x {FP64_FLOP_PER_SM_CLK} FLOP/clk (2 DFMA) x {float(mhz):.0f} MHz "
                  f"({src})")


def make_workload(name):
    import synth

    w = WORKLOADS[name]
    if w["kind"] == "water":
        return synth.water(w["n"], seed=w["seed"]), w["eps"]
    if w["kind"] == "dense":
        return synth.dense_blocks(w["n"], w["bs"], seed=w["seed"]), w["eps"]
    if w["kind"] == "sparse":
        return synth.sparse_random(w["n"], w["bs"], w["occ"], seed=w["seed"]), w["eps"]
    return synth.amorphous(w["n"], seed=w["seed"]), w["eps"]


def replica_aggregate(local_ms, local_flop, dist=None, device="cpu"):
    """Replicas only: every rank runs its own multiplies on its own GPU (no
    data-path collective). The job time is the slowest rank's; the job's
    throughput is all ranks' FLOPs over that time (GFLOP/s)."""
    import torch

    t = torch.tensor([local_ms, local_flop], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized():
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        fsum = t[1:].clone()
        dist.all_reduce(fsum, op=dist.ReduceOp.SUM)
        ms, flop = float(tmax.item()), float(fsum.item())
    else:
        ms, flop = float(local_ms), float(local_flop)
    return ms, flop / (ms / 1e3) / 1e9


def norm_product_percentile(A, pct, sample=2_000_000, seed=0):
    """eps at a percentile of the candidate norm products nrm(A_ik) nrm(A_kj)
    (numpy Frobenius norms over a random sample of candidates): a threshold
    that makes the filter drop about pct percent of the products."""
    off = np.zeros(A.nblk + 1, np.int64)
    lens = A.row_sizes.astype(np.int64)[A.blk_row] * A.col_sizes.astype(np.int64)[A.blk_col]
    np.cumsum(lens, out=off[1:])
    sq = np.add.reduceat(A.values * A.values, off[:-1]) if A.nblk else np.zeros(0)
    nrm = np.sqrt(sq)
    rng = np.random.default_rng(seed)
    row_start = np.searchsorted(A.blk_row, np.arange(A.nbr + 1))
    a = rng.integers(0, A.nblk, sample)
    k = A.blk_col[a]
    cnt = row_start[k + 1] - row_start[k]
    ok = cnt > 0
    b = row_start[k[ok]] + (rng.random(int(ok.sum())) * cnt[ok]).astype(np.int64)
    return float(np.percentile(nrm[a[ok]] * nrm[b], pct))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for ln in open(self.path):
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(A, eps, budget_s=12.0, nthreads=None, ref_rows=None):
    """The CPU oracle (as it stands) on the first block rows of the workload,
    sized to about budget_s seconds. Returns (dict, rows, result)."""
    import oracle

    oracle.build()
    nthreads = nthreads or max(1, os.cpu_count() or 1)
    # probe: a small slice to estimate the rate
    probe_rows = max(1, min(A.nbr, 64))
    t0 = time.perf_counter()
    r = oracle.multiply(A, A, eps=eps, rows=(0, probe_rows), nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-3)
    rate_rows = probe_rows / dt
    nrows = ref_rows or int(min(A.nbr, max(probe_rows, rate_rows * budget_s)))
    t0 = time.perf_counter()
    r = oracle.multiply(A, A, eps=eps, rows=(0, nrows), nthreads=nthreads)
    dt = time.perf_counter() - t0
    gflops = r.flops / dt / 1e9
    info = {"value": round(gflops, 3), "unit": "GFLOP/s", "cores": nthreads, "kind": "oracle",
            "sample": f"C block rows 0..{nrows} of {A.nbr} ({r.flops / 1e9:.2f} GFLOP, {dt:.1f} s, "
                      f"OpenMP over block rows)", "cpu_model": cpu_model()}
    # one thread on a sample of about 3 s
    probe1 = max(1, min(A.nbr, 16))
    t0 = time.perf_counter()
    oracle.multiply(A, A, eps=eps, rows=(0, probe1), nthreads=1)
    rows1 = int(min(A.nbr, max(probe1, probe1 / max(time.perf_counter() - t0, 1e-3) * 3.0)))
    t0 = time.perf_counter()
    r1 = oracle.multiply(A, A, eps=eps, rows=(0, rows1), nthreads=1)
    dt1 = time.perf_counter() - t0
    info["single_thread"] = {"value": round(r1.flops / dt1 / 1e9, 3), "unit": "GFLOP/s",
                             "sample": f"C block rows 0..{rows1} ({r1.flops / 1e9:.2f} GFLOP, {dt1:.1f} s)"}
    return info, nrows, r


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    A, eps = make_workload(args.workload)
    import oracle

    oracle.build()
    nthreads = max(1, os.cpu_count() or 1)
    # size one step to about 2 s of oracle work
    probe = max(1, min(A.nbr, 32))
    t0 = time.perf_counter()
    oracle.multiply(A, A, eps=eps, rows=(0, probe), nthreads=nthreads)
    rate = probe / max(time.perf_counter() - t0, 1e-3)
    rows = int(min(A.nbr, max(probe, rate * 2.0)))
    for _ in range(args.warmup):
        oracle.multiply(A, A, eps=eps, rows=(0, rows), nthreads=nthreads)
    times, flops = [], 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.multiply(A, A, eps=eps, rows=(0, rows), nthreads=nthreads)
        times.append(time.perf_counter() - t0)
        flops = r.flops
    tot = sum(times)
    value = flops * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64", "sample_rows": rows},
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"C block rows 0..{rows} of {A.nbr} per step"},
        "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def timed_multiplies(ctx, dA, dC, eps, steps, warmup, stream, **kw):
    """Per-step device times (CUDA events on the launch stream) of steps
    multiplies C = A.A after warmup untimed ones, and the context's profile."""
    import torch

    for _ in range(warmup):
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stream=stream, **kw)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    ctx.profile(True)
    for k in range(steps):
        ev[k][0].record(stream)
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stream=stream, **kw)
        ev[k][1].record(stream)
    stream.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    return [a.elapsed_time(b) for a, b in ev], prof


def split_slice_bytes(A, precision):
    """Operand slice bytes of C = A.A (left and right layouts, rows padded
    along k to 16 bytes: 8 BF16 or 4 TF32 values)."""
    rs = A.row_sizes.astype(np.int64)
    r, c = rs[A.blk_row], A.col_sizes.astype(np.int64)[A.blk_col]

    def up(x, q):
        return (x + q - 1) // q * q
    if precision == "bf16x3":
        return 3 * 2 * int((r * up(c, 8) + c * up(r, 8)).sum())
    return 2 * 4 * int((r * up(c, 4) + c * up(r, 4)).sum())


def measure_variants(ctx, A, dA, dC, eps, flops, local, sample=None, steps=10, warmup=3):
    """The other configurations of the benchmark, measured in the same process
    after the headline: the split precisions on the same water system (both
    kernels; errors against the oracle on the CPU baseline's block rows), the
    mixed-size amorphous system in the launch modes, and a reduced serving
    replay. Each with its own clock samples."""
    import torch

    import synth

    s = torch.cuda.Stream()
    out = {}
    hbm = measured_peak("hbm_gbs", 6800.0)
    bf16 = measured_peak("bf16_tflops", 1900.0)
    split = {}
    for prec in ("bf16x3", "tf32x2"):
        for kname, knum in (("blocks", 1), ("chunks", 2), ("panel", 0)):
            kw = dict(precision=PRECISIONS[prec], split_kernel=knum)
            with ClockSampler(local) as clk:
                per, prof = timed_multiplies(ctx, dA, dC, eps, steps, warmup, s, **kw)
            num_ms = prof.ms_numeric / max(prof.multiplies, 1)
            ms = statistics.median(per)
            nnz_c = dC.nblocks()[1]
            nbytes = 8 * nnz_c + split_slice_bytes(A, prec)
            pairs = 6 if prec == "bf16x3" else 3
            # tensor peak of the slices' type: BF16 measured; TF32 at the nominal
            # ratio 1.1 / 2.25 of it
            tpeak = bf16[0] * (1.0 if prec == "bf16x3" else 1.1 / 2.25)
            e = {"value": round(flops / (ms / 1e3) / 1e9, 2), "unit": "GFLOP/s (FP64-equivalent)",
                 "ms_p50": round(ms, 4), "numeric_ms": round(num_ms, 4),
                 "vs_fp64_path": None,
                 "roofline_hbm": {"achieved_gbs": round(nbytes / (num_ms / 1e3) / 1e9, 1),
                                  "peak_gbs": hbm[0], "frac": round(nbytes / (num_ms / 1e3) / 1e9 / hbm[0], 4),
                                  "algorithmic": "C written once + operand slices read once"},
                 "roofline_tensor": {"achieved_tflops": round(pairs * flops / (num_ms / 1e3) / 1e12, 2),
                                     "peak_tflops": round(tpeak, 1),
                                     "frac": round(pairs * flops / (num_ms / 1e3) / 1e12 / tpeak, 4),
                                     "algorithmic": f"{pairs} slice products x 2mnk per kept product"},
                 "clocks": clk.summary()}
            if sample is not None:
                rows, ref = sample
                gr, gc = dC.pattern()
                gv = dC.values()
                nb = int(np.searchsorted(gr, rows))
                nv = len(ref.values)
                if np.array_equal(gr[:nb], ref.blk_row) and np.array_equal(gc[:nb], ref.blk_col):
                    d = gv[:nv] - ref.values
                    e["rel_frobenius_err"] = float(np.linalg.norm(d) / np.linalg.norm(ref.values))
                    e["max_abs_err"] = float(np.max(np.abs(d)))
                    e["max_abs_value"] = float(np.max(np.abs(ref.values)))
                    e["error_sample"] = f"C block rows 0..{rows} against the oracle (FP64)"
                else:
                    e["pattern_differs_on_sample"] = True
            split[f"{prec}_{kname}"] = e
    out["split_water"] = split

    # the filter at work: the same water system with eps at the 30th percentile
    # of the candidate norm products (the headline's eps drops nothing)
    feps = norm_product_percentile(A, 30.0)
    dC3 = ctx.empty(A.row_sizes, A.col_sizes)
    st3 = ctx.multiply(1.0, dA, dA, 0.0, dC3, feps, stats=True, blocking=True)
    with ClockSampler(local) as clk:
        per, prof = timed_multiplies(ctx, dA, dC3, feps, steps, warmup, s)
    ms = statistics.median(per)
    out["filter_active_water"] = {
        "workload": "water2048, eps at the 30th percentile of the candidate norm products",
        "eps": feps, "candidates": st3.candidates, "kept": st3.kept, "dropped": st3.dropped,
        "c_blocks": st3.c_blocks, "gflop_kept_per_multiply": round(st3.flops / 1e9, 4),
        "value": round(st3.flops / (ms / 1e3) / 1e9, 2), "unit": "filtered GFLOP/s",
        "ms_p50": round(ms, 4), "numeric_ms": round(prof.ms_numeric / max(prof.multiplies, 1), 4),
        "clocks": clk.summary()}
    dC3.destroy()

    # mixed block sizes: one persistent launch vs one launch per shape class
    B2 = synth.amorphous(4096, seed=2)
    dB2 = ctx.from_blocks(B2)
    dC2 = ctx.empty(B2.row_sizes, B2.col_sizes)
    st2 = ctx.multiply(1.0, dB2, dB2, 0.0, dC2, 1e-8, stats=True)
    amo = {"workload": "amorphous4096 (block sizes 5/9/13/23/32), eps 1e-8",
           "gflop_per_multiply": round(st2.flops / 1e9, 3)}
    for name, kw in (("persistent", dict(launch=0)), ("per_stack", dict(launch=1)),
                     ("persistent_graph_autotune", dict(launch=0, graph=True, autotune=True))):
        with ClockSampler(local) as clk:
            per, prof = timed_multiplies(ctx, dB2, dC2, 1e-8, 5, 3, s, **kw)
        ms = statistics.median(per)
        amo[name] = {"value": round(st2.flops / (ms / 1e3) / 1e9, 2), "unit": "GFLOP/s",
                     "ms_p50": round(ms, 3), "clocks": clk.summary()}
    dB2.destroy()
    dC2.destroy()
    out["amorphous"] = amo

    # serving: a reduced replay of the request stream
    with ClockSampler(local) as clk:
        sv = serve_measure(100, 12, 4, 48.0)
    sv["clocks"] = clk.summary()
    out["serving"] = sv
    return out


def serve_measure(requests, pool_n, slots, budget_gb, seed=4):
    """Serving: C = A.A for a stream of independent water systems of different
    sizes (log-uniform 32..1024 molecules), replayed with Poisson arrivals at
    0.8 x the measured sequential capacity, as a saturating burst, and with
    Poisson arrivals at 0.8 x the server's burst capacity, against sequential
    per-call execution. Returns the measurements as a dict."""
    import synth
    from paper_1705_10218_gb300 import Context, Server

    rng = np.random.default_rng(seed)
    eps = 1e-10
    sizes = np.rint(np.exp(rng.uniform(np.log(32), np.log(1024), pool_n))).astype(int)
    pool = [synth.water(int(n), seed=1000 + p) for p, n in enumerate(sizes)]
    pick = rng.integers(0, pool_n, requests)
    gflop = []

    # sequential per-call execution through the C ABI: upload, multiply with the
    # result stored into page-locked host memory by the device (the fastest
    # per-call read-back), release
    import torch

    ctx = Context(0)
    nnz_of = {}
    for p in sorted(set(pick.tolist())):  # result sizes, for the page-locked buffer
        A = pool[p]
        dA = ctx.from_blocks(A)
        dC = ctx.empty(A.row_sizes, A.col_sizes)
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True)
        nnz_of[p] = dC.nblocks()[1]
        dA.destroy()
        dC.destroy()
    host = torch.empty(max(nnz_of.values()), dtype=torch.float64, pin_memory=True).numpy()
    lat_seq = []
    t0 = time.perf_counter()
    for r in range(requests):
        A = pool[pick[r]]
        ts = time.perf_counter()
        dA = ctx.from_blocks(A)
        dC = ctx.empty(A.row_sizes, A.col_sizes)
        st = ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stats=True, host_out=host)
        if st.c_nnz and not np.isfinite(host[st.c_nnz - 1]):
            raise RuntimeError("non-finite result")
        dA.destroy()
        dC.destroy()
        lat_seq.append((time.perf_counter() - ts) * 1e3)
        gflop.append(st.flops / 1e9)
    t_seq = time.perf_counter() - t0
    ctx.close()
    cap = requests / t_seq

    srv = Server(0, slots=slots, hbm_budget=int(budget_gb * (1 << 30)))
    # steady state: every distinct system once through the server first (its
    # page-locked result pool and the device-memory cache are then warm)
    # requests are submitted borrowed (bsm_server_submit_borrowed): the pool's
    # arrays stay alive, so the values need no copy at submission
    warm = [srv.submit(pool[p], eps, borrow=True) for p in sorted(set(pick.tolist()))]
    while warm:
        srv.progress()
        for i in list(warm):
            if srv.poll(i)[0] >= 2:
                srv.release(i)
                warm.remove(i)

    def replay(arrivals):
        lat, order, parts = [], [], []
        ids = [None] * requests
        nxt, done = 0, 0
        t0 = time.perf_counter()
        while done < requests:
            now = time.perf_counter() - t0
            k = 0  # a client thread would submit concurrently: interleave with progress
            while nxt < requests and arrivals[nxt] <= now and k < 8:
                ids[nxt] = srv.submit(pool[pick[nxt]], eps, borrow=True)
                order.append(nxt)
                nxt += 1
                k += 1
            if srv.progress() == 0:
                continue
            # admission is by deadline, not FIFO: any outstanding request may be done
            for r in list(order):
                state, l_ms, _, _ = srv.poll(ids[r])
                if state >= 2:
                    # the result is in host memory: used in place, then released
                    rows, cols, vals = srv.result(ids[r])
                    if len(vals) and not np.isfinite(vals[-1]):
                        raise RuntimeError("non-finite result")
                    parts.append(srv.timing(ids[r]))
                    srv.release(ids[r])
                    lat.append(l_ms)
                    order.remove(r)
                    done += 1
        makespan = time.perf_counter() - t0
        return lat, makespan, srv.info()["bytes_peak"], np.asarray(parts)

    def poisson(rate):
        gaps = rng.exponential(1.0 / rate, requests)
        return np.cumsum(gaps) - gaps[0]

    # the same requests through the server one at a time (each submitted once
    # the one before is done): the server's own latency without contention
    lat_1, parts_1 = [], []
    for r in range(requests):
        rid = srv.submit(pool[pick[r]], eps, borrow=True)
        while srv.poll(rid)[0] < 2:
            srv.progress()
        lat_1.append(srv.poll(rid)[1])
        parts_1.append(srv.timing(rid))
        srv.release(rid)
    parts_1 = np.asarray(parts_1)

    lam = 0.8 * cap
    b0 = srv.info()["batches"]
    lat_p, span_p, peak_p, parts_p = replay(poisson(lam))
    b1 = srv.info()["batches"]
    lat_b, span_b, peak_b, parts_b = replay(np.zeros(requests))
    b2 = srv.info()["batches"]
    lam_s = 0.8 * requests / span_b  # 0.8 x the server's own capacity
    lat_s, span_s, peak_s, parts_s = replay(poisson(lam_s))
    b3 = srv.info()["batches"]
    srv.close()

    def pct(x, q):
        return round(float(np.percentile(np.asarray(x), q)), 3)

    def split(parts):  # medians of the time in submit, queued and running
        return {k: pct(parts[:, c], 50) for c, k in enumerate(("submit_p50_ms", "wait_p50_ms",
                                                               "run_p50_ms"))}

    tot_gflop = float(np.sum(gflop))
    return {
        "config": {"workload": "water requests, 32..1024 molecules log-uniform", "requests": requests,
                   "distinct_systems": pool_n, "slots": slots, "budget_gb": budget_gb,
                   "eps": eps, "total_gflop": round(tot_gflop, 2),
                   "submission": "borrowed (bsm_server_submit_borrowed: values read from the "
                                 "caller's array when the request runs)"},
        "sequential": {"multiplies_per_s": round(cap, 3), "p50_ms": pct(lat_seq, 50),
                       "p99_ms": pct(lat_seq, 99), "gflop_per_s": round(tot_gflop / t_seq, 2)},
        "server_one_at_a_time": {"p50_ms": pct(lat_1, 50), "p99_ms": pct(lat_1, 99),
                                 **split(parts_1)},
        "poisson": {"arrival_rate_per_s": round(lam, 3), "multiplies_per_s": round(requests / span_p, 3),
                    "p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99), "peak_gb": round(peak_p / 2**30, 3),
                    "batches": b1 - b0, **split(parts_p)},
        "burst": {"multiplies_per_s": round(requests / span_b, 3), "p50_ms": pct(lat_b, 50),
                  "p99_ms": pct(lat_b, 99), "gflop_per_s": round(tot_gflop / span_b, 2),
                  "peak_gb": round(peak_b / 2**30, 3), "batches": b2 - b1, **split(parts_b)},
        "poisson_at_server_rate": {"arrival_rate_per_s": round(lam_s, 3),
                                   "multiplies_per_s": round(requests / span_s, 3),
                                   "p50_ms": pct(lat_s, 50), "p99_ms": pct(lat_s, 99),
                                   "peak_gb": round(peak_s / 2**30, 3), "batches": b3 - b2,
                                   **split(parts_s)},
    }


def serve_bench(args):
    """The request-loop benchmark on its own: one JSON line."""
    m = serve_measure(args.requests, args.serve_pool, args.slots, args.budget_gb)
    line = {
        "metric": "multiplies/s + p50/p99 latency (serving, continuous batching)",
        "value": m["burst"]["multiplies_per_s"], "unit": "multiplies/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic", **m}
    print(json.dumps(line), flush=True)
    return 0


def next_bench(args):
    """The next items beside the multiply, on the device, one JSON line:
    the post-multiplication filter and the block-sparse add on the water2048
    result, and the sign iteration of Eq. 3 (Newton-Schulz, two filtered
    multiplies per iteration plus the post filter) on water512."""
    import torch

    import synth
    from paper_1705_10218_gb300 import Context
    from paper_1705_10218_gb300.sign import block_identity

    torch.cuda.set_device(0)
    ctx = Context(0)
    out = {"metric": "next items: post filter, block-sparse add (GB/s), sign iteration (GFLOP/s)",
           "n_gpus": 1, "dtype": "f64", "data": "synthetic", "impl": "ours"}

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # post filter and add on C = A.A (water2048)
    A, eps = make_workload("water2048")
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True)
    nb0, nnz0 = dC.nblocks()
    r, c = dC.pattern()
    v = dC.values()
    lens = A.row_sizes.astype(np.int64)[r] * A.col_sizes.astype(np.int64)[c]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    nrm = np.sqrt(np.add.reduceat(v * v, off[:-1]))
    feps = float(np.percentile(nrm, 30))
    times, kept = [], 0
    for k in range(args.warmup + args.steps):
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True)
        dt = wall(lambda: dC.filter(feps))
        if k >= args.warmup:
            times.append(dt)
    nb1, nnz1 = dC.nblocks()
    fbytes = 8 * nnz0 + 16 * nnz1  # norms read every value; kept values read and written
    ms = 1e3 * statistics.median(times)
    out["post_filter"] = {"workload": "water2048 C = A.A", "eps": feps, "blocks_before": nb0,
                          "blocks_after": nb1, "ms": round(ms, 3),
                          "gb_per_s": round(fbytes / (ms / 1e3) / 1e9, 1),
                          "algorithmic": "8 B per value (norms) + 16 B per kept value (copy)"}
    times = []
    ctx.multiply(1.0, dA, dA, 0.0, dC, eps, blocking=True)
    for k in range(args.warmup + args.steps):
        dt = wall(lambda: ctx.add(1.0, dA, 1.0, dC))
        if k >= args.warmup:
            times.append(dt)
    nb2, nnz2 = dC.nblocks()
    abytes = 8 * (len(A.values) + nnz0 + nnz2)
    ms = 1e3 * statistics.median(times)
    out["add"] = {"workload": "water2048: C = C + A", "ms": round(ms, 3),
                  "gb_per_s": round(abytes / (ms / 1e3) / 1e9, 1),
                  "algorithmic": "A and C read once, the sum written once"}
    dA.destroy()
    dC.destroy()

    # sign iteration (Eq. 3) on a gapped water-like matrix: H = A + D with D =
    # +100 on the O atoms' diagonal and -100 on the H atoms' (two groups of
    # eigenvalues, standing for occupied and virtual states, with a gap wide
    # enough that sign(H) decays with distance as in an insulator), X0 = H / g
    # with g the largest absolute row sum (Gershgorin), so the spectrum of X0
    # lies in (-1, 1). The filters keep the iterates sparse (linear scaling).
    S = synth.water(args.sign_molecules, seed=1)
    vals = S.values.copy()
    rsz = S.row_sizes.astype(np.int64)
    lens = rsz[S.blk_row] * S.col_sizes.astype(np.int64)[S.blk_col]
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    for b in np.nonzero(S.blk_row == S.blk_col)[0]:
        n = int(S.row_sizes[S.blk_row[b]])
        vals[off[b] + np.arange(n) * (n + 1)] += 100.0 if n == 13 else -100.0
    row_off = np.zeros(S.nbr + 1, np.int64)
    np.cumsum(rsz, out=row_off[1:])
    blk = np.repeat(np.arange(S.nblk), lens)
    within = np.arange(len(vals)) - off[blk]
    rows = row_off[S.blk_row[blk]] + within % rsz[S.blk_row[blk]]
    g = float(np.bincount(rows, weights=np.abs(vals), minlength=int(row_off[-1])).max())
    vals /= g
    sizes = S.row_sizes
    X = ctx.matrix(sizes, sizes, S.blk_row, S.blk_col, vals)
    eps_s, feps_s = 1e-6, 1e-4
    its = []
    for it in range(args.sign_iters):
        T = block_identity(ctx, sizes, 3.0)
        s1 = ctx.multiply(-1.0, X, X, 1.0, T, eps_s, stats=True)  # 3I - X^2
        Xn = ctx.empty(sizes, sizes)
        s2 = ctx.multiply(0.5, X, T, 0.0, Xn, eps_s, stats=True)  # X (3I - X^2) / 2
        tf = wall(lambda: Xn.filter(feps_s))
        T.destroy()
        X.destroy()
        X = Xn
        nb, nz = X.nblocks()
        ms = s1.ms_total + s2.ms_total
        its.append({"iter": it + 1, "gflop": round((s1.flops + s2.flops) / 1e9, 2),
                    "multiply_ms": round(ms, 2), "filter_ms": round(1e3 * tf, 2),
                    "gflop_per_s": round((s1.flops + s2.flops) / (ms / 1e3) / 1e9, 1),
                    "x_blocks": nb, "x_block_occupancy": round(nb / (S.nbr * S.nbr), 4),
                    "dropped_products": s1.dropped + s2.dropped})
    # convergence: || X^2 - I ||_F / sqrt(N)
    Y = ctx.empty(sizes, sizes)
    ctx.multiply(1.0, X, X, 0.0, Y, 0.0, blocking=True)
    ctx.add(-1.0, block_identity(ctx, sizes), 1.0, Y)
    idem = float(np.linalg.norm(Y.values()) / np.sqrt(sizes.sum()))
    tot_f = sum(i["gflop"] for i in its)
    tot_ms = sum(i["multiply_ms"] for i in its)
    out["sign_iteration"] = {
        "workload": f"water{args.sign_molecules} (N = {int(sizes.sum())}), X0 = (A + D) / g: D = +100 (O) "
                    f"/ -100 (H) on the diagonal, g the largest absolute row sum",
        "eps": eps_s, "post_filter_eps": feps_s, "a_block_occupancy": round(S.nblk / S.nbr ** 2, 4),
        "iterations": its, "gflop_per_s": round(tot_f / (tot_ms / 1e3), 1),
        "idempotency_error": idem}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water2048", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--launch", default="persistent", choices=["persistent", "per_stack"])
    ap.add_argument("--eps", type=float, default=None, help="filter threshold (default: the workload's)")
    ap.add_argument("--eps-percentile", type=float, default=None,
                    help="filter threshold at this percentile of the candidate norm products")
    ap.add_argument("--graph", action="store_true", help="replay the multiply as a CUDA graph")
    ap.add_argument("--autotune", action="store_true", help="tune the FP64 kernel variants first")
    ap.add_argument("--fp64-kernel", default=None, choices=sorted(FP64_KERNELS),
                    help="force one FP64 numeric kernel (default: the library's choice)")
    ap.add_argument("--split-kernel", default=None, choices=sorted(SPLIT_KERNELS),
                    help="force a split-precision kernel (default: the library's choice)")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default: --steps; 0 skips the end-to-end leg)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other configurations (split precisions, amorphous, serving)")
    ap.add_argument("--serve", action="store_true", help="the request-loop benchmark instead")
    ap.add_argument("--next", action="store_true",
                    help="post filter, block-sparse add and sign iteration instead")
    ap.add_argument("--sign-molecules", type=int, default=2048)
    ap.add_argument("--sign-iters", type=int, default=8)
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--serve-pool", type=int, default=48)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=48.0)
    args = ap.parse_args()
    if args.serve:
        return serve_bench(args)
    if args.next:
        return next_bench(args)
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1705_10218_gb300 import Context

    A, eps = make_workload(args.workload)
    if args.eps is not None:
        eps = args.eps
    if args.eps_percentile is not None:
        eps = norm_product_percentile(A, args.eps_percentile)
    prec = PRECISIONS[args.precision]
    launch = 0 if args.launch == "persistent" else 1
    ctx = Context(local)
    dA = ctx.from_blocks(A)
    dC = ctx.empty(A.row_sizes, A.col_sizes)
    fk = None if args.fp64_kernel is None else FP64_KERNELS[args.fp64_kernel][0]
    kw = dict(precision=prec, launch=launch, graph=args.graph, autotune=args.autotune, fp64_kernel=fk)
    if args.split_kernel is not None:
        kw["split_kernel"] = SPLIT_KERNELS[args.split_kernel]
    st = ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stats=True,
                      **{k: v for k, v in kw.items() if k != "graph"})
    flops = st.flops
    s = torch.cuda.Stream()
    for _ in range(args.warmup):
        ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stream=s, **kw)
    s.synchronize()
    # A and C larger than L2 together: no flush; else a 256 MB buffer is written
    # between timed steps (outside the timed intervals) so each step starts cold
    a_bytes, c_bytes = 8 * len(A.values), 8 * dC.nblocks()[1]
    flush = None
    if a_bytes + c_bytes < 2 * L2_BYTES:
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    l2_note = (f"A {a_bytes / 1e6:.0f} MB, C {c_bytes / 1e6:.0f} MB: "
               + ("L2 flushed between steps (256 MB written)" if flush is not None
                  else "inputs larger than the 129 MB L2; no flush"))
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            if flush is not None:
                with torch.cuda.stream(s):
                    flush.fill_(k)
            ev[k][0].record(s)
            ctx.multiply(1.0, dA, dA, 0.0, dC, eps, stream=s, **kw)
            ev[k][1].record(s)
        s.synchronize()
        torch.cuda.synchronize()
    clocks = clk.summary()
    if dist is not None:
        dist.barrier()
    per_step = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = sum(per_step)
    prof = ctx.profile_read()
    ctx.profile(False)
    launches = prof.launches
    total_ms, value = replica_aggregate(total_ms, flops * args.steps, dist, device="cuda")
    nb_c, nnz_c = dC.nblocks()

    # dominant kernel: the numeric phase (one launch per multiply). In graph
    # replay the phases are not timed separately: the whole multiply is used.
    if prof.multiplies > 0:
        num_ms = prof.ms_numeric / prof.multiplies
        kname = (FP64_KERNELS[FP64_BY_NUMBER[prof.last_fp64_kernel]][1] if args.precision == "fp64"
                 else SPLIT_KERNEL_SYMBOLS.get(prof.last_split_kernel, "k_numeric_split_pipe"))
    else:
        num_ms = total_ms / args.steps
        kname = "whole multiply (CUDA graph replay)"
    phase = {"norms": round(prof.ms_norms / max(prof.multiplies, 1), 4),
             "symbolic": round(prof.ms_symbolic / max(prof.multiplies, 1), 4),
             "numeric": round(num_ms, 4)}
    # the integer / streaming phases against their own units: the norms read A's
    # values once (A = B); the symbolic phase (count, scan, fill) visits every
    # candidate product
    phase_rates = None
    if prof.multiplies > 0 and args.precision == "fp64":
        phase_rates = {
            "norms_gb_per_s": round(8 * len(A.values) / (phase["norms"] / 1e3) / 1e9, 1),
            "symbolic_gcandidates_per_s": round(st.candidates / (phase["symbolic"] / 1e3) / 1e9, 2)}
    if args.precision == "fp64":
        achieved = flops / (num_ms / 1e3) / 1e9
        fp64_peak, fp64_src = fp64_peak_gflops(torch.cuda.get_device_properties(local).multi_processor_count,
                                               clocks)
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(fp64_peak, 1),
                "unit": "GFLOP/s", "frac": round(achieved / fp64_peak, 4),
                "traffic": (measured_traffic(FP64_BY_NUMBER[prof.last_fp64_kernel], args.workload)
                            if prof.multiplies > 0 and args.eps_percentile is None else None),
                "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + write.sum)",
                "kernel": kname, "peak_source": fp64_src,
                "algorithmic": "2*m*n*k over kept products per launch", "phase_ms": phase,
                "phase_rates": phase_rates}
    else:
        # compulsory bytes of the numeric kernel: C written once (FP64) and the
        # operand slices read once (A = B: left and right layouts)
        rs = A.row_sizes.astype(np.int64)
        r, c = rs[A.blk_row], A.col_sizes.astype(np.int64)[A.blk_col]
        # rows padded along k to 16 bytes (8 BF16 / 4 TF32 values), per layout
        def up(x, q):
            return (x + q - 1) // q * q
        if args.precision == "bf16x3":
            slice_bytes = 3 * 2 * int((r * up(c, 8) + c * up(r, 8)).sum())
        else:
            slice_bytes = 2 * 4 * int((r * up(c, 4) + c * up(r, 4)).sum())
        nbytes = 8 * nnz_c + slice_bytes
        achieved = nbytes / (num_ms / 1e3) / 1e9
        peak = measured_peak("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak[0], "unit": "GB/s",
                "frac": round(achieved / peak[0], 4), "traffic": None, "kernel": kname,
                "peak_source": peak[1], "algorithmic": f"{nbytes} B per launch (C write + operand slices)",
                "phase_ms": phase}

    # end to end through the C ABI with host buffers: A's block list and
    # values from pinned host memory, the multiply, C's values stored into
    # pinned host memory by the device as they are computed.
    e2e = None
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    if args.e2e_steps > 0:
        pin_vals = torch.empty(len(A.values), dtype=torch.float64, pin_memory=True).numpy()
        pin_vals[:] = A.values
        pin_out = torch.empty(nnz_c, dtype=torch.float64, pin_memory=True).numpy()
        rs, cs, br, bc = A.row_sizes, A.col_sizes, A.blk_row, A.blk_col
        Ce = ctx.empty(rs, cs)
        Ae = [ctx.empty(rs, cs), ctx.empty(rs, cs)]

        def e2e_steps(k):
            # step i's input goes into handle i % 2 while the multiply of step
            # i - 1 (on the other handle) runs; each step ends when its result
            # is in host memory
            Ae[0].assign(br, bc, pin_vals)
            for i in range(k):
                ctx.multiply(1.0, Ae[i % 2], Ae[i % 2], 0.0, Ce, eps, precision=prec, launch=launch,
                             fp64_kernel=fk, host_out=pin_out)
                if i + 1 < k:
                    Ae[(i + 1) % 2].assign(br, bc, pin_vals)
                ctx.sync()

        e2e_steps(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps(args.e2e_steps)
        dt = time.perf_counter() - t0
        for M in Ae:
            M.destroy()
        # the host copy is the result: check it on a sample against the device values
        chk = Ce.values()
        idx = np.random.default_rng(0).integers(0, nnz_c, 1_000_000) if nnz_c else np.zeros(0, int)
        if not np.array_equal(pin_out[idx], chk[idx]):
            raise RuntimeError("end-to-end host copy differs from the device result")
        h2d = pin_vals.nbytes + br.nbytes + bc.nbytes + rs.nbytes + cs.nbytes
        e2e = {"value": round(flops * args.e2e_steps / dt / 1e9, 3), "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(pin_out.nbytes),
               "ms_per_step": round(dt / args.e2e_steps * 1e3, 3),
               "path": "bsm_mat_assign of A's block list and values from pinned host memory "
                       "into two reused handles in turn (step i+1's upload while step i's "
                       "multiply runs), bsm_multiply with opts.host_values (C's values stored "
                       "into pinned host memory by the device), bsm_sync every step"}
        Ce.destroy()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, rows, r = cpu_baseline(A, eps)
        # the GPU result on the same block rows, for the record
        gr, gc = dC.pattern()
        gv = dC.values()
        nb = int(np.searchsorted(gr, rows))
        same = np.array_equal(gr[:nb], r.blk_row) and np.array_equal(gc[:nb], r.blk_col)
        nv = len(r.values)
        err = float(np.linalg.norm(gv[:nv] - r.values) / np.linalg.norm(r.values)) if same else None
        cpu["gpu_pattern_equal_on_sample"] = bool(same)
        cpu["gpu_rel_err_on_sample"] = err
        if same and nv:
            cpu["gpu_max_abs_err_on_sample"] = float(np.max(np.abs(gv[:nv] - r.values)))
            cpu["max_abs_value_on_sample"] = float(np.max(np.abs(r.values)))

    variants = None
    if rank == 0 and world == 1 and not args.no_variants and args.workload == "water2048" \
            and args.precision == "fp64":
        sample = None
        if cpu is not None and cpu.get("gpu_pattern_equal_on_sample"):
            sample = (rows, r)
        variants = measure_variants(ctx, A, dA, dC, eps, flops, local, sample)
        fp64_ms = total_ms / args.steps
        for e in variants["split_water"].values():
            e["vs_fp64_path"] = round(fp64_ms / e["ms_p50"], 3)

    if rank == 0:
        srt = sorted(per_step)
        p99 = srt[min(len(srt) - 1, int(np.ceil(0.99 * len(srt))) - 1)]
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "atoms": A.nbr, "dimension": int(A.row_sizes.sum()),
                       "eps": eps, "precision": args.precision, "launch": args.launch,
                       "split_kernel": args.split_kernel,
                       "graph": bool(args.graph), "autotune": bool(args.autotune),
                       "fp64_kernel": (FP64_BY_NUMBER.get(prof.last_fp64_kernel)
                                       if args.precision == "fp64" else None),
                       "a_blocks": A.nblk, "c_blocks": nb_c, "c_nnz": nnz_c,
                       "kept_products": st.kept, "dropped_products": st.dropped,
                       "gflop_per_multiply": round(flops / 1e9, 4),
                       "l2": l2_note,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "multiplies_per_s": round(1e3 * args.steps * world / total_ms, 3),
            "latency_ms": {"p50": round(statistics.median(per_step), 4), "p99": round(p99, 4),
                           "min": round(min(per_step), 4), "max": round(max(per_step), 4)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches - 0),
            "clocks": clocks,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
