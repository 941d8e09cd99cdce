"""Benchmark of the exhaustive k-SNP MI search on one GB300.

One step = one whole search (enumerate every combination, count its
contingency table, score it, keep the exact top-N) over a dataset resident
in HBM.  Prints one JSON line.

    python bench.py [--steps K] [--warmup W] [--workload NAME] [--path auto|tc|popc]
    python bench.py --impl reference ...   # the CPU oracle on the host cores

The main figure is the order-3 workload (2000 SNPs x 4000 samples) on the
fastest exact counting path (tensor cores); the popcount path and the order-4
workload (500 SNPs x 8192 samples) are measured beside it.  Under torchrun
with N > 1 each rank runs the same search on its own GPU (independent
replicas, weak scaling); the reported value sums the ranks' work over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "combination-samples/sec at orders 2-4 (INT8-TC vs popcount path); top-N recall at k=5"
UNIT = "combination-samples/s"
DEFAULT_WORKLOAD = "order3_2000snp_4000"
# integer-pipe roofline of the popcount path: POPC executes on the XU pipe,
# 16 results per SM per clock (measured: 15.1/clk/SM), 152 SMs, 2070 MHz max
POPC_PER_SM_CLK = 16
N_SMS = 152
SM_MAX_MHZ = 2070.0
# FP8 dense rate = 2 x BF16 dense (nominal 4.5 vs 2.25 PFLOP/s)
FP8_OVER_BF16 = 2.0


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return dict(bf16=p["bf16_tflops"], bf16_sustained=p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                    hbm=p["hbm_gbs"], source="measured")
    except (OSError, KeyError, ValueError):
        return dict(bf16=1900.0, bf16_sustained=1700.0, hbm=6800.0, source="fallback")


def workload_desc(name, d, k, top_n):
    return dict(workload=name, order=k, n_snps=d.n_snps, n_samples=d.n_samples, n_cases=d.n_cases,
                n_controls=d.n_samples - d.n_cases, top_n=top_n, data="synthetic HWE, seeded")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        out.update(sm_mhz=statistics.median(loaded) if loaded else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out



def oracle_range_rate(d, k, top_n, target_s):
    """Time the oracle, as it stands, on a rank range sized to ~target_s."""
    from oracle import oracle as O
    total = O.binom(d.n_snps, k)
    r = min(total, 20000)
    t0 = time.perf_counter()
    O.search(d.geno, d.pheno, k, top_n, rank_begin=0, rank_end=r, with_counts=False)
    dt = time.perf_counter() - t0
    for _ in range(3):            # grow the range until it takes about target_s
        if dt >= target_s / 2 or r >= total:
            break
        r = min(total, int(r * target_s / max(dt, 1e-3)))
        t0 = time.perf_counter()
        O.search(d.geno, d.pheno, k, top_n, rank_begin=0, rank_end=r, with_counts=False)
        dt = time.perf_counter() - t0
    return r, dt, total


def cpu_baseline(d, k, top_n, target_s=15.0):
    from oracle import oracle as O
    r, dt, total = oracle_range_rate(d, k, top_n, target_s)
    return dict(value=r * d.n_samples / dt, unit=UNIT, cores=O.max_threads(), kind="oracle",
                sample=f"lexicographic ranks [0, {r}) of the {total} combinations ({dt:.1f} s)")


def run_reference(args):
    """Reference arm: the CPU oracle timed on this host's cores."""
    if _env_int("RANK", 0) != 0:
        return 0
    from oracle import oracle as O
    from paper_2201_02460_gb300 import synth
    d, k, top_n = synth.make_workload(args.workload)
    total = O.binom(d.n_snps, k)
    threads = O.max_threads()
    r, dt, _ = oracle_range_rate(d, k, top_n, 10.0)
    for _ in range(args.warmup):
        O.search(d.geno, d.pheno, k, top_n, rank_begin=0, rank_end=min(total, r // 10 + 1), with_counts=False)
    times = []
    for s in range(args.steps):
        r0 = (s * r) % max(1, total - r + 1)
        t0 = time.perf_counter()
        O.search(d.geno, d.pheno, k, top_n, rank_begin=r0, rank_end=r0 + r, with_counts=False)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = args.steps * r * d.n_samples / t
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * t / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=workload_desc(args.workload, d, k, top_n),
                cpu_baseline=dict(value=value, unit=UNIT, cores=threads, kind="oracle",
                                  sample=f"each step: {r} consecutive lexicographic ranks of {total}"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def time_search(epi, ctx, ds, k, top_n, path, steps, warmup, flush, stream):
    """Device time of `steps` searches (L2 flushed between them, not timed),
    the counting kernel's own event time, and the library's launches."""
    import torch
    for _ in range(warmup):
        epi.search(ds, k, top_n, path=path)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.kernel_launches()
    ctx.profile_begin()
    res = None
    for s in range(steps):
        flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        res = epi.search(ds, k, top_n, path=path)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    waits = ctx.profile_waits()
    kern_ms, kern_n = ctx.profile_end()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    return dict(t_ms=t_ms, kern_ms=kern_ms / max(kern_n, 1), launches=ctx.kernel_launches() - launches0,
                res=res, waits=waits)


def measure_batch(epi, ctx, synth, n_div, steps=2):
    """The 64-dataset batched configuration (orders 2-4, 1000-16000 samples,
    case fraction 0.3-0.7, top-20 each) with SNP counts divided by n_div: one
    epi_search_batched call per step (graph captured during the warm-up)."""
    import torch
    specs = synth.batch_specs()
    dss, orders, tops, work = [], [], [], 0
    for sp in specs:
        n = max(sp["order"] + 2, sp["n_snps"] // n_div)
        d = synth.make_dataset(n, sp["n_cases"], sp["n_controls"], seed=sp["seed"], maf_lo=sp["maf_lo"])
        dss.append(epi.Dataset(ctx, d.geno, d.pheno))
        orders.append(sp["order"])
        tops.append(sp["top_n"])
        work += math.comb(n, sp["order"]) * d.n_samples
    epi.search_batched(ctx, dss, orders, tops)          # warm-up: builds and captures the graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        epi.search_batched(ctx, dss, orders, tops)
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / steps
    for ds in dss:
        ds.close()
    return dict(value=work / t, ms_per_step=1e3 * t, datasets=len(specs), combination_samples=work,
                snp_divisor=n_div, timing="host wall clock around the synchronous batched call")


def measure_training(epi, ctx, peaks, rows=8192, steps=50, n_in=25, hidden=256):
    """Training throughput of the proposer network: AdamW steps on one
    resident batch (forward, backward, optimiser), the three hidden x hidden
    products on the tensor cores.  Work per row: 2 flop per multiply-add of
    the forward (n_in h + h^2 + h) and backward (n_in h + 2 h^2 + 3 h)
    products."""
    import torch
    net = epi.MLP(ctx, n_in, hidden, seed=2)
    X = (torch.rand(rows, n_in, device="cuda") * -8.0).contiguous()
    t = torch.randn(rows, device="cuda")
    for _ in range(3):
        net.train_step(X, t, 1e-4, 0.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        net.train_step(X, t, 1e-4, 0.0)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / steps
    flops = 2.0 * rows * (2 * n_in * hidden + 3 * hidden * hidden + 4 * hidden)
    net.close()
    return dict(rows_per_step=rows, ms_per_step=sec * 1e3, rows_per_s=rows / sec, tflops=flops / sec / 1e12,
                frac_of_bf16_peak=flops / sec / 1e12 / peaks["bf16"],
                note="whole AdamW step on a resident batch, CUDA events; 2*(2*in*h + 3*h^2 + 4*h) flop per row")


def measure_count_variants(epi, ctx, synth, flush, stream):
    """The GPU counterpart of the paper's popcount comparison (Table 1): every
    order-3 table of the first 500 SNPs of the 2000 x 4000 workload counted
    with the POPC instruction, a byte lookup table in shared memory, and the
    binary tensor-core MMA (AND + POPC), each run twice (the second timed);
    paper work 3^k (W1 + W0) 32-bit word operations per combination, against
    the POPC pipe's rate.  The FP8 tensor-core search of the same dataset is
    timed beside them (it also scores and selects)."""
    import torch
    d, k, top_n = synth.make_workload("order3_2000snp_4000", n_snps=500)
    ds = epi.Dataset(ctx, d.geno, d.pheno)
    W = 4 * (-(-d.n_cases // 128) + -(-(d.n_samples - d.n_cases) // 128))
    ops = math.comb(d.n_snps, k) * 3 ** k * W
    peak = N_SMS * POPC_PER_SM_CLK * SM_MAX_MHZ * 1e6
    out = {}
    sums = set()
    for v in ("popc", "lut", "mma_b1"):
        epi.count_variant(ds, k, v)
        r = epi.count_variant(ds, k, v)
        sums.add(r["checksum"])
        out[v] = dict(ms=r["ms"], word_ops_per_s=ops / (r["ms"] / 1e3), frac_of_popc_peak=ops / (r["ms"] / 1e3) / peak)
    m = time_search(epi, ctx, ds, k, top_n, "tc", 2, 1, flush, stream)
    out["tc_fp8_search"] = dict(ms=m["t_ms"] / 2, word_ops_per_s=ops / (m["t_ms"] / 2 / 1e3),
                                note="whole search (count, score, top-N), paper work in the same units")
    ds.close()
    out["checksums_agree"] = len(sums) == 1
    out["workload"] = f"order 3, {d.n_snps} SNPs x {d.n_samples} samples, every table"
    return out


def measure_batch_full(epi, ctx, synth, peaks, tc_rate, stream):
    """The 64-dataset batched configuration at its configured sizes (SNPs
    ~ U{100..1000}, samples ~ U{1000..16000}, case fraction ~ U[0.3, 0.7],
    orders ~ U{2, 3, 4}, top-20 each): the autotuner first runs once per size
    bucket, then one epi_search_batched call (its first: the graph is captured
    and launched) is timed with CUDA events on the context's stream.  The
    scheduler efficiency is the time every dataset would take alone at its
    path's peak (paper work: 2*3^k*m flop per combination on the tensor path
    against the measured MMA rate, 3^k*(W1+W0) word operations on the popcount
    path against the POPC rate), summed, over the measured time."""
    import torch
    specs = synth.batch_specs()
    dss, orders, tops, data = [], [], [], []
    for sp in specs:
        d = synth.make_dataset(sp["n_snps"], sp["n_cases"], sp["n_controls"], seed=sp["seed"], maf_lo=sp["maf_lo"])
        dss.append(epi.Dataset(ctx, d.geno, d.pheno))
        orders.append(sp["order"])
        tops.append(sp["top_n"])
        data.append(d)
    # autotune one dataset per (order, log2 SNPs, log2 sample words) bucket
    t0 = time.perf_counter()
    chosen = {}
    for ds, d, k in zip(dss, data, orders):
        wt = 4 * (-(-d.n_cases // 128) + -(-(d.n_samples - d.n_cases) // 128))
        key = (k, d.n_snps.bit_length() - 1, wt.bit_length() - 1)
        if key not in chosen:
            chosen[key] = epi.autotune(ds, k)
    tune_s = time.perf_counter() - t0
    tc_peak = (2.0 * tc_rate[0]["mac_per_clk_sm"] * N_SMS * SM_MAX_MHZ * 1e6 if tc_rate
               else FP8_OVER_BF16 * peaks["bf16"] * 1e12)
    popc_peak = N_SMS * POPC_PER_SM_CLK * SM_MAX_MHZ * 1e6
    work = 0
    ideal_s = 0.0
    for d, k in zip(data, orders):
        wt = 4 * (-(-d.n_cases // 128) + -(-(d.n_samples - d.n_cases) // 128))
        key = (k, d.n_snps.bit_length() - 1, wt.bit_length() - 1)
        total = math.comb(d.n_snps, k)
        work += total * d.n_samples
        if chosen[key]["path"] == "tc":
            ideal_s += 2.0 * total * 3 ** k * d.n_samples / tc_peak
        else:
            ideal_s += total * 3 ** k * wt / popc_peak
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    epi.search_batched(ctx, dss, orders, tops)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    for ds in dss:
        ds.close()
    paths = {}
    for (k, _, _), c in chosen.items():
        nm = f"order{k}/{c['path']}"
        paths[nm] = paths.get(nm, 0) + 1
    return dict(value=work / t, ms_per_step=1e3 * t, datasets=len(specs), combination_samples=work,
                scheduler_efficiency=ideal_s / t, ideal_seconds=ideal_s, autotune_seconds=tune_s,
                tuned_buckets=paths,
                timing="CUDA events on the context's stream around the first batched call (graph capture and "
                       "launch; capture is host work of milliseconds)")


def measure_mlp_inference(epi, ctx, peaks):
    """Throughput of the proposer network's fused BF16 tensor-core inference
    on 2^24 resident rows of 25 features."""
    import torch
    net = epi.MLP(ctx, 25, 256, seed=1)
    out = {}
    # the network alone on resident rows: fused BF16 tensor-core inference
    X = torch.randn(1 << 24, 25, device="cuda") - 4.0
    net.forward(X)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        net.forward(X)
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / 3
    flops = X.shape[0] * 2.0 * (25 * 256 + 256 * 256 + 256)
    out["mlp_inference"] = dict(rows_per_s=X.shape[0] / t, tflops=flops / t / 1e12,
                                frac_of_bf16_peak=flops / t / 1e12 / peaks["bf16"],
                                note="2*(25*256+256*256+256) flop per row; K of layer 1 padded to 32 on the device")
    net.close()
    return out


def comb_shift(d, k):
    """Class shift of the tensor path's combined-class variant, 0 where the
    separate-class variant runs (the rule include/epi.h states for
    EPI_TC_AUTO)."""
    m1, m0 = d.n_cases, d.n_samples - d.n_cases
    if k != 3:
        return 0
    p = 1
    while p < 15 and (1 << p) <= m0:
        p += 1
    return p if p <= 14 and m1 * (1 << p) + m0 < (1 << 23) else 0


def tc_executed_flops(d, k):
    """Multiply-adds the tensor-core counting kernel issues for a whole search,
    x 2.  The items are the M tiles of ppt prefixes that start in panel c
    times the N tiles after c (the kernel's item table), each over the padded
    K of both classes (128-individual stages).  Separate classes: N tiles of
    64 last SNPs, every MMA M128 x N128.  Combined classes: N tiles of 128
    last SNPs, the MMA's N cut to the columns below 2 n (steps of 16)."""
    n = d.n_snps
    ppt = 1 if 3 ** (k - 1) > 32 else 4 * (32 // 3 ** (k - 1))
    comb = comb_shift(d, k) != 0
    kj = 128 if comb else 64
    cols = 0
    for c in range(k - 2, n - 1):
        t0 = -(-math.comb(c, k - 1) // ppt)
        t1 = -(-math.comb(c + 1, k - 1) // ppt)
        if t1 == t0:
            continue
        # the N tiles of an M tile whose first prefix lies in panel c
        per_m = 0
        for u in range(-(-(n - 1 - c) // kj)):
            j0 = c + 1 + u * kj
            live = 2 * (n - j0)
            per_m += min(2 * kj, -(-live // 16) * 16) if comb else 2 * kj
        cols += (t1 - t0) * per_m
    kt = 32 * 4 * (-(-d.n_cases // 128) + -(-(d.n_samples - d.n_cases) // 128))
    return 2.0 * cols * 128 * kt


def roofline(kind, d, k, kern_ms, peaks, tc_rate=None):
    total = math.comb(d.n_snps, k)
    if kind == "tc":
        # algorithmic (paper) work: 3^k cells x m individuals multiply-adds
        # per combination; executed: the MMAs the kernel issues (two genotype
        # columns of the last SNP, padded rows and K)
        flops = 2.0 * total * (3 ** k) * d.n_samples
        achieved = flops / (kern_ms / 1e3) / 1e12
        executed = tc_executed_flops(d, k) / (kern_ms / 1e3) / 1e12
        fp8_conv = FP8_OVER_BF16 * peaks["bf16"]
        comb = comb_shift(d, k) != 0
        if tc_rate:
            # the measured rate of the kernel's own MMA, at the maximum SM clock
            r = tc_rate[1 if comb else 0]
            shape = "E5M2 M128 N256 K32" if comb else "E4M3 M128 N128 K32"
            peak = 2.0 * r["mac_per_clk_sm"] * N_SMS * SM_MAX_MHZ * 1e6 / 1e12
            note = (f"peak = measured FP8 {shape} tcgen05.mma rate, {r['mac_per_clk_sm']:.0f} "
                    f"MAC/clk/SM x 152 SMs x 2070 MHz (probe ran at {r['sm_mhz']:.0f} MHz: "
                    f"{r['tflops']:.0f} TFLOP/s); work 2*3^k*m flop per combination; "
                    f"{'combined' if comb else 'separate'}-class variant")
        else:
            peak = fp8_conv
            note = f"FP8 (E4M3) dense = 2 x {peaks['source']} burst BF16; work 2*3^k*m flop per combination"
        return dict(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    traffic=None, kernel="tc_search_kernel", kernel_ms=kern_ms,
                    executed_tflops=executed, executed_frac=executed / peak,
                    frac_vs_2x_bf16=achieved / fp8_conv, note=note)
    W = ((d.n_cases + 127) // 128 + (d.n_samples - d.n_cases + 127) // 128) * 4
    ops = total * (3 ** k) * W
    achieved = ops / (kern_ms / 1e3) / 1e12
    executed = popc_executed_ops(d, k, W) / (kern_ms / 1e3) / 1e12
    peak = N_SMS * POPC_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    return dict(bound="alu", achieved=achieved, peak=peak, unit="Tops/s", frac=achieved / peak, traffic=None,
                kernel="popc_pair_kernel" if k >= 6 else "popc_search_kernel", kernel_ms=kern_ms,
                executed_tops=executed, executed_frac=executed / peak,
                note="32-bit AND+POPC word operations, 3^k cells x (W1+W0) words per combination (paper "
                     "work; executed: the POPCs the kernel issues, the other cells by subtraction); "
                     "peak = 152 SMs x 16 POPC/clk x 2070 MHz")


def popc_executed_ops(d, k, W):
    """32-bit POPC word operations the popcount kernels issue for a whole
    search: the (k-1)-prefix kernel counts two genotype rows of the last SNP
    per prefix row (the third by subtraction); the (k-2)-prefix kernel of
    orders 6-8 counts the four joint rows of the last two SNPs per prefix row,
    and per prefix its row totals and the single counts of every following
    SNP's genotype-0/1 rows (rank ranges split between CTAs add a little, and
    the pairs its screen passes are counted a second time, not included)."""
    n, total = d.n_snps, math.comb(d.n_snps, k)
    if k < 6:
        return total * 2 * 3 ** (k - 1) * W
    per_prefix = sum(math.comb(c, k - 3) * (2 * (n - 1 - c) + 1) for c in range(k - 3, n - 2))
    return 3 ** (k - 2) * W * (4 * total + per_prefix)


def run_ours(args):
    import torch

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)

    from paper_2201_02460_gb300 import build as B
    B.build()
    from paper_2201_02460_gb300 import epi, synth

    peaks = measured_peaks()
    over = {"n_snps": args.n_snps} if args.n_snps else {}
    d, k, top_n = synth.make_workload(args.workload, **over)
    ctx = epi.Context(local)
    ds = epi.Dataset(ctx, d.geno, d.pheno)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    total = math.comb(d.n_snps, k)
    units = total * d.n_samples
    path = args.path
    tc_ok = 2 <= k <= 4 and 0 < d.n_cases < d.n_samples
    kind = "tc" if (path == "tc" or (path == "auto" and tc_ok and k >= 3)) else "popc"

    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        main_m = time_search(epi, ctx, ds, k, top_n, path, args.steps, args.warmup, flush, stream)
    clocks = clk.summary()
    t_ms = main_m["t_ms"]
    if world > 1:
        tt = torch.tensor([t_ms], dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    value = world * units * args.steps / (t_ms / 1e3)
    res = main_m["res"]
    # the roofline's denominator: the tensor pipe's rate for the counting MMA
    tc_rate = {s: ctx.tc_rate(shape=s) for s in (0, 1)} if kind == "tc" or not args.no_compare else None

    # end to end through the C-ABI: host genotypes in, host records out
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ds2 = epi.Dataset(ctx, d.geno, d.pheno)
        epi.search(ds2, k, top_n, path=path)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        ds2.close()
    e2e_t = statistics.median(e2e_times)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=t_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype=(("f8e5m2 0/1 operands (classes combined), f32 accumulate" if comb_shift(d, k)
                        else "f8e4m3 0/1 operands, f32 accumulate") if kind == "tc" else "u32"),
                data="synthetic",
                config=dict(**workload_desc(args.workload, d, k, top_n), path=path, counting=kind,
                            l2="flushed between steps (256 MiB write)", parallelism="replicas"),
                e2e=dict(value=units / e2e_t, unit=UNIT, h2d_bytes_per_step=int(d.geno.nbytes + d.pheno.nbytes),
                         d2h_bytes_per_step=int(top_n * epi.RESULT_DTYPE.itemsize + top_n * 2 * 3 ** k * 4),
                         seconds=e2e_t),
                roofline=roofline(kind, d, k, main_m["kern_ms"], peaks, tc_rate),
                gpu_launches=int(main_m["launches"]), clocks=clocks,
                top1=dict(snps=[int(x) for x in res.combs[0]], mi=float(res.mi[0]), planted=list(d.planted)))
    if kind == "tc" and main_m["waits"].get("mma_loop"):
        w = main_m["waits"]
        line["tc_wait_fractions"] = {k2: round(v / w["mma_loop"], 4) for k2, v in w.items() if k2 != "unused4"}

    # the other counting path and the order-4 workload, measured beside it
    if not args.no_compare and world == 1:
        comp = {}
        other = "popc" if kind == "tc" else ("tc" if tc_ok else None)
        if other:
            m2 = time_search(epi, ctx, ds, k, top_n, other, 2, 1, flush, stream)
            comp[f"{args.workload}/{other}"] = dict(value=units / (m2["t_ms"] / 2 / 1e3), ms_per_step=m2["t_ms"] / 2,
                                                     roofline=roofline(other, d, k, m2["kern_ms"], peaks, tc_rate))
        if args.workload != "order4_500snp_8192":
            d4, k4, n4 = synth.make_workload("order4_500snp_8192")
            ds4 = epi.Dataset(ctx, d4.geno, d4.pheno)
            u4 = math.comb(d4.n_snps, k4) * d4.n_samples
            m4 = time_search(epi, ctx, ds4, k4, n4, "tc", 2, 1, flush, stream)
            comp["order4_500snp_8192/tc"] = dict(value=u4 / (m4["t_ms"] / 2 / 1e3), ms_per_step=m4["t_ms"] / 2,
                                                 roofline=roofline("tc", d4, k4, m4["kern_ms"], peaks, tc_rate))
            if not args.quick:
                # one step (about 28 s): the popcount path on the same workload
                p4 = time_search(epi, ctx, ds4, k4, n4, "popc", 1, 0, flush, stream)
                comp["order4_500snp_8192/popc"] = dict(value=u4 / (p4["t_ms"] / 1e3), ms_per_step=p4["t_ms"],
                                                       roofline=roofline("popc", d4, k4, p4["kern_ms"], peaks))
            ds4.close()
        if args.workload != "order2_200snp_1600":
            # the order-2 workload (200 SNPs x 1600 samples): launch-bound,
            # reported without a roofline
            d2, k2, n2 = synth.make_workload("order2_200snp_1600")
            ds2w = epi.Dataset(ctx, d2.geno, d2.pheno)
            u2 = math.comb(d2.n_snps, k2) * d2.n_samples
            m2w = time_search(epi, ctx, ds2w, k2, n2, "auto", 20, 3, flush, stream)
            r2 = m2w["res"]
            comp["order2_200snp_1600/auto"] = dict(value=u2 / (m2w["t_ms"] / 20 / 1e3), ms_per_step=m2w["t_ms"] / 20,
                                                   kernel_ms=m2w["kern_ms"],
                                                   top1=[int(x) for x in r2.combs[0]], planted=list(d2.planted))
            ds2w.close()
        # thresholded output (every combination above an MI threshold; here
        # the 100th best of the top-N search): all scores on the popcount path
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt, nt = epi.search_threshold(ds, k, float(res.mi[-1]), capacity=1000)
        torch.cuda.synchronize()
        tt = time.perf_counter() - t0
        comp[f"{args.workload}/threshold"] = dict(value=units / tt, seconds=tt, threshold=float(res.mi[-1]),
                                                 found=int(nt), matches_top_n=bool(nt == len(res)))
        if args.workload != "order8_23snp_2048":
            # the order-8 row of Table 2 (popcount path, global prefix tables)
            d8, k8, n8 = synth.make_workload("order8_23snp_2048")
            ds8 = epi.Dataset(ctx, d8.geno, d8.pheno)
            u8 = math.comb(d8.n_snps, k8) * d8.n_samples
            m8 = time_search(epi, ctx, ds8, k8, n8, "popc", 2, 1, flush, stream)
            comp["order8_23snp_2048/popc"] = dict(value=u8 / (m8["t_ms"] / 2 / 1e3), ms_per_step=m8["t_ms"] / 2,
                                                  cells_per_s=math.comb(d8.n_snps, k8) * 3 ** k8 / (m8["t_ms"] / 2 / 1e3),
                                                  roofline=roofline("popc", d8, k8, m8["kern_ms"], peaks))
            ds8.close()
        comp["count_variants/order3_500snp_4000"] = measure_count_variants(epi, ctx, synth, flush, stream)
        comp["batch64/auto"] = measure_batch(epi, ctx, synth, args.batch_div)
        if not args.quick:
            comp["batch64_full/auto"] = measure_batch_full(epi, ctx, synth, peaks, tc_rate, stream)
        from paper_2201_02460_gb300 import proposer_eval
        comp["proposer_order5/mlp_inference"] = measure_mlp_inference(epi, ctx, peaks)["mlp_inference"]
        comp["proposer_order5/mlp_training"] = measure_training(epi, ctx, peaks)
        comp["proposer_order5/mlp_training_65536"] = measure_training(epi, ctx, peaks, rows=65536, steps=20)
        if not args.quick:
            # 2000 SNPs x 4000 samples with a planted 5-SNP parity: a trained
            # network against the heuristic, recall of the candidate space's
            # exact top-100
            comp["proposer_order5/eval_2000snp_4000"] = proposer_eval.evaluate_large(ctx)
        if args.proposer_eval:
            comp["proposer_order5/recall_200snp_2000"] = proposer_eval.evaluate(ctx)
        else:
            q = proposer_eval.quick(ctx)
            comp["proposer_order5/recall_200snp_2000_quick"] = q
            # the metric's second part: recall@100 of the exhaustive order-5
            # top-100 among the proposer's top-100 (30 features, network)
            best = [r for r in q["results"] if r["ranking"] == "network"]
            line["recall_k5"] = dict(value=best[-1]["recall_at_100"], budget=best[-1]["budget"],
                                     by_budget={str(r["budget"]): r["recall_at_100"] for r in best},
                                     heuristic={str(r["budget"]): r["recall_at_100"] for r in q["results"]
                                                if r["ranking"] == "heuristic"},
                                     workload="200 SNPs x 2000 samples, held-out synthetic dataset, "
                                              "T = 65536 expanded triples")
        line["compare"] = comp

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(d, k, top_n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    faulthandler.enable()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--path", default="auto", choices=["popc", "tc", "auto"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the other path and the order-4 workload")
    ap.add_argument("--quick", action="store_true",
                    help="skip the order-4 popcount leg (~28 s) and the full 64-dataset batch (~2 min)")
    ap.add_argument("--n-snps", type=int, default=None, help="smaller SNP count (profiling captures)")
    ap.add_argument("--batch-div", type=int, default=3, help="SNP-count divisor of the 64-dataset batch")
    ap.add_argument("--proposer-eval", action="store_true",
                    help="also train the order-5 proposer and measure its recall (several minutes)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
