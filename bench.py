"""Benchmark: FP64-accurate GEMM on one GB300 (or N independent replicas).

One step = one FP64-accurate product C = A B, N = P = M = 8192, entries
+-2^E (1 + f) with E uniform in [-20, 19] (log-uniform magnitudes, random
sign), through the library's split-precision path (mm_emulated, 8 BF16
slices, tcgen05): split of A and B, slice products, exact recombination.
The same line reports the plain FP64 product (mm_naive, FP64 tensor-core MMA)
on the same inputs, the measured normwise error of both on sampled rows, the
dominant kernel against its roofline, an end-to-end number through the C ABI
with host buffers, and the CPU oracle timed on this machine's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it runs under torchrun as N independent replicas (the product does
not exchange data between GPUs), barriers and synchronises around the timed
region and reports the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "split-precision vs plain FP64 GEMM TFLOP/s at rel ∞-err ≤1e-14; serve p50/p99 ms"
N = P = M = 8192
SLICES = 8
KIND = 0  # MM_SLICE_BF16
WORKLOAD = "fp64-accurate GEMM 8192x8192x8192, log-uniform |a| in 2^-20..2^20 with random sign"
DOMINANT = "emu_slice_gemm_tcgen05"
PROFILE_FILE = os.path.join(ROOT, "profiles", "emu_slice_gemm_tcgen05_8192.json")
KERNEL_SRC = os.path.join(ROOT, "paper_1106_1347_gb300", "csrc", "slice_gemm.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--n", type=int, default=8192, help="N = P = M (profiling runs use a smaller case)")
    ap.add_argument("--quick", action="store_true", help="only the timed product (for profiler captures)")
    ap.add_argument("--fp8", type=int, default=0, metavar="S",
                    help="profiling runs: time S FP8-E4M3 slices instead of 8 BF16 ones (with --quick)")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-baseline-requests", type=int, default=2000)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the slice sweep, the 4096x16384x4096 shape and the badly scaled errors")
    ap.add_argument("--variants-n", type=int, default=1, help="0: skip the per-method FP64 sweep and the paper's table")
    ap.add_argument("--fp64-only", action="store_true",
                    help="only the per-method FP64 timings at n = --n, one run each (profiling runs)")
    ap.add_argument("--detail", default=os.path.join(ROOT, "bench_detail.json"),
                    help="file that receives every section of the run (the printed line carries summaries)")
    ap.add_argument("--grouped-only", type=int, default=0, metavar="COUNT",
                    help="profiling runs: only the grouped launch of COUNT serving-shaped products")
    ap.add_argument("--method", default="",
                    help="profiling runs: one method at n = --n, a warm-up and one timed call (naive, kahan, "
                         "naive_unrolled_4, winograd, strassen, strassen_winograd, strassen_paper, "
                         "strassen_winograd_paper, strassen_emulated_1, emulated_8)")
    ap.add_argument("--no-cpu-table", action="store_true", help="skip the CPU oracle's run of the paper's test")
    ap.add_argument("--cpu-table-repeats", type=int, default=10)
    args = ap.parse_args()
    global N, P, M, WORKLOAD, SLICES, KIND, DOMINANT
    if args.fp8:
        if not args.quick:
            ap.error("--fp8 is for profiling runs: use it with --quick")
        SLICES, KIND, DOMINANT = args.fp8, 1, "emu_slice_gemm_tcgen05_fp8"
    if args.n != 8192:
        N = P = M = args.n
        WORKLOAD = WORKLOAD.replace("8192x8192x8192", f"{N}x{N}x{N}")
    return args


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(ms, device):
    """The slowest rank's time: every rank gets the MAX over all ranks (one
    all-reduce of a scalar; no data-path collective -- the ranks are replicas)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flop_per_step, steps, world, ms):
    """Weak scaling: every rank runs `steps` steps of its own replica, so the job
    completes world * steps * flop_per_step in the slowest rank's time."""
    return flop_per_step * steps * world / (ms * 1e-3) / 1e12


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_tflops(a, b, seconds, threads):
    """Times the CPU oracle's NaivStandard (the paper's plain FP64 product) on a
    row sample of the workload, rows split across `threads` Python threads (the
    ctypes call releases the GIL).  Returns (TFLOP/s, rows, threads, elapsed)."""
    import numpy as np

    import oracle

    oracle.build()
    t0 = time.perf_counter()
    oracle.naiv_standard(a[:1], b)
    one_row = max(time.perf_counter() - t0, 1e-3)
    rows = int(max(threads, min(a.shape[0], seconds * threads / one_row)))
    rows -= rows % threads
    rows = max(rows, threads)
    blocks = np.array_split(np.arange(rows), threads)
    def work(idx):
        oracle.naiv_standard(a[idx[0]: idx[-1] + 1], b)
    ths = [threading.Thread(target=work, args=(blk,)) for blk in blocks]
    t0 = time.perf_counter()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    el = time.perf_counter() - t0
    return 2.0 * rows * b.shape[0] * b.shape[1] / el / 1e12, rows, threads, el


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        # nvidia-smi's start-up (driver and device enumeration) comes before its
        # first sample; the timed region starts only once that sample is in, so
        # the start-up does not overlap it.
        self._reader = threading.Thread(target=self._read, daemon=True)
        self._reader.start()
        deadline = time.time() + 10.0
        while not self.lines and time.time() < deadline and self.proc.poll() is None:
            time.sleep(0.01)
        time.sleep(0.1)
        return self

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self._reader.join(timeout=5)
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def source_hash(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def dominant_traffic(ntiles_scale=1.0):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    try:
        prof = json.load(open(PROFILE_FILE))
    except (OSError, ValueError):
        return None
    if prof.get("kernel_source_sha256_16") != source_hash(KERNEL_SRC):
        return None
    return prof.get("dram_bytes_per_launch_full_size")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_inputs():
    import synthetic as S

    a = S.loguniform(N, P, S.stream_seed(3, 0))
    b = S.loguniform(P, M, S.stream_seed(3, 1))
    return a, b


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    a, b = make_inputs()
    cores = host_cores()
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_tflops(a, b, per_step / 4, cores)
    vals, rows_used, t_total = [], 0, 0.0
    for _ in range(args.steps):
        v, rows, thr, el = cpu_oracle_tflops(a, b, per_step, cores)
        vals.append(v)
        rows_used = rows
        t_total += el
    value = statistics.median(vals)
    sample = f"{rows_used} of {N} rows of C per step (all {P}x{M} of B), NaivStandard, {cores} threads over row blocks"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "P": P, "M": M, "oracle": "NaivStandard (plain C, sequential sums)"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sampled_error(c_dev, a, b, norm_a, norm_b, rows, truth=None):
    """max over sampled rows i of sum_j |C_ij - T_ij| / (||A|| ||B||), T the
    oracle's Dot2 product on those rows (a sample of the inf-norm's rows)."""
    import numpy as np

    import oracle

    if truth is None:
        truth = oracle.dot2_product(a[rows], b)
    got = c_dev[rows].cpu().numpy() if hasattr(c_dev, "cpu") else c_dev[rows]
    return float(np.abs(got - truth).sum(axis=1).max() / (norm_a * norm_b))


def timed(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def slice_sweep(ta, tb, a, b, norm_a, norm_b, rows, truth):
    """The emulated product at the bench shape for every slice count 3..8 with
    BF16 slices (beta = 7) and 3..10 with FP8-E4M3 slices (beta = 5,
    kind::f8f6f4): FP64-equivalent TFLOP/s (2NPM / t) and the sampled normwise
    error."""
    import torch

    import paper_1106_1347_gb300 as mm

    n, p, m = a.shape[0], a.shape[1], b.shape[1]
    c = torch.empty((n, m), dtype=torch.float64, device=ta.device)
    out = {}
    for kind, label in ((mm.SLICE_BF16, "bf16"), (mm.SLICE_FP8E4M3, "fp8_e4m3")):
        res = {}
        for s in range(3, 11 if kind == mm.SLICE_FP8E4M3 else 9):
            ms = timed(lambda: mm.emulated(ta, tb, nslices=s, kind=kind, out=c), 3)
            res[str(s)] = {"ms": ms, "tflops": 2.0 * n * p * m / (ms * 1e-3) / 1e12,
                           "slice_pairs": s * (s + 1) // 2,
                           "rel_inf_err_sampled": sampled_error(c, a, b, norm_a, norm_b, rows, truth)}
        out[label] = res
    return out


def tall_inner_shape(dev):
    """N = M = 4096, P = 16384, log-uniform entries, 8 slices."""
    import numpy as np
    import torch

    import paper_1106_1347_gb300 as mm
    import synthetic as S

    n, p, m = 4096, 16384, 4096
    a = S.loguniform(n, p, S.stream_seed(3, 2))
    b = S.loguniform(p, m, S.stream_seed(3, 3))
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    c = torch.empty((n, m), dtype=torch.float64, device=dev)
    ms = timed(lambda: mm.emulated(ta, tb, nslices=8, out=c), 5)
    norm_a, norm_b = float(mm.norm_inf(ta).item()), float(mm.norm_inf(tb).item())
    rows = np.arange(0, n, n // 4)[:4]
    return {"N": n, "P": p, "M": m, "slices": 8, "ms": ms, "tflops": 2.0 * n * p * m / (ms * 1e-3) / 1e12,
            "slice_gemm_tflops_bf16": 36 * 2.0 * n * p * m / (ms * 1e-3) / 1e12,
            "rel_inf_err_sampled": sampled_error(c, a, b, norm_a, norm_b, rows)}


def strassen_over_emulated(ta, tb, a, b, norm_a, norm_b, rows, truth):
    """Strassen / Strassen-Winograd levels over the emulated product (8 BF16
    slices): 8192^3 on the bench inputs with 0..2 levels (sampled error), and
    16384^3 with 0..2 levels on the bench inputs tiled 2 x 2 (time only).
    TFLOP/s is 2NPM / t throughout."""
    import torch

    import paper_1106_1347_gb300 as mm

    res = {}
    n = a.shape[0]
    c = torch.empty((n, n), dtype=torch.float64, device=ta.device)
    for variant, label in ((0, "strassen"), (1, "strassen_winograd")):
        for levels in (0, 1, 2):
            if variant == 1 and levels == 0:
                continue
            name = "emulated" if levels == 0 else f"{label}_{levels}"
            ms = timed(lambda: mm.strassen_emulated(ta, tb, variant=variant, levels=levels, nslices=8, out=c), 3)
            res.setdefault("8192", {})[name] = {
                "ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                "rel_inf_err_sampled": sampled_error(c, a, b, norm_a, norm_b, rows, truth)}
    del c
    torch.cuda.empty_cache()
    big = 2 * n
    ta2 = ta.repeat(2, 2)
    tb2 = tb.flip(0).repeat(2, 2)
    c2 = torch.empty((big, big), dtype=torch.float64, device=ta.device)
    for variant, label in ((0, "strassen"), (1, "strassen_winograd")):
        for levels in (0, 1, 2):
            if variant == 1 and levels == 0:
                continue
            name = "emulated" if levels == 0 else f"{label}_{levels}"
            ms = timed(lambda: mm.strassen_emulated(ta2, tb2, variant=variant, levels=levels, nslices=8, out=c2), 2)
            res.setdefault(str(big), {})[name] = {"ms": ms, "tflops": 2.0 * big ** 3 / (ms * 1e-3) / 1e12}
            torch.cuda.empty_cache()
    del ta2, tb2, c2
    torch.cuda.empty_cache()
    res["inputs"] = "8192: the bench's log-uniform A, B; 16384: A tiled 2x2, B row-reversed and tiled 2x2"
    return res


def grouped_vs_single(dev, count=256):
    """`count` products with the serving stream's shapes (N, P, M log-uniform on
    [32, 4096]), 8 BF16 slices: one grouped launch per kernel against one
    mm_emulated call per product, device-resident operands."""
    import torch

    import paper_1106_1347_gb300 as mm
    import synthetic as S

    trace = S.serving_trace(count, S.stream_seed(4, 7), mean_gap_s=0.0)
    a_pool = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(4, 0))).to(dev)
    b_pool = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(4, 1))).to(dev)
    pairs = [(a_pool[:r["N"], :r["P"]], b_pool[:r["P"], :r["M"]]) for r in trace]
    outs = [torch.empty((r["N"], r["M"]), dtype=torch.float64, device=dev) for r in trace]
    flop = sum(2.0 * r["N"] * r["P"] * r["M"] for r in trace)
    # Back-to-back calls: the host side of a call (argument checks, the problem
    # table and its tensor maps) overlaps the device work of the one before;
    # `host_ms` is that host side alone, timed once after a synchronize.
    ms_group = timed(lambda: mm.emulated_group(pairs, nslices=8, outs=outs), 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mm.emulated_group(pairs, nslices=8, outs=outs)
    host_ms = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()
    with mm.profile() as prof:  # per-kernel device time of one more grouped launch
        mm.emulated_group(pairs, nslices=8, outs=outs)
        torch.cuda.synchronize()
    kernels = {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.stats.items()}
    # Useful and padded work of the slice product: 36 pair products per 2NPM, tiles of
    # 128 x 64 outputs and K-blocks of 32.
    padded = sum(2.0 * -(-r["N"] // 128) * 128 * -(-r["M"] // 64) * 64 * -(-r["P"] // 32) * 32 for r in trace)
    gemm_ms = kernels.get("emu_group_slice_gemm_tcgen05")

    def singles():
        for (ta, tb), c in zip(pairs, outs):
            mm.emulated(ta, tb, nslices=8, out=c)

    ms_single = timed(singles, 3)
    return {"problems": count, "dims": "N, P, M log-uniform [32, 4096]", "slices": 8, "gflop": flop / 1e9,
            "grouped": {"ms": ms_group, "tflops": flop / (ms_group * 1e-3) / 1e12, "host_ms_per_call": host_ms,
                        "kernel_ms": kernels,
                        "slice_gemm_pair_tflops_useful": (36 * flop / (gemm_ms * 1e-3) / 1e12) if gemm_ms else None,
                        "slice_gemm_pair_tflops_padded": (36 * padded / (gemm_ms * 1e-3) / 1e12) if gemm_ms else None,
                        "padding_efficiency": flop / padded},
            "one_call_each": {"ms": ms_single, "tflops": flop / (ms_single * 1e-3) / 1e12}}


def autotuner(dev):
    """The library's autotuner on a few shape buckets: the Strassen depth at
    4096^3 for both variants, and the emulated product's format x Strassen-
    Winograd levels x tile width for several tiers and shapes (one narrow),
    against the models' choices (the tuned table lives in this process only)."""
    import torch

    import paper_1106_1347_gb300 as mm
    import synthetic as S

    mm.tune_clear()
    out = {"strassen": {}, "emulated": []}
    a = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(1, 0))).to(dev)
    b = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(1, 1))).to(dev)
    for variant, name in ((0, "strassen"), (1, "strassen_winograd")):
        depth, ms = mm.tune_strassen(a, b, variant=variant)
        out["strassen"][name] = {"n": 4096, "depth": depth, "ms": ms, "tflops": 2.0 * 4096 ** 3 / (ms * 1e-3) / 1e12}
    del a, b
    for (n, p, m), tier in (((1024, 1024, 1024), 1e-14), ((1024, 1024, 1024), 1e-6), ((4096, 4096, 4096), 1e-9),
                            ((4096, 4096, 4096), 1e-12), ((8192, 8192, 8192), 1e-14), ((8192, 8192, 32), 1e-14)):
        a = torch.from_numpy(S.loguniform(n, p, S.stream_seed(3, 0))).to(dev)
        b = torch.from_numpy(S.loguniform(p, m, S.stream_seed(3, 1))).to(dev)
        model, _ = mm.emulated_choice(n, p, m, tier)
        kind, slices, levels, ms, tile = mm.tune_emulated(a, b, tier=tier)
        out["emulated"].append({"n": n, "p": p, "m": m, "tier": tier,
                                "tuned": {"format": kind, "slices": slices, "levels": levels, "tile": tile},
                                "ms": ms, "tflops": 2.0 * n * p * m / (ms * 1e-3) / 1e12,
                                "model": {"format": model[0], "slices": model[1], "levels": model[2],
                                          "tile": model[3]}})
        del a, b
        torch.cuda.empty_cache()
    mm.tune_clear()
    out["formats"] = "0 = BF16 slices, 1 = FP8-E4M3 slices"
    return out


def badly_scaled_errors(dev, n=2048, nrows=64):
    """Rows of A times 10^u, columns of B times 10^v (u, v uniform [-6, 6]):
    normwise error ||C - T||/(||A|| ||B||) and componentwise
    max |C - T|_ij / (|A| |B|)_ij of every method on sampled rows, T the oracle's
    Dot2 product."""
    import numpy as np
    import torch

    import oracle
    import paper_1106_1347_gb300 as mm
    import synthetic as S

    a, b = S.badly_scaled(n, S.stream_seed(2, 0), S.stream_seed(2, 1))
    ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    rows = np.linspace(0, n - 1, nrows).astype(np.int64)
    truth = oracle.dot2_product(a[rows], b)
    absab = np.abs(a[rows]) @ np.abs(b)
    na, nb = float(np.abs(a).sum(axis=1).max()), float(np.abs(b).sum(axis=1).max())
    runs = {
        "naive": lambda: mm.naive(ta, tb),
        "kahan": lambda: mm.kahan(ta, tb),
        "winograd": lambda: mm.winograd(ta, tb),
        "winograd_scaled": lambda: mm.winograd_scaled(ta, tb),
        "strassen": lambda: mm.strassen(ta, tb),
        "strassen_winograd": lambda: mm.strassen_winograd(ta, tb),
        "emulated_8_slices": lambda: mm.emulated(ta, tb, nslices=8),
    }
    if hasattr(mm, "winograd_rowcol_scaled"):
        runs["winograd_rowcol_scaled"] = lambda: mm.winograd_rowcol_scaled(ta, tb)
    out = {}
    for name, fn in runs.items():
        got = fn()[rows].cpu().numpy()
        diff = np.abs(got - truth)
        out[name] = {"normwise": float(diff.sum(axis=1).max() / (na * nb)),
                     "componentwise": float((diff / np.maximum(absab, np.finfo(float).tiny)).max())}
    return {"n": n, "rows_sampled": nrows, "scaling": "rows of A x 10^u, columns of B x 10^v, u, v in [-6, 6]",
            "reference": "oracle Dot2 product", "errors": out}


def serve_bench(dev, requests, budget_gb, baseline_requests, sweep_requests=3000):
    """The serving stream: `requests` products with N, P, M log-uniform on
    [32, 4096], entries uniform [-1, 1], tiers 1e-14 / 1e-6 half and half.
    1) saturated: every request submitted at t = 0 -> throughput;
    2) Poisson arrivals at 0.7x that rate -> p50 / p99 latency;
    3) like for like at one accuracy (every request at the 1e-14 tier): the
       plain FP64 kernel one request at a time and the emulated server, each
       paced at 0.7x its own saturated rate over the whole trace (the FP64
       arm's rate from its first `baseline_requests`), and the emulated server
       at the FP64 arm's arrival rate."""
    import torch

    import synthetic as S
    from paper_1106_1347_gb300 import serving

    a_pool = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(4, 0))).pin_memory()
    b_pool = torch.from_numpy(S.uniform(4096, 4096, S.stream_seed(4, 1))).pin_memory()
    c_pool = torch.empty((8192, 8192), dtype=torch.float64).pin_memory()
    budget = int(budget_gb * (1 << 30))
    # The host link the requests' operands cross: pinned copies of 512 MiB each way.
    probe_h = torch.empty(1 << 26, dtype=torch.float64).pin_memory()
    probe_d = torch.empty(1 << 26, dtype=torch.float64, device=dev)
    up_ms = timed(lambda: probe_d.copy_(probe_h, non_blocking=True), 3)
    down_ms = timed(lambda: probe_h.copy_(probe_d, non_blocking=True), 3)
    link = {"h2d_gbs": probe_h.nbytes / (up_ms * 1e-3) / 1e9, "d2h_gbs": probe_h.nbytes / (down_ms * 1e-3) / 1e9}
    del probe_h, probe_d
    sat_trace = S.serving_trace(requests, S.stream_seed(4, 2), mean_gap_s=0.0)

    def warm():
        # In a long-lived process a paced replay could meet one stall of 10-60 ms
        # (at a new server's first batches, or mid-replay), more often the
        # longer the process had run or idled before it, with the GPU at its
        # maximum clock throughout; the ~45 requests caught in it set p99.  So
        # the latency replays run first, before the long light-load replays of
        # the like-for-like comparison, each after the same short saturated
        # burst.
        with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as w:
            serving.replay(w, sat_trace[:1000], a_pool, b_pool, c_pool)

    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st_sat, _, rc_sat = serving.replay(srv, sat_trace, a_pool, b_pool, c_pool)
    rate = st_sat["completed"] / max(st_sat["busy_s"], 1e-9)
    up_bytes = sum(8.0 * (r["N"] * r["P"] + r["P"] * r["M"]) for r in sat_trace)
    down_bytes = sum(8.0 * r["N"] * r["M"] for r in sat_trace)
    # Time the copies alone would take, one direction after the other, at the measured link rates.
    copy_s = up_bytes / (link["h2d_gbs"] * 1e9) + down_bytes / (link["d2h_gbs"] * 1e9)
    paced = S.serving_trace(requests, S.stream_seed(4, 2), mean_gap_s=1.0 / (0.7 * rate))
    warm()
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st, comps, rc = serving.replay(srv, paced, a_pool, b_pool, c_pool)
    # Latency against load: shorter Poisson streams at other fractions of the saturated rate.
    sweep = {}
    for frac in (0.3, 0.5, 1.0):
        tr = S.serving_trace(sweep_requests, S.stream_seed(4, 3), mean_gap_s=1.0 / (frac * rate))
        warm()
        with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
            st_f, _, rc_f = serving.replay(srv, tr, a_pool, b_pool, c_pool)
        sweep[str(frac)] = {"arrival_rate_rps": frac * rate, "p50_ms": st_f["p50_ms"], "p99_ms": st_f["p99_ms"],
                            "completed": st_f["completed"], "status": rc_f}
    # The same two runs when each request takes the cheaper of BF16 and FP8 slices for its tier.
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True,
                        method=serving.METHOD_EMULATED_AUTO) as srv:
        st_sat_a, _, rc_sat_a = serving.replay(srv, sat_trace, a_pool, b_pool, c_pool)
    rate_a = st_sat_a["completed"] / max(st_sat_a["busy_s"], 1e-9)
    paced_a = S.serving_trace(requests, S.stream_seed(4, 2), mean_gap_s=1.0 / (0.7 * rate_a))
    warm()
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True,
                        method=serving.METHOD_EMULATED_AUTO) as srv:
        st_a, _, rc_a = serving.replay(srv, paced_a, a_pool, b_pool, c_pool)
    # Like for like at one accuracy: every request at the 1e-14 tier, each arm paced at 0.7x the rate
    # it sustains itself (the FP64 arm's rate measured on a prefix of the trace), plus the emulated
    # arm at the FP64 arm's arrival rate.
    strict = lambda gap: S.serving_trace(requests, S.stream_seed(4, 5), mean_gap_s=gap, tiers=(1e-14, 1e-14))
    with serving.Server(budget, method=serving.METHOD_FP64) as srv:
        st_fs, _, rc_fs = serving.replay(srv, strict(0.0)[:baseline_requests], a_pool, b_pool, c_pool)
    rate_f = st_fs["completed"] / max(st_fs["busy_s"], 1e-9)
    with serving.Server(budget, method=serving.METHOD_FP64) as srv:
        st_fp, _, rc_fp = serving.replay(srv, strict(1.0 / (0.7 * rate_f)), a_pool, b_pool, c_pool)
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st_es, _, rc_es = serving.replay(srv, strict(0.0), a_pool, b_pool, c_pool)
    rate_e = st_es["completed"] / max(st_es["busy_s"], 1e-9)
    warm()
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st_ep, _, rc_ep = serving.replay(srv, strict(1.0 / (0.7 * rate_e)), a_pool, b_pool, c_pool)
    warm()
    with serving.Server(budget, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st_ef, _, rc_ef = serving.replay(srv, strict(1.0 / (0.7 * rate_f)), a_pool, b_pool, c_pool)

    def arm(st_sat_x, st_paced_x, rate_x, rc_x):
        return {"saturated_requests_per_s": rate_x,
                "saturated_tflops": st_sat_x["flops"] / max(st_sat_x["busy_s"], 1e-9) / 1e12,
                "paced": {"arrival_rate_rps": 0.7 * rate_x, "requests": st_paced_x["completed"],
                          "p50_ms": st_paced_x["p50_ms"], "p99_ms": st_paced_x["p99_ms"],
                          "mean_ms": st_paced_x["mean_ms"], "max_ms": st_paced_x["max_ms"],
                          "requests_per_s": st_paced_x["completed"] / max(st_paced_x["busy_s"], 1e-9),
                          "status": rc_x}}

    like_for_like = {
        "tier": 1e-14, "requests": requests,
        "fp64_one_at_a_time": dict(arm(st_fs, st_fp, rate_f, rc_fp), saturated_on=f"first {baseline_requests}"),
        "emulated": arm(st_es, st_ep, rate_e, rc_ep),
        "emulated_at_fp64_rate": {"arrival_rate_rps": 0.7 * rate_f, "p50_ms": st_ef["p50_ms"],
                                  "p99_ms": st_ef["p99_ms"], "mean_ms": st_ef["mean_ms"],
                                  "max_ms": st_ef["max_ms"], "completed": st_ef["completed"], "status": rc_ef},
    }
    flop_all = st["flops"]
    # A 1 GiB budget, where admission binds: the largest requests (about 1.5 GB with
    # their split workspace) can never fit and are rejected, the rest queue for memory.
    small = 1 << 30
    tr = S.serving_trace(sweep_requests, S.stream_seed(4, 4), mean_gap_s=0.0)
    with serving.Server(small, max_batch=256, nstreams=4, use_graphs=True) as srv:
        st_s, comps_s, rc_s = serving.replay(srv, tr, a_pool, b_pool, c_pool)
    tight = {"budget_gb": 1.0, "requests": len(tr), "completed": st_s["completed"], "rejected": st_s["rejected"],
             "requests_per_s": st_s["completed"] / max(st_s["busy_s"], 1e-9),
             "p50_ms": st_s["p50_ms"], "p99_ms": st_s["p99_ms"], "peak_arena_gb": st_s["peak_arena_bytes"] / 2 ** 30,
             "status": rc_s}
    return {
        "requests": requests, "budget_gb": budget_gb, "dims": "N, P, M log-uniform [32, 4096]",
        "tiers": "1e-14 (8 slices) / 1e-6 (5 slices), 50/50",
        "host_link": link,
        "saturated": {"requests_per_s": rate, "tflops": st_sat["flops"] / max(st_sat["busy_s"], 1e-9) / 1e12,
                      "batches": st_sat["batches"], "graph_replays": st_sat["graph_replays"], "status": rc_sat,
                      "h2d_gb": up_bytes / 1e9, "d2h_gb": down_bytes / 1e9, "busy_s": st_sat["busy_s"],
                      "copy_bound_s": copy_s,
                      "note": "copy_bound_s: the operand and result copies alone at the measured link rates, one "
                              "direction after the other"},
        "paced": {"arrival_rate_rps": 0.7 * rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                  "mean_ms": st["mean_ms"], "max_ms": st["max_ms"], "completed": st["completed"],
                  "tflops": flop_all / max(st["busy_s"], 1e-9) / 1e12, "batches": st["batches"],
                  "graph_replays": st["graph_replays"], "peak_arena_gb": st["peak_arena_bytes"] / 2 ** 30,
                  "status": rc},
        "like_for_like_1e-14": like_for_like,
        "auto_format": {"formats": "1e-14: 8 BF16 slices; 1e-6: 6 FP8-E4M3 slices",
                        "saturated": {"requests_per_s": rate_a,
                                      "tflops": st_sat_a["flops"] / max(st_sat_a["busy_s"], 1e-9) / 1e12,
                                      "status": rc_sat_a},
                        "paced": {"arrival_rate_rps": 0.7 * rate_a, "p50_ms": st_a["p50_ms"], "p99_ms": st_a["p99_ms"],
                                  "completed": st_a["completed"], "status": rc_a}},
        "load_sweep": sweep, "budget_1gb_saturated": tight,
        "latency": "submit -> result in pinned host memory (H2D copies, product, D2H copy)",
    }


def fp64_peak(local, target_ms=150.0):
    """The FP64 pipe's rate measured on this GPU by the library's probe
    (mm_probe_fp64_peak: independent DFMA chains, and independent mma.sync f64
    accumulators), with the SM clock sampled while it runs."""
    import paper_1106_1347_gb300 as mm

    with ClockSampler(local) as clk:
        dfma, dmma = mm.probe_fp64_peak(target_ms)
    return {"dfma_tflops": dfma, "dmma_tflops": dmma, "clocks": clk.summary(),
            "how": f"mm_probe_fp64_peak, each kernel timed over >= {target_ms:.0f} ms with CUDA events"}


FP64_SWEEP = (256, 1024, 2047, 2048, 4095, 4096, 8192)


def variants_bench(dev, peak, sizes=FP64_SWEEP, reps=None):
    """Each FP64 method at n^3 for n in `sizes` (uniform [-1, 1] inputs; odd n
    exercise Winograd's odd-P term): TFLOP/s as 2n^3/t and, for the methods
    with a fixed operation count, the fraction of the FP64 pipe kept busy
    against the probe's rate for the instruction the kernel issues (`peak`,
    from fp64_peak)."""
    import torch

    import paper_1106_1347_gb300 as mm
    import synthetic as S

    # FP64-pipe operations (an FMA, DADD or DMUL each, or 1/256 of an m8n8k4 MMA)
    # issued per reported flop (2n^3 per product): naive 1 MMA-FMA per 2 flop; the
    # ordered naive sum 1 DMUL + 1 DADD per k; unrolled by 4, per group of four k
    # 4 DMUL + 3 DADD inside the group + 1 DADD into aux (2 per k); Kahan 1 DMUL +
    # 4 DADD per k; Winograd 2 DADD + 1 FMA per pair of k.
    pipe = {"naive": 0.5, "naive_ordered": 1.0, "naive_unrolled_4": 1.0, "kahan": 2.5, "winograd": 0.75,
            "winograd_scaled": 0.75, "winograd_rowcol_scaled": 0.75}
    ops_rate = {"dmma": peak["dmma_tflops"] / 2.0, "dfma": peak["dfma_tflops"] / 2.0}  # 1e12 FP64-pipe ops/s
    by_size = {}
    for n in sizes:
        a = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 0))).to(dev)
        b = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 1))).to(dev)
        c = torch.empty((n, n), dtype=torch.float64, device=dev)
        runs = {
            "naive": lambda: mm.naive(a, b, out=c),
            "naive_ordered": lambda: mm.naive_unrolled(a, b, unroll=1, out=c),
            "naive_unrolled_4": lambda: mm.naive_unrolled(a, b, unroll=4, out=c),
            "kahan": lambda: mm.kahan(a, b, out=c),
            "winograd": lambda: mm.winograd(a, b, out=c),
            "winograd_scaled": lambda: mm.winograd_scaled(a, b, out=c),
            "winograd_rowcol_scaled": lambda: mm.winograd_rowcol_scaled(a, b, out=c),
            "strassen": lambda: mm.strassen(a, b, out=c),
            "strassen_winograd": lambda: mm.strassen_winograd(a, b, out=c),
            "strassen_paper_rule": lambda: mm.strassen(a, b, cutoff=0, out=c),
            "strassen_winograd_paper_rule": lambda: mm.strassen_winograd(a, b, cutoff=0, out=c),
            "emulated_8_slices": lambda: mm.emulated(a, b, nslices=8, out=c),
        }
        out = {}
        for name, fn in runs.items():
            try:
                ms = timed(fn, reps or (1 if n >= 4095 else 3))
            except mm.MMError as exc:  # a depth the library refuses (reported, not hidden)
                out[name] = {"status": exc.status}
                continue
            tf = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
            entry = {"ms": ms, "tflops": tf}
            if name in pipe:  # fraction of the FP64 pipe kept busy
                entry["fp64_pipe_frac"] = tf * pipe[name] / ops_rate["dmma" if name == "naive" else "dfma"]
            out[name] = entry
        by_size[str(n)] = out
        del a, b, c
    return {"inputs": "uniform [-1, 1]", "fp64_peak": peak,
            "pipe_frac_against": "naive: the mma.sync f64 probe; the others: the DFMA probe", "by_size": by_size}


def paper_table(dev, sizes=(200, 400, 800), repeats=10):
    """The paper's own test (section 'Tests'): C = A (8A) for a random n x n A,
    every method timed over `repeats` runs, and NormInf(N - C) with N the
    NaivKahan result -- the same table on the GPU.  NaivOnArray runs the
    ordered naive kernel (its arithmetic is NaivStandard's); Strassen uses the
    paper's padding rule."""
    import torch

    import paper_1106_1347_gb300 as mm
    import synthetic as S

    table = {}
    for n in sizes:
        a_h, b_h = S.paper_pair(n, S.stream_seed(5, n))
        a = torch.from_numpy(a_h).to(dev)
        b = torch.from_numpy(b_h).to(dev)
        ref = mm.kahan(a, b)
        methods = {
            "NaivKahan (N)": lambda: mm.kahan(a, b),
            "NaivStandard": lambda: mm.naive_unrolled(a, b, unroll=1),
            "NaivOnArray": lambda: mm.naive_unrolled(a, b, unroll=1),
            "NaivLoopUnrollingTwo": lambda: mm.naive_unrolled(a, b, unroll=2),
            "NaivLoopUnrollingThree": lambda: mm.naive_unrolled(a, b, unroll=3),
            "NaivLoopUnrollingFour": lambda: mm.naive_unrolled(a, b, unroll=4),
            "StrassenNaiv": lambda: mm.strassen(a, b, cutoff=0),
            "StrassenWinograd": lambda: mm.strassen_winograd(a, b, cutoff=0),
            "WinogradOriginal": lambda: mm.winograd(a, b),
            "WinogradScaled": lambda: mm.winograd_scaled(a, b),
            "naive (FP64 DMMA)": lambda: mm.naive(a, b),
            "emulated, 8 BF16 slices": lambda: mm.emulated(a, b, nslices=8),
        }
        rows = {}
        for name, fn in methods.items():
            ms = timed(fn, repeats)
            c = fn()
            err = float(mm.norm_inf(ref - c).item())
            rows[name] = {"time_s": ms * 1e-3, "gflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "norm_inf_N_minus_C": err}
        table[str(n)] = rows
    return {"workload": "C = A (8A), A uniform [-1, 1]", "repeats": repeats, "time": "mean of one product", "n": table}


def paper_table_cpu(sizes=(200, 400, 800), repeats=10):
    """The paper's own test (section 'Tests') on this machine's host cores with
    the CPU oracle (plain C, -O2, no FMA contraction): C = A (8A) for a random
    n x n A, each method single-threaded and timed over `repeats` runs, and
    NormInf(N - C) with N the NaivKahan result.  The ten methods run at the
    same time, one thread each, each thread pinned to its own core when there
    are enough; the time is the mean of one product."""
    import numpy as np

    import oracle
    import synthetic as S

    oracle.build()
    methods = {
        "NaivKahan (N)": oracle.naiv_kahan,
        "NaivStandard": oracle.naiv_standard,
        "NaivOnArray": oracle.naiv_on_array,
        "NaivLoopUnrollingTwo": oracle.naiv_unrolled_2,
        "NaivLoopUnrollingThree": oracle.naiv_unrolled_3,
        "NaivLoopUnrollingFour": oracle.naiv_unrolled_4,
        "StrassenNaiv": lambda x, y: oracle.strassen_naiv(x, y),
        "StrassenWinograd": lambda x, y: oracle.strassen_winograd(x, y),
        "WinogradOriginal": oracle.winograd_original,
        "WinogradScaled": lambda x, y: oracle.winograd_scaled(x, y)[0],
    }
    try:
        cores = sorted(os.sched_getaffinity(0))
    except AttributeError:
        cores = []
    pin = len(cores) >= len(methods)
    table = {}
    for n in sizes:
        a, b = S.paper_pair(n, S.stream_seed(5, n))
        results, times = {}, {}

        def work(idx, name, fn):
            if pin:
                os.sched_setaffinity(0, {cores[idx]})  # the calling thread only
            t0 = time.perf_counter()
            for _ in range(repeats):
                c = fn(a, b)
            times[name] = (time.perf_counter() - t0) / repeats
            results[name] = c

        ths = [threading.Thread(target=work, args=(i, nm, fn)) for i, (nm, fn) in enumerate(methods.items())]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        ref = results["NaivKahan (N)"]
        table[str(n)] = {nm: {"time_s": times[nm], "gflops": 2.0 * n ** 3 / times[nm] / 1e9,
                              "norm_inf_N_minus_C": oracle.norm_inf(np.asarray(ref) - np.asarray(results[nm]))}
                         for nm in methods}
    if pin:
        os.sched_setaffinity(0, set(cores))
    return {"workload": "C = A (8A), A uniform [-1, 1]", "repeats": repeats, "time": "mean of one product",
            "threads": f"{len(methods)} methods at once, one thread each" + (", pinned to own cores" if pin else ""),
            "host_cores": host_cores(), "n": table}


def compact_line(core, sections):
    """The one JSON line the bench prints: the contract's keys (`core`) plus a
    short summary of each section; every section in full goes to the detail
    file.  Stays a few KB whatever the sections hold."""
    def get(d, *path):
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def rnd(x, n=4):
        return float(f"{x:.{n}g}") if isinstance(x, float) else x

    line = dict(core)
    e2e = sections.get("e2e")
    if e2e:
        line["e2e"] = {k: e2e[k] for k in ("value", "unit", "ms_per_step", "ms_mean", "ms_min", "ms_max", "steps",
                                          "statistic", "h2d_bytes_per_step", "d2h_bytes_per_step", "call")
                       if k in e2e}
    if "cpu_baseline" in sections:
        cb = sections["cpu_baseline"]
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample") if k in cb}
    summary = {}
    if "plain_fp64" in sections:
        pf = sections["plain_fp64"]
        summary["plain_fp64"] = {k: rnd(pf[k]) for k in ("value", "unit", "ms", "rel_inf_err_sampled",
                                                           "fp64_pipe_frac") if k in pf}
    if "accuracy" in sections:
        summary["accuracy"] = {k: sections["accuracy"][k] for k in ("rel_inf_err_sampled", "target")}
    if "fp64_peak" in sections:
        fp = sections["fp64_peak"]
        summary["fp64_peak_tflops"] = {"dfma": rnd(fp["dfma_tflops"]), "dmma": rnd(fp["dmma_tflops"]),
                                       "sm_mhz": get(fp, "clocks", "sm_mhz")}
    sv = sections.get("serving")
    if sv:
        lfl = sv.get("like_for_like_1e-14", {})
        summary["serving"] = {
            "requests": sv.get("requests"),
            "saturated_rps": rnd(get(sv, "saturated", "requests_per_s")),
            "paced_0.7x": {"p50_ms": rnd(get(sv, "paced", "p50_ms")), "p99_ms": rnd(get(sv, "paced", "p99_ms"))},
            "1e-14_fp64_one_at_a_time": {"p50_ms": rnd(get(lfl, "fp64_one_at_a_time", "paced", "p50_ms")),
                                         "p99_ms": rnd(get(lfl, "fp64_one_at_a_time", "paced", "p99_ms")),
                                         "saturated_rps": rnd(get(lfl, "fp64_one_at_a_time",
                                                                  "saturated_requests_per_s"))},
            "1e-14_emulated": {"p50_ms": rnd(get(lfl, "emulated", "paced", "p50_ms")),
                               "p99_ms": rnd(get(lfl, "emulated", "paced", "p99_ms")),
                               "saturated_rps": rnd(get(lfl, "emulated", "saturated_requests_per_s"))},
            "1e-14_emulated_at_fp64_rate": {"p50_ms": rnd(get(lfl, "emulated_at_fp64_rate", "p50_ms")),
                                            "p99_ms": rnd(get(lfl, "emulated_at_fp64_rate", "p99_ms"))},
        }
    gv = sections.get("grouped_vs_single")
    if gv:
        summary["grouped_256"] = {"tflops": rnd(get(gv, "grouped", "tflops")),
                                  "one_call_each_tflops": rnd(get(gv, "one_call_each", "tflops"))}
    at = sections.get("autotuner")
    if at:
        summary["autotuner"] = {k: v.get("depth") for k, v in at.get("strassen", {}).items()}
    sh = sections.get("shape_4096x16384x4096")
    if sh:
        summary["shape_4096x16384x4096_tflops"] = rnd(sh.get("tflops"))
    se = sections.get("strassen_over_emulated")
    if se:
        summary["strassen_winograd_1_over_emulated_8192_tflops"] = rnd(get(se, "8192", "strassen_winograd_1",
                                                                            "tflops"))
    if summary:
        line["summary"] = summary
    return line


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1106_1347_gb300 as mm
    from paper_1106_1347_gb300 import build as mmbuild

    rank, world, local = dist_env()
    serving = None
    if world == 1 and not args.quick and not args.no_serve:
        # The serving benchmark runs first, in a process of its own, before this
        # one opens a CUDA context: another process holding an idle context (20 GB
        # on the device, 2 GB pinned) doubled the serving loop's p99 (0.7x: 6.1 ->
        # 12.1 ms; 0.3x: 2.2 -> 4.5 ms), and this process holds far more later.
        serving = serve_in_own_process(local, args)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mmbuild.build()
    a, b = make_inputs()
    ta = torch.from_numpy(a).to(dev)
    tb = torch.from_numpy(b).to(dev)
    c = torch.empty((N, M), dtype=torch.float64, device=dev)
    ws_bytes = mm.lib().mm_emulated_workspace_bytes(N, P, M, KIND, SLICES, 1e-14)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = mm.lib()
    import ctypes

    def step(out=c):
        rc = lib.mm_emulated(N, P, M, ctypes.c_void_p(ta.data_ptr()), P, ctypes.c_void_p(tb.data_ptr()), M,
                             ctypes.c_void_p(out.data_ptr()), M, KIND, SLICES, 1e-14, ctypes.c_void_p(ws.data_ptr()),
                             ws_bytes, ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise RuntimeError(lib.mm_last_error().decode())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk, mm.profile() as prof:
        torch.cuda.synchronize()
        e0.record(stream)
        marks[0].record(stream)
        for i in range(args.steps):
            step()
            marks[i + 1].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    per_step = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    flop = 2.0 * N * P * M
    value = whole_job_tflops(flop, args.steps, world, ms)

    # Dominant kernel against its roofline (events bracket each launch on its stream).
    launches, kms = prof.stats.get(DOMINANT, (0, 0.0))
    pairs = SLICES * (SLICES + 1) // 2
    pk, pk_kind = peaks()
    tensor_flop_per_launch = pairs * flop
    achieved = tensor_flop_per_launch / (kms / max(launches, 1) * 1e-3) / 1e12 if launches else None
    # The burst figure was taken at the maximum SM clock, the sustained one under the
    # power cap: take the one whose conditions the clock record of this run matches.
    clk_rec = clk.summary()
    capped = ("sw_power_cap" in clk_rec["reasons"] or
              (clk_rec["sm_mhz"] is not None and
               clk_rec["sm_mhz"] < 0.95 * (clk_rec["sm_max_mhz"] or pk.get("sm_max_mhz") or 0)))
    peak_key = "bf16_tflops_sustained" if capped else "bf16_tflops"
    peak = pk.get(peak_key) or pk.get("bf16_tflops")
    other_key = "bf16_tflops" if capped else "bf16_tflops_sustained"
    other = pk.get(other_key)
    peak_source = f"{pk_kind} {peak_key} (clocks during the run: " + \
        ("power-capped or below max)" if capped else "at max SM clock, no power cap)")
    if KIND == 1:  # FP8: the measured BF16 peak times the nominal FP8/BF16 ratio (4.5 / 2.25)
        peak, peak_source = 2.0 * peak, peak_source + " x 2 (nominal FP8/BF16 ratio)"
        other = 2.0 * other if other else None
    fmt = "FP8-E4M3" if KIND == 1 else "BF16"
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": dominant_traffic() if KIND == 0 else None,
                "kernel": DOMINANT, "peak_source": peak_source,
                f"frac_of_{other_key}": (achieved / other) if (achieved and other) else None,
                "algorithmic_unit": f"{pairs} slice pairs x 2NPM {fmt} flops per launch"}
    gpu_launches = sum(v[0] for v in prof.stats.values())
    kernel_ms = {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.stats.items()}

    out = {}
    rows = np.arange(0, N, N // 4)[:4]
    if not args.quick:
        # End to end through the C ABI with host buffers (mm_emulated_host), on
        # every rank with its own pinned A, B, C: the copies of A and B up and of
        # C back run inside the call, overlapped with the products of other row
        # blocks.  Per-step events; each rank's value is its median step (the
        # paper's statistic: the host link sees sporadic stalls of several ms that
        # a mean of ten steps would carry), and the whole job's is the slowest
        # rank's.
        ha = torch.from_numpy(a).pin_memory()
        hb = torch.from_numpy(b).pin_memory()
        hc = torch.empty((N, M), dtype=torch.float64).pin_memory()
        hws_bytes = lib.mm_emulated_host_workspace_bytes(N, P, M, 0, SLICES, 1e-14)
        hws = torch.empty(hws_bytes, dtype=torch.uint8, device=dev)

        def e2e_step():
            rc = lib.mm_emulated_host(N, P, M, ctypes.c_void_p(ha.data_ptr()), P, ctypes.c_void_p(hb.data_ptr()), M,
                                      ctypes.c_void_p(hc.data_ptr()), M, 0, SLICES, 1e-14,
                                      ctypes.c_void_p(hws.data_ptr()), hws_bytes, ctypes.c_void_p(stream.cuda_stream))
            if rc != 0:
                raise RuntimeError(lib.mm_last_error().decode())

        e2e_steps = max(10, min(20, args.steps))
        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        gm = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
        with ClockSampler(local) as clk_e2e:
            gm[0].record(stream)
            for i in range(e2e_steps):
                e2e_step()
                gm[i + 1].record(stream)
            torch.cuda.synchronize()
        e2e_each = [gm[i].elapsed_time(gm[i + 1]) for i in range(e2e_steps)]
        e2e_ms = max_over_ranks(statistics.median(e2e_each), dev)
        if not np.array_equal(hc[rows].numpy(), c[rows].cpu().numpy()):
            raise RuntimeError("host-operand product differs from the device call")
        out["e2e"] = {"value": whole_job_tflops(flop, 1, world, e2e_ms), "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                      "steps": e2e_steps,
                      "statistic": "median of per-step CUDA-event times" + (", slowest rank" if world > 1 else ""),
                      "ms_mean": statistics.mean(e2e_each), "ms_min": min(e2e_each), "ms_max": max(e2e_each),
                      "ms_each": [round(x, 3) for x in e2e_each], "clocks": clk_e2e.summary(),
                      "h2d_bytes_per_step": int(world * (a.nbytes + b.nbytes)),
                      "d2h_bytes_per_step": int(world * N * M * 8),
                      "call": "mm_emulated_host (pinned host A, B, C; copies overlapped with row-block products)"}
        del hws, ha, hb, hc
        torch.cuda.empty_cache()

    # Single-GPU sections (rank 0 of a one-rank run): accuracy, the plain FP64
    # product, the other configurations, serving and the CPU baseline.
    if rank == 0 and world == 1 and not args.quick:
        norm_a = float(mm.norm_inf(ta).item())
        norm_b = float(mm.norm_inf(tb).item())
        import oracle

        truth = oracle.dot2_product(a[rows], b)
        err_emu = sampled_error(c, a, b, norm_a, norm_b, rows, truth)
        cn = torch.empty_like(c)
        mm.naive(ta, tb, out=cn)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(2):
            mm.naive(ta, tb, out=cn)
        f1.record(stream)
        torch.cuda.synchronize()
        plain_ms = f0.elapsed_time(f1) / 2
        err_plain = sampled_error(cn, a, b, norm_a, norm_b, rows, truth)
        out["plain_fp64"] = {"value": flop / (plain_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms": plain_ms,
                             "kernel": "gemm_f64_dmma (mma.sync m8n8k4 f64)", "rel_inf_err_sampled": err_plain}
        out["accuracy"] = {"rel_inf_err_sampled": err_emu, "rows_sampled": [int(r) for r in rows],
                           "target": 1e-14, "reference": "oracle Dot2 product on the sampled rows"}
        del cn

        # The FP64 pipe's own rate, measured here (denominator of the FP64 fractions).
        out["fp64_peak"] = fp64_peak(local)
        pk64 = out["fp64_peak"]["dmma_tflops"]
        out["plain_fp64"]["fp64_pipe_frac"] = out["plain_fp64"]["value"] / pk64 if pk64 else None
        out["plain_fp64"]["fp64_pipe_frac_against"] = "mma.sync f64 probe"

        if serving is not None:
            out["serving"] = serving
        if args.variants_n > 0:
            out["fp64_methods"] = variants_bench(dev, out["fp64_peak"])
            out["paper_table"] = paper_table(dev)
        if not args.no_configs:
            out["slice_sweep"] = slice_sweep(ta, tb, a, b, norm_a, norm_b, rows, truth)
            out["shape_4096x16384x4096"] = tall_inner_shape(dev)
            out["badly_scaled_2048"] = badly_scaled_errors(dev)
            out["grouped_vs_single"] = grouped_vs_single(dev)
            out["autotuner"] = autotuner(dev)
            out["strassen_over_emulated"] = strassen_over_emulated(ta, tb, a, b, norm_a, norm_b, rows, truth)
            torch.cuda.empty_cache()

        cores = host_cores()
        v, rows_used, thr, el = cpu_oracle_tflops(a, b, args.cpu_seconds, cores)
        v1, rows1, _, el1 = cpu_oracle_tflops(a, b, min(4.0, args.cpu_seconds), 1)
        out["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
                               "sample": f"{rows_used} of {N} rows of C (NaivStandard, plain C), {el:.1f} s",
                               "single_thread": {"value": v1, "unit": "TFLOP/s", "cores": 1,
                                                 "sample": f"{rows1} rows of C, {el1:.1f} s (the paper-like figure)"}}
        if not args.no_cpu_table and args.variants_n > 0:
            out["paper_table_cpu"] = paper_table_cpu(repeats=args.cpu_table_repeats)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    core = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "step_ms": {"median": statistics.median(per_step), "min": min(per_step), "max": max(per_step)},
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp8" if KIND == 1 else "bf16", "data": "synthetic",
        "precision": (f"{SLICES} {fmt} slices, exact FP32 TMEM chunks, exact int64 recombination"
                      + ("" if KIND == 1 else " (FP64-accurate)")),
        "config": {"workload": WORKLOAD, "N": N, "P": P, "M": M, "slices": SLICES, "beta": 5 if KIND == 1 else 7,
                   "parallelism": "replicas" if world > 1 else "single", "l2": "inputs (1 GiB) larger than L2"},
        "roofline": roofline,
        "kernel_ms_per_launch": kernel_ms, "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
    }
    if "fp64_peak" in out:
        pk64 = out["fp64_peak"]["dmma_tflops"]
        core["vs_fp64_peak"] = {"fp64_peak_tflops": pk64, "ratio": value / world / pk64 if pk64 else None,
                                "note": "2NPM/t per GPU against the FP64 rate measured in this run (mm_probe_fp64_peak)"}
    line = compact_line(core, out)
    detail = dict(line)
    detail.update(out)
    detail["step_ms_each"] = [round(x, 4) for x in per_step]
    try:
        with open(args.detail, "w") as f:
            json.dump(detail, f, indent=1)
        line["detail"] = os.path.relpath(args.detail, ROOT)
    except OSError as exc:
        print(f"bench: could not write {args.detail}: {exc}", file=sys.stderr)
    print(json.dumps(line), flush=True)


def serve_in_own_process(local, args):
    """The serving benchmark in a process of its own, as a server would run: a
    long-lived benchmark process (tens of GB of allocations behind it) showed
    sporadic host-side stalls of 30-100 ms that a fresh process does not, and
    the serving loop's latencies are host-driven.  Same GPU, same trace."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only", "--serve-requests", str(args.serve_requests),
           "--serve-budget-gb", str(args.serve_budget_gb),
           "--serve-baseline-requests", str(args.serve_baseline_requests)]
    visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=visible.split(",")[local] if visible else str(local))
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"serving benchmark failed:\n{r.stderr[-4000:]}")
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["process"] = "own process (bench.py --serve-only), same GPU"
    return res


def main():
    args = parse()
    if args.serve_only:
        import torch

        from paper_1106_1347_gb300 import build as mmbuild

        mmbuild.build()
        print(json.dumps(serve_bench(torch.device("cuda", 0), args.serve_requests, args.serve_budget_gb,
                                     args.serve_baseline_requests)), flush=True)
        return
    if args.fp64_only:
        import torch

        from paper_1106_1347_gb300 import build as mmbuild

        mmbuild.build()
        # profiling runs: every FP64 method once (after one warm-up) at n = --n
        print(json.dumps(variants_bench(torch.device("cuda", 0), fp64_peak(0), (args.n,), reps=1)), flush=True)
        return
    if args.method:
        import torch

        import paper_1106_1347_gb300 as mm
        import synthetic as S
        from paper_1106_1347_gb300 import build as mmbuild

        mmbuild.build()
        calls = {"naive": lambda a, b: mm.naive(a, b), "kahan": lambda a, b: mm.kahan(a, b),
                 "naive_unrolled_4": lambda a, b: mm.naive_unrolled(a, b, unroll=4),
                 "winograd": lambda a, b: mm.winograd(a, b), "strassen": lambda a, b: mm.strassen(a, b),
                 "strassen_winograd": lambda a, b: mm.strassen_winograd(a, b),
                 "strassen_paper": lambda a, b: mm.strassen(a, b, cutoff=0),
                 "strassen_winograd_paper": lambda a, b: mm.strassen_winograd(a, b, cutoff=0),
                 "strassen_emulated_1": lambda a, b: mm.strassen_emulated(a, b, variant=1, levels=1, nslices=8),
                 "emulated_8": lambda a, b: mm.emulated(a, b, nslices=8)}
        if args.method not in calls:
            raise SystemExit(f"unknown --method {args.method}")
        n = args.n
        if "emulated" in args.method:  # the bench's log-uniform inputs
            a = torch.from_numpy(S.loguniform(n, n, S.stream_seed(3, 0))).cuda()
            b = torch.from_numpy(S.loguniform(n, n, S.stream_seed(3, 1))).cuda()
        else:
            a = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 0))).cuda()
            b = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 1))).cuda()
        fn = calls[args.method]
        ms = timed(lambda: fn(a, b), 1)
        print(json.dumps({"method": args.method, "n": n, "ms": ms, "tflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e12}),
              flush=True)
        return
    if args.grouped_only:
        import torch

        from paper_1106_1347_gb300 import build as mmbuild

        mmbuild.build()
        print(json.dumps(grouped_vs_single(torch.device("cuda", 0), args.grouped_only)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
