"""Benchmark: useful TFLOP/s of the block-sparse product on one GB300 per rank.

Workload (one step = one pass of the whole device path: tile exponents, slicing,
tensor-core contraction, recombination and epilogue): the dense square product
of order 16384 with nonuniform block sizes drawn uniform-integer in [64, 256] on
rows, columns and inner dimension, entries U[-1,1] in FP64 -- the paper's
nonuniformly blocked square matrices (Sec. 4.1) at single-GPU scale. The headline
path is the 6-slice split-bfloat16 mode (FP32 tensor-core accumulation, FP64
recombination); the plain FP64 path is timed beside it on the same inputs, and
the split result is compared with it (the FP64 path reproduces the CPU oracle bit
for bit, so that error is the error against the oracle).

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the product does not need
any exchange between GPUs); the reported value is the sum over ranks divided by
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "useful TFLOP/s (nonzero-tile flops) & % of peak; split vs FP64 at <=1e-11 rel err"
PROFILE_FILE = os.path.join(ROOT, "profiles", "split_mma_kernel_nonuniform_dense.txt")
# exponents, scales, scale classes, slices, contraction
def kernels_per_execute(P, plan, mode, split_scale=0):
    """Kernels one bsmm_execute launches: FP64 the tile kernel; split modes the exponent
    (and line exponent), scale, class, pack and contraction kernels; plus the split-k
    reduction when the plan cut a k-list."""
    red = int(P.bsmm_plan_ksplit(plan)["n_regions"] > 0)
    return (1 if mode == P.BSMM_FP64 else 5 + int(split_scale)) + red


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=16384, help="matrix order")
    ap.add_argument("--single-n", type=int, default=0,
                    help="banded / clustered / uniform / thin workloads: another order (small cases for profiling; "
                         "0 = the workload's own)")
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--cluster", type=int, default=-1,
                    help="split modes: CTAs per column-block group (-1 = the planner's choice, 0 = library "
                         "default 1; batches use the default)")
    ap.add_argument("--store-warps", type=int, default=0, choices=[0, 1, 2],
                    help="split modes: contraction kernel with C store warps (0 = library's choice, 1 = never, "
                         "2 = always)")
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-cublas", action="store_true",
                    help="dense workload: skip the cuBLAS DGEMM reference point (torch.matmul float64)")
    ap.add_argument("--no-learned", action="store_true",
                    help="dense workload: skip the learned-schedule comparison on the clustered workload")
    ap.add_argument("--workload", default="dense", choices=["dense", "batch", "uniform", "banded", "banded_wide",
                                                                "clustered", "thin"],
                    help="dense: the 16384 nonuniform dense product (headline); batch: 256 independent products of "
                         "uneven size, separate launches vs one graph-replayed batch launch, before and after "
                         "autotuning; uniform: N=2048, blocks 128, Bernoulli(0.5) masks (FP64 path); banded / "
                         "banded_wide: N=32768 band |i-j|<=6 with distance-decaying values (FP64 vs split-fp16); "
                         "clustered: M=N=24576, K=49152 clustered masks, learned vs flop-count schedule; thin: "
                         "M=N=512, K=524288 dense (few C tiles, long inner sums), split k against uncut k-lists")
    ap.add_argument("--ksplit", type=int, default=0,
                    help="split k for every plan: 0 = the library's automatic choice (split modes only), "
                         "-1 = automatic in FP64 mode too, 1 = never, n = n pieces")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--split-scale", default="tile", choices=["tile", "rows"],
                    help="split modes: one power-of-two scale per tile, or per row of A and column of B")
    ap.add_argument("--trans", default="none", choices=["none", "a", "b", "ab"],
                    help="dense workload: supply A and/or B as the transposed block matrix (C = A'^T B, A B'^T)")
    ap.add_argument("--other-slices", type=int, nargs="*", default=[3, 4, 5],
                    help="slice counts also timed on the dense workload, each with its error against FP64")
    ap.add_argument("--c128-slices", type=int, nargs="*", default=[6],
                    help="dense workload: slice counts timed with complex elements on the N/2 nonuniform dense "
                         "product (same flops per element pair x4), each with its error against cuBLAS ZGEMM")
    ap.add_argument("--f32-slices", type=int, nargs="*", default=[4, 6],
                    help="dense workload: slice counts timed with float32 elements (the same values rounded "
                         "to float32), each with its error against the FP64 result")
    return ap.parse_args()


def workload_name(n):
    return f"nonuniform_dense N={n} blocks U-int[64,256] (rows=cols=inner), dense masks, U[-1,1] FP64"


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def kernel_source_hash():
    """Hash of the contraction kernel's sources with comments and blank space removed, so a
    comment-only edit keeps the recorded DRAM counters valid and a code edit does not."""
    h = hashlib.sha256()
    for f in ("split.cu", "bsmm_internal.h"):
        with open(os.path.join(ROOT, "paper_1504_05046_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the contraction kernel from the committed ncu summary,
    valid only while the kernel source is unchanged since the capture."""
    try:
        vals = {}
        with open(PROFILE_FILE) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_hash") != kernel_source_hash():
            return None
        return float(vals["dram_bytes_per_full_launch"])
    except Exception:
        return None


def aggregate(t, work, device):
    """Whole-job figures over the ranks of an initialised process group (else this
    rank's): the slowest rank's time and the summed work."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t), float(work)
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    ww = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ww.item())


def make_inputs(n, seed):
    import bsmm_gen as G
    prob = G.make_problem("nonuniform_dense", seed, n, lo=64, hi=256)
    return prob


def run_reference(args, rank):
    """The CPU oracle as it stands, on the host cores: each step computes a bounded
    sample (whole C tile rows of the workload) and reports useful TFLOP/s."""
    import bsmm_gen as G
    import oracle
    prob = make_inputs(args.n, args.seed)
    cs, _, _ = oracle.structure(prob)
    rows = pick_rows(prob, 1)
    sub, subcs = row_subproblem(prob, cs, rows)
    off, tot = G.layout_arena(subcs, sub.row_sizes, sub.col_sizes)
    _, _, fl = oracle.structure(sub)
    C = np.zeros(tot)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.bsmm(sub, subcs, C, off)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    tot_t = sum(times)
    val = fl * len(times) / tot_t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.n), "sample": f"C tile row {rows[0]} of {prob.M} "
                       f"({sub.row_sizes.sum()} rows x {prob.col_sizes.sum()} cols, full inner dim)"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"one C tile row per step ({fl / 1e9:.1f} GFLOP)"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def pick_rows(prob, count):
    return list(range(min(count, prob.M)))


def row_subproblem(prob, cs, rows):
    """The C tile rows `rows` of the product as a problem of its own (same inner and
    column tilings, the A tiles of those rows)."""
    import bsmm_gen as G
    r = prob.row_sizes[rows]
    am = prob.a_mask[rows]
    a_off, a_tot = G.layout_arena(am, r, prob.inner_sizes)
    A = np.zeros(a_tot)
    for ii, i in enumerate(rows):
        for k in range(prob.K):
            if am[ii, k]:
                n = int(r[ii]) * int(prob.inner_sizes[k])
                A[a_off[ii, k]:a_off[ii, k] + n] = prob.A[prob.a_off[i, k]:prob.a_off[i, k] + n]
    sub = G.Problem(prob.name + "_rows", r, prob.col_sizes, prob.inner_sizes, am, prob.b_mask, a_off, prob.b_off, A,
                    prob.B, prob.alpha, prob.beta)
    return sub, cs[rows]


def cpu_baseline(prob, cs, Cgpu, c_off, seconds):
    """Oracle on host cores over whole C tile rows until `seconds` have passed; also
    returns the max relative error of the GPU result on those rows."""
    import bsmm_gen as G
    import oracle
    done_fl, done_t, errs, nrows = 0.0, 0.0, [], 0
    for i in range(prob.M):
        sub, subcs = row_subproblem(prob, cs, [i])
        off, tot = G.layout_arena(subcs, sub.row_sizes, sub.col_sizes)
        C = np.zeros(tot)
        _, _, fl = oracle.structure(sub)
        t0 = time.perf_counter()
        oracle.bsmm(sub, subcs, C, off)
        done_t += time.perf_counter() - t0
        done_fl += fl
        nrows += 1
        # compare with the GPU's row
        num = den = 0.0
        for j in range(prob.N):
            if subcs[0, j]:
                n = int(sub.row_sizes[0]) * int(prob.col_sizes[j])
                g = Cgpu[c_off[i, j]:c_off[i, j] + n]
                o = C[off[0, j]:off[0, j] + n]
                num += float(np.sum((g - o) ** 2))
                den += float(np.sum(o ** 2))
        errs.append((num / den) ** 0.5 if den else 0.0)
        if done_t >= seconds:
            break
    return {"value": done_fl / done_t / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nrows} C tile row(s) of {prob.M} ({done_fl / 1e9:.1f} GFLOP, full inner dimension), "
                      f"{done_t:.1f} s"}, max(errs) if errs else None


def run_batch(args, rank, world):
    """256 independent square products (n ~ U-int[512, 8192], blocks U-int[32, 192], one
    tile density d ~ U[0.1, 1] per product, U[-1,1] entries), 6-slice split-bfloat16:
    the whole batch per step, as 256 separate launches, as one persistent batch launch
    replayed from a CUDA graph with the default launch shape, and the same after the
    library's autotuner picked the shape."""
    import torch
    import bsmm_gen as G
    import paper_1504_05046_gb300 as P
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    t_gen = time.perf_counter()
    probs = G.make_batch(args.batch_count, args.seed + rank)
    t_gen = time.perf_counter() - t_gen
    s = args.slices
    plans, items = [], []
    F = 0.0
    for p in probs:
        pl = P.bsmm_plan(p.row_sizes, p.col_sizes, p.inner_sizes, p.a_mask, p.b_mask, mode=P.BSMM_SPLIT_BF16,
                         nslices=s, ksplit=args.ksplit)
        q = P.bsmm_plan_query(pl)
        F += q["useful_flops"]
        off, tot = G.layout_arena(q["c_mask"], p.row_sizes, p.col_sizes)
        d = lambda x: torch.from_numpy(x if x.size else np.zeros(2, x.dtype)).to(dev)
        items.append(dict(A=d(p.A), B=d(p.B), ao=d(p.a_off), bo=d(p.b_off), co=d(off),
                          C=torch.zeros(max(tot, 1), dtype=torch.float64, device=dev)))
        plans.append(pl)
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def separate():
        for pl, it in zip(plans, items):
            P.bsmm_execute(pl, 1.0, it["A"], it["ao"], it["B"], it["bo"], 0.0, it["C"], it["co"])

    batch = P.bsmm_batch_create(plans)
    P.bsmm_batch_set_args(batch, [1.0] * len(plans), [it["A"] for it in items], [it["ao"] for it in items],
                          [it["B"] for it in items], [it["bo"] for it in items], [0.0] * len(plans),
                          [it["C"] for it in items], [it["co"] for it in items])

    def capture():
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            P.bsmm_batch_execute(batch)
        torch.cuda.synchronize()
        return g

    for _ in range(args.warmup):
        separate()
    torch.cuda.synchronize()
    ms_sep = timed(separate, args.steps)
    g = capture()
    for _ in range(args.warmup):
        g.replay()
    ms_batch = timed(g.replay, args.steps)
    default_bins = P.bsmm_batch_query(batch)["bins"]
    t_tune = time.perf_counter()
    chosen, tune_ms = P.bsmm_batch_autotune(batch, reps=2)
    t_tune = time.perf_counter() - t_tune
    g = capture()
    for _ in range(args.warmup):
        g.replay()
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    ms_tuned = timed(g.replay, args.steps)
    clocks = clk.stop()
    ms_sep, _ = aggregate(ms_sep, 0.0, dev)
    ms_batch, _ = aggregate(ms_batch, 0.0, dev)
    ms_tuned, F = aggregate(ms_tuned, F, dev)
    P.bsmm_batch_status_device(batch)
    space = P.bsmm_tune_space(P.BSMM_SPLIT_BF16, s)
    tf = lambda ms: F / (ms * 1e-3) / 1e12
    launches_per_step = P.bsmm_batch_kernels(batch)
    line = {"metric": METRIC, "value": tf(ms_tuned), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_tuned, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"batch of {len(plans)} products, n ~ U-int[512,8192], blocks U-int[32,192], "
                                   f"density ~ U[0.1,1], U[-1,1] FP64", "mode": f"split_bf16 s={s}",
                       "useful_flops_per_step": F, "seed": args.seed, "generation_s": t_gen},
            "batch_graph_autotuned": {"value": tf(ms_tuned), "ms_per_step": ms_tuned, "chosen": chosen,
                                      "tuning_s": t_tune,
                                      "candidates_ms": {f"cluster={c['cluster']} stages={c['stages']} "
                                                        f"store_warps={c['store_warps']}": m
                                                        for c, m in zip(space, tune_ms)}},
            "batch_graph_default": {"value": tf(ms_batch), "ms_per_step": ms_batch, "bins": default_bins},
            "separate_launches": {"value": tf(ms_sep), "ms_per_step": ms_sep, "launches_per_step":
                                  sum(kernels_per_execute(P, pl, P.BSMM_SPLIT_BF16) for pl in plans)},
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))


SINGLE = {
    "uniform": dict(recipe="uniform_bernoulli", n=2048, kw=dict(block=128, density=0.5), mode="BSMM_SPLIT_BF16",
                    head="fp64", desc="uniform_bernoulli N=2048 blocks 128, Bernoulli(0.5) masks, U[-1,1] FP64, beta=0"),
    "banded": dict(recipe="banded_decay", n=32768, kw=dict(lo=32, hi=256, band=6), mode="BSMM_SPLIT_FP16", head="split",
                   desc="banded_decay N=32768 blocks U-int[32,256], |i-j|<=6, N(0,1)exp(-|i-j|/2)"),
    "banded_wide": dict(recipe="banded_decay_wide", n=32768, kw=dict(lo=32, hi=256, band=6), mode="BSMM_SPLIT_FP16",
                        head="split", desc="banded_decay_wide N=32768 blocks U-int[32,256], |i-j|<=6, "
                                           "N(0,1)exp(-2.3|i-j|)"),
    "clustered": dict(recipe="clustered", n=24576, kw=dict(lo=16, hi=512, nclusters=40, cluster_density=0.10),
                      mode="BSMM_SPLIT_BF16", head="split",
                      desc="clustered M=N=24576 K=49152, log-uniform blocks [16,512], 40 clusters at 10%, U[-1,1]"),
    "thin": dict(recipe="thin_dense", n=512, kw=dict(lo=64, hi=256, k_factor=1024), mode="BSMM_SPLIT_BF16",
                 head="split", desc="thin_dense M=N=512 K=524288, blocks U-int[64,256], dense, U[-1,1] "
                                    "(few C tiles, long inner sums)"),
}

# position of the contraction kernel in bsmm_plan_kernel_ms (the reduction, if any, follows)
CONTRACTION_INDEX = {"split": 2, "fp64": 0}


def fp64_roofline(P, pk, achieved):
    """The FP64 path against its unit count x clock (152 SMs x 2 FP64 FMA per clock x 2 flops
    x the maximum SM clock) and against the rates measured in this run on every SM (DFMA
    chains, the FP64 mma.sync, and for reference the INT8 mma.sync)."""
    rates = P.bsmm_measure_rates()
    peak = 152 * 2 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_def": "152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
            "measured_dfma_tflops": rates["dfma"], "frac_of_measured_dfma": achieved / rates["dfma"],
            "measured_dmma_tflops": rates["dmma"], "frac_of_measured_dmma": achieved / rates["dmma"],
            "measured_int8_mma_sync_tops": rates["imma"],
            "measured_def": "bsmm_measure_rates in this run: DFMA chains, FP64 mma.sync m8n8k4, INT8 mma.sync "
                            "m16n8k32, each on every SM"}


def timed_steps(plan, run, steps, warmup):
    """Mean step time (ms, CUDA events on the current stream) of `steps` runs after
    `warmup` untimed ones, and each kernel's mean device time over the timed runs (read
    once afterwards from the plan's events)."""
    import torch
    import paper_1504_05046_gb300 as P
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    P.bsmm_plan_kernel_ms(plan)  # the per-kernel means below cover the timed steps only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ks = P.bsmm_plan_kernel_ms(plan)
    P.bsmm_status_device(plan)
    return e0.elapsed_time(e1) / steps, ks


def learned_vs_flops(setup, seed, steps, warmup, dev):
    """The learned schedule against the flop-count schedule on one product: the cost model
    is trained on unit timings of three other inputs of the same recipe (3 timed runs
    each, 2000 Adam steps on the GPU), then the product is timed under both schedules.
    `setup(seed, **opt)` plans a product and returns (prob, plan, q, t, run). Returns the
    record, the product's (plan, t, run) under the learned schedule, its timing and the
    clocks sampled while it was timed."""
    import torch
    import paper_1504_05046_gb300 as P
    from paper_1504_05046_gb300 import costmodel as CM
    rows = []
    for ts in (seed + 101, seed + 102, seed + 103):
        _, tplan, _, _, trun = setup(ts, record_timings=1)
        trun()
        rows.append(CM.training_rows(tplan, CM.unit_times(tplan, trun, repeats=3)))
        del tplan
    mlp, loss = CM.fit(rows, steps=2000, lr=3e-3)
    prob, plan, q, t, run = setup(seed, record_timings=1)
    run()
    times = CM.unit_times(plan, run, repeats=3)
    CM.apply_flops(plan)
    ms_flops, k_flops = timed_steps(plan, run, steps, warmup)
    ref = t["C"].clone()
    CM.apply(plan, mlp)
    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    ms_mlp, k_mlp = timed_steps(plan, run, steps, warmup)
    clocks = clk.stop()
    same = bool((t["C"] == ref).all())
    feats, flops = P.bsmm_plan_features(plan)
    y = torch.zeros(len(feats), dtype=torch.float32, device=dev)
    P.bsmm_mlp_predict(mlp, torch.from_numpy(feats).to(dev), y)
    ci = CONTRACTION_INDEX["split"]
    rec = {"makespan_ms_flop_count": k_flops[ci], "makespan_ms_mlp": k_mlp[ci], "step_ms_flop_count": ms_flops,
           "step_ms_mlp": ms_mlp, "makespan_gain": 1.0 - k_mlp[ci] / k_flops[ci], "bits_identical": same,
           "train_loss": loss,
           "log_rms_err_flop_count": CM.prediction_error(plan, times, np.maximum(flops, 1.0)),
           "log_rms_err_mlp": CM.prediction_error(plan, times, np.exp(y.cpu().numpy().astype(np.float64))),
           "train_inputs": "3 other seeds of the same workload, 3 timed runs each",
           "timing": f"mean of {steps} steps after {warmup} warm-up steps, per schedule"}
    return rec, (prob, plan, q, t, run), (ms_mlp, k_mlp), clocks


def single_setup(args, w, dev):
    """setup(seed, mode, **opt) for one of the SINGLE workloads: the seeded product
    planned (profile events on) with its device arenas; returns (prob, plan, q, t, run)."""
    import torch
    import bsmm_gen as G
    import paper_1504_05046_gb300 as P

    def setup(seed, mode, **opt):
        if mode != P.BSMM_FP64:
            opt.setdefault("split_scale", int(args.split_scale == "rows"))
            opt.setdefault("cluster", args.cluster)
            opt.setdefault("store_warps", args.store_warps)
        opt.setdefault("ksplit", args.ksplit)
        prob = G.make_problem(w["recipe"], seed, args.single_n or w["n"], **w["kw"])
        plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask, mode=mode,
                           nslices=args.slices, profile=1, **opt)
        q = P.bsmm_plan_query(plan)
        off, tot = G.layout_arena(q["c_mask"], prob.row_sizes, prob.col_sizes)
        d = lambda x: torch.from_numpy(x if x.size else np.zeros(2, x.dtype)).to(dev)
        t = dict(A=d(prob.A), B=d(prob.B), ao=d(prob.a_off), bo=d(prob.b_off), co=d(off),
                 C=torch.zeros(max(tot, 1), dtype=torch.float64, device=dev))
        run = lambda: P.bsmm_execute(plan, 1.0, t["A"], t["ao"], t["B"], t["bo"], 0.0, t["C"], t["co"])
        return prob, plan, q, t, run
    return setup


def run_single(args, rank, world):
    """One of the other workloads: the split path (and, for the clustered one, the
    learned schedule against the flop-count schedule) and the FP64 path on the same
    inputs, each timed over the steps with CUDA events; the split result compared with
    the FP64 result over the whole C."""
    import torch
    import paper_1504_05046_gb300 as P
    w = SINGLE[args.workload]
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    s = args.slices
    mode = getattr(P, w["mode"])
    setup = single_setup(args, w, dev)

    def timed(plan, run, steps):
        return timed_steps(plan, run, steps, args.warmup)

    extra = {}
    seed = args.seed + rank
    if args.workload == "clustered":
        # learned schedule against the flop-count schedule (the split path's headline)
        rec, (prob, plan, q, t, run), (ms_split, k_split), clocks = learned_vs_flops(
            lambda sd, **o: setup(sd, mode, **o), seed, args.steps, args.warmup, dev)
        extra["learned_schedule"] = rec
    else:
        prob, plan, q, t, run = setup(seed, mode)
        clk = ClockSampler(dev.index)
        clk.start()
        time.sleep(0.3)
        ms_split, k_split = timed(plan, run, args.steps)
        clocks = clk.stop()
    Csplit = t["C"].clone()
    # FP64 takes automatic cuts only when asked (they change its rounding): the thin
    # workload asks, to show split k on both paths
    prob64, plan64, _, t64, run64 = setup(seed, P.BSMM_FP64,
                                          **({"ksplit": -1} if args.workload == "thin" and args.ksplit == 0 else {}))
    ms64, k64 = timed(plan64, run64, args.steps if w["head"] == "fp64" else max(1, args.fp64_steps))
    if args.workload == "thin":
        # split k (Sec. 3.2, Fig. 2) against uncut k-lists on the same inputs, both paths
        def uncut(mode, steps, ref, cut_plan, cut_ms):
            _, plan1, _, t1, run1 = setup(seed, mode, ksplit=1)
            ms1, k1 = timed(plan1, run1, steps)
            ks = P.bsmm_plan_ksplit(cut_plan)
            d = {"cut_ms": cut_ms, "uncut_ms": ms1, "speedup": ms1 / cut_ms, "regions_cut": ks["n_regions"],
                 "pieces": ks["n_pieces"], "units_cut": int(len(ks["pieces"])),
                 "units_uncut": int(P.bsmm_plan_query(plan1)["n_units"]), "uncut_kernel_ms": k1}
            if mode == P.BSMM_FP64:
                d["rel_diff_cut_vs_uncut"] = float(torch.linalg.norm(t1["C"] - ref) / torch.linalg.norm(t1["C"]))
            else:
                d["bits_identical_cut_vs_uncut"] = bool((t1["C"] == ref).all())
            del plan1, t1
            return d
        extra["split_k"] = {"split_path": uncut(mode, args.steps, Csplit, plan, ms_split),
                            "fp64_path": uncut(P.BSMM_FP64, max(1, args.fp64_steps), t64["C"], plan64, ms64)}
    ms_split, _ = aggregate(ms_split, 0.0, dev)
    ms64, F = aggregate(ms64, q["useful_flops"], dev)
    c64 = t64["C"]
    err = float(torch.linalg.norm(Csplit - c64) / torch.linalg.norm(c64))
    tf = lambda ms: F / (ms * 1e-3) / 1e12
    pk, pk_src = peaks()
    head_split = w["head"] == "split"
    cis, cif = CONTRACTION_INDEX["split"], CONTRACTION_INDEX["fp64"]
    split = {"value": tf(ms_split), "ms_per_step": ms_split, "kernel_ms": k_split,
             "mode": f"{w['mode'][5:].lower()} s={s}" + (", scale per row/column" if args.split_scale == "rows" else ""),
             "rel_err_vs_fp64": err}
    fp64 = {"value": tf(ms64), "ms_per_step": ms64, "kernel_ms": k64}
    pair = s * (s + 1) / 2 * F
    if head_split:
        roof = {"bound": "tensor", "kernel": "split_mma_kernel", "achieved": pair / (k_split[cis] * 1e-3) / 1e12,
                "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s", "traffic": None,
                "peak_source": f"{pk_src} bf16_tflops_sustained (MEASURED_PEAKS.json)",
                "launch": P.bsmm_plan_form(plan)}
    else:
        roof = dict(fp64_roofline(P, pk, F / (k64[cif] * 1e-3) / 1e12), kernel="fp64_tile_kernel", traffic=None)
    roof["frac"] = roof["achieved"] / roof["peak"]
    head = split if head_split else fp64
    line = {"metric": METRIC, "value": head["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if head_split and "BF16" in w["mode"] else
            ("f16" if head_split else "f64"), "data": "synthetic",
            "config": {"workload": w["desc"] + (f" (order {args.single_n} instead)" if args.single_n else ""),
                       "useful_flops_per_step": F, "seed": seed,
                       "headline_path": "split" if head_split else "fp64"},
            "split_path": split, "fp64_path": fp64, "roofline": roof, "gpu_launches":
                (kernels_per_execute(P, plan, mode, args.split_scale == "rows") if head_split
                 else kernels_per_execute(P, plan64, P.BSMM_FP64)) * args.steps, "clocks": clocks}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "batch":
        run_batch(args, rank, world)
    elif args.workload in SINGLE:
        run_single(args, rank, world)
    else:
        run_dense(args, rank, world, local)
    if world > 1:
        dist.destroy_process_group()


def densify(torch, arena_t, offs, rows, cols, dev):
    """Gather a tile-by-tile arena into the dense matrix (a library reference point's input,
    not part of the measured path); tiles absent from offs (-1) stay zero."""
    ro = np.concatenate([[0], np.cumsum(rows.astype(np.int64))])
    cc = np.concatenate([[0], np.cumsum(cols.astype(np.int64))])
    out = torch.zeros((int(ro[-1]), int(cc[-1])), dtype=arena_t.dtype, device=dev)
    for u in range(len(rows)):
        for v in range(len(cols)):
            if offs[u, v] < 0:
                continue
            nn = int(rows[u]) * int(cols[v])
            out[ro[u]:ro[u + 1], cc[v]:cc[v + 1]] = arena_t[offs[u, v]:offs[u, v] + nn].view(int(rows[u]), int(cols[v]))
    return out


def cublas_dgemm_line(P, torch, prob, A, B, C64, c_off, dev, stream):
    """cuBLAS DGEMM (torch.matmul float64) of the densified operands of the dense product: a
    library reference point for the FP64 path, with its error against that path's result
    and cuBLAS's FP64 emulation setting as the environment gives it."""
    Ad = densify(torch, A, prob.a_off, prob.row_sizes, prob.inner_sizes, dev)
    Bd = densify(torch, B, prob.b_off, prob.inner_sizes, prob.col_sizes, dev)
    Cd = torch.matmul(Ad, Bd)  # warm-up
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    torch.matmul(Ad, Bd, out=Cd)
    g1.record(stream)
    torch.cuda.synchronize()
    ms = g0.elapsed_time(g1)
    del Ad, Bd
    ref = densify(torch, C64, c_off, prob.row_sizes, prob.col_sizes, dev)
    err = float(torch.linalg.norm(Cd - ref) / torch.linalg.norm(ref))
    del Cd, ref
    n = int(prob.row_sizes.sum()), int(prob.inner_sizes.sum()), int(prob.col_sizes.sum())
    flops = 2.0 * n[0] * n[1] * n[2]
    return {"value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms": ms,
            "rel_err_vs_fp64_path": err,
            "emulation": os.environ.get("CUBLAS_EMULATION_STRATEGY", "unset (cuBLAS default)"),
            "what": "torch.matmul float64 of the densified dense operands, one timed call after one "
                    "warm-up; a library reference point, not part of the measured path"}


def complex_line(args, P, G, torch, dev, stream):
    """Complex elements on the N/2 nonuniform dense product: split-mode throughput in
    useful flops (8 r c q per triple) and the error against cuBLAS ZGEMM of the dense
    operands (a library reference point, not part of the measured path)."""
    n2 = args.n // 2
    pc = G.as_complex(make_inputs(n2, args.seed + 7), args.seed + 7)
    d = lambda x: torch.from_numpy(x).to(dev)
    Ac, Bc, ao, bo = d(pc.A), d(pc.B), d(pc.a_off), d(pc.b_off)
    cs = np.ones((pc.M, pc.N), np.uint8)
    off, tot = G.layout_arena(cs, pc.row_sizes, pc.col_sizes)
    co = d(off)
    # dense reference: the arenas are tile by tile; gather them into dense matrices
    dense = lambda arena_t, offs, rows, cols: densify(torch, arena_t, offs, rows, cols, dev)
    ref = dense(Ac, pc.a_off, pc.row_sizes, pc.inner_sizes) @ dense(Bc, pc.b_off, pc.inner_sizes, pc.col_sizes)
    out = {"workload": f"nonuniform_dense N={n2} blocks U-int[64,256], complex128 entries (re and im U[-1,1])"}
    for s2 in args.c128_slices:
        plan = P.bsmm_plan(pc.row_sizes, pc.col_sizes, pc.inner_sizes, pc.a_mask, pc.b_mask,
                           mode=P.BSMM_SPLIT_BF16, nslices=s2, elem=P.BSMM_C128, profile=1)
        F = P.bsmm_plan_query(plan)["useful_flops"]
        C = torch.zeros(tot, dtype=torch.complex128, device=dev)
        for _ in range(2):
            P.bsmm_execute(plan, 1.0, Ac, ao, Bc, bo, 0.0, C, co)
        P.bsmm_plan_kernel_ms(plan)  # kernel means over the timed executes only
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(3):
            P.bsmm_execute(plan, 1.0, Ac, ao, Bc, bo, 0.0, C, co)
        g1.record(stream)
        torch.cuda.synchronize()
        P.bsmm_status_device(plan)
        ms = g0.elapsed_time(g1) / 3
        got = dense(C, off, pc.row_sizes, pc.col_sizes)
        err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        out[f"s={s2}"] = {"value": F / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms,
                          "useful_flops_per_step": F, "rel_err_vs_zgemm": err,
                          "kernel_ms": P.bsmm_plan_kernel_ms(plan)}
        del plan, C
    return out


def run_dense(args, rank, world, local):
    """The headline workload: the 16384 nonuniform dense product, 6-slice split-bf16."""
    import torch
    import torch.distributed as dist
    import bsmm_gen as G
    import paper_1504_05046_gb300 as P

    def barrier():
        if world > 1:
            dist.barrier()

    prob0 = make_inputs(args.n, args.seed + rank)
    ta, tb = "a" in args.trans, "b" in args.trans
    prob = G.transposed_storage(prob0, ta, tb) if (ta or tb) else prob0
    tr = dict(transa=int(ta), transb=int(tb))
    sc = dict(split_scale=int(args.split_scale == "rows"))
    s = args.slices
    plan = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                       mode=P.BSMM_SPLIT_BF16, nslices=s, profile=1, cluster=args.cluster, ksplit=args.ksplit, **tr,
                       store_warps=args.store_warps, **sc)
    q = P.bsmm_plan_query(plan)
    F = q["useful_flops"]
    cs = q["c_mask"]
    c_off, c_tot = G.layout_arena(cs, prob.row_sizes, prob.col_sizes)
    dev = torch.device("cuda", local)
    A = torch.from_numpy(prob.A).to(dev)
    B = torch.from_numpy(prob.B).to(dev)
    ao = torch.from_numpy(prob.a_off).to(dev)
    bo = torch.from_numpy(prob.b_off).to(dev)
    co = torch.from_numpy(c_off).to(dev)
    C = torch.zeros(c_tot, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
    torch.cuda.synchronize()
    P.bsmm_status_device(plan)

    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    P.bsmm_plan_kernel_ms(plan)  # start the per-kernel means at the first timed step
    per_step = kernels_per_execute(P, plan, P.BSMM_SPLIT_BF16, sc["split_scale"])
    # an event between consecutive steps as well (recording one adds no wait), for the
    # median and spread of the step times beside the mean over the whole timed region
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = ev[0], ev[-1]
    launches = 0
    e0.record(stream)
    for i in range(args.steps):
        P.bsmm_execute(plan, 1.0, A, ao, B, bo, 0.0, C, co)
        launches += per_step
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    # each kernel's mean device time over the timed steps, from the events the library
    # recorded around its launches on this stream (read once, after the timed region)
    kms = [P.bsmm_plan_kernel_ms(plan)]
    ms = e0.elapsed_time(e1) / args.steps
    steps_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms_max, F_all = aggregate(ms, F, dev)
    value = F_all / (ms_max * 1e-3) / 1e12
    P.bsmm_status_device(plan)
    Csplit = C.cpu().numpy()

    # per-kernel live times (CUDA events on the launching stream)
    kk = np.array(kms)
    k_names = ["split_exp_scale_class_kernels", "split_pack_kernel", "split_mma_kernel"]
    k_avg = {nm: float(kk[:, i].mean()) for i, nm in enumerate(k_names)}
    t_mma = k_avg["split_mma_kernel"] * 1e-3
    pk, pk_src = peaks()
    pair_flops = s * (s + 1) / 2 * F
    mma_tflops = pair_flops / t_mma / 1e12
    peak_tc = pk["bf16_tflops_sustained"]
    traffic = profiled_traffic()
    roofline = {"bound": "tensor", "kernel": "split_mma_kernel", "achieved": mma_tflops, "peak": peak_tc,
                "unit": "TFLOP/s", "frac": mma_tflops / peak_tc, "traffic": traffic,
                "peak_source": f"{pk_src} bf16_tflops_sustained (MEASURED_PEAKS.json)",
                "achieved_def": f"{s * (s + 1) // 2} slice-pair products x useful flops per launch / mean launch time",
                "kernel_ms": k_avg, "launch": P.bsmm_plan_form(plan)}
    if traffic:  # the recorded DRAM bytes per launch over this run's launch time, against the copy peak
        roofline["dram_gbs"] = traffic / t_mma / 1e9
        roofline["dram_frac_of_measured_copy_peak"] = roofline["dram_gbs"] / pk["hbm_gbs"]

    extra = {}
    if rank == 0 and not args.no_fp64:
        plan64 = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                             mode=P.BSMM_FP64, profile=1, **tr)
        C64 = torch.zeros_like(C)
        P.bsmm_execute(plan64, 1.0, A, ao, B, bo, 0.0, C64, co)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            P.bsmm_execute(plan64, 1.0, A, ao, B, bo, 0.0, C64, co)
        f1.record(stream)
        torch.cuda.synchronize()
        P.bsmm_status_device(plan64)
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        c64 = C64.cpu().numpy()
        d = Csplit - c64
        err = float(np.linalg.norm(d) / np.linalg.norm(c64))
        v64 = F / (ms64 * 1e-3) / 1e12
        extra["fp64_path"] = {"value": v64, "unit": "TFLOP/s", "ms_per_step": ms64,
                              "roofline": fp64_roofline(P, pk, v64)}
        extra["split_rel_err_vs_fp64"] = err
        extra["split_speedup_vs_fp64"] = ms64 / ms_max
        if not args.no_cublas and not (ta or tb):
            extra["cublas_dgemm"] = cublas_dgemm_line(P, torch, prob, A, B, C64, c_off, dev, stream)
        # the other slice counts on the same inputs: throughput and error against the FP64 result
        modes = {}
        for s2 in args.other_slices:
            if s2 == s:
                continue
            plan2 = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                                mode=P.BSMM_SPLIT_BF16, nslices=s2, cluster=args.cluster, **tr, **sc)
            C2 = torch.zeros_like(C)
            for _ in range(2):
                P.bsmm_execute(plan2, 1.0, A, ao, B, bo, 0.0, C2, co)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(3):
                P.bsmm_execute(plan2, 1.0, A, ao, B, bo, 0.0, C2, co)
            g1.record(stream)
            torch.cuda.synchronize()
            P.bsmm_status_device(plan2)
            ms2 = g0.elapsed_time(g1) / 3
            e2 = float(np.linalg.norm(C2.cpu().numpy() - c64) / np.linalg.norm(c64))
            modes[f"s={s2}"] = {"value": F / (ms2 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms2,
                                "rel_err_vs_fp64": e2, "bar": {3: 1e-5}.get(s2)}
            del plan2, C2
        extra["split_modes"] = modes
        # float32 elements (the same values rounded to float32): throughput and error against FP64
        if args.f32_slices and not (ta or tb):
            p32 = G.as_float32(prob)
            A32, B32 = torch.from_numpy(p32.A).to(dev), torch.from_numpy(p32.B).to(dev)
            ao32, bo32 = torch.from_numpy(p32.a_off).to(dev), torch.from_numpy(p32.b_off).to(dev)
            C32 = torch.zeros(c_tot, dtype=torch.float32, device=dev)
            f32 = {}
            for s2 in args.f32_slices:
                plan2 = P.bsmm_plan(prob.row_sizes, prob.col_sizes, prob.inner_sizes, prob.a_mask, prob.b_mask,
                                    mode=P.BSMM_SPLIT_BF16, nslices=s2, cluster=args.cluster, elem=P.BSMM_F32,
                                    profile=1, **sc)
                for _ in range(2):
                    P.bsmm_execute_f32(plan2, 1.0, A32, ao32, B32, bo32, 0.0, C32, co)
                P.bsmm_plan_kernel_ms(plan2)  # kernel means over the timed executes only
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                for _ in range(3):
                    P.bsmm_execute_f32(plan2, 1.0, A32, ao32, B32, bo32, 0.0, C32, co)
                g1.record(stream)
                torch.cuda.synchronize()
                P.bsmm_status_device(plan2)
                ms2 = g0.elapsed_time(g1) / 3
                e2 = float(np.linalg.norm(C32.cpu().numpy().astype(np.float64) - c64) / np.linalg.norm(c64))
                f32[f"s={s2}"] = {"value": F / (ms2 * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms2,
                                  "rel_err_vs_fp64": e2, "kernel_ms": P.bsmm_plan_kernel_ms(plan2)}
                del plan2
            extra["float32_elements"] = {"modes": f32, "inputs": "the float64 inputs rounded to float32; error "
                                         "against the FP64 product of the float64 inputs"}
            del A32, B32, C32
        # complex elements: the N/2 product of the same recipe with complex128 entries
        if args.c128_slices and not (ta or tb):
            extra["complex_elements"] = complex_line(args, P, G, torch, dev, stream)
        del plan64, C64
        # the learned schedule against the flop-count schedule on the clustered workload
        if not args.no_learned and not (ta or tb):
            w = SINGLE["clustered"]
            cl_setup = single_setup(args, w, dev)
            rec, (cprob, cplan, cq, ct, crun), _, _ = learned_vs_flops(
                lambda sd, **o: cl_setup(sd, P.BSMM_SPLIT_BF16, **o), args.seed, 5, args.warmup, dev)
            rec["workload"] = w["desc"]
            extra["learned_schedule_clustered"] = rec
            del cplan, ct, crun

    # end to end through the public C ABI with host buffers (pinned)
    e2e = None
    if args.e2e_steps > 0:
        hA = torch.from_numpy(prob.A).pin_memory()
        hB = torch.from_numpy(prob.B).pin_memory()
        hC = torch.zeros(c_tot, dtype=torch.float64).pin_memory()
        hao = torch.from_numpy(prob.a_off).pin_memory()
        hbo = torch.from_numpy(prob.b_off).pin_memory()
        hco = torch.from_numpy(c_off).pin_memory()
        P.bsmm_execute_host(plan, 1.0, hA, hao, hB, hbo, 0.0, hC, hco)
        # one product at a time (each call returns with C on the host)
        barrier()
        t0 = time.perf_counter()
        for _ in range(2):
            P.bsmm_execute_host(plan, 1.0, hA, hao, hB, hbo, 0.0, hC, hco)
        dt_sync, _ = aggregate((time.perf_counter() - t0) / 2, 0.0, dev)
        # products in flight: the copies of one overlap the kernels of the one before
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            P.bsmm_execute_host_async(plan, 1.0, hA, hao, hB, hbo, 0.0, hC, hco)
        P.bsmm_host_wait(plan)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        dt_max, _ = aggregate(dt, 0.0, dev)
        P.bsmm_status_device(plan)
        h2d = (prob.A.nbytes + prob.B.nbytes + prob.a_off.nbytes + prob.b_off.nbytes + c_off.nbytes)
        e2e = {"value": F_all / dt_max / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(c_tot * 8),
               "ms_per_step": dt_max * 1e3, "steps": args.e2e_steps,
               "api": "bsmm_execute_host_async x steps, then bsmm_host_wait (pinned host arenas; every step "
                      "copies A, B and the offset tables in and C out)",
               "one_at_a_time": {"value": F_all / dt_sync / 1e12, "ms_per_step": dt_sync * 1e3,
                                 "api": "bsmm_execute_host"}}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu, row_err = cpu_baseline(prob0, cs, Csplit, c_off, args.cpu_seconds)
        extra["split_rel_err_vs_oracle_sampled_rows"] = row_err

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": workload_name(args.n) + ("" if args.trans == "none" else
                                                                 f", operands supplied transposed: {args.trans}"),
                           "mode": f"split_bf16 s={s} (fp32 tensor-core accumulate,"
                           " exact int64 diagonal combine, fp64 recombination)" +
                           (", one scale per row of A and column of B" if args.split_scale == "rows" else ""),
                           "useful_flops_per_step": F,
                           "l2": "inputs larger than L2 (A and B 2.1 GB each), no flush",
                           "parallelism": f"replicas x{world}", "seed": args.seed},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "step_ms": {"mean": ms, "median": statistics.median(steps_ms), "min": min(steps_ms),
                            "max": max(steps_ms), "rank": "this rank's (0) timed steps"}}
        line.update(extra)
        print(json.dumps(line))


if __name__ == "__main__":
    main()
