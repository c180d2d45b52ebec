"""Benchmark of the connected-sum hot path on B300.

Headline workload: SU(6) symmetric square-lattice Hubbard model, mu = 0.1, L = 32, t = 1,
beta = 6, U = 1, orders n drawn uniformly from 4..12 per configuration, 2 x 10^5
configurations (sites uniform on the torus, tau uniform in [0, beta), seed 3), FP64, tables
of 1024 tau points.  One step = one launch of the CUDA-graph plan that holds the device
planner, the propagator gather and the whole DP (seed, clow extension, loop closing, sink)
as one persistent launch over every order, inputs resident in HBM.

The other forms of the path (FP64 / mixed / double-float at orders 4, 8 and 10, the
gradient at order 10, one configuration per launch, and the NEXT modes) are timed on the
same GPU after the headline, each with its own clock record; see `measure_forms`.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--no-extras]
Prints ONE JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2507_12349_b300 import inputs as I  # noqa: E402

WORKLOAD = "su6_sym_uneven_n4_12"
METRIC = "connected-sum configs/s at order n (FP64 vs mixed), roofline fraction, grad overhead"
UNIT = "configs/s"
NOMINAL_FP64_TFLOPS = 1.25
FP64_FMA_PER_CLK_SM = 2.0      # FP64 FMA lanes per clock per SM (ncu pipe counters of the FMA probe)
FP32_FMA_PER_CLK_SM = 128.0
# FP32 instructions a double-float term needs at least (the Dot2 step: 1 multiply, 3 FMA,
# 8 additions; the first term of a dot product fewer): the FP32-pipe floor of that mode.
DF64_FP32_PER_TERM = 11.5
# FP32 instructions of one term of the mixed mode's compensated loop close (FMA TwoProduct with
# the cross term, TwoSum, error accumulation).
MIXED_CLOSE_FP32_PER_TERM = 11.0


def measured_hbm_gbs():
    """HBM copy bandwidth measured on the B300s (MEASURED_PEAKS.json beside this file),
    else the earlier single B300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--no-extras", action="store_true", help="only the headline workload (for launch lists)")
    p.add_argument("--form-steps", type=int, default=10, help="timed steps of each order-4/8/10 form (median)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of each CPU oracle sample")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline (profiling runs)")
    p.add_argument("--n-cfg", type=int, default=0, help="smaller configuration count (profiling runs only)")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=sorted(k for k, v in I.WORKLOADS.items() if isinstance(v.model, I.Model) and not v.det),
                   help="profiling runs only: run this workload's DP instead of the headline")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "df64"], help="profiling runs only")
    p.add_argument("--grad", action="store_true",
                   help="profiling runs only: time the gradient call (adjoint DP) instead of the forward")
    p.add_argument("--bipartite", action="store_true",
                   help="profiling runs only: time the honeycomb workload's bipartite step (gather + DP)")
    p.add_argument("--det", action="store_true",
                   help="profiling runs only: time the SU(2) determinant-weight step (gather + DP, Alg. 1) "
                        "of the order-10 Zeeman workload")
    p.add_argument("--subsets", action="store_true",
                   help="profiling runs only: time the all-subsets call (c(S) and a(S) of every vertex subset) "
                        "on the order-8 SU(4) workload's gathered matrices")
    p.add_argument("--order", type=int, default=0, help="with --bipartite or --det: order of the configurations")
    p.add_argument("--probe", action="store_true",
                   help="print the GPU's FP64 FMA rates (by chains per thread and warps per SM) and the DRAM rate "
                        "of scattered 512-byte row traffic (by warps per SM and rows in flight), one JSON line each")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


# ------------------------------------------------------------------ CPU oracle (reported baseline)

def _oracle_model_args(w):
    from oracle import propagators as P
    model = w.model
    tabs = P.model_tables(model)
    wt, sig = 1, list(model.sigma)
    if model.symmetric:
        tabs, wt, sig = tabs[:1], model.n_flavors, sig[:1]
    return tabs, wt, (sig if any(sig) else None)


def oracle_values(w, cfgs, absmode=False, prec="d", nthreads=0):
    """Oracle connected sums of `cfgs` (numpy gather + the C DP in double, or `prec`, OpenMP
    over configurations), any mix of orders.  Returns (values, threads used)."""
    import oracle as O
    from oracle import propagators as P
    tabs, wt, sig = _oracle_model_args(w)
    Ms = P.gather(tabs, cfgs, w.model.L, w.model.beta)
    vals = np.zeros(cfgs.n_cfg)
    threads = 1
    for n in np.unique(cfgs.order):
        idx = np.flatnonzero(cfgs.order == n)
        hi, lo, threads = O.dp_batch(np.stack([Ms[i] for i in idx]), sig, wt, absmode=absmode, prec=prec,
                                     nthreads=nthreads)
        vals[idx] = hi + lo
    return vals, threads


def det_oracle_values(w, cfgs, absmode=False):
    """Oracle SU(2) determinant-weight sums (numpy gather + the C DP of Alg. 1 in double) of
    `cfgs`, one configuration at a time."""
    import oracle as O
    from oracle import propagators as P
    tabs = P.model_tables(w.model)
    return np.array([O.det_clow(M, absmode=absmode) for M in P.gather(tabs, cfgs, w.model.L, w.model.beta)])


def cpu_oracle_rate(w, budget_s: float, nthreads: int = 0):
    """Oracle on a bounded sample of the workload: the first configurations of its seeded
    stream, as many as `budget_s` seconds allow (estimated from a probe of 9).  Returns
    (configs/s, threads, sample size, oracle values)."""
    probe = I.workload_configs(w, 9)
    t0 = time.perf_counter()
    oracle_values(w, probe, nthreads=nthreads)
    per_cfg = (time.perf_counter() - t0) / 9.0
    n = int(min(w.n_cfg, max(9, budget_s / max(per_cfg, 1e-7))))
    cfgs = I.workload_configs(w, n)
    t0 = time.perf_counter()
    vals, threads = oracle_values(w, cfgs, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n / dt, threads, n, vals


def brute_rate_order4(budget_s: float):
    """Tier-0 oracle (every decorated cover enumerated, union-find connectivity) on the
    order-4 SU(2) workload, one configuration at a time on one core."""
    import oracle as O
    from oracle import propagators as P
    w = I.WORKLOADS["su2_sym_n4"]
    tabs = P.model_tables(w.model)
    cfgs = I.workload_configs(w, 400)
    Ms = P.gather(tabs, cfgs, w.model.L, w.model.beta)
    t0 = time.perf_counter()
    k = 0
    while k < len(Ms) and time.perf_counter() - t0 < budget_s:
        O.brute(O.tiled(Ms[k]))   # both flavors' (equal) matrices: loop weight = the flavor sum
        k += 1
    return k / (time.perf_counter() - t0), k


def cpu_baseline(w, budget_s: float):
    """The oracle as it stands on the host's cores: tier 2 (the merged DP in double) on every
    visible core and on one core, plus tier 0 (brute force) at order 4."""
    rate, threads, n, vals = cpu_oracle_rate(w, budget_s)
    rate1, _, n1, _ = cpu_oracle_rate(w, budget_s / 2, nthreads=1)
    brute, nb = brute_rate_order4(min(5.0, budget_s / 2))
    base = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {n} configurations of the {w.name} workload (numpy gather + the C merged "
                      f"DP in double, OpenMP over configurations)",
            "host_cores_visible": host_cores(),
            "value_1core": rate1, "sample_1core": f"the first {n1} configurations, one thread",
            "brute_force_order4": {"value": brute, "unit": UNIT, "cores": 1, "configs": nb,
                                   "workload": "su2_sym_n4",
                                   "kind": "oracle tier 0: every decorated cover of 8 points, union-find"}}
    return base, vals


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = I.WORKLOADS[WORKLOAD]
    budget = max(1.0, 90.0 / max(1, args.steps + 1))
    for _ in range(args.warmup):
        cpu_oracle_rate(w, min(budget, 2.0))
    rates, sample, threads = [], 0, 1
    t_start = time.perf_counter()
    for _ in range(args.steps):
        r, threads, sample, _ = cpu_oracle_rate(w, budget)
        rates.append(r)
    wall = time.perf_counter() - t_start
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": "4..12", "n_flavors": 6, "n_cfg_sample": sample, "L": 32,
                   "beta": 6.0, "n_tau": 1024, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"the first {sample} configurations of the uneven order-4..12 SU(6) workload "
                                   f"per step (numpy gather + C DP in double, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU helpers

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms (read-only)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    gpu = 0

    def __init__(self, gpu_index: int | None = None):
        self.gpu = ClockSampler.gpu if gpu_index is None else gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


class Peaks:
    """Roofline denominators at a sampled SM clock: the FP64 and FP32 pipes from unit counts
    (148 SMs x lanes per clock x 2 flop), HBM from the measured copy bandwidth."""

    def __init__(self, sms: int):
        self.sms = sms
        self.hbm_gbs, self.hbm_src = measured_hbm_gbs()

    def clk(self, clocks) -> float:
        return (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2032.0

    def fp64(self, clocks) -> float:
        return self.sms * FP64_FMA_PER_CLK_SM * 2.0 * self.clk(clocks) * 1e6

    def fp32_lane_ops(self, clocks) -> float:
        return self.sms * FP32_FMA_PER_CLK_SM * self.clk(clocks) * 1e6

    def fp32(self, clocks) -> float:
        return 2.0 * self.fp32_lane_ops(clocks)


def dp_counts(B, order: np.ndarray, n_mat: int, state_bytes: int):
    """Algorithmic work of the DP over a batch: FP64-equivalent flops (2 per multiply-add of
    the extension dot products and loop-closing sums over reachable states; shift points
    ride on the shifted diagonal and add no work), the loop-closing flops alone, and the
    layer traffic of the kernels (every reachable state written once and read once)."""
    flops = close = traffic = 0.0
    for n in np.unique(order):
        s = B.cos_structure(int(n))
        cnt = int((order == n).sum()) * n_mat
        flops += cnt * 2.0 * (s.fma_ext + s.fma_close)
        close += cnt * 2.0 * s.fma_close
        traffic += cnt * 2.0 * s.states * state_bytes
    return {"flops": flops, "close_flops": close, "traffic": traffic}


STATE_BYTES = {"fp64": 8, "mixed": 4, "df64": 8}


def flush_l2(buf):
    buf.add_(1.0)


def time_steps(torch, fn, steps, flush):
    """Per-step CUDA-event times on the current stream (L2 flushed before each step, untimed)."""
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    return times


def timed_form(torch, fn, steps, flush, warm=1):
    """A form's timing: `warm` untimed calls, then `steps` event-timed steps with the clocks
    sampled over them.  Returns (median seconds, all step times, clock record)."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    sampler = ClockSampler()
    sampler.start()
    time.sleep(0.25)
    ts = time_steps(torch, fn, steps, flush)
    clocks = sampler.stop()
    return statistics.median(ts), ts, clocks


def rooflines(r, counts, t, prec, peaks, clocks):
    """Add the form's roofline fractions: FP64 -> the FP64 pipe; mixed -> the FP64 pipe for
    the close, the FP32 pipe for the extension and HBM for the layer traffic (whichever is
    lowest binds); double-float -> the FP32 floor of its compensated terms and HBM."""
    hbm = counts["traffic"] / t / 1e9
    r["dram_gbs_model"] = hbm
    r["frac_hbm"] = hbm / peaks.hbm_gbs
    if prec == "fp64":
        r["tflops"] = counts["flops"] / t / 1e12
        r["frac_fp64_peak"] = counts["flops"] / t / peaks.fp64(clocks)
    elif prec == "mixed":
        # FP32 instructions the mode needs at least: one FMA per extension term and, per close
        # term, the compensated step (1 multiply, 2 FMA, 8 additions)
        ext_fma = (counts["flops"] - counts["close_flops"]) / 2.0
        fp32_inst = ext_fma + MIXED_CLOSE_FP32_PER_TERM * counts["close_flops"] / 2.0
        r["fp32_ext_tflops"] = 2.0 * ext_fma / t / 1e12
        r["frac_fp32_floor"] = fp32_inst / t / peaks.fp32_lane_ops(clocks)
        r["binding_roof"] = "hbm" if r["frac_hbm"] >= r["frac_fp32_floor"] else "fp32"
        r["frac_binding_roof"] = max(r["frac_hbm"], r["frac_fp32_floor"])
    else:
        terms = counts["flops"] / 2.0
        r["tflops_equiv"] = counts["flops"] / t / 1e12
        r["frac_fp32_floor"] = terms * DF64_FP32_PER_TERM / t / peaks.fp32_lane_ops(clocks)
        r["binding_roof"] = "hbm" if r["frac_hbm"] >= r["frac_fp32_floor"] else "fp32"
        r["frac_binding_roof"] = max(r["frac_hbm"], r["frac_fp32_floor"])
    return r


# ------------------------------------------------------------------ native arm

def native_arm(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ClockSampler.gpu = local
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2507_12349_b300 import binding as B
    B.lib()

    w = I.WORKLOADS[args.workload]
    n_cfg = args.n_cfg if args.n_cfg > 0 else w.n_cfg
    # weak scaling: every rank takes its own configurations of the seeded stream
    from paper_2507_12349_b300 import shard
    cfgs = I.workload_configs(w, n_cfg, first_cfg=shard.weak_block(n_cfg, rank)[0])
    tabs = B.tables_for(w.model)
    d_order, d_offset, d_site, d_tau = B.configs_to_device(cfgs)
    inf = tabs.info()
    n_mat = inf.n_mat
    n_max = int(cfgs.order.max())
    loop_weight = w.model.n_flavors if inf.symmetric else 1
    sigma = list(inf.sigma)[:n_mat]
    sigma = sigma if any(sigma) else None
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2 (126 MB)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = Peaks(sms)
    counts = dp_counts(B, cfgs.order, n_mat, STATE_BYTES[args.precision])
    graph = args.workload == WORKLOAD and not args.grad
    plan = None
    if graph:
        # the headline's launch form: planner + gather + DP frozen into one CUDA graph
        plan = B.cos_plan_create_batch(tabs, n_max, d_order, d_offset, d_site, d_tau, args.precision, out)
        step = plan.launch
        kernel = "dp_forward_kernel<double> (CUDA-graph step: 4 planner kernels, gather, DP)"
        launches_per_step = 6
    else:
        # profiling runs of another workload: gather, then the DP call on the gathered matrices
        stride = n_mat * n_max * n_max
        d_moff = torch.arange(n_cfg, dtype=torch.int64, device="cuda") * stride
        d_M = torch.empty(n_cfg * stride, dtype=torch.float64, device="cuda")
        if args.grad:
            d_gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
            d_gM = torch.empty_like(d_M)
            d_gsig = torch.empty(n_cfg, n_mat, dtype=torch.float64, device="cuda")

        def step():
            B.cos_gather(tabs, d_order, d_offset, d_site, d_tau, d_moff, d_M)
            if args.grad:
                B.cos_connected_sum_matrices_grad(n_max, d_order, d_moff, n_mat, loop_weight, sigma, d_M, d_gout,
                                                  out, d_gM, d_gsig)
            else:
                B.cos_connected_sum_matrices(n_max, d_order, d_moff, n_mat, loop_weight, sigma, d_M,
                                             args.precision, out)
        kernel = ("dp_adjoint_kernel (step: gather + the gradient call)" if args.grad else
                  "dp_forward_kernel<%s> (step: gather + planner + DP)" % args.precision)
        launches_per_step = 1 + 4 + (1 if not args.grad else 1)

    for _ in range(max(3, args.warmup)):
        step()
    B.cos_sync_status()
    if plan is not None:
        plan.status()

    # FMA probe on this GPU (reported beside the unit-count peak below)
    probe = B.measure_peak(0)

    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    times = time_steps(torch, step, args.steps, lambda: flush_l2(flush_buf))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    B.cos_sync_status()
    if plan is not None:
        plan.status()
    total = sum(times)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    value = world * n_cfg * args.steps / total
    step_mean = total / args.steps
    head_out = out.cpu().numpy()
    # The gradient call runs the forward sweep and its reverse: two multiply-adds (Obar and dM)
    # per forward multiply-add, so three times the forward's algorithmic flops.
    flops_step = counts["flops"] * (3 if args.grad else 1)
    fp64_peak = peaks.fp64(clocks)
    achieved = flops_step / step_mean
    hbm_model = counts["traffic"] / step_mean / 1e9

    # end to end through the public call with host buffers (pinned), copies inside the region
    h_in = [torch.tensor(x).pin_memory() for x in (cfgs.order, cfgs.offset, cfgs.site, cfgs.tau)]
    h_out = torch.empty(n_cfg, dtype=torch.float64).pin_memory()
    dev_in = (d_order, d_offset, d_site, d_tau)
    e_out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")

    def e2e_step():
        for dst, src in zip(dev_in, h_in):
            dst.copy_(src, non_blocking=True)
        if plan is not None:
            plan.launch()
            h_out.copy_(out, non_blocking=True)
        else:
            B.cos_connected_sum_batch(tabs, n_max, *dev_in, args.precision, e_out)
            h_out.copy_(e_out, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e2e_times = time_steps(torch, e2e_step, max(2, min(args.steps, 4)), lambda: flush_l2(flush_buf))
    B.cos_sync_status()
    h2d = sum(x.numel() * x.element_size() for x in h_in)
    d2h = h_out.numel() * h_out.element_size()
    e2e_mean = statistics.mean(e2e_times)
    if world > 1:   # the job's end-to-end time is the slowest rank's
        te = torch.tensor([e2e_mean], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        e2e_mean = float(te.item())
    e2e_value = world * n_cfg / e2e_mean
    if plan is not None:
        plan.close()

    extras, keep = {}, {}
    # the other forms and the CPU baseline are single-GPU measurements (N = 1 only)
    if not args.no_extras and world == 1:
        extras, keep = measure_forms(torch, B, flush_buf, peaks, args.form_steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_mean, "ms_per_step_median": 1e3 * statistics.median(times),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32 extension / f64 close",
                                                       "df64": "f32 pairs (df64)"}[args.precision], "data": "synthetic",
        "config": {"workload": args.workload,
                   "n": (f"{w.n_lo}..{w.n_hi} uniform" if w.n_lo != w.n_hi else w.n_lo),
                   "n_flavors": w.model.n_flavors, "n_cfg_per_gpu": n_cfg,
                   "L": w.model.L, "beta": w.model.beta, "U": w.model.U, "mu": list(w.model.mu),
                   "alpha": list(w.model.alpha), "n_tau": w.model.n_tau, "precision": args.precision,
                   "launch": "one CUDA-graph launch per step" if graph else "gather + DP call per step",
                   "full_size": n_cfg == w.n_cfg,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"configs sharded x{world}"},
        "roofline": {"bound": "alu", "pipe": "fp64 fma", "achieved": achieved / 1e12,
                     "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "peak_source": (f"unit count: {sms} SMs x {FP64_FMA_PER_CLK_SM} FP64 FMA/clk/SM x 2 flop x "
                                     f"{peaks.clk(clocks):.0f} MHz (median SM clock in the timed region); "
                                     f"MEASURED_PEAKS.json has no FP64 figure"),
                     "probe_tflops": probe / 1e12,
                     "peak_nominal": NOMINAL_FP64_TFLOPS, "frac_of_nominal": achieved / 1e12 / NOMINAL_FP64_TFLOPS,
                     "kernel": kernel,
                     "achieved_over": "the whole timed step (event pair around each step); the DP kernel is "
                                      "over 99 % of it, so this is a lower bound on the kernel's own rate",
                     "flops_per_launch": flops_step,
                     "launch_ms": step_mean * 1e3,
                     "traffic": counts["traffic"],
                     "traffic_source": "model: every reachable DP state written once and read once "
                                       "(cos_structure states x lanes x state bytes x 2); ncu DRAM bytes of the "
                                       "same launch are the cross-check",
                     # the other roof: the modelled DRAM rate of the same launch against the copy bandwidth
                     "dram_gbs": hbm_model, "hbm_peak_gbs": peaks.hbm_gbs, "hbm_peak_source": peaks.hbm_src,
                     "dram_frac": hbm_model / peaks.hbm_gbs},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "wall_s_timed_region": t_wall,
    }
    if args.grad:
        line["roofline"]["traffic"] = None
        line["roofline"]["traffic_source"] = "gradient: the kept forward layers and the adjoint ring (not modelled)"
    if extras:
        line["forms"] = extras
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"], line["accuracy"] = oracle_leg(w, args.cpu_seconds, head_out, keep, args)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    tabs.close()


def error_stats(got, ref, mass=None):
    got, ref = np.asarray(got), np.asarray(ref)
    rel = np.abs(got - ref) / np.abs(ref)
    out = {"configs": int(len(ref)), "median_rel_err": float(np.median(rel)), "max_rel_err": float(np.max(rel))}
    if mass is not None:
        em = np.abs(got - ref) / mass
        kap = mass / np.abs(ref)
        out.update({"max_err_over_mass": float(np.max(em)), "median_kappa": float(np.median(kap)),
                    "max_kappa": float(np.max(kap))})
        ok = kap <= 1e5
        if ok.any():
            out["max_rel_err_kappa_le_1e5"] = float(np.max(rel[ok]))
    return out


def oracle_leg(w, budget, head_out, keep, args):
    """The CPU oracle on the host cores: its throughput on a bounded sample of the headline
    workload, and the error of the GPU results of the same configurations against it; the
    other forms' results against the FP64 (or long-double) oracle, per configuration."""
    base, vals = cpu_baseline(w, budget)
    n = len(vals)
    cfgs = I.workload_configs(w, n)
    mass, _ = oracle_values(w, cfgs, absmode=True)
    acc = {f"{w.name}_{args.precision}_vs_oracle": error_stats(head_out[:n], vals, mass)}
    for name, (wname, got) in keep.items():
        wk = I.WORKLOADS[wname]
        if name.endswith("_by_order"):
            acc[name] = accuracy_by_order(wk, got[0], got[1])
            continue
        if name.endswith("_vs_oracle_ld"):
            k = min(len(got), 64)
            cfgs = I.workload_configs(wk, k)
            ref, _ = oracle_values(wk, cfgs, prec="ld")
            mass, _ = oracle_values(wk, cfgs, absmode=True)
            acc[name] = error_stats(got[:k], ref, mass)
            continue
        if wk.det:
            k = min(len(got), 8)
            cfgs = I.workload_configs(wk, k)
            acc[name] = error_stats(got[:k], det_oracle_values(wk, cfgs), det_oracle_values(wk, cfgs, True))
            continue
        k = min(len(got), 160)
        cfgs = I.workload_configs(wk, k)
        ref, _ = oracle_values(wk, cfgs)
        mass, _ = oracle_values(wk, cfgs, absmode=True)
        acc[name] = error_stats(got[:k], ref, mass)
    return base, acc


def sample_by_order(w, n_total, per_order=8, span=4000):
    """The first `per_order` configurations of each order within the first `span` of the
    seeded stream: {n: indices}."""
    cfgs = I.workload_configs(w, min(n_total, span))
    return {n: [c for c in range(cfgs.n_cfg) if int(cfgs.order[c]) == n][:per_order]
            for n in range(w.n_lo, w.n_hi + 1)}


def gathered_matrices(torch, B, w, idx):
    """The GPU gather's matrices [k][n_mat][n][n] of configurations idx (one order), so that
    the oracle's DP runs on the very inputs of the GPU DP."""
    cfgs = I.workload_configs(w, max(idx) + 1).subset(idx)
    tabs = B.tables_for(w.model)
    n_mat = tabs.info().n_mat
    n = int(cfgs.order[0])
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.matrix_offsets(cfgs.order, n_mat), device="cuda")
    M = torch.empty(len(idx) * n_mat * n * n, dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, moff, M)
    B.cos_sync_status()
    tabs.close()
    return M.cpu().numpy().reshape(len(idx), n_mat, n, n)


def accuracy_by_order(w, got, mats):
    """FP64 error of an uneven-order batch per order n against the long-double oracle DP on
    the same gathered matrices: the growth of the DP's cancellation error with the order."""
    import oracle as O
    sig = list(w.model.sigma)
    wt = 1
    if w.model.symmetric:
        wt, sig = w.model.n_flavors, sig[:1]
    sig = sig if any(sig) else None
    out = {}
    for n, (idx, Ms) in sorted(mats.items()):
        hi, lo, _ = O.dp_batch(Ms, sig, wt, prec="ld", nthreads=0)
        mass = O.dp_batch(Ms, sig, wt, absmode=True, nthreads=0)[0]
        out[str(n)] = error_stats(np.asarray(got)[idx], hi + lo, mass)
    return out


# ------------------------------------------------------------------ forms

def measure_forms(torch, B, flush_buf, peaks, steps):
    """The other forms of the path on the same GPU, each timed over `steps` event-timed steps
    (median) with its own clock record: FP64 vs mixed vs double-float at orders 8 and 10,
    order 4 as a plain call and as a graph launch, the adjoint at order 10 against its
    forward, the plain FP64 form with one configuration per launch, and the NEXT modes
    (all subsets, bipartite, determinant weights; fewer steps).  Returns the measurements
    and the GPU outputs kept for the oracle leg's error statistics."""
    res, keep = {}, {}
    flush = lambda: flush_l2(flush_buf)

    def run(name, prec, graph=False, n_cfg=None):
        w = I.WORKLOADS[name]
        cfgs = I.workload_configs(w, n_cfg)
        tabs = B.tables_for(w.model)
        d = B.configs_to_device(cfgs)
        out = torch.empty(cfgs.n_cfg, dtype=torch.float64, device="cuda")
        nmax = int(cfgs.order.max())
        n_mat = tabs.info().n_mat
        if graph:
            plan = B.cos_plan_create_batch(tabs, nmax, *d, prec, out)
            fn = plan.launch
        else:
            fn = lambda: B.cos_connected_sum_batch(tabs, nmax, *d, prec, out)
        t, ts, clocks = timed_form(torch, fn, steps, flush)
        if graph:
            plan.status()
            plan.close()
        B.cos_sync_status()
        tabs.close()
        counts = dp_counts(B, cfgs.order, n_mat, STATE_BYTES[prec])
        r = {"configs": cfgs.n_cfg, "configs_per_s": cfgs.n_cfg / t, "ms_median": t * 1e3,
             "ms_min": min(ts) * 1e3, "ms_max": max(ts) * 1e3, "steps": len(ts), "clocks": clocks,
             "launch_shape_n_max": dict(zip(("warps", "ctas_per_sm", "prefetch"), B.cos_get_tuning(nmax, prec, n_mat)))}
        rooflines(r, counts, t, prec, peaks, clocks)
        if graph:
            r["cuda_graph"] = True
        return r, out.cpu().numpy()

    # SU(2) symmetric, order 4, 10^4 configurations: latency- and launch-bound (about 15 us of
    # FP64 work), one plain call and one CUDA-graph plan launch
    res["su2_n4_fp64"], _ = run("su2_sym_n4", "fp64")
    res["su2_n4_fp64_graph"], _ = run("su2_sym_n4", "fp64", graph=True)
    # SU(4), mu broken, order 8, 10^5 configurations: FP64, mixed, double-float
    res["su4_n8_fp64"], keep_f8 = run("su4_mu_broken_n8", "fp64")
    keep["su4_n8_fp64_vs_fp64_oracle"] = ("su4_mu_broken_n8", keep_f8)
    res["su4_n8_mixed"], keep_n8 = run("su4_mu_broken_n8", "mixed")
    keep["su4_n8_mixed_vs_fp64_oracle"] = ("su4_mu_broken_n8", keep_n8)
    res["su4_n8_df64"], keep_df8 = run("su4_mu_broken_n8", "df64")
    keep["su4_n8_df64_vs_fp64_oracle"] = ("su4_mu_broken_n8", keep_df8)
    # SU(3) with shifts, order 10, 10^5 configurations: mixed (the workload's precision), FP64, df64
    res["su3_shift_n10_mixed"], keep_n10 = run("su3_shift_mixed_n10", "mixed")
    keep["su3_shift_n10_mixed_vs_fp64_oracle"] = ("su3_shift_mixed_n10", keep_n10)
    res["su3_shift_n10_fp64"], keep_f10 = run("su3_shift_mixed_n10", "fp64")
    keep["su3_shift_n10_fp64_vs_oracle_ld"] = ("su3_shift_mixed_n10", keep_f10)
    res["su3_shift_n10_df64"], keep_df10 = run("su3_shift_mixed_n10", "df64")
    keep["su3_shift_n10_df64_vs_fp64_oracle"] = ("su3_shift_mixed_n10", keep_df10)
    res["su3_shift_n10_mixed"]["speedup_vs_fp64"] = (res["su3_shift_n10_mixed"]["configs_per_s"]
                                                     / res["su3_shift_n10_fp64"]["configs_per_s"])
    res["su3_shift_n10_df64"]["speedup_vs_fp64"] = (res["su3_shift_n10_df64"]["configs_per_s"]
                                                    / res["su3_shift_n10_fp64"]["configs_per_s"])
    # the headline's outputs per order against the oracle DP on the same gathered matrices
    wu = I.WORKLOADS[WORKLOAD]
    cu = I.workload_configs(wu, 4000)
    tabs = B.tables_for(wu.model)
    d = B.configs_to_device(cu)
    out_u = torch.empty(cu.n_cfg, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_batch(tabs, 12, *d, "fp64", out_u)
    B.cos_sync_status()
    tabs.close()
    mats = {n: (idx, gathered_matrices(torch, B, wu, idx)) for n, idx in sample_by_order(wu, 4000).items() if idx}
    keep["su6_uneven_fp64_by_order"] = (WORKLOAD, (out_u.cpu().numpy(), mats))
    res["su4_n10_adjoint"] = measure_adjoint(torch, B, flush, peaks, steps)
    res["su4_n8_fp64_one_config_per_launch"] = measure_one_per_launch(torch, B)
    # NEXT modes: fewer steps each (their sizes match the rows above)
    nsteps = max(2, steps // 3)
    res["su4_n8_all_subsets_fp64"] = measure_subsets(torch, B, flush, nsteps)
    for prec in ("fp64", "df64", "mixed"):
        hb = measure_bipartite(torch, B, flush, I.WORKLOADS["hc_su2_af_n8"].n_cfg, prec, nsteps)
        if prec == "fp64":
            hb["frac_fp64_peak"] = hb["tflops"] * 1e12 / peaks.fp64(hb["clocks"])
        elif prec == "df64":
            hb["frac_fp32_floor"] = hb["tflops"] * 1e12 / 2.0 * DF64_FP32_PER_TERM / peaks.fp32_lane_ops(hb["clocks"])
        res[f"hc_su2_af_n8_bipartite_{prec}"] = hb
    det, det_out = measure_det(torch, B, flush, peaks, nsteps)
    res.update(det)
    keep["su2_zeeman_n10_det_fp64_vs_oracle"] = ("su2_zeeman_det_n10", det_out)
    res.update(measure_grad_high_orders(torch, B, flush, peaks, nsteps))
    return res, keep


def measure_grad_high_orders(torch, B, flush, peaks, steps, n_cfg=2368):
    """Gradient at orders 11 and 12 (the adjoint workload's model, SU(4) with mu broken;
    2368 configurations = 296 batches, two waves of one CTA per SM): the automatic plan, which
    checkpoints layers where the free memory cannot hold every CTA's layers, against every
    layer kept with the grid the memory allows."""
    w = I.WORKLOADS["su4_adjoint_n10"]
    # start from the memory a fresh process would see: the earlier forms' workspaces released
    B.cos_release_workspace()
    torch.cuda.empty_cache()
    tabs = B.tables_for(w.model)
    res = {}
    for n in (11, 12):
        cfgs = I.make_configs(w.model, n, n, n_cfg, seed=40 + n)
        d = B.configs_to_device(cfgs)
        gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
        out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
        fn = lambda: B.cos_connected_sum_grad(tabs, n, *d, gout, out)
        r = {"configs": n_cfg, "steps": steps}
        fl = dp_counts(B, cfgs.order, 4, 8)["flops"]
        for mode, key in (("0", "every_layer_kept"), ("", "automatic")):
            if mode:
                os.environ["COS_GRAD_CHECKPOINT"] = mode
            else:
                os.environ.pop("COS_GRAD_CHECKPOINT", None)
            t, _, clocks = timed_form(torch, fn, steps, flush)
            B.cos_sync_status()
            r[key] = {"grad_configs_per_s": n_cfg / t, "ms_median": t * 1e3, "clocks": clocks,
                      "frac_fp64_peak_3x_forward": 3 * fl / t / peaks.fp64(clocks)}
        os.environ.pop("COS_GRAD_CHECKPOINT", None)
        mask, store, rec = B.cos_grad_checkpoint_plan(n, 0)
        s = B.cos_structure(n)
        r["speedup_automatic_vs_kept"] = r["automatic"]["grad_configs_per_s"] / r["every_layer_kept"]["grad_configs_per_s"]
        r["layer_storage_per_cta_gb"] = s.slots * 32 * 8 / 1e9
        r["least_storage_plan"] = {"checkpoint_layers": [l for l in range(2, 2 * n + 1) if mask >> l & 1],
                                   "storage_fraction": store / s.slots,
                                   "recompute_fraction_of_forward": rec / (s.fma_ext + s.fma_close)}
        res[f"su4_n{n}_grad_fp64"] = r
    tabs.close()
    return res


def measure_adjoint(torch, B, flush, peaks, steps):
    """Gradient overhead on the adjoint workload (SU(4), mu broken, n = 10, 5 x 10^4
    configurations): the gradient call (forward recomputed + reverse DP + chain rule to mu,
    alpha) against the forward call on the same configurations, each timed over `steps`."""
    w = I.WORKLOADS["su4_adjoint_n10"]
    cfgs = I.workload_configs(w)
    n_cfg = cfgs.n_cfg
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
    gmu = torch.empty(n_cfg, 4, dtype=torch.float64, device="cuda")
    gal = torch.empty_like(gmu)
    fwd = lambda: B.cos_connected_sum_batch(tabs, 10, *d, "fp64", out)
    grad = lambda: B.cos_connected_sum_grad(tabs, 10, *d, gout, gmu=gmu, galpha=gal)
    tf, _, cf = timed_form(torch, fwd, steps, flush)
    tg, tgs, cg = timed_form(torch, grad, steps, flush)
    B.cos_sync_status()
    tabs.close()
    fl = dp_counts(B, cfgs.order, 4, 8)["flops"]
    return {"configs": n_cfg, "forward_configs_per_s": n_cfg / tf, "grad_configs_per_s": n_cfg / tg,
            "grad_overhead": tg / tf, "forward_ms_median": tf * 1e3, "grad_ms_median": tg * 1e3,
            "grad_ms_min": min(tgs) * 1e3, "steps": steps,
            "grad_tflops": 3 * fl / tg / 1e12, "frac_fp64_peak": 3 * fl / tg / peaks.fp64(cg),
            "forward_frac_fp64_peak": fl / tf / peaks.fp64(cf),
            "work": "gradient = forward recompute + reverse sweep (2 multiply-adds per forward one): 3x the "
                    "forward's algorithmic flops",
            "clocks_forward": cf, "clocks": cg}


def measure_one_per_launch(torch, B):
    """The plain FP64 per-configuration form: one configuration per call, no graph (200
    calls of the order-8 SU(4) workload)."""
    w = I.WORKLOADS["su4_mu_broken_n8"]
    cfgs = I.workload_configs(w, 200)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    zero = torch.zeros(1, dtype=torch.int64, device="cuda")
    per = []
    for c in range(200):
        o = int(cfgs.offset[c])
        per.append((d[0][c:c + 1], zero, d[2][o:o + 8], d[3][o:o + 8]))
    B.cos_connected_sum_batch(tabs, 8, *per[0], "fp64", out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for a in per:
        B.cos_connected_sum_batch(tabs, 8, *a, "fp64", out)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    B.cos_sync_status()
    tabs.close()
    return {"configs": 200, "configs_per_s": 200 / t}


def measure_subsets(torch, B, flush, steps):
    """All-subsets mode on the order-8 SU(4) workload: c(S) of all 255 vertex subsets and
    a(S) by the GPU subset exponential, against the plain call (c(V) only) on the same
    gathered matrices.  Also the root-0 by-product (c(S) for S containing vertex 0)."""
    w = I.WORKLOADS["su4_mu_broken_n8"]
    cfgs = I.workload_configs(w)
    n_cfg = cfgs.n_cfg
    tabs = B.tables_for(w.model)
    n_mat = tabs.info().n_mat
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.matrix_offsets(cfgs.order, n_mat), device="cuda")
    M = torch.empty(int(n_cfg * n_mat * 64), dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, d[0], d[1], d[2], d[3], moff, M)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    c = torch.empty(n_cfg * 256, dtype=torch.float64, device="cuda")
    a = torch.empty_like(c)
    plain = lambda: B.cos_connected_sum_matrices(8, d[0], moff, n_mat, 1, None, M, "fp64", out)
    root0 = lambda: B.cos_connected_sum_subsets(8, d[0], moff, n_mat, 1, None, M, "fp64", c, None, False)
    full = lambda: B.cos_connected_sum_subsets(8, d[0], moff, n_mat, 1, None, M, "fp64", c, a, True)
    tp, _, _ = timed_form(torch, plain, steps, flush)
    t0, _, _ = timed_form(torch, root0, steps, flush)
    tf, _, clocks = timed_form(torch, full, steps, flush)
    B.cos_sync_status()
    tabs.close()
    return {"configs": n_cfg, "plain_configs_per_s": n_cfg / tp, "root0_configs_per_s": n_cfg / t0,
            "all_subsets_configs_per_s": n_cfg / tf, "all_subsets_cost_vs_plain": tf / tp,
            "root0_cost_vs_plain": t0 / tp, "steps": steps, "clocks": clocks}


def measure_bipartite(torch, B, flush, n_cfg, precision, steps):
    """Honeycomb workload (SU(2), antiferromagnetic staggered shift, n = 8; sublattices summed
    per vertex by the sublattice-resolved DP): gather + bipartite DP from vertex coordinates."""
    w = I.WORKLOADS["hc_su2_af_n8"]
    cfgs = I.workload_configs(w, n_cfg)
    tabs = B.honeycomb_tables_for(w.model)
    n_mat = tabs.info().n_mat
    d = B.configs_to_device(cfgs)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    fn = lambda: B.cos_connected_sum_bipartite_batch(tabs, 8, *d, precision, out)
    t, _, clocks = timed_form(torch, fn, steps, flush)
    B.cos_sync_status()
    s = B.cos_bipartite_structure(8)
    fl = n_cfg * n_mat * 2.0 * (s.fma_ext + s.fma_close)
    tabs.close()
    return {"configs": n_cfg, "configs_per_s": n_cfg / t, "tflops": fl / t / 1e12, "ms_median": t * 1e3,
            "assignments_per_config": 256, "steps": steps, "clocks": clocks}


def det_fma(B, n: int) -> int:
    """Multiply-adds of one spin block of the determinant-weight DP at order n: those of the
    merged structure minus the first loop's step onto vertex 0, which Alg. 1 does not take
    (one per endpoint state of every mask with vertex 0 half-visited: k other visited
    vertices give max(k, 1) endpoints, and C(n-1, k) 2^k masks have k)."""
    s = B.cos_structure(n)
    saved = sum(math.comb(n - 1, k) * 2 ** k * max(k, 1) for k in range(n))
    return s.fma_ext - saved + s.fma_close


def measure_det(torch, B, flush, peaks, steps):
    """SU(2) determinant weights by the DP without cycle factors (Alg. 1): the order-10 square
    workload with a Zeeman-split chemical potential (gather + DP on the same matrices in
    FP64, double-float and mixed precision, against the CoS DP of the same two matrices, which
    returns 2^n times the same sum), and the honeycomb order-8 workload's matrices (bipartite,
    against the CoS bipartite DP).  Returns the forms and the FP64 output for the accuracy."""
    res = {}
    w = I.WORKLOADS["su2_zeeman_det_n10"]
    n_cfg, n = w.n_cfg, 10
    cfgs = I.workload_configs(w)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.matrix_offsets(cfgs.order, 2), device="cuda")
    M = torch.empty(n_cfg * 2 * n * n, dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, moff, M)
    outs = {p: torch.empty(n_cfg, dtype=torch.float64, device="cuda") for p in ("fp64", "df64", "mixed", "cos")}
    fns = {p: (lambda p=p: B.cos_connected_det_matrices(n, d[0], moff, None, M, p, outs[p]))
           for p in ("fp64", "df64", "mixed")}
    fns["cos"] = lambda: B.cos_connected_sum_matrices(n, d[0], moff, 2, 1, None, M, "fp64", outs["cos"])
    ts, cl = {}, {}
    for p, f in fns.items():
        ts[p], _, cl[p] = timed_form(torch, f, steps, flush)
    B.cos_sync_status()
    # c_det against c_CoS / 2^n on the same matrices, read at once and again after the gradient and
    # all-subsets calls below (which must leave both outputs untouched)
    rel_vs_cos = lambda: float(np.max(np.abs(outs["fp64"].cpu().numpy() - outs["cos"].cpu().numpy() / 2.0 ** n)
                                      / np.abs(outs["fp64"].cpu().numpy())))
    first_diff = rel_vs_cos()
    fl = n_cfg * 2 * 2.0 * det_fma(B, n)
    for p in ("fp64", "df64", "mixed"):
        r = {"configs": n_cfg, "configs_per_s": n_cfg / ts[p], "ms_median": ts[p] * 1e3,
             "cost_vs_cos_fp64": ts[p] / ts["cos"], "steps": steps, "clocks": cl[p]}
        if p == "fp64":
            r["tflops"] = fl / ts[p] / 1e12
            r["frac_fp64_peak"] = fl / ts[p] / peaks.fp64(cl[p])
        elif p == "df64":
            r["frac_fp32_floor"] = fl / 2.0 * DF64_FP32_PER_TERM / ts[p] / peaks.fp32_lane_ops(cl[p])
        else:
            s = B.cos_structure(n)
            r["frac_hbm"] = n_cfg * 2 * 2.0 * s.states * 4 / ts[p] / 1e9 / peaks.hbm_gbs
        res[f"su2_zeeman_n10_det_{p}"] = r
    # gradient (reverse sweep of the determinant weights): dc/dM and dc/dalpha of every configuration
    gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
    gM = torch.empty_like(M)
    ga = torch.empty(n_cfg, 2, dtype=torch.float64, device="cuda")
    gfn = lambda: B.cos_connected_det_matrices_grad(n, d[0], moff, None, M, gout, None, gM, ga)
    tg, _, cg = timed_form(torch, gfn, steps, flush)
    B.cos_sync_status()
    # every vertex subset: c(S) and a(S) = det(A_up[S]) det(A_dn[S]) (CDet's set of minors)
    cs = torch.empty(n_cfg << n, dtype=torch.float64, device="cuda")
    as_ = torch.empty_like(cs)
    sfn = lambda: B.cos_connected_det_subsets(n, d[0], moff, None, M, cs, as_, True)
    tsub, _, csub = timed_form(torch, sfn, steps, flush)
    B.cos_sync_status()
    res["su2_zeeman_n10_det_all_subsets_fp64"] = {"configs": n_cfg, "configs_per_s": n_cfg / tsub,
                                                  "ms_median": tsub * 1e3, "cost_vs_plain": tsub / ts["fp64"],
                                                  "steps": steps, "clocks": csub}
    del cs, as_
    res["su2_zeeman_n10_det_grad_fp64"] = {"configs": n_cfg, "grad_configs_per_s": n_cfg / tg, "ms_median": tg * 1e3,
                                           "grad_overhead": tg / ts["fp64"],
                                           "frac_fp64_peak": 3 * fl / tg / peaks.fp64(cg), "steps": steps,
                                           "clocks": cg}
    got = outs["fp64"].cpu().numpy()
    res["su2_zeeman_n10_det_fp64"]["max_rel_diff_vs_cos_over_2n"] = first_diff
    res["su2_zeeman_n10_det_fp64"]["max_rel_diff_vs_cos_over_2n_after_grad_and_subsets"] = rel_vs_cos()
    tabs.close()
    # bipartite: the honeycomb workload's gathered matrices, det vs CoS bipartite sweep
    hw = I.WORKLOADS["hc_su2_af_n8"]
    hc = I.workload_configs(hw)
    htabs = B.honeycomb_tables_for(hw.model)
    hd = B.configs_to_device(hc)
    hmoff = torch.as_tensor(B.bipartite_matrix_offsets(hc.order, 2), device="cuda")
    M4 = torch.empty(hc.n_cfg * 2 * 16 * 16, dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(htabs, *hd, hmoff, M4)
    hout = torch.empty(hc.n_cfg, dtype=torch.float64, device="cuda")
    al = [list(r) for r in hw.model.sigma2]
    hfns = {"det_fp64": lambda: B.cos_connected_det_bipartite_matrices(8, hd[0], hmoff, al, M4, "fp64", hout),
            "det_df64": lambda: B.cos_connected_det_bipartite_matrices(8, hd[0], hmoff, al, M4, "df64", hout),
            "det_mixed": lambda: B.cos_connected_det_bipartite_matrices(8, hd[0], hmoff, al, M4, "mixed", hout),
            "cos_fp64": lambda: B.cos_connected_sum_bipartite_matrices(8, hd[0], hmoff, 2, 1, None, M4, "fp64", hout)}
    ht, hcl = {}, {}
    for k, f in hfns.items():
        ht[k], _, hcl[k] = timed_form(torch, f, steps, flush)
    B.cos_sync_status()
    htabs.close()
    for k in ("det_fp64", "det_df64", "det_mixed"):
        res[f"hc_su2_af_n8_{k}"] = {"configs": hc.n_cfg, "configs_per_s": hc.n_cfg / ht[k], "ms_median": ht[k] * 1e3,
                                    "cost_vs_cos_fp64": ht[k] / ht["cos_fp64"], "steps": steps, "clocks": hcl[k]}
    # every vertex subset of both bipartite sweeps: c(S) of all 255 subsets (8 rooted derived
    # problems per configuration) and a(S) by the subset exponential, against the plain call
    hcs = torch.empty(hc.n_cfg * 256, dtype=torch.float64, device="cuda")
    has = torch.empty_like(hcs)
    sfns = {"cos_fp64": lambda: B.cos_connected_sum_bipartite_subsets(8, hd[0], hmoff, 2, 1, None, M4, hcs, has),
            "det_fp64": lambda: B.cos_connected_det_bipartite_subsets(8, hd[0], hmoff, al, M4, hcs, has)}
    for k, f in sfns.items():
        tsk, _, ck = timed_form(torch, f, steps, flush)
        B.cos_sync_status()
        res[f"hc_su2_af_n8_{k.split('_')[0]}_all_subsets_fp64"] = {
            "configs": hc.n_cfg, "configs_per_s": hc.n_cfg / tsk, "ms_median": tsk * 1e3,
            "cost_vs_plain": tsk / ht[k], "steps": steps, "clocks": ck}
    del hcs, has
    # gradients of both bipartite sweeps (reverse sweep over every kept layer)
    hg = torch.ones(hc.n_cfg, dtype=torch.float64, device="cuda")
    gM4 = torch.empty_like(M4)
    gs2 = torch.empty(hc.n_cfg, 2, 2, dtype=torch.float64, device="cuda")
    gfns = {"cos_fp64": lambda: B.cos_connected_sum_bipartite_matrices_grad(8, hd[0], hmoff, 2, 1, None, M4, hg,
                                                                            None, gM4, gs2),
            "det_fp64": lambda: B.cos_connected_det_bipartite_matrices_grad(8, hd[0], hmoff, al, M4, hg, None,
                                                                            gM4, gs2)}
    for k, f in gfns.items():
        tgk, _, ck = timed_form(torch, f, steps, flush)
        B.cos_sync_status()
        res[f"hc_su2_af_n8_{k.split('_')[0]}_grad_fp64"] = {"configs": hc.n_cfg, "grad_configs_per_s": hc.n_cfg / tgk,
                                                           "ms_median": tgk * 1e3, "grad_overhead": tgk / ht[k],
                                                           "steps": steps, "clocks": ck}
    return res, got


# ------------------------------------------------------------------ profiling arms

def bipartite_arm(args):
    """Profiling runs of the bipartite path alone: the honeycomb workload's gather + DP from
    vertex coordinates, at its order or --order, --n-cfg configurations, CUDA-event timing;
    with --grad the gradient call instead (FP64); with --subsets, gather + the all-subsets
    mode (c(S) and a(S) of every subset, FP64)."""
    import torch
    from paper_2507_12349_b300 import binding as B
    B.lib()
    w = I.WORKLOADS["hc_su2_af_n8"]
    n = args.order if args.order > 0 else w.n_lo
    n_cfg = args.n_cfg if args.n_cfg > 0 else w.n_cfg
    cfgs = I.make_configs(w.model, n, n, n_cfg, w.seed)
    tabs = B.honeycomb_tables_for(w.model)
    n_mat = tabs.info().n_mat
    d = B.configs_to_device(cfgs)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    fn = lambda: B.cos_connected_sum_bipartite_batch(tabs, n, *d, args.precision, out)
    if args.grad:   # the gradient from vertex coordinates: gather, reverse sweep, chain rule to mu, alpha
        gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
        gmu = torch.empty(n_cfg, tabs.info().n_flavors, dtype=torch.float64, device="cuda")
        gal = torch.empty_like(gmu)
        fn = lambda: B.cos_connected_sum_bipartite_grad(tabs, n, *d, gout, out, gmu=gmu, galpha=gal)
    if args.subsets:
        moff = torch.as_tensor(B.bipartite_matrix_offsets(cfgs.order, n_mat), device="cuda")
        M4 = torch.empty(n_cfg * n_mat * 4 * n * n, dtype=torch.float64, device="cuda")
        c = torch.empty(n_cfg << n, dtype=torch.float64, device="cuda")
        a = torch.empty_like(c)
        info = tabs.info()   # the tables' shift weights and loop weight, as the batch call uses them
        sig2 = [[info.sigma2[l][s] for s in range(2)] for l in range(n_mat)]
        wt = info.n_flavors if info.symmetric else 1

        def fn():
            B.cos_gather_bipartite(tabs, *d, moff, M4)
            B.cos_connected_sum_bipartite_subsets(n, d[0], moff, n_mat, wt, sig2, M4, c, a)
    for _ in range(max(1, args.warmup)):
        fn()
    B.cos_sync_status()
    ts = time_steps(torch, fn, args.steps, lambda: flush_l2(flush_buf))
    B.cos_sync_status()
    s = B.cos_bipartite_structure(n)
    t = statistics.mean(ts)
    fl = n_cfg * n_mat * 2.0 * (s.fma_ext + s.fma_close)
    print(json.dumps({"metric": ("bipartite all-subsets configs/s (c(S), a(S) of every subset)" if args.subsets else
                                 "bipartite gradient configs/s (honeycomb, dc/dmu and dc/dalpha)" if args.grad else
                                 "bipartite connected-sum configs/s (honeycomb, sublattices summed)"),
                      "value": n_cfg / t, "unit": "configs/s", "order": n, "configs": n_cfg,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                      "tflops": None if (args.subsets or args.grad) else fl / t / 1e12,
                      "dtype": "f64" if args.subsets else {"fp64": "f64", "df64": "f32 pairs (df64)"}.get(
                          args.precision, args.precision)}), flush=True)
    tabs.close()


def subsets_arm(args):
    """Profiling runs of the all-subsets mode alone: gather + cos_connected_sum_subsets with
    all roots and a(S) on --n-cfg configurations of the order-8 SU(4) workload."""
    import torch
    from paper_2507_12349_b300 import binding as B
    B.lib()
    w = I.WORKLOADS["su4_mu_broken_n8"]
    n = w.n_lo
    n_cfg = args.n_cfg if args.n_cfg > 0 else w.n_cfg
    cfgs = I.workload_configs(w, n_cfg)
    tabs = B.tables_for(w.model)
    n_mat = tabs.info().n_mat
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.matrix_offsets(cfgs.order, n_mat), device="cuda")
    M = torch.empty(n_cfg * n_mat * n * n, dtype=torch.float64, device="cuda")
    c = torch.empty(n_cfg << n, dtype=torch.float64, device="cuda")
    a = torch.empty_like(c)
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def fn():
        B.cos_gather(tabs, *d, moff, M)
        B.cos_connected_sum_subsets(n, d[0], moff, n_mat, 1, None, M, "fp64", c, a, True)
    for _ in range(max(1, args.warmup)):
        fn()
    B.cos_sync_status()
    ts = time_steps(torch, fn, args.steps, lambda: flush_l2(flush_buf))
    B.cos_sync_status()
    t = statistics.mean(ts)
    print(json.dumps({"metric": "all-subsets connected sums configs/s (c(S), a(S) of every subset)",
                      "value": n_cfg / t, "unit": "configs/s", "order": n, "configs": n_cfg,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "dtype": "f64"}),
          flush=True)
    tabs.close()


def det_arm(args):
    """Profiling runs of the determinant-weight path alone: the SU(2) Zeeman workload's gather
    + DP without cycle factors, at its order or --order, --n-cfg configurations."""
    import torch
    from paper_2507_12349_b300 import binding as B
    B.lib()
    w = I.WORKLOADS["su2_zeeman_det_n10"]
    n = args.order if args.order > 0 else w.n_lo
    n_cfg = args.n_cfg if args.n_cfg > 0 else w.n_cfg
    cfgs = I.make_configs(w.model, n, n, n_cfg, w.seed)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.matrix_offsets(cfgs.order, 2), device="cuda")
    M = torch.empty(n_cfg * 2 * n * n, dtype=torch.float64, device="cuda")
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def fn():
        B.cos_gather(tabs, *d, moff, M)
        B.cos_connected_det_matrices(n, d[0], moff, None, M, args.precision, out)
    for _ in range(max(1, args.warmup)):
        fn()
    B.cos_sync_status()
    ts = time_steps(torch, fn, args.steps, lambda: flush_l2(flush_buf))
    B.cos_sync_status()
    t = statistics.mean(ts)
    fl = n_cfg * 2 * 2.0 * det_fma(B, n)
    print(json.dumps({"metric": "SU(2) determinant-weight connected-sum configs/s (Alg. 1)",
                      "value": n_cfg / t, "unit": "configs/s", "order": n, "configs": n_cfg,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                      "tflops": fl / t / 1e12, "dtype": {"fp64": "f64", "df64": "f32 pairs (df64)"}.get(
                          args.precision, args.precision)}), flush=True)
    tabs.close()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.probe:
        import torch
        from paper_2507_12349_b300 import binding as B
        torch.cuda.set_device(0)
        for r in B.probe_sweep():
            print(json.dumps(r), flush=True)
    elif args.bipartite:
        bipartite_arm(args)
    elif args.det:
        det_arm(args)
    elif args.subsets:
        subsets_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
