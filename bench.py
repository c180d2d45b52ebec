"""Benchmark of the connected-sum hot path on B300.

Workload (the configuration the metric is quoted on): SU(4) square-lattice
Hubbard model with flavor-dependent chemical potentials mu = (-0.3, -0.1, 0.1,
0.3), L = 16, t = 1, beta = 4, U = 1.5, order n = 8, 10^5 configurations with
sites uniform on the torus and tau uniform in [0, beta) (seed 1), FP64,
per-flavor tables of 1024 tau points.  One step = propagator gather + the
whole DP (seed, clow extension, loop closing, sink) for all 10^5
configurations, inputs resident in HBM.

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

WORKLOAD = "su4_mu_broken_n8"
METRIC = "connected-sum configs/s at order n (FP64 vs mixed), roofline fraction, grad overhead"
UNIT = "configs/s"
NOMINAL_FP64_TFLOPS = 1.25
# DRAM bytes (read + write) of dp_forward_kernel<double, 320> per configuration of the headline
# workload: ncu dram__bytes_read.sum + dram__bytes_write.sum on a 5 000-configuration launch
# (8.917 GB + 7.099 GB, profiles/dp_forward_fp64_su4_n8.md); traffic grows in proportion
# to the configurations of a launch.
HEADLINE_DRAM_BYTES_PER_CFG = (8.917352e9 + 7.098890e9) / 5000
FP64_FMA_PER_CLK_SM = 2.0


def measured_hbm_gbs():
    """HBM copy bandwidth measured on the B300s (MEASURED_PEAKS.json beside this file),
    else the earlier single B300 measurement."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
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
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU oracle sample")
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
                        "on the headline workload's gathered matrices")
    p.add_argument("--order", type=int, default=0, help="with --bipartite or --det: order of the configurations")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ CPU oracle (reported baseline)

def oracle_values(w, cfgs, absmode=False, prec="d"):
    """Oracle connected sums (numpy gather + C DP in double, or `prec`, OpenMP) of `cfgs` (one
    order)."""
    import oracle as O
    from oracle import propagators as P
    model = w.model
    tabs = P.model_tables(model)
    wt, sig = 1, list(model.sigma)
    if model.symmetric:
        tabs, wt, sig = tabs[:1], model.n_flavors, sig[:1]
    sig = sig if any(sig) else None
    Ms = np.stack(P.gather(tabs, cfgs, model.L, model.beta))
    hi, lo, threads = O.dp_batch(Ms, sig, wt, absmode=absmode, prec=prec, nthreads=0)
    return hi + lo, threads


def det_oracle_values(w, cfgs, absmode=False):
    """Oracle SU(2) determinant-weight sums (numpy gather + the C DP of Alg. 1 in double) of
    `cfgs`, one configuration at a time."""
    import oracle as O
    from oracle import propagators as P
    tabs = P.model_tables(w.model)
    return np.array([O.det_clow(M, absmode=absmode) for M in P.gather(tabs, cfgs, w.model.L, w.model.beta)])


def cpu_oracle_rate(w, budget_s: float, n_limit: int | None = None):
    """Oracle on a bounded sample of the workload (the first configurations of its seeded
    stream).  Returns (configs/s, threads, sample size, oracle values)."""
    probe = I.workload_configs(w, 8)
    t0 = time.perf_counter()
    oracle_values(w, probe)
    per_cfg = (time.perf_counter() - t0) / 8.0
    n = max(8, int(budget_s / max(per_cfg, 1e-6)))
    if n_limit:
        n = min(n, n_limit)
    n = min(n, w.n_cfg)
    cfgs = I.workload_configs(w, n)
    t0 = time.perf_counter()
    vals, threads = oracle_values(w, cfgs)
    dt = time.perf_counter() - t0
    return n / dt, threads, n, vals


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
        "config": {"workload": WORKLOAD, "n": 8, "n_flavors": 4, "n_cfg_sample": sample, "L": 16, "beta": 4.0,
                   "n_tau": 1024, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{sample} configurations of the n=8 SU(4) workload per step "
                                   f"(numpy gather + C DP in double, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU helpers

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms (read-only)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
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


def algorithmic_flops(B, order: np.ndarray, n_mat: int, shifts: bool) -> float:
    """FP64-equivalent flops the DP must do: 2 per multiply-add of the extension dot products
    and loop-closing sums over reachable states (shift points ride on the shifted diagonal of
    the extension matrices and add no work)."""
    del shifts
    total = 0.0
    for n in np.unique(order):
        s = B.cos_structure(int(n))
        cnt = int((order == n).sum())
        total += cnt * n_mat * 2.0 * (s.fma_ext + s.fma_close)
    return total


def flush_l2(buf):
    buf.add_(1.0)


def time_steps(torch, fn, steps, flush):
    """Per-step CUDA-event times (flush between steps, untimed)."""
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


def native_arm(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2507_12349_b300 import binding as B
    B.lib()

    w = I.WORKLOADS[args.workload]
    n_cfg = args.n_cfg if args.n_cfg > 0 else w.n_cfg
    # weak scaling: every rank takes its own 10^5 configurations of the seeded stream
    cfgs = I.workload_configs(w, n_cfg, first_cfg=rank * n_cfg)
    tabs = B.tables_for(w.model)
    d_order, d_offset, d_site, d_tau = B.configs_to_device(cfgs)
    inf = tabs.info()
    n_mat = inf.n_mat
    n_max = int(cfgs.order.max())
    loop_weight = w.model.n_flavors if inf.symmetric else 1
    sigma = list(inf.sigma)[:n_mat]
    sigma = sigma if any(sigma) else None
    stride = n_mat * n_max * n_max
    d_moff = torch.arange(n_cfg, dtype=torch.int64, device="cuda") * stride
    d_M = torch.empty(n_cfg * stride, dtype=torch.float64, device="cuda")
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    if args.grad:
        d_gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
        d_gM = torch.empty_like(d_M)
        d_gsig = torch.empty(n_cfg, n_mat, dtype=torch.float64, device="cuda")
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2 (126 MB)
    stream = torch.cuda.current_stream()

    # a step, with CUDA events between the gather and the DP (same stream)
    dp_times = []

    def step():
        B.cos_gather(tabs, d_order, d_offset, d_site, d_tau, d_moff, d_M)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        if args.grad:
            B.cos_connected_sum_matrices_grad(n_max, d_order, d_moff, n_mat, loop_weight, sigma, d_M, d_gout, out,
                                              d_gM, d_gsig)
        else:
            B.cos_connected_sum_matrices(n_max, d_order, d_moff, n_mat, loop_weight, sigma, d_M, args.precision,
                                         out)
        ev1.record(stream)
        dp_times.append((ev0, ev1))

    for _ in range(max(3, args.warmup)):
        step()
    B.cos_sync_status()
    dp_times.clear()

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
    total = sum(times)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    value = world * n_cfg * args.steps / total
    # FP64 roofline denominator from unit counts and the clock seen in the timed region: the
    # FP64 pipe retires 2 FMA lanes per clock per SM (ncu: the FMA probe issues 1.68 FP64
    # lanes per SM-cycle at 84.2 % sm__pipe_fp64_cycles_active), 2 flop per FMA.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2032.0
    fp64_peak = sms * FP64_FMA_PER_CLK_SM * 2.0 * clk * 1e6
    peak_source = (f"unit count: {sms} SMs x {FP64_FMA_PER_CLK_SM} FP64 FMA/clk/SM x 2 flop x "
                   f"{clk:.0f} MHz (median SM clock in the timed region)")
    dp_avg = statistics.mean(a.elapsed_time(b) * 1e-3 for a, b in dp_times)
    # The gradient call runs the forward sweep and its reverse: two multiply-adds (Obar and dM)
    # per forward multiply-add, so three times the forward's algorithmic flops.
    flops_launch = algorithmic_flops(B, cfgs.order, n_mat, sigma is not None) * (3 if args.grad else 1)
    achieved = flops_launch / dp_avg
    traffic = (HEADLINE_DRAM_BYTES_PER_CFG * n_cfg
               if args.workload == WORKLOAD and args.precision == "fp64" and not args.grad else None)
    hbm_gbs, hbm_src = measured_hbm_gbs()

    # end to end through the public call with host buffers (pinned), copies inside the region
    h_order = torch.tensor(cfgs.order).pin_memory()
    h_offset = torch.tensor(cfgs.offset).pin_memory()
    h_site = torch.tensor(cfgs.site).pin_memory()
    h_tau = torch.tensor(cfgs.tau).pin_memory()
    h_out = torch.empty(n_cfg, dtype=torch.float64).pin_memory()
    e_order, e_offset, e_site, e_tau = (torch.empty_like(x, device="cuda") for x in (h_order, h_offset, h_site, h_tau))
    e_out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")

    def e2e_step():
        for dst, src in ((e_order, h_order), (e_offset, h_offset), (e_site, h_site), (e_tau, h_tau)):
            dst.copy_(src, non_blocking=True)
        B.cos_connected_sum_batch(tabs, n_max, e_order, e_offset, e_site, e_tau, args.precision, e_out)
        h_out.copy_(e_out, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_times = time_steps(torch, e2e_step, max(2, min(args.steps, 5)), lambda: flush_l2(flush_buf))
    B.cos_sync_status()
    h2d = sum(x.numel() * x.element_size() for x in (h_order, h_offset, h_site, h_tau))
    d2h = h_out.numel() * h_out.element_size()
    e2e_mean = statistics.mean(e2e_times)
    if world > 1:   # the job's end-to-end time is the slowest rank's
        te = torch.tensor([e2e_mean], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        e2e_mean = float(te.item())
    e2e_value = world * n_cfg / e2e_mean
    head_out = out.cpu().numpy()
    extras, keep = {}, {}
    # the other forms and the CPU baseline are single-GPU measurements (N = 1 only)
    if not args.no_extras and world == 1:
        extras, keep = measure_forms(torch, B, flush_buf, fp64_peak, sms * 128 * clk * 1e6)

    launches_per_step = 1 + 4 + 1   # gather, 4 planner kernels, DP
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32 extension / f64 close",
                                                       "df64": "f32 pairs (df64)"}[args.precision], "data": "synthetic",
        "config": {"workload": args.workload, "n": n_max, "n_flavors": w.model.n_flavors, "n_cfg_per_gpu": n_cfg,
                   "L": w.model.L, "beta": w.model.beta, "U": w.model.U, "mu": list(w.model.mu),
                   "alpha": list(w.model.alpha), "n_tau": w.model.n_tau, "precision": args.precision,
                   "full_size": n_cfg == w.n_cfg,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"configs sharded x{world}"},
        "roofline": {"bound": "alu", "pipe": "fp64 fma", "achieved": achieved / 1e12,
                     "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "peak_source": peak_source, "probe_tflops": probe / 1e12,
                     "peak_nominal": NOMINAL_FP64_TFLOPS, "frac_of_nominal": achieved / 1e12 / NOMINAL_FP64_TFLOPS,
                     "kernel": ("dp_adjoint_kernel<sigma grad>" if args.grad else
                                "dp_forward_kernel<%s>" % {"fp64": "double", "mixed": "float",
                                                           "df64": "df64"}[args.precision]),
                     "flops_per_launch": flops_launch,
                     "launch_ms": dp_avg * 1e3,
                     "traffic": traffic,
                     "traffic_source": "ncu DRAM bytes of a 5000-configuration launch, scaled by configurations",
                     # the other roof: DRAM rate of the same launch against the measured copy bandwidth
                     "dram_gbs": (traffic / dp_avg / 1e9) if traffic else None,
                     "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": hbm_src,
                     "dram_frac": (traffic / dp_avg / 1e9 / hbm_gbs) if traffic else None},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "wall_s_timed_region": t_wall,
    }
    if extras:
        line["forms"] = extras
    if rank == 0:
        if not args.no_cpu and world == 1:
            line["cpu_baseline"], line["accuracy"] = oracle_leg(w, args.cpu_seconds, head_out, keep)
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
        out.update({"max_err_over_mass": float(np.max(em)), "median_kappa": float(np.median(mass / np.abs(ref))),
                    "max_kappa": float(np.max(mass / np.abs(ref)))})
    return out


def oracle_leg(w, budget, head_out, keep):
    """The CPU oracle on the host cores: its throughput on a bounded sample of the headline
    workload, and the error of the GPU results of the same configurations against it (FP64
    headline; mixed-precision forms against the FP64 oracle, per configuration)."""
    rate, threads, n, vals = cpu_oracle_rate(w, budget)
    base = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} configurations of the n=8 SU(4) workload (numpy gather + C DP in double, OpenMP)"}
    mass, _ = oracle_values(w, I.workload_configs(w, n), absmode=True)
    acc = {"su4_n8_fp64_vs_oracle": error_stats(head_out[:n], vals, mass)}
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


def measure_adjoint(torch, B, flush_buf, n_cfg):
    """Gradient overhead on the adjoint workload (SU(4), mu broken, n = 10): the gradient call
    (forward recomputed with every layer kept + reverse DP + chain rule to mu, alpha) against
    the forward call on the same configurations."""
    w = I.WORKLOADS["su4_adjoint_n10"]
    cfgs = I.workload_configs(w, n_cfg)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
    gmu = torch.empty(n_cfg, 4, dtype=torch.float64, device="cuda")
    gal = torch.empty_like(gmu)
    fwd = lambda: B.cos_connected_sum_batch(tabs, 10, *d, "fp64", out)
    grad = lambda: B.cos_connected_sum_grad(tabs, 10, *d, gout, gmu=gmu, galpha=gal)
    fwd()
    grad()      # full-size warm-up: sizes every workspace before the timed calls
    B.cos_sync_status()
    tf = statistics.mean(time_steps(torch, fwd, 1, lambda: flush_l2(flush_buf)))
    tg = statistics.mean(time_steps(torch, grad, 1, lambda: flush_l2(flush_buf)))
    B.cos_sync_status()
    tabs.close()
    fl = 3 * algorithmic_flops(B, cfgs.order, 4, False)   # forward sweep + reverse (2 multiply-adds per edge)
    return {"configs": n_cfg, "forward_configs_per_s": n_cfg / tf, "grad_configs_per_s": n_cfg / tg,
            "grad_overhead": tg / tf, "grad_tflops": fl / tg / 1e12}


def measure_subsets(torch, B, flush_buf, n_cfg):
    """All-subsets mode on the headline workload (SU(4), mu broken, n = 8): c(S) of all 255
    vertex subsets and a(S) by the GPU subset exponential, against the plain call (c(V) only)
    on the same gathered matrices.  Also the root-0 by-product (c(S) for S containing vertex 0)."""
    w = I.WORKLOADS[WORKLOAD]
    cfgs = I.workload_configs(w, n_cfg)
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
    for f in (plain, root0, full):
        f()
    B.cos_sync_status()
    tp, t0, tf = (statistics.mean(time_steps(torch, f, 2, lambda: flush_l2(flush_buf))) for f in (plain, root0, full))
    B.cos_sync_status()
    tabs.close()
    return {"configs": n_cfg, "plain_configs_per_s": n_cfg / tp, "root0_configs_per_s": n_cfg / t0,
            "all_subsets_configs_per_s": n_cfg / tf, "all_subsets_cost_vs_plain": tf / tp,
            "root0_cost_vs_plain": t0 / tp}


def measure_bipartite(torch, B, flush_buf, n_cfg, precision="fp64"):
    """Honeycomb workload (SU(2), antiferromagnetic staggered shift, n = 8; sublattices summed
    per vertex by the sublattice-resolved DP): gather + bipartite DP from vertex coordinates."""
    w = I.WORKLOADS["hc_su2_af_n8"]
    cfgs = I.workload_configs(w, n_cfg)
    tabs = B.honeycomb_tables_for(w.model)
    n_mat = tabs.info().n_mat
    d = B.configs_to_device(cfgs)
    out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
    fn = lambda: B.cos_connected_sum_bipartite_batch(tabs, 8, *d, precision, out)
    fn()
    B.cos_sync_status()
    t = statistics.mean(time_steps(torch, fn, 2, lambda: flush_l2(flush_buf)))
    B.cos_sync_status()
    s = B.cos_bipartite_structure(8)
    fl = n_cfg * n_mat * 2.0 * (s.fma_ext + s.fma_close)
    tabs.close()
    return {"configs": n_cfg, "configs_per_s": n_cfg / t, "tflops": fl / t / 1e12, "ms": t * 1e3,
            "assignments_per_config": 256}


def det_fma(B, n: int) -> int:
    """Multiply-adds of one spin block of the determinant-weight DP at order n: those of the
    merged structure minus the first loop's step onto vertex 0, which Alg. 1 does not take
    (one per endpoint state of every mask with vertex 0 half-visited: k other visited
    vertices give max(k, 1) endpoints, and C(n-1, k) 2^k masks have k)."""
    s = B.cos_structure(n)
    saved = sum(math.comb(n - 1, k) * 2 ** k * max(k, 1) for k in range(n))
    return s.fma_ext - saved + s.fma_close


def measure_det(torch, B, flush_buf, fp64_peak: float, fp32_lane_ops: float):
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
    for f in fns.values():
        f()
    B.cos_sync_status()
    ts = {p: statistics.mean(time_steps(torch, f, 2, lambda: flush_l2(flush_buf))) for p, f in fns.items()}
    B.cos_sync_status()
    fl = n_cfg * 2 * 2.0 * det_fma(B, n)
    for p in ("fp64", "df64", "mixed"):
        r = {"configs": n_cfg, "configs_per_s": n_cfg / ts[p], "ms": ts[p] * 1e3,
             "cost_vs_cos_fp64": ts[p] / ts["cos"]}
        if p == "fp64":
            r["tflops"] = fl / ts[p] / 1e12
            r["frac_fp64_peak"] = fl / ts[p] / fp64_peak
        elif p == "df64":
            r["frac_fp32_floor"] = fl / 2.0 * DF64_FP32_PER_TERM / ts[p] / fp32_lane_ops
        else:
            s = B.cos_structure(n)
            r["frac_fp64_peak_close"] = n_cfg * 2 * 2.0 * s.fma_close / ts[p] / fp64_peak
        res[f"su2_zeeman_n10_det_{p}"] = r
    # gradient (reverse sweep of the determinant weights): dc/dM and dc/dalpha of every configuration
    gout = torch.ones(n_cfg, dtype=torch.float64, device="cuda")
    gM = torch.empty_like(M)
    ga = torch.empty(n_cfg, 2, dtype=torch.float64, device="cuda")
    gfn = lambda: B.cos_connected_det_matrices_grad(n, d[0], moff, None, M, gout, None, gM, ga)
    gfn()
    B.cos_sync_status()
    tg = statistics.mean(time_steps(torch, gfn, 1, lambda: flush_l2(flush_buf)))
    B.cos_sync_status()
    # every vertex subset: c(S) and a(S) = det(A_up[S]) det(A_dn[S]) (CDet's set of minors)
    cs = torch.empty(n_cfg << n, dtype=torch.float64, device="cuda")
    as_ = torch.empty_like(cs)
    sfn = lambda: B.cos_connected_det_subsets(n, d[0], moff, None, M, cs, as_, True)
    sfn()
    B.cos_sync_status()
    tsub = statistics.mean(time_steps(torch, sfn, 1, lambda: flush_l2(flush_buf)))
    B.cos_sync_status()
    res["su2_zeeman_n10_det_all_subsets_fp64"] = {"configs": n_cfg, "configs_per_s": n_cfg / tsub,
                                                  "ms": tsub * 1e3, "cost_vs_plain": tsub / ts["fp64"]}
    del cs, as_
    res["su2_zeeman_n10_det_grad_fp64"] = {"configs": n_cfg, "grad_configs_per_s": n_cfg / tg, "ms": tg * 1e3,
                                           "grad_overhead": tg / ts["fp64"],
                                           "frac_fp64_peak": 3 * fl / tg / fp64_peak}
    got = outs["fp64"].cpu().numpy()
    cos = outs["cos"].cpu().numpy()
    res["su2_zeeman_n10_det_fp64"]["max_rel_diff_vs_cos_over_2n"] = float(np.max(np.abs(got - cos / 2.0 ** n) / np.abs(got)))
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
    for f in hfns.values():
        f()
    B.cos_sync_status()
    ht = {k: statistics.mean(time_steps(torch, f, 2, lambda: flush_l2(flush_buf))) for k, f in hfns.items()}
    B.cos_sync_status()
    htabs.close()
    for k in ("det_fp64", "det_df64", "det_mixed"):
        res[f"hc_su2_af_n8_{k}"] = {"configs": hc.n_cfg, "configs_per_s": hc.n_cfg / ht[k], "ms": ht[k] * 1e3,
                                    "cost_vs_cos_fp64": ht[k] / ht["cos_fp64"]}
    # every vertex subset of both bipartite sweeps: c(S) of all 255 subsets (8 rooted derived
    # problems per configuration) and a(S) by the subset exponential, against the plain call
    hcs = torch.empty(hc.n_cfg * 256, dtype=torch.float64, device="cuda")
    has = torch.empty_like(hcs)
    sfns = {"cos_fp64": lambda: B.cos_connected_sum_bipartite_subsets(8, hd[0], hmoff, 2, 1, None, M4, hcs, has),
            "det_fp64": lambda: B.cos_connected_det_bipartite_subsets(8, hd[0], hmoff, al, M4, hcs, has)}
    for k, f in sfns.items():
        f()
        B.cos_sync_status()
        tsk = statistics.mean(time_steps(torch, f, 1, lambda: flush_l2(flush_buf)))
        B.cos_sync_status()
        res[f"hc_su2_af_n8_{k.split('_')[0]}_all_subsets_fp64"] = {
            "configs": hc.n_cfg, "configs_per_s": hc.n_cfg / tsk, "ms": tsk * 1e3, "cost_vs_plain": tsk / ht[k]}
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
        f()
        B.cos_sync_status()
        tgk = statistics.mean(time_steps(torch, f, 1, lambda: flush_l2(flush_buf)))
        B.cos_sync_status()
        res[f"hc_su2_af_n8_{k.split('_')[0]}_grad_fp64"] = {"configs": hc.n_cfg, "grad_configs_per_s": hc.n_cfg / tgk,
                                                           "ms": tgk * 1e3, "grad_overhead": tgk / ht[k]}
    return res, got


# FP32 instructions a double-float term needs at least (the Dot2 step: 1 multiply, 3 FMA,
# 8 additions; the first term of a dot product fewer): the FP32-pipe floor of that mode.
DF64_FP32_PER_TERM = 11.5


def close_flops(B, order: np.ndarray, n_mat: int) -> float:
    """FP64 flops of the loop-closing sums alone (2 per close multiply-add)."""
    total = 0.0
    for n in np.unique(order):
        s = B.cos_structure(int(n))
        total += int((order == n).sum()) * n_mat * 2.0 * s.fma_close
    return total


def measure_forms(torch, B, flush_buf, fp64_peak: float, fp32_lane_ops: float):
    """The other forms of the path on the same GPU: FP64 vs mixed vs double-float (df64)
    precision at orders 8 and 10,
    the uneven-order batch as one persistent launch in a CUDA graph (autotuned shapes), the
    adjoint, and the plain FP64 form with one configuration per launch.  Returns the
    measurements and the GPU outputs kept for the oracle leg's error statistics."""
    res, keep = {}, {}

    def run(name, n_cfg, prec, steps=2, graph=False):
        w = I.WORKLOADS[name]
        cfgs = I.workload_configs(w, n_cfg)
        tabs = B.tables_for(w.model)
        d = B.configs_to_device(cfgs)
        out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
        nmax = int(cfgs.order.max())
        n_mat = tabs.info().n_mat
        if graph:
            plan = B.cos_plan_create_batch(tabs, nmax, *d, prec, out)
            fn = plan.launch
        else:
            fn = lambda: B.cos_connected_sum_batch(tabs, nmax, *d, prec, out)
            fn()
        B.cos_sync_status()
        ts = time_steps(torch, fn, steps, lambda: flush_l2(flush_buf))
        if graph:
            plan.status()
            plan.close()
        B.cos_sync_status()
        fl = algorithmic_flops(B, cfgs.order, n_mat, any(w.model.sigma))
        t = statistics.mean(ts)
        tabs.close()
        r = {"configs": n_cfg, "configs_per_s": n_cfg / t, "tflops": fl / t / 1e12, "ms": t * 1e3,
             "launch_shape_n_max": dict(zip(("warps", "ctas_per_sm", "prefetch"), B.cos_get_tuning(nmax, prec, n_mat)))}
        # roofline of the form: FP64 pipe (FP64), FP64 pipe for the close (mixed), FP32 floor
        # of the compensated terms (double-float); peaks from the headline's clock sample
        if prec == "fp64":
            r["frac_fp64_peak"] = fl / t / fp64_peak
        elif prec == "mixed":
            cf = close_flops(B, cfgs.order, n_mat)
            r["fp64_close_tflops"] = cf / t / 1e12
            r["frac_fp64_peak_close"] = cf / t / fp64_peak
        else:
            terms = fl / 2.0
            r["frac_fp32_floor"] = terms * DF64_FP32_PER_TERM / t / fp32_lane_ops
        if graph:
            r["cuda_graph"] = True
        return r, out.cpu().numpy()

    # SU(2) symmetric, order 4, 10^4 configurations: latency- and launch-bound (about 15 us of
    # FP64 work), one plain call and one CUDA-graph plan launch
    res["su2_n4_fp64"], _ = run("su2_sym_n4", 10_000, "fp64", steps=5)
    res["su2_n4_fp64_graph"], _ = run("su2_sym_n4", 10_000, "fp64", steps=5, graph=True)
    res["su4_n8_mixed"], keep_n8 = run("su4_mu_broken_n8", 100_000, "mixed")
    keep["su4_n8_mixed_vs_fp64_oracle"] = ("su4_mu_broken_n8", keep_n8)
    res["su3_shift_n10_mixed"], keep_n10 = run("su3_shift_mixed_n10", 100_000, "mixed")
    keep["su3_shift_n10_mixed_vs_fp64_oracle"] = ("su3_shift_mixed_n10", keep_n10)
    res["su3_shift_n10_fp64"], keep_f10 = run("su3_shift_mixed_n10", 100_000, "fp64", steps=1)
    keep["su3_shift_n10_fp64_vs_oracle_ld"] = ("su3_shift_mixed_n10", keep_f10)
    res["su4_n8_df64"], keep_df8 = run("su4_mu_broken_n8", 100_000, "df64")
    keep["su4_n8_df64_vs_fp64_oracle"] = ("su4_mu_broken_n8", keep_df8)
    res["su3_shift_n10_df64"], keep_df10 = run("su3_shift_mixed_n10", 100_000, "df64", steps=1)
    keep["su3_shift_n10_df64_vs_fp64_oracle"] = ("su3_shift_mixed_n10", keep_df10)
    res["su6_uneven_n4_12_fp64_graph"], keep_un = run("su6_sym_uneven_n4_12", 200_000, "fp64", steps=1, graph=True)
    wu = I.WORKLOADS["su6_sym_uneven_n4_12"]
    mats = {n: (idx, gathered_matrices(torch, B, wu, idx)) for n, idx in sample_by_order(wu, 200_000).items() if idx}
    keep["su6_uneven_fp64_by_order"] = ("su6_sym_uneven_n4_12", (keep_un, mats))
    adj = measure_adjoint(torch, B, flush_buf, 50_000)
    adj["frac_fp64_peak"] = adj["grad_tflops"] * 1e12 / fp64_peak
    res["su4_n10_adjoint"] = adj
    res["su4_n8_all_subsets_fp64"] = measure_subsets(torch, B, flush_buf, 100_000)
    hb = measure_bipartite(torch, B, flush_buf, I.WORKLOADS["hc_su2_af_n8"].n_cfg)
    hb["frac_fp64_peak"] = hb["tflops"] * 1e12 / fp64_peak
    res["hc_su2_af_n8_bipartite_fp64"] = hb
    hd = measure_bipartite(torch, B, flush_buf, I.WORKLOADS["hc_su2_af_n8"].n_cfg, "df64")
    hd["frac_fp32_floor"] = hd["tflops"] * 1e12 / 2.0 * DF64_FP32_PER_TERM / fp32_lane_ops
    res["hc_su2_af_n8_bipartite_df64"] = hd
    res["hc_su2_af_n8_bipartite_mixed"] = measure_bipartite(torch, B, flush_buf, I.WORKLOADS["hc_su2_af_n8"].n_cfg,
                                                            "mixed")
    det, det_out = measure_det(torch, B, flush_buf, fp64_peak, fp32_lane_ops)
    res.update(det)
    keep["su2_zeeman_n10_det_fp64_vs_oracle"] = ("su2_zeeman_det_n10", det_out)
    # plain FP64 per-configuration form: one configuration per call, no graph
    w = I.WORKLOADS[WORKLOAD]
    cfgs = I.workload_configs(w, 200)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    per = []
    for c in range(200):
        o = int(cfgs.offset[c])
        per.append((d[0][c:c + 1], torch.zeros(1, dtype=torch.int64, device="cuda"), d[2][o:o + 8], d[3][o:o + 8]))
    B.cos_connected_sum_batch(tabs, 8, *per[0], "fp64", out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for a in per:
        B.cos_connected_sum_batch(tabs, 8, *a, "fp64", out)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    res["su4_n8_fp64_one_config_per_launch"] = {"configs": 200, "configs_per_s": 200 / t}
    B.cos_sync_status()
    tabs.close()
    return res, keep


def bipartite_arm(args):
    """Profiling runs of the bipartite path alone: the honeycomb workload's gather + DP from
    vertex coordinates, at its order or --order, --n-cfg configurations, CUDA-event timing;
    with --subsets, gather + the all-subsets mode (c(S) and a(S) of every subset, FP64)."""
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
                                 "bipartite connected-sum configs/s (honeycomb, sublattices summed)"),
                      "value": n_cfg / t, "unit": "configs/s", "order": n, "configs": n_cfg,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
                      "tflops": None if args.subsets else fl / t / 1e12,
                      "dtype": "f64" if args.subsets else {"fp64": "f64", "df64": "f32 pairs (df64)"}.get(
                          args.precision, args.precision)}), flush=True)
    tabs.close()


def subsets_arm(args):
    """Profiling runs of the all-subsets mode alone: gather + cos_connected_sum_subsets with
    all roots and a(S) on --n-cfg configurations of the headline workload (SU(4), n = 8)."""
    import torch
    from paper_2507_12349_b300 import binding as B
    B.lib()
    w = I.WORKLOADS[WORKLOAD]
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
