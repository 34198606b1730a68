#!/usr/bin/env python
"""Benchmark of the spin-adapted two-site DMRG hot path on GB300.

Metric: H_eff matvec GFLOP/s (planner-counted flops of the nonzero block products,
FP64) and the time of the sweep step that contains it.  One step = one micro-iteration
at the middle site pair of the workload: Eq. 25 (TT -> S), the H_eff diagonal and
term tables, Davidson with a fixed number of iterations (each one H_eff matvec), the
decomposition and truncation of Eqs. 26-28 to D, and the operator update in the
step's direction (alternating right / left, so both updates are timed).

Default workload: L=28 orbitals, N=12, S=0, Ag, D2h irreps 8/3/3/2/6/2/2/2 (contiguous),
random integrals (h: N(0,0.5) off-diagonal within an irrep, diagonal -2..0; V = sum over
84 symmetric factor matrices with N(0,0.3) entries), D_SU(2) = 2500, initial MPS of
Sec. 4.3 (seed 2415028) brought to mixed canonical form at sites (13, 14).

Multi-GPU: replicas only (the path does not shard across GPUs); each rank runs the same
workload and value sums the ranks' flops over the max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff matvec GFLOP/s + sweep time, mixed vs FP64 on 1 GB300 at |ΔE|≤1e-6 Eh"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="random28")
    p.add_argument("--D", type=int, default=None)
    p.add_argument("--davidson-iters", type=int, default=12)
    p.add_argument("--precision", type=int, default=0, choices=[0, 1],
                   help="0: FP64 block products; 1: split-TF32 tensor cores + FP64 finish")
    p.add_argument("--fp64-iters", type=int, default=2,
                   help="FP64 Davidson iterations that finish each mixed-precision step")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def fp64_peak_measured():
    """FP64 roof on this GPU: cuBLAS DGEMM 8192^3 throughput (best of 3), measured here
    because the driver's peak file carries HBM and bf16 only."""
    import torch
    n = 8192
    a = torch.randn(n, n, device="cuda", dtype=torch.float64)
    b = torch.randn(n, n, device="cuda", dtype=torch.float64)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(); torch.matmul(a, b); e.record(); torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (s.elapsed_time(e) * 1e-3) / 1e9)
    del a, b
    torch.cuda.empty_cache()
    return best  # GFLOP/s


def setup_context(args):
    from paper_1312_2415_gb300 import Context
    from workloads import make_problem
    cfg, h, V = make_problem(args.workload)
    D = args.D or cfg["D"]
    L, N = cfg["L"], cfg["N"]
    ctx = Context(L, cfg["group_irreps"], N, cfg["two_S"], cfg["irrep"], group=7)
    ctx.set_integrals(h, V)
    # tolerance below attainable precision: every step runs exactly davidson_iters
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-14, args.davidson_iters)
    ctx.set_precision(args.precision, args.fp64_iters)
    ctx.init_mps(cfg.get("seed", 1))
    center = L // 2 - 1
    ctx.canonicalize(center)
    return ctx, cfg, D, center


def run_gb300(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    peak64 = fp64_peak_measured()
    ctx, cfg, D, center = setup_context(args)
    n_x, _ = ctx.layout(center)
    for w in range(args.warmup):
        ctx.sweep_step(center, 1 if w % 2 == 0 else -1, D)
    torch.cuda.synchronize()
    st0 = ctx.stats()
    clk = ClockSampler(torch.cuda.current_device())
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    energies = []
    for k in range(args.steps):
        e, wd, it, ok = ctx.sweep_step(center, 1 if (args.warmup + k) % 2 == 0 else -1, D)
        energies.append(e)
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    st1 = ctx.stats()
    flops = st1["matvec_flops"] - st0["matvec_flops"]
    t_max = allreduce_max(ms, world)
    flops_all = allreduce_sum(flops, world)
    value = flops_all / (t_max * 1e-3) / 1e9
    launches = int(st1["kernels_launched"] - st0["kernels_launched"])
    nmv = st1["k_launches"] - st0["k_launches"]
    k1 = (st1["k_phase1_ms"] - st0["k_phase1_ms"]) / max(nmv, 1)
    k2 = (st1["k_phase2_ms"] - st0["k_phase2_ms"]) / max(nmv, 1)
    f1 = (st1["k_phase1_flops"] - st0["k_phase1_flops"]) / max(nmv, 1)
    f2 = (st1["k_phase2_flops"] - st0["k_phase2_flops"]) / max(nmv, 1)
    dom, fl, kms = ("phase2 (left-block operators)", f2, k2) if k2 >= k1 else ("phase1 (right-block operators)", f1, k1)
    achieved = fl / (kms * 1e-3) / 1e9
    roof = {"bound": "alu", "kernel": "k_grouped_gemm " + dom, "achieved": achieved / 1e3,
            "peak": peak64 / 1e3, "unit": "TFLOP/s", "frac": achieved / peak64,
            "traffic": None, "peak_source": "FP64 cuBLAS DGEMM 8192^3 measured by bench.py on this GPU",
            "launch_ms": kms, "flops_per_launch": fl,
            "matvec_kernel_gflops": (f1 + f2) / ((k1 + k2) * 1e-3) / 1e9}
    # one marked matvec after the timed region (an NVTX range for kernel profilers)
    import numpy as np
    xprof = torch.tensor(ctx.tt_to_x(center), dtype=torch.float64, device="cuda")
    yprof = torch.empty_like(xprof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("matvec")
    ctx.matvec(center, xprof, yprof)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ctx, center, D, args, n_x)
    out = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: random integrals L={cfg['L']} N={cfg['N']} S=0 Ag "
                               f"D2h 8/3/3/2/6/2/2/2, D_SU(2)={D}, middle sites ({center},{center + 1})",
                   "L": cfg["L"], "N": cfg["N"], "D": D, "site": center, "two_site_elements": n_x,
                   "davidson_iters_per_step": args.davidson_iters,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (renormalised operators of both environments, several GB)"},
        "matvecs": nmv, "micro_iteration_s": t_max / args.steps / 1e3,
        "energy_last": energies[-1] if energies else None,
        "clocks": clocks, "gpu_launches": launches, "roofline": roof,
    }
    if e2e:
        out["e2e"] = e2e
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(bounded_seconds=15.0)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(ctx, center, D, args, n_x):
    """Same steps through the host-pointer C ABI: x crosses host<->device every step
    (tt_to_x to pinned host, Davidson from / to host, truncation from host)."""
    import numpy as np
    import torch
    x = torch.empty(n_x, dtype=torch.float64).pin_memory().numpy()
    st0 = ctx.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ctx.tt_to_x(center, x)
        ctx.davidson(center, x)
        ctx.truncate(center, 1 if k % 2 == 0 else -1, D, x)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st1 = ctx.stats()
    flops = st1["matvec_flops"] - st0["matvec_flops"]
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": 2 * 8 * n_x,
            "d2h_bytes_per_step": 2 * 8 * n_x + 8,
            "path": "dmrg_tt_to_x / dmrg_davidson / dmrg_truncate with host buffers"}


def oracle_sample():
    """The oracle's H_eff matvec (P^T H P applied to x) at the middle site pair of the
    L=8 Hubbard chain with D=64: the largest member of the workload family the oracle
    evaluates in seconds (determinant expansion of the two-site basis)."""
    from oracle import dmrg as odmrg
    from oracle import mps as om
    from workloads import hubbard_chain, uniform_pm1
    L, N = 8, 8
    h, V = hubbard_chain(L, 1.0, 4.0)
    irr = [0] * L
    m = om.right_canonicalize(om.random_mps(irr, N, 0, 0, 64, uniform_pm1(2415001, 10 ** 6)))
    i = L // 2 - 1
    for k in range(i):
        om.svd_truncate(m, k, om.tt_to_x(m, k), 10 ** 9, "right")
    prob = odmrg.Problem(h, V, irr, N, 0, 0)
    return prob, m, i


def sample_flops():
    """Planner-counted flops of one matvec of the oracle sample (the metric's unit)."""
    from paper_1312_2415_gb300 import Context
    from tests.mps_io import mps_to_bytes
    import numpy as np
    prob, m, i = oracle_sample()
    ctx = Context(prob.L, prob.irreps, prob.N, 0, 0)
    ctx.set_integrals(prob.h, prob.V)
    ctx.set_mps(mps_to_bytes(m))
    n, _ = ctx.layout(i)
    ctx.matvec(i, np.ones(n))
    return ctx.stats()["last_matvec_flops"]


def cpu_baseline(bounded_seconds=15.0, flops=None):
    from oracle import dmrg as odmrg
    from oracle import mps as om
    import numpy as np
    prob, m, i = oracle_sample()
    if flops is None:
        flops = sample_flops()
    x = om.tt_to_x(m, i)
    t0 = time.perf_counter()
    n = 0
    while True:
        odmrg.matvec(prob, m, i, x)
        n += 1
        if time.perf_counter() - t0 > bounded_seconds:
            break
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return {"value": flops * n / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle H_eff matvecs (P^T H P, determinant basis) at sites (3,4) of "
                      f"the L=8 Hubbard chain, D=64, {dt:.1f} s; flops counted by the planner "
                      f"for the same matvec ({flops:.3e})"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import dmrg as odmrg
    from oracle import mps as om
    import numpy as np
    prob, m, i = oracle_sample()
    try:
        flops = sample_flops()
    except Exception:
        flops = None
    x = om.tt_to_x(m, i)
    for _ in range(args.warmup):
        odmrg.matvec(prob, m, i, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        odmrg.matvec(prob, m, i, x)
    dt = time.perf_counter() - t0
    value = (flops * args.steps / dt / 1e9) if flops else None
    cb = {"value": value, "unit": "GFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "oracle H_eff matvec (P^T H P) at sites (3,4) of the L=8 Hubbard chain, D=64"}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "oracle sample: L=8 Hubbard chain, D=64, "
                                                       "middle sites, one H_eff matvec per step"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
