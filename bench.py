#!/usr/bin/env python
"""Benchmark of the spin-adapted two-site DMRG hot path on GB300.

Metric: H_eff matvec GFLOP/s (planner-counted flops of the nonzero block products) and
the time of the sweep step that contains it, for the mixed-precision path (block
products on the tensor cores in split TF32 with FP32 accumulation, Davidson finished
in FP64) against the FP64 path on the same state, with the energy difference of the
two.  One step = one micro-iteration at the middle site pair of the workload: Eq. 25
(TT -> S), the H_eff diagonal and term tables, Davidson with a fixed number of
iterations, the decomposition and truncation of Eqs. 26-28 to D, and the operator
update in the step's direction (alternating right / left, so both updates are timed).

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
    p.add_argument("--precision", type=int, default=1, choices=[0, 1],
                   help="headline path: 1 = split-TF32 tensor cores + FP64 finish, 0 = FP64")
    p.add_argument("--fp64-iters", type=int, default=1,
                   help="FP64 Davidson iterations that finish each mixed-precision step")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison steps")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip both macro-iterations (the headline steps then run on the initial MPS)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64-sweep", action="store_true", help="skip the FP64 macro-iteration")
    p.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 steps on the swept state")
    p.add_argument("--e2e-steps", type=int, default=5, help="steps of the host-buffer e2e run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batch32 summary of the default line")
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


def aggregate(flops, ms, world):
    """Whole-job throughput of replicas: all ranks' flops over the slowest rank's time."""
    t_max = allreduce_max(ms, world)
    return allreduce_sum(flops, world) / (t_max * 1e-3) / 1e9, t_max


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def fp64_peak_measured():
    """FP64 roof on this GPU: cuBLAS DGEMM 8192^3 throughput (best of 3), measured here
    because the measured-peaks file carries HBM and bf16 only."""
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


def tf32_peak_measured():
    """TF32 tensor roof on this GPU: cuBLAS FP32 GEMM 8192^3 with TF32 allowed (best of 3),
    measured here because the measured-peaks file carries HBM and bf16 only."""
    import torch
    n = 8192
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(n, n, device="cuda", dtype=torch.float32)
        b = torch.randn(n, n, device="cuda", dtype=torch.float32)
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(3):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(); torch.matmul(a, b); e.record(); torch.cuda.synchronize()
            best = max(best, 2.0 * n ** 3 / (s.elapsed_time(e) * 1e-3) / 1e9)
        del a, b
        torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return best  # GFLOP/s


def block_histogram(table):
    """Block-size histogram of a two-site layout (rows dL, columns dR of every block)."""
    import numpy as np
    edges = [1, 8, 16, 32, 64, 128, 256, 512, 10 ** 9]
    out = {}
    for name, col in (("dL", 9), ("dR", 10)):
        v = table[:, col]
        out[name] = {f"{edges[k]}-{edges[k + 1] - 1 if edges[k + 1] < 10 ** 9 else 'max'}":
                     int(((v >= edges[k]) & (v < edges[k + 1])).sum()) for k in range(len(edges) - 1)}
    out["blocks"] = int(table.shape[0])
    out["largest"] = [int(table[:, 9].max()), int(table[:, 10].max())]
    out["elements_in_blocks_above_64"] = int((table[:, 9] * table[:, 10] * ((table[:, 9] > 64) | (table[:, 10] > 64))).sum())
    return out


def setup_context(args):
    from paper_1312_2415_gb300 import Context
    from workloads import make_problem
    cfg, h, V = make_problem(args.workload)
    D = args.D or cfg["D"]
    L, N = cfg["L"], cfg["N"]
    ctx = Context(L, cfg["group_irreps"], N, cfg["two_S"], cfg["irrep"], group=7)
    ctx.set_integrals(h, V)
    fixed_iters(ctx, D, args.davidson_iters)
    ctx.set_precision(args.precision, args.fp64_iters)
    ctx.init_mps(cfg.get("seed", 1))
    center = L // 2 - 1
    ctx.canonicalize(center)
    return ctx, cfg, D, center


def fixed_iters(ctx, D, iters):
    # tolerance below attainable precision: every Davidson runs exactly `iters` iterations
    # (a mixed-precision Davidson stops at its own accuracy, then runs the FP64 finish)
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-14, iters)


class Walker:
    """Sites and directions of a sweep that bounces between sites lo and hi (right to hi,
    then left to lo, ...): each step's site is the neighbour of the last one, or the same
    site where the sweep turns, as in a macro-iteration (Sec. 4.2)."""

    def __init__(self, lo, hi):
        self.lo, self.hi, self.site, self.dir = lo, hi, lo, 1

    def peek(self):
        if self.dir > 0:
            return (self.site + 1, 1) if self.site < self.hi else (self.site, -1)
        return (self.site - 1, -1) if self.site > self.lo else (self.site, 1)

    def step(self, ctx, D):
        nxt = self.peek()
        ctx.set_next_site(nxt[0])
        out = ctx.sweep_step(self.site, self.dir, D)
        self.site, self.dir = nxt
        return out


def window(center):
    return center - 5, center + 4


def timed_steps(ctx, walker, D, steps, warmup, clk=None, world=1):
    """warmup + steps micro-iterations of a sweep between two sites around the middle
    (Walker); the timed region is bracketed by barriers, synchronisation and CUDA
    events."""
    import torch
    for _ in range(warmup):
        walker.step(ctx, D)
    torch.cuda.synchronize()
    st0 = ctx.stats()
    barrier(world)
    torch.cuda.synchronize()
    if clk:
        clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("steps")
    ev0.record()
    energies = []
    for _ in range(steps):
        e, wd, it, ok = walker.step(ctx, D)
        energies.append(e)
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop() if clk else None
    ms = ev0.elapsed_time(ev1)
    st1 = ctx.stats()
    delta = {k: st1[k] - st0[k] for k in st1}
    return ms, delta, energies, clocks


def step_breakdown(delta, steps):
    """Where a step's time goes: host wall clock of table planning (including the
    tensor-core tables), truncation (Eqs. 26-28) and operator update, and the device time
    (CUDA events) of the matvec kernels of both precisions; per step, in ms."""
    k = max(steps, 1)
    return {"host_plan": delta["t_plan_ms"] / k, "truncation": delta["t_trunc_ms"] / k,
            "operator_update": delta["t_update_ms"] / k,
            "mixed_matvecs_device": (delta["tc_phase1_ms"] + delta["tc_phase2_ms"]) / k,
            "fp64_matvecs_device": (delta["k_phase1_ms"] + delta["k_phase2_ms"]) / k,
            "mixed_matvecs": delta["tc_matvecs"] / k, "fp64_matvecs": delta["k_launches"] / k}


def matvec_kernel_rates(delta):
    """Device-time GFLOP/s of the matvec kernels by precision (CUDA events around them)."""
    out = {}
    if delta["tc_matvecs"] > 0:
        t = delta["tc_phase1_ms"] + delta["tc_phase2_ms"]
        out["mixed"] = {"matvecs": int(delta["tc_matvecs"]), "ms_per_matvec": t / delta["tc_matvecs"],
                        "gflops": delta["tc_flops"] / (t * 1e-3) / 1e9,
                        "phase1_ms": delta["tc_phase1_ms"] / delta["tc_matvecs"],
                        "phase2_ms": delta["tc_phase2_ms"] / delta["tc_matvecs"]}
    if delta["k_launches"] > 0:
        t = delta["k_phase1_ms"] + delta["k_phase2_ms"]
        f = delta["k_phase1_flops"] + delta["k_phase2_flops"]
        out["fp64"] = {"matvecs": int(delta["k_launches"]), "ms_per_matvec": t / delta["k_launches"],
                       "gflops": f / (t * 1e-3) / 1e9,
                       "phase1_ms": delta["k_phase1_ms"] / delta["k_launches"],
                       "phase2_ms": delta["k_phase2_ms"] / delta["k_launches"]}
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the mixed
# matvec's main kernel from one ncu capture (a smaller case scaled to a full launch by the
# units processed, as the profile summary states), keyed by the workload and the SHA-256
# prefix of the kernel source it was taken with: a changed kernel reports traffic null.
# DRAM bytes per launch of k_tc_matvec (dram__bytes_read.sum + dram__bytes_write.sum, one
# ncu pass, every launch of the timed steps of the default run), keyed by workload and
# the kernel source it was measured on (a changed kernel reports null):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none --nvtx
#       --nvtx-include "steps/" -k regex:k_tc_matvec -c 48 --csv
#       python bench.py --no-fp64 --no-e2e --no-cpu-baseline --no-batch
NCU_TRAFFIC = {
    (("random28", 2500), "f73a6011045fa39d"): {
        "bytes": 4.06e10, "how": "mean over the 48 launches of the timed steps (3.39e10 .. 4.55e10), ncu one pass"},
}


def kernel_source_hash():
    """Hash of the fused kernel's code (comments and blank space left out, so that a
    comment change keeps a measured figure valid)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "paper_1312_2415_gb300", "csrc", "kernels_tc.cu")
    code = re.sub(r"//[^\n]*", "", open(path).read())
    code = re.sub(r"\s+", " ", code)
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def roofline_mixed(delta, peaks, peak_tf32, workload=None):
    """Main kernel of the mixed-precision matvec against both of its roofs: HBM with the
    algorithmic bytes of a matvec (every operator block it reads, once, in its FP32
    mirror, x read and y written once, in FP64), and the TF32 tensor pipe with the
    method's flops (2 m k n per block product, one product per block pair however many
    split products run).  `bound` is the roof that gives the longer time; `frac` is
    achieved / peak on that roof; the other roof is reported beside it."""
    nm = max(delta["tc_matvecs"], 1)
    ms = delta["tc_phase2_ms"] / nm
    byts = delta["tc_phase2_bytes"] / nm
    fl = delta["tc_phase2_flops"] / nm
    if "hbm_gbs" in peaks:
        hbm, hsrc = peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)"
    else:
        hbm, hsrc = 6800.0, "profiling recipe fallback 6.8 TB/s (of fallback)"
    t_hbm, t_tc = byts / (hbm * 1e9), fl / (peak_tf32 * 1e9)
    gbs = byts / (ms * 1e-3) / 1e9
    tfs = fl / (ms * 1e-3) / 1e12
    tr = NCU_TRAFFIC.get((workload, kernel_source_hash())) if workload else None
    traffic = tr["bytes"] if tr else None
    hbm_roof = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "peak_source": hsrc}
    tc_roof = {"achieved": tfs, "peak": peak_tf32 / 1e3, "unit": "TFLOP/s", "frac": tfs / (peak_tf32 / 1e3),
               "peak_source": "cuBLAS FP32 GEMM with TF32, 8192^3, measured by bench.py in this run (of measured)"}
    main, other = (tc_roof, hbm_roof) if t_tc >= t_hbm else (hbm_roof, tc_roof)
    return {"bound": "tensor" if t_tc >= t_hbm else "hbm", "kernel": "k_tc_matvec (fused split-TF32 block "
            "products: x D^T in tensor memory, then C W, per output tile)",
            "achieved": main["achieved"], "peak": main["peak"], "unit": main["unit"], "frac": main["frac"],
            "traffic": traffic, "traffic_source": tr["how"] if tr else None,
            "peak_source": main["peak_source"], "launch_ms": ms,
            "algorithmic_bytes": byts, "method_flops": fl,
            "other_roof": {"bound": "hbm" if main is tc_roof else "tensor", **other}}


def roofline_fp64(delta, peak64):
    nmv = max(delta["k_launches"], 1)
    k1, k2 = delta["k_phase1_ms"] / nmv, delta["k_phase2_ms"] / nmv
    f1, f2 = delta["k_phase1_flops"] / nmv, delta["k_phase2_flops"] / nmv
    name, fl, kms = ("k_grouped_gemm phase 2", f2, k2) if k2 >= k1 else ("k_grouped_gemm phase 1", f1, k1)
    achieved = fl / (kms * 1e-3) / 1e9
    return {"bound": "alu", "kernel": name, "achieved": achieved / 1e3, "peak": peak64 / 1e3,
            "unit": "TFLOP/s", "frac": achieved / peak64, "traffic": None,
            "peak_source": "FP64 cuBLAS DGEMM 8192^3 measured by bench.py on this GPU"}


def energy_agreement(ctx, center, D, args):
    """Both Davidsons from the same two-site vector (no truncation in between), converged
    to 1e-9: the FP64 eigenvalue and the mixed-precision one (FP64 Rayleigh quotient
    after the FP64 finishing iterations).  Also the Rayleigh quotient of the FP64
    eigenvector through the tensor-core matvec against the FP64 one: the bias of the
    tensor cores' FP32 accumulation, which is why energies (and the renormalised
    operators, which enter H itself) stay FP64."""
    import numpy as np
    import torch
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-9, 300)
    x0 = torch.tensor(ctx.tt_to_x(center), dtype=torch.float64, device="cuda")
    out = {}
    for name, prec, fi in (("fp64", 0, 0), ("mixed", 1, args.fp64_iters)):
        ctx.set_precision(prec, fi)
        x = x0.clone()
        st0 = ctx.stats()
        t0 = time.perf_counter()
        e, it, ok = ctx.davidson(center, x)
        torch.cuda.synchronize()
        st1 = ctx.stats()
        out[name] = {"energy": e, "iterations": it, "converged": bool(ok), "s": time.perf_counter() - t0,
                     "tc_matvecs": int(st1["tc_matvecs"] - st0["tc_matvecs"]),
                     "fp64_matvecs": int(st1["k_launches"] - st0["k_launches"])}
        if name == "fp64":
            x64 = x.clone()
    out["abs_diff_eh"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"])
    out["target_eh"] = 1e-6
    y = torch.empty_like(x64)
    rq = {}
    for name, prec in (("fp64", 0), ("tensor_core", 1)):
        ctx.set_precision(prec, 0)
        ctx.matvec(center, x64, y)
        torch.cuda.synchronize()
        rq[name] = (x64 @ y).item() / (x64 @ x64).item()
    out["rayleigh_quotient_tensor_core_minus_fp64_eh"] = rq["tensor_core"] - rq["fp64"]
    ctx.set_precision(args.precision, args.fp64_iters)
    return out


def converged_agreement():
    """The metric's |dE| <= 1e-6 Eh on converged DMRG: the L=12 random-integral system
    (N=12, S=0, D2h irreps round-robin, D_SU(2)=500), macro-iterations until the energy
    changes by less than 1e-10 Eh (at most 4), Davidson tolerance 1e-9, both precisions
    from the same initial MPS; the mixed path runs the tensor-core Davidson, then FP64
    Davidson iterations to the tolerance.  With the seconds of each solve."""
    import torch
    from paper_1312_2415_gb300 import Context
    from workloads import make_problem
    cfg, h, V = make_problem("random12")
    out = {"workload": f"random12: random integrals L={cfg['L']} N={cfg['N']} S=0 Ag, D2h round-robin, "
                       f"D_SU(2)={cfg['D']}, solved to convergence (E_conv 1e-10 Eh, at most 4 macro-iterations, "
                       "Davidson tolerance 1e-9)"}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        ctx = Context(cfg["L"], cfg["group_irreps"], cfg["N"], cfg["two_S"], cfg["irrep"], group=7,
                      precision=prec)
        ctx.set_integrals(h, V)
        ctx.set_schedule([cfg["D"]], [1e-10], [4], [0.0], 1e-9, 200)
        ctx.set_precision(prec, 0)
        ctx.init_mps(cfg["seed"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        emin, elast = ctx.solve()
        torch.cuda.synchronize()
        s = time.perf_counter() - t0
        st = ctx.stats()
        out[name] = {"energy": emin, "energy_last": elast, "s": s, "tc_matvecs": int(st["tc_matvecs"]),
                     "davidson_iterations": int(st["davidson_iters"])}
        ctx.close()
    out["abs_diff_eh"] = abs(out["mixed"]["energy"] - out["fp64"]["energy"])
    out["target_eh"] = 1e-6
    out["speedup_mixed_vs_fp64"] = out["fp64"]["s"] / out["mixed"]["s"]
    return out


def sweep_time(ctx, L, D, precision, fp64_iters, iters):
    """One macro-iteration (Sec. 4.2: sites 0..L-2 right, then L-2..0 left) at fixed D,
    fixed Davidson iterations per step, from the state the context holds (right-canonical
    form first); returns a record with the seconds of both half sweeps, the energy of the
    last step and the lowest one (Sec. 4.3), and the step count."""
    import torch
    ctx.set_precision(precision, fp64_iters)
    fixed_iters(ctx, D, iters)
    ctx.canonicalize(0)
    torch.cuda.synchronize()
    out, es = [], []
    for sites, d in ((range(0, L - 1), 1), (range(L - 2, -1, -1), -1)):
        t0 = time.perf_counter()
        for i in sites:
            last = (d > 0 and i == L - 2) or (d < 0 and i == 0)
            ctx.set_next_site(i if last else i + d)
            e, wd, it, ok = ctx.sweep_step(i, d, D)
            es.append(e)
        torch.cuda.synchronize()
        out.append(time.perf_counter() - t0)
    return {"macro_s": out[0] + out[1], "right_s": out[0], "left_s": out[1], "energy_last": es[-1],
            "energy_min": min(es), "steps": len(es)}


# 32 independent instances of uneven size for the batched launch: Hubbard chains
# (t=1, U=4, C1) L = 8..24 and random-integral systems (D2h, round-robin irreps, built as
# the L=12 system) L = 10..20, N = L, S in {0, 1}, D_SU(2) in {64..1024}
BATCH_HUB_L = [8, 10, 12, 14, 16, 18, 20, 22, 24]
BATCH_RND_L = [10, 12, 14, 16, 18, 20]
BATCH_D = [64, 128, 256, 512, 1024]


def batch_instances():
    out = []
    for k in range(32):
        kind = "hubbard" if k % 2 == 0 else "random"
        L = BATCH_HUB_L[(k // 2) % len(BATCH_HUB_L)] if kind == "hubbard" else BATCH_RND_L[(k // 2) % len(BATCH_RND_L)]
        out.append((kind, L, 0 if (k // 4) % 2 == 0 else 2, BATCH_D[k % len(BATCH_D)], 2415300 + k))
    return out


def batch_contexts(args):
    """The 32 instances at their middle pairs, tables prepared, start vectors (Eq. 25)."""
    import torch
    from paper_1312_2415_gb300 import Context
    from workloads import hubbard_chain, random_integrals, round_robin_irreps
    ctxs, sites, xs, ys = [], [], [], []
    for kind, L, tS, D, seed in batch_instances():
        if kind == "hubbard":
            irr, (h, V), group = [0] * L, hubbard_chain(L, 1.0, 4.0), 0
        else:
            irr = round_robin_irreps(L)
            (h, V), group = random_integrals(irr, seed), 7
        c = Context(L, irr, L, tS, 0, group=group)
        c.set_integrals(h, V)
        fixed_iters(c, D, args.davidson_iters)
        c.set_precision(1, args.fp64_iters)
        c.init_mps(seed)
        i = L // 2 - 1
        c.canonicalize(i)
        x = torch.tensor(c.tt_to_x(i), dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        c.matvec(i, x, y)  # prepares the instance's tables
        ctxs.append(c); sites.append(i); xs.append(x); ys.append(y)
    torch.cuda.synchronize()
    return ctxs, sites, xs, ys


def batch_summary(args):
    """The batch32 matvecs for the default line: one batched persistent launch (fixed
    tile shape, no autotuner) against the instances one at a time, 3 timed runs each."""
    import torch
    from paper_1312_2415_gb300 import Batch
    t0 = time.perf_counter()
    ctxs, sites, xs, ys = batch_contexts(args)

    def timed(fn, k=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    def sequential():
        for c, i, x, y in zip(ctxs, sites, xs, ys):
            c.matvec(i, x, y)
    seq_ms = timed(sequential)
    b = Batch(ctxs, sites, autotune=False)
    bat_ms = timed(lambda: b.run(xs, ys))
    flops = b.info()["flops"]
    b.close()
    for c in ctxs:
        c.close()
    return {"workload": "batch32 (32 instances, Hubbard L=8..24 and random-integral L=10..20, N=L, S in {0,1}, "
                        "D in {64..1024}, middle sites; the initial MPS of Sec. 4.3)",
            "batched_ms": bat_ms, "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / bat_ms,
            "batched_gflops": flops / (bat_ms * 1e-3) / 1e9, "flops_per_matvec_set": flops,
            "s": time.perf_counter() - t0, "details": "python bench.py --workload batch32 (autotuner, batched Davidson)"}


def run_batch(args):
    """batch32: the mixed-precision matvecs of 32 instances, one at a time (one grouped
    launch sequence per instance) against one batched, graph-replayed launch sequence
    over all of them; value = their summed flops over the batched time."""
    import torch
    from paper_1312_2415_gb300 import Batch
    torch.cuda.set_device(0)
    t_setup = time.perf_counter()
    ctxs, sites, xs, ys = batch_contexts(args)
    t_setup = time.perf_counter() - t_setup

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def sequential():
        for c, i, x, y in zip(ctxs, sites, xs, ys):
            c.matvec(i, x, y)
    seq_ms = timed(sequential)
    b = Batch(ctxs, sites, autotune=True)
    info = b.info()
    clk = ClockSampler(torch.cuda.current_device())
    l0 = ctxs[0].stats()["kernels_launched"]
    clk.start()
    bat_ms = timed(lambda: b.run(xs, ys))
    clocks = clk.stop()
    launches = int(ctxs[0].stats()["kernels_launched"] - l0)
    flops = info["flops"]
    out = {"metric": METRIC, "value": flops / (bat_ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": bat_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3-f32acc", "data": "synthetic",
           "config": {"workload": "batch32: 32 instances, Hubbard L=8..24 and random-integral L=10..20, "
                                  "N=L, S in {0,1}, D in {64..1024}, middle sites, one matvec each per step",
                      "instances": [list(q[:4]) for q in batch_instances()], "flops_per_step": flops,
                      "l2": "inputs of the larger instances exceed L2"},
           "sequential": {"ms_per_step": seq_ms, "value": flops / (seq_ms * 1e-3) / 1e9,
                          "what": "the same 32 matvecs one instance at a time (their own launches)"},
           "speedup_vs_sequential": seq_ms / bat_ms, "autotune": info, "setup_s": t_setup,
           "clocks": clocks, "gpu_launches": launches}
    out["davidson"] = batch_davidson_timing(ctxs, sites, b, [q[3] for q in batch_instances()])
    print(json.dumps(out), flush=True)
    b.close()


def batch_davidson_timing(ctxs, sites, b, Ds, tol=1e-4, max_iter=200):
    """Davidson for every instance from Eq. 25's start vector to ||r|| <= tol: in lockstep
    through dmrg_batch_davidson (one batched matvec and one launch per vector operation
    per iteration, FP64 Rayleigh quotient of each result) against one dmrg_davidson per
    instance (tensor-core matvecs, then one FP64 iteration); wall clock of each, and the
    largest energy difference between the two."""
    import numpy as np
    import torch
    starts = [torch.tensor(c.tt_to_x(i), dtype=torch.float64, device="cuda") for c, i in zip(ctxs, sites)]
    for c, D in zip(ctxs, Ds):
        c.set_schedule([D], [0.0], [1], [0.0], tol, max_iter)
        c.set_precision(1, 1)
    xs = [s.clone() for s in starts]
    b.davidson(xs, tol=tol, max_iter=max_iter, fp64_energy=True)  # warm-up
    xs = [s.clone() for s in starts]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eb, itb, cvb = b.davidson(xs, tol=tol, max_iter=max_iter, fp64_energy=True)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    es, its = [], []
    t0 = time.perf_counter()
    for c, i, s in zip(ctxs, sites, starts):
        x = s.clone()
        e, it, ok = c.davidson(i, x)
        es.append(e)
        its.append(it)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    diff = np.abs(np.array(es) - eb)
    return {"batched_s": t_bat, "sequential_s": t_seq, "speedup_vs_sequential": t_seq / t_bat,
            "iterations_batched": [int(v) for v in itb], "iterations_sequential": its,
            "converged": int(np.sum(cvb)), "energies_within_1e-6_eh": int(np.sum(diff <= 1e-6)),
            "instances": len(es), "max_abs_energy_diff_eh": float(np.max(diff)),
            "note": "an instance whose two runs differ converged to another eigenstate from the same start "
                    "(Davidson from Eq. 25 of the initial MPS at tolerance 1e-4)",
            "tol": tol}


def rdm_cpu_baseline(bounded_seconds=10.0):
    """The oracle's RDMs (determinant expansion of the state + E_pq products) of an L=8,
    N=8, D2h random-integral state at D=60, repeated for a bounded time."""
    from oracle import mps as om
    from oracle.rdm import mps_state, rdm_from_vector
    from workloads import round_robin_irreps, uniform_pm1
    irr = round_robin_irreps(8)
    m = om.right_canonicalize(om.random_mps(irr, 8, 0, 0, 60, uniform_pm1(5, 10 ** 6)))
    t0 = time.perf_counter()
    n = 0
    while True:
        rdm_from_vector(*mps_state(m))
        n += 1
        if time.perf_counter() - t0 > bounded_seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": dt / n, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} oracle RDM evaluations of an L=8, N=8, S=0, D2h state at D=60 "
                      f"(the oracle cannot expand the L=16 state), {dt:.1f} s"}


def run_rdm(args):
    """random16: the spin-summed 1- and 2-RDMs (dE/dh, dE/dV) of an L=16, N=16, S=0, D2h
    random-integral state at D=1000 (the initial MPS of Sec. 4.3): one step = one
    dmrg_rdm pass (the adjoint of the H_eff matvec at every site pair, the centre moving
    right), outputs in device memory."""
    import numpy as np
    import torch
    from paper_1312_2415_gb300 import Context
    from workloads import make_problem
    torch.cuda.set_device(0)
    cfg, h, V = make_problem("random16")
    L, D = cfg["L"], args.D or cfg["D"]
    ctx = Context(L, cfg["group_irreps"], cfg["N"], cfg["two_S"], cfg["irrep"], group=7)
    ctx.set_integrals(h, V)
    fixed_iters(ctx, D, args.davidson_iters)
    ctx.init_mps(cfg["seed"])
    gamma = torch.empty((L, L), dtype=torch.float64, device="cuda")
    Gamma = torch.empty((L,) * 4, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ctx.rdm(gamma, Gamma)
    torch.cuda.synchronize()
    st0 = ctx.stats()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.rdm(gamma, Gamma)
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st1 = ctx.stats()
    flops = (st1["rdm_flops"] - st0["rdm_flops"]) / args.steps
    plan_ms = (st1["t_plan_ms"] - st0["t_plan_ms"]) / args.steps
    launches = int(st1["kernels_launched"] - st0["kernels_launched"])
    out = {"metric": "1-/2-RDM pass (dE/dh, dE/dV by the adjoint of the H_eff matvec)",
           "value": ms * 1e-3, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"random16: random integrals L={L} N={cfg['N']} S=0 Ag D2h round-robin, "
                                  f"D_SU(2)={D}, initial MPS of Sec. 4.3 (seed {cfg['seed']}), outputs "
                                  f"gamma (L^2) and Gamma (L^4) on the device",
                      "l2": "operators and two-site objects exceed L2"},
           "gflops": flops / (ms * 1e-3) / 1e9, "flops_per_step": flops,
           "host_plan_ms_per_step": plan_ms, "clocks": clocks, "gpu_launches": launches}
    if not args.no_e2e:
        g_h, G_h = np.zeros((L, L)), np.zeros((L,) * 4)
        t0 = time.perf_counter()
        ctx.rdm(g_h, G_h)
        dt = time.perf_counter() - t0
        out["e2e"] = {"value": dt, "unit": "s", "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": 8 * (L * L + L ** 4)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = rdm_cpu_baseline()
    print(json.dumps(out), flush=True)


def run_gb300(args):
    """The headline workload (random28, D=2500).  Order of the run:
    1. one mixed-precision macro-iteration from the initial MPS of Sec. 4.3 (the metric's
       mixed sweep time); its end state is the swept state the headline steps use;
    2. one FP64 macro-iteration from the same initial MPS with the same Davidson settings
       (the FP64 sweep time);
    3. the timed micro-iterations at the middle pair of the swept state (value), the same
       steps on the FP64 path, the converged-Davidson energy agreement at that pair (and
       the tensor-core Rayleigh quotient's bias), the energy agreement of converged DMRG
       in both precisions on the L=12 system, the roofline of the matvec kernel, and e2e
       through the host-buffer C ABI."""
    import torch
    if args.workload == "batch32":
        return run_batch(args)
    if args.workload == "random16":
        return run_rdm(args)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    peaks = measured_peaks()
    peak64 = fp64_peak_measured()
    peak_tf32 = tf32_peak_measured()
    ctx, cfg, D, center = setup_context(args)
    L = cfg["L"]
    mixed = args.precision == 1
    # 1-2: macro-iterations from the initial state (the metric's sweep time)
    ctx.canonicalize(0)
    start = ctx.get_mps()
    sweeps = {"what": "one macro-iteration (L-1 steps right, L-1 left) from the initial MPS of Sec. 4.3 "
                      f"at fixed D, {args.davidson_iters} Davidson iterations per step; both precisions "
                      "start from the same state"}
    if not args.no_sweep:
        sweeps["mixed" if mixed else "fp64"] = sweep_time(ctx, L, D, args.precision, args.fp64_iters,
                                                          args.davidson_iters)
        swept = ctx.get_mps()
        if mixed and not args.no_fp64 and not args.no_fp64_sweep:
            ctx.set_mps(start)
            sweeps["fp64"] = sweep_time(ctx, L, D, 0, 0, args.davidson_iters)
            # not the agreement criterion: one unconverged macro-iteration from a random
            # MPS at fixed Davidson iterations amplifies matvec rounding into different
            # trajectories (converged_agreement and energy_agreement carry the criterion)
            sweeps["trajectory_difference"] = {
                "abs_diff_last_eh": abs(sweeps["mixed"]["energy_last"] - sweeps["fp64"]["energy_last"]),
                "abs_diff_min_eh": abs(sweeps["mixed"]["energy_min"] - sweeps["fp64"]["energy_min"])}
            sweeps["speedup_mixed_vs_fp64"] = sweeps["fp64"]["macro_s"] / sweeps["mixed"]["macro_s"]
        ctx.set_mps(swept)
        state = "the state one mixed macro-iteration at D leaves (swept state)"
    else:
        state = "the initial MPS of Sec. 4.3"
    ctx.set_precision(args.precision, args.fp64_iters)
    fixed_iters(ctx, D, args.davidson_iters)
    ctx.canonicalize(center)
    n_x, table = ctx.layout(center)
    hist = block_histogram(table)
    lo, hi = window(center)
    ctx.canonicalize(lo)
    swept_state = ctx.get_mps()
    # 3: headline steps on that state
    clk = ClockSampler(torch.cuda.current_device())
    ms, delta, energies, clocks = timed_steps(ctx, Walker(lo, hi), D, args.steps, args.warmup, clk, world)
    value, t_max = aggregate(delta["matvec_flops"], ms, world)
    launches = int(delta["kernels_launched"])
    rates = matvec_kernel_rates(delta)
    roof = roofline_mixed(delta, peaks, peak_tf32, (args.workload, D)) if mixed else roofline_fp64(delta, peak64)
    fp64 = None
    if not args.no_fp64 and mixed:
        ctx.set_mps(swept_state)
        ctx.set_precision(0, 0)
        k64 = max(1, min(args.steps, args.fp64_steps))
        ms64, d64, e64, _ = timed_steps(ctx, Walker(lo, hi), D, k64, 1)
        r64 = matvec_kernel_rates(d64)
        fp64 = {"steps": k64, "ms_per_step": ms64 / k64, "step_breakdown_ms": step_breakdown(d64, k64),
                "value": d64["matvec_flops"] / (ms64 * 1e-3) / 1e9, "unit": "GFLOP/s",
                "matvec": r64.get("fp64"), "roofline": roofline_fp64(d64, peak64)}
        ctx.set_precision(args.precision, args.fp64_iters)
    ctx.set_mps(swept_state)
    ctx.canonicalize(center)
    acc = energy_agreement(ctx, center, D, args) if not args.no_fp64 else None
    conv = converged_agreement() if not args.no_fp64 and not args.no_sweep else None
    batch = batch_summary(args) if not args.no_batch and world == 1 else None
    # one marked matvec in each precision after the timed region (NVTX range for profilers)
    xprof = torch.tensor(ctx.tt_to_x(center), dtype=torch.float64, device="cuda")
    yprof = torch.empty_like(xprof)
    for prec in (args.precision, 0):
        ctx.set_precision(prec, args.fp64_iters)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("matvec")
        ctx.matvec(center, xprof, yprof)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ctx.set_precision(args.precision, args.fp64_iters)
    fixed_iters(ctx, D, args.davidson_iters)
    e2e = None
    if not args.no_e2e:
        ctx.set_mps(swept_state)
        e2e = run_e2e(ctx, Walker(lo, hi), D, args)
    out = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32x3-f32acc+f64" if mixed else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: random integrals L={L} N={cfg['N']} S=0 Ag "
                               f"D2h 8/3/3/2/6/2/2/2, D_SU(2)={D}, micro-iterations of a sweep between sites "
                               f"{lo} and {hi} (both directions) of " + state,
                   "L": L, "N": cfg["N"], "D": D, "sites": [lo, hi], "middle_site": center,
                   "two_site_elements_middle": n_x,
                   "davidson_iters_per_step": args.davidson_iters,
                   "precision": ("split-TF32 tensor-core block products (FP32 data and accumulation) in "
                                 f"Davidson, then {args.fp64_iters} FP64 Davidson iteration(s)") if mixed
                                else "FP64 block products",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (renormalised operators of both environments, several GB)",
                   "block_histogram": hist},
        "matvec": rates, "fp64": fp64, "energy_agreement": acc, "converged_agreement": conv, "sweep": sweeps, "batch32": batch,
        "micro_iteration_s": t_max / args.steps / 1e3,
        "step_breakdown_ms": step_breakdown(delta, args.steps),
        "energy_last": energies[-1] if energies else None,
        "clocks": clocks, "gpu_launches": launches, "roofline": roof,
        "peaks_measured_here": {"fp64_gflops": peak64, "tf32_gflops": peak_tf32,
                                "how": "cuBLAS through torch.matmul, 8192^3, best of 3 (FP64; FP32 with TF32 "
                                       "allowed)"},
    }
    if e2e:
        out["e2e"] = e2e
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(bounded_seconds=15.0)
            out["cpu_baseline"]["single_core"] = single_core_baseline(5.0)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(ctx, walker, D, args):
    """The headline steps through the host-buffer C ABI (stream 0): dmrg_tt_to_x into
    pinned host memory, dmrg_davidson from and to it, dmrg_truncate from it and
    dmrg_update_operators: the work of dmrg_sweep_step (Eq. 25, Davidson, Eqs. 26-28, the
    operator update), with the two-site vector crossing host <-> device every step; the
    energy is read back on the host.  Same sweep window as the headline steps."""
    import torch
    steps = max(1, min(args.steps, args.e2e_steps))
    buf = [torch.empty(0, dtype=torch.float64).pin_memory()]

    def one():
        i, d = walker.site, walker.dir
        n, _ = ctx.layout(i)
        if buf[0].numel() < n:  # one pinned buffer, grown when a site needs more
            buf[0] = torch.empty(2 * n, dtype=torch.float64).pin_memory()
        x = buf[0][:n].numpy()
        ctx.tt_to_x(i, x)
        e, it, ok = ctx.davidson(i, x)
        ctx.truncate(i, d, D, x)
        ctx.update_operators(i, d)
        walker.site, walker.dir = walker.peek()
        return n

    one()  # warm-up step (tables, environments)
    st0 = ctx.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(steps):
        nbytes += one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st1 = ctx.stats()
    flops = st1["matvec_flops"] - st0["matvec_flops"]
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "steps": steps, "s_per_step": dt / steps,
            "h2d_bytes_per_step": 2 * 8 * nbytes // steps, "d2h_bytes_per_step": 2 * 8 * nbytes // steps + 8,
            "path": "dmrg_tt_to_x / dmrg_davidson / dmrg_truncate / dmrg_update_operators with host "
                    "buffers (the work of dmrg_sweep_step)"}


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


# Planner-counted flops of one H_eff matvec of the oracle sample (n = 1764 two-site
# elements): the block products over nonzero blocks that the GPU path issues for the
# same problem, counted by the host planner (a count, not a computed result).
SAMPLE_FLOPS = 3493410.0


def cpu_baseline(bounded_seconds=15.0, flops=None):
    from oracle import dmrg as odmrg
    from oracle import mps as om
    import numpy as np
    prob, m, i = oracle_sample()
    if flops is None:
        flops = SAMPLE_FLOPS
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


def single_core_baseline(bounded_seconds=5.0):
    """The same oracle sample with the BLAS / OpenMP thread pools of a fresh process held
    to one thread (the 1-core figure beside the all-cores one); None if it cannot run."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline(bounded_seconds=%r)))" % (ROOT, float(bounded_seconds)))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=bounded_seconds * 4 + 120)
        if r.returncode != 0:
            return None
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": d["value"], "unit": d["unit"], "cores": 1, "sample": d["sample"]}
    except Exception:
        return None


def run_reference(args):
    """The reference arm: the oracle (plain FP64 CPU program) on the host cores.  It can
    only evaluate the L=8 member of the workload family (dense projection through the
    determinant basis), so each step is one oracle matvec of that sample."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import dmrg as odmrg
    from oracle import mps as om
    from workloads import CONFIGS
    prob, m, i = oracle_sample()
    x = om.tt_to_x(m, i)
    for _ in range(args.warmup):
        odmrg.matvec(prob, m, i, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        odmrg.matvec(prob, m, i, x)
    dt = time.perf_counter() - t0
    value = SAMPLE_FLOPS * args.steps / dt / 1e9
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    cfg = CONFIGS[args.workload]
    sample = ("one oracle H_eff matvec (P^T H P, determinant basis) per step at sites (3,4) of the "
              "L=8 Hubbard chain, D=64 (n=1764): the oracle cannot evaluate the L=28 problem")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "hubbard8: Hubbard chain L=8 N=8 S=0 C1 t=1 U=4, D_SU(2)=64, sites (3,4), "
                                  "one oracle H_eff matvec per step",
                      "stands_in_for": f"{args.workload}: random integrals L={cfg['L']} N={cfg['N']} S=0 Ag "
                                       f"D2h 8/3/3/2/6/2/2/2, D_SU(2)={args.D or cfg['D']}, middle sites (the "
                                       "GPU arm's workload, beyond the oracle's dense projection)",
                      "sample": sample},
           "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
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
