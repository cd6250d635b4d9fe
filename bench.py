#!/usr/bin/env python
"""Benchmark: PCG solve of the space-time least-squares heat-equation system.

One step = one complete solve A u = F from u = 0 to ||r|| / ||F|| <= 1e-8
(preconditioner setup excluded; it runs once per context) on the workload
"cube3d_p3_n64": (0,1)^3 x (0,1), degree 3 splines, 64 elements per
direction, N = 18,125,250 unknowns, F ~ U[-1,1] (seed 1809100264).

Metric: solved degrees of freedom per second (DoF/s), whole job.  The
headline form is the mixed one (BF16 tensor-core preconditioner inside a
flexible CG, FP64 residual and inner products); the FP64 form is measured on
the same workload and reported in "fp64_form".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (under torchrun) every rank solves its own copy of the
workload (replicas; the method has no data-path exchange on one node) and
value = N_dof * steps * ranks / max-over-ranks time.  --impl reference times
the CPU oracle (numpy/scipy FP64 PCG with the FD preconditioner) on the host
cores: each step is one PCG iteration of the same workload, and the solve
time is extrapolated with the iteration count of the solve.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="cube3d_p3_n64", d=3, p=3, n_el=64, T=1.0, tol=1e-8, tag=4,
                text="3D space + time cube, degree 3, 64 elements per direction, "
                     "N = 18,125,250, F ~ U[-1,1] seed 1809100264, CG tol 1e-8 from u = 0")
# Iterations of the FP64 PCG on this workload (checked by tests/test_gpu_bench_config.py)
FP64_ITERS = 17
PAPER_DOFS = 18125250 / 227.93  # Table 1, p = 3, n_sub = 64: serial Matlab, i7-5820K (context)
METRIC = "PCG solve DoF/s (mixed BF16-preconditioned FCG vs FP64 PCG, rel. residual 1e-8)"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return {"hbm_gbs": pk["hbm_gbs"], "bf16_tflops": pk["bf16_tflops"],
                "bf16_tflops_sustained": pk.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


# FP64 peak: nominal 1.25 TFLOP/s per GB300 (152 SMs); a DFMA probe on this machine
# measured 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def fd_flops(S):
    return 4.0 * S.N * (sum(S.n_s) + S.n_t) + S.N


def apply_A_flops(S, p):
    # banded products per DoF of the factored A x (3 + 6 + 5 spatial, 2 in time)
    products = {1: 2 + 2, 2: 3 + 4 + 2, 3: 3 + 6 + 5 + 2}[S.d]
    return 2.0 * (2 * p + 1) * products * S.N


def timed_solves(S, F, u, tol, steps, warmup, world, device, timing):
    import torch
    for _ in range(warmup):
        S.solve(F, tol, 500, out=u)
    S.enable_timing(timing)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = S.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos = []
    for _ in range(steps):
        _, info = S.solve(F, tol, 500, out=u)
        infos.append(info[0])
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    launches = S.launch_count() - l0
    phases = S.phase_times() if timing else None
    S.enable_timing(False)
    return ms, infos, launches, phases


def roofline_entry(kind, ms, count, S, p, peaks):
    if count == 0 or ms <= 0:
        return None
    per = ms / count * 1e-3
    if kind == "precond_fp64":
        ach = fd_flops(S) / per / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "FD apply (FP64 mode products)",
                "peak_source": "nominal FP64 (1.25 TFLOP/s)", "avg_ms": per * 1e3}
    if kind == "precond_mixed":
        ach = 16.0 * S.N / per / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "FD apply (tensor-core mode products)",
                "peak_source": peaks["source"] + " hbm_gbs", "avg_ms": per * 1e3}
    if kind == "apply_A":
        ach = apply_A_flops(S, p) / per / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "A x (FP64 banded mode products)",
                "peak_source": "nominal FP64 (1.25 TFLOP/s)", "avg_ms": per * 1e3}
    if kind == "cg_vectors":
        return None
    return None


def cpu_baseline_sample(F, iters):
    """Oracle FP64 PCG on the same workload, on the host cores: setup + 1 iteration,
    extrapolated to `iters` iterations."""
    from oracle.system import STProblem
    from oracle.fd import FD
    import numpy as np
    W = WORKLOAD
    t0 = time.perf_counter()
    prob = STProblem(W["d"], W["p"], W["n_el"], W["T"])
    fd = FD(prob)
    t_setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    r = F.copy()
    z = fd.apply(r)
    q = prob.apply_A_kron(z)
    alpha = (r @ z) / (z @ q)
    x = alpha * z
    r -= alpha * q
    _ = np.linalg.norm(r)
    t_iter = time.perf_counter() - t1
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    solve_s = t_setup + iters * t_iter
    del x
    return {"value": prob.N / solve_s, "unit": "DoF/s", "cores": cores, "kind": "oracle",
            "sample": "oracle setup (%.1f s) + one PCG iteration (%.1f s) on the full workload, "
                      "extrapolated to %d iterations" % (t_setup, t_iter, iters),
            "solve_s_extrapolated": solve_s}


def run_ours(args):
    import numpy as np
    import torch
    import paper_1809_10026_gb300 as stls
    from paper_1809_10026_gb300 import synth

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    peaks = load_peaks()
    W = WORKLOAD
    forms = [args.precision]
    if args.precision != "fp64":
        forms.append("fp64")
    F_host = synth.uniform(18125250, W["tag"])
    F = torch.from_numpy(F_host).to(device)
    results = {}
    sampler = ClockSampler(local)
    for form in forms:
        S = stls.Solver(W["d"], W["p"], W["n_el"], W["T"], precision=form, device=device)
        u = torch.empty_like(F)
        steps = args.steps if form == forms[0] else max(1, min(args.steps, args.fp64_steps))
        if form == forms[0]:
            sampler.start()
        ms, infos, launches, _ = timed_solves(S, F, u, W["tol"], steps, args.warmup, world, device, False)
        if form == forms[0]:
            clocks = sampler.stop()
        ms_max = max_over_ranks(ms, world, device)
        _, _, _, phases = timed_solves(S, F, u, W["tol"], steps, 0, world, device, True)
        results[form] = dict(S=S, u=u, ms=ms_max, infos=infos, launches=launches, phases=phases,
                             steps=steps)
    main = results[forms[0]]
    S = main["S"]
    N = S.N
    value = N * main["steps"] * world / (main["ms"] * 1e-3)
    # roofline: dominant phase of the headline form, and the preconditioner apply
    ph = main["phases"]
    p = W["p"]
    pre_kind = "precond_fp64" if forms[0] == "fp64" else "precond_mixed"
    entries = {"precond": roofline_entry(pre_kind, ph["precond"][0], ph["precond"][1], S, p, peaks),
               "apply_A": roofline_entry("apply_A", ph["apply_A"][0], ph["apply_A"][1], S, p, peaks)}
    dominant = max(("precond", "apply_A"), key=lambda k: ph[k][0])
    total_ph = sum(v[0] for v in ph.values())
    # end to end through the host-pointer C entry point (pinned host buffers)
    Fh = torch.from_numpy(F_host).pin_memory()
    uh = torch.empty_like(Fh).pin_memory()
    for _ in range(args.warmup):
        S.solve_host_ptr(Fh.data_ptr(), uh.data_ptr(), W["tol"], 500)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(main["steps"]):
        S.solve_host_ptr(Fh.data_ptr(), uh.data_ptr(), W["tol"], 500)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device)
    barrier(world)
    it = main["infos"][-1]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "DoF/s",
        "n_gpus": world,
        "steps": main["steps"],
        "warmup": args.warmup,
        "ms_per_step": main["ms"] / main["steps"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / PAPER_DOFS,
        "dtype": "f64" if forms[0] == "fp64" else forms[0] + "+f64",
        "data": "synthetic",
        "config": {"workload": W["name"], "description": W["text"], "form": forms[0],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (145 MB FP64 vectors, 129 MB L2)",
                   "iterations": it["iters"], "true_rel_res": it["true_rel_res"]},
        "roofline": dict(entries[dominant] or {}, phase=dominant,
                         phase_share=ph[dominant][0] / total_ph if total_ph else None),
        "precond_roofline": entries["precond"],
        "phase_ms_per_solve": {k: v[0] / main["steps"] for k, v in ph.items()},
        "e2e": {"value": N * main["steps"] * world / e2e_s, "unit": "DoF/s",
                "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "gpu_launches": main["launches"],
        "clocks": clocks,
        "paper_context": {"dofs": PAPER_DOFS, "note": "Table 1, p=3, n_sub=64: 13 it / 227.93 s, serial "
                                                      "Matlab FP64 on i7-5820K incl. setup, manufactured RHS"},
    }
    if "fp64" in results and forms[0] != "fp64":
        r64 = results["fp64"]
        S64 = r64["S"]
        ph64 = r64["phases"]
        line["fp64_form"] = {"value": N * r64["steps"] * world / (r64["ms"] * 1e-3), "unit": "DoF/s",
                             "ms_per_step": r64["ms"] / r64["steps"], "steps": r64["steps"],
                             "iterations": r64["infos"][-1]["iters"],
                             "precond_roofline": roofline_entry("precond_fp64", ph64["precond"][0],
                                                                ph64["precond"][1], S64, p, peaks),
                             "apply_A_roofline": roofline_entry("apply_A", ph64["apply_A"][0],
                                                                ph64["apply_A"][1], S64, p, peaks)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(F_host, FP64_ITERS)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from oracle.system import STProblem
    from oracle.fd import FD
    from paper_1809_10026_gb300 import synth
    W = WORKLOAD
    t0 = time.perf_counter()
    prob = STProblem(W["d"], W["p"], W["n_el"], W["T"])
    fd = FD(prob)
    t_setup = time.perf_counter() - t0
    F = synth.uniform(prob.N, W["tag"])
    # textbook PCG (the oracle's), one iteration per step
    x = np.zeros_like(F)
    r = F.copy()
    z = fd.apply(r)
    p = z.copy()
    rz = r @ z

    def iteration():
        nonlocal x, r, z, p, rz
        q = prob.apply_A_kron(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = fd.apply(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new

    for _ in range(args.warmup):
        iteration()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        iteration()
    t_iter = (time.perf_counter() - t1) / args.steps
    solve_s = t_setup + FP64_ITERS * t_iter
    value = prob.N / solve_s
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "DoF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_iter * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": value / PAPER_DOFS,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": W["name"], "description": W["text"], "form": "fp64 oracle PCG (CPU)"},
        "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                         "sample": "each step is one oracle PCG iteration on the full workload; solve time "
                                   "= setup %.1f s + %d iterations x %.2f s" % (t_setup, FP64_ITERS, t_iter)},
        "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16"], default="bf16")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
