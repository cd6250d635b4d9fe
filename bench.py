#!/usr/bin/env python
"""Benchmark: PCG solve of the space-time least-squares heat-equation system.

One step = one complete solve A u = F from u = 0 to ||r|| / ||F|| <= 1e-8
(context setup excluded: it runs once per context and is reported as
setup_ms) on the workload
"cube3d_p3_n64": (0,1)^3 x (0,1), degree 3 splines, 64 elements per
direction, N = 18,125,250 unknowns, F ~ U[-1,1] (seed 1809100264).

Metric: solved degrees of freedom per second (DoF/s), whole job.  The
headline form is the mixed one of this workload: TF32 tensor-core
preconditioner apply with FP32 accumulation, FP64 outer residual F - A u
(iterative refinement around a flexible CG in FP32 with compensated inner
products; the outer steps before the last take a provisional residual with
the double-float A x).  The other forms are measured on the same workload in
the same run and reported under "forms": the same with every outer residual
in FP64 ("_ir64"), BF16 refinement (both residual variants), the strict
TF32 and BF16 forms (flexible CG with FP64 vectors, FP64 A x, only the
preconditioner in TF32/BF16) and the FP64 PCG.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision tf32|bf16|fp64] [--no-refine] [--fp64-residuals]
                  [--forms a,b,...]

Also in the line: "sweep", the degree sweep of this workload's size (p = 2..6
with 67 - p elements per direction, N = 18,125,250 for every p) in the
headline form and the FP64 PCG; and "errors_vs_oracle", the relative error
||u - u_oracle|| / ||u_oracle|| of every form's solution, u_oracle from the
oracle's FP64 PCG on the host cores to a residual of 1e-12 (run after the GPU
timing; the same run gives the CPU baseline's measured time to 1e-8).

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
# Iterations of the FP64 PCG on this workload (measured on the GPU; the CPU
# baseline extrapolates one oracle iteration by this count)
FP64_ITERS = 17
PAPER_DOFS = 18125250 / 227.93  # Table 1, p = 3, n_sub = 64: serial Matlab, i7-5820K (context)
# The line carries the DoF/s (value), the solve time (ms_per_step), the mixed
# forms beside the FP64 one (forms) and the preconditioner's roofline
METRIC = "PCG DoF/s & solve time, mixed vs FP64 at 1e-8 residual; precond apply %roofline"
# form name -> (precision, refine, every outer residual in FP64); the "_ir"
# forms take provisional double-float outer residuals before the last one,
# the "_ir64" forms take every outer residual in FP64
FORMS = {"bf16_ir": ("bf16", True, False), "tf32_ir": ("tf32", True, False),
         "bf16_ir64": ("bf16", True, True), "tf32_ir64": ("tf32", True, True),
         "bf16_fcg": ("bf16", False, False), "tf32_fcg": ("tf32", False, False),
         "fp64_pcg": ("fp64", False, False)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return {"hbm_gbs": pk["hbm_gbs"], "bf16_tflops": pk["bf16_tflops"],
                "bf16_tflops_sustained": pk.get("bf16_tflops_sustained"), "source": "measured",
                "sm_max_mhz": pk.get("sm_max_mhz", 2070.0)}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback", "sm_max_mhz": 2070.0}


# FP64 peak: nominal 1.25 TFLOP/s per GB300 (152 SMs); a DFMA probe on this machine
# measured 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
# FP32 CUDA-core peak: SMs x 128 FMA/clk x 2 flop x maximum SM clock; this default
# is GB300's 152 SMs at 2.07 GHz, and run_ours replaces it by the device's SM
# count and the maximum SM clock of MEASURED_PEAKS.json (fp32_peak_tflops)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def fp32_peak_tflops(sms, sm_mhz):
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


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


def replica_rate(units, steps, world, ms_max):
    """Whole-job throughput of `world` replicas that each processed `units` per
    step for `steps` steps, the slowest taking `ms_max` milliseconds."""
    return units * steps * world / (ms_max * 1e-3)


def fd_flops(S):
    return 4.0 * S.N * (sum(S.n_s) + S.n_t) + S.N


def apply_A_flops(S, p, p_t=None):
    """Banded products per DoF of the fused A x: 3 + 6 (directions 1, 2) + 4
    (direction 3) + 2 (time) = 15 in three spatial directions, 3 + 4 + 2 = 9 in
    two; each is 2(2p+1) flops per DoF (the L_s x of the last time slice is
    not counted)."""
    p_t = p if p_t is None else p_t
    spatial = {1: 3, 2: 3 + 4, 3: 3 + 6 + 4}[S.d]
    return 2.0 * (2 * p + 1) * spatial * S.N + 2.0 * (2 * p_t + 1) * 2 * S.N


def timed_solves(S, F, u, tol, steps, warmup, world, timing):
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


# ncu DRAM bytes (read + write) per operation on this workload, from the
# captures summarised under profiles/ (ncu flushes the caches before every
# kernel, so intermediate tensors that stay in L2 in a normal run count as DRAM
# reads there); None where no capture of the current kernels exists.
TRAFFIC = {
    # fused BF16 FD apply with FP32 in/out: 5 kernels, 234.8 MB read + 19.1 MB written
    ("precond", "bf16", True): 253888256,
    # TF32 FD apply inside the inner loop: 8 rotation passes, 649.7 MB read + 133.9 MB written
    ("precond", "tf32", True): 783665536,
    # FP32 A x of the inner loop (slice kernel, fused direction 3 + time with (p, A p)):
    # 398.7 MB read + 211.3 MB written; the same kernels serve both refinement forms
    ("apply_A_f32", "tf32", True): 610040042,
    ("apply_A_f32", "bf16", True): 610040042,
}


def roofline_entry(phase, ms, count, S, p, peaks, refine):
    """Roofline of one operation (the kernels between two phase events), from
    the CUDA-event phase times of the timed solves."""
    if count == 0 or ms <= 0:
        return None
    per = ms / count * 1e-3
    hbm = peaks["hbm_gbs"]
    src = peaks["source"] + " hbm_gbs"
    if phase == "precond" and S.precision == "fp64":
        ach = fd_flops(S) / per / 1e12
        e = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "kernel": "FD apply, FP64 mode products", "peak_source": "nominal FP64 1.25 TFLOP/s"}
    elif phase == "precond":
        # vectors in and out: FP32 inside the refinement form, FP64 in the strict form
        nbytes = (8.0 if refine else 16.0) * S.N
        ach = nbytes / per / 1e9
        e = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
             "kernel": "FD apply, %s tensor-core mode products (%s in/out)"
                       % (S.precision, "FP32" if refine else "FP64"),
             "algorithmic_bytes": nbytes, "peak_source": src}
    elif phase == "apply_A":
        ach = apply_A_flops(S, p) / per / 1e12
        e = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "kernel": "A x, FP64 fused banded mode products", "peak_source": "nominal FP64 1.25 TFLOP/s"}
    elif phase == "apply_A_f32":
        ach = apply_A_flops(S, p) / per / 1e12
        f32 = peaks.get("fp32_tflops", FP32_PEAK_TFLOPS)
        e = {"bound": "alu", "achieved": ach, "peak": f32, "unit": "TFLOP/s",
             "kernel": "A x, FP32 fused banded mode products",
             "peak_source": peaks.get("fp32_source", "FP32 FMA units x max SM clock (152 x 128 x 2 x 2.07 GHz)")}
    elif phase == "apply_A_df":
        # 12 FP32 operations per banded term (an FMA counts as one operation)
        ops = 12 * apply_A_flops(S, p) / 2
        ach = ops / per / 1e12
        f32 = peaks.get("fp32_tflops", FP32_PEAK_TFLOPS)
        e = {"bound": "alu", "achieved": ach, "peak": f32 / 2, "unit": "Top/s",
             "kernel": "A x, double-float fused banded mode products (with the split of u)",
             "peak_source": "FP32 operations: SMs x 128 lanes x max SM clock"}
    else:
        return None
    e["frac"] = e["achieved"] / e["peak"]
    e["traffic"] = TRAFFIC.get((phase, S.precision, refine))
    e["avg_ms"] = per * 1e3
    e["launch_ops"] = count
    return e


def run_form(stls, name, W, F, args, world, sampler=None):
    import torch
    precision, refine, fp64_res = FORMS[name]
    t0 = time.perf_counter()
    S = stls.Solver(W["d"], W["p"], W["n_el"], W["T"], precision=precision, refine=refine,
                    fp64_residuals=fp64_res,
                    device=F.device)
    setup_ms = (time.perf_counter() - t0) * 1e3  # host eigendecompositions, uploads, workspace
    u = torch.empty_like(F)
    steps = args.steps if sampler is not None else max(1, min(args.steps, args.form_steps))
    if sampler is not None:
        sampler.start()
    ms, infos, launches, _ = timed_solves(S, F, u, W["tol"], steps, args.warmup, world, False)
    clocks = sampler.stop() if sampler is not None else None
    ms_max = max_over_ranks(ms, world, F.device)
    _, _, _, phases = timed_solves(S, F, u, W["tol"], 1, 0, world, True)
    return dict(S=S, u=u, ms=ms_max, infos=infos, launches=launches, phases=phases, steps=steps,
                clocks=clocks, precision=precision, refine=refine, setup_ms=setup_ms,
                u_host=u.cpu().numpy())


def sweep_entry(stls, p, form, F, args, world):
    """One solve form on the degree-sweep workload of degree p (67 - p elements
    per direction, the N of the main workload)."""
    W = dict(WORKLOAD, p=p, n_el=67 - p)
    r = run_form(stls, form, W, F, args, world)
    S, ph = r["S"], r["phases"]
    total = sum(v[0] for v in ph.values())
    it = r["infos"][-1]
    out = {"form": form, "n_el": W["n_el"], "value": replica_rate(S.N, r["steps"], world, r["ms"]),
           "unit": "DoF/s", "ms_per_step": r["ms"] / r["steps"], "steps": r["steps"],
           "iterations": it["iters"], "outer": it["outer"], "true_rel_res": it["true_rel_res"],
           "phase_share": {k: v[0] / total for k, v in ph.items() if v[1]} if total else None,
           "phase_ms_per_solve": {k: v[0] for k, v in ph.items() if v[1]}}
    S.close()
    return out


def oracle_iteration_times(F):
    """(setup s, one PCG iteration s, N) of the oracle's FP64 PCG on the workload."""
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
    del x
    return t_setup, t_iter, prob.N


def oracle_reference_solve(F, tol_ref=1e-12, tol=1e-8):
    """The oracle's FP64 PCG (oracle.solve.pcg with the FD preconditioner and
    the Kronecker-factored A) on the workload to tol_ref, on all host cores.
    Returns (u, seconds from setup start to the first iterate with residual
    <= tol, iterations to tol, iterations to tol_ref, setup seconds)."""
    from oracle.system import STProblem
    from oracle.fd import FD
    from oracle.solve import pcg
    W = WORKLOAD
    t0 = time.perf_counter()
    prob = STProblem(W["d"], W["p"], W["n_el"], W["T"])
    fd = FD(prob)
    t_setup = time.perf_counter() - t0
    stamps = []  # entry of every preconditioner call: call k + 1 starts right after iteration k

    def apply_P(r):
        stamps.append(time.perf_counter())
        return fd.apply(r)

    u, its, hist = pcg(prob.apply_A_kron, apply_P, F, tol_ref, 400)
    t_end = time.perf_counter()
    k_tol = next(k for k, h in enumerate(hist) if h <= tol)
    t_tol = (stamps[k_tol] if k_tol < len(stamps) else t_end) - t0
    return u, t_tol, k_tol, its, t_setup


def single_thread_sample(iters, timeout_s=240):
    """The same sample with one host thread (BLAS and OpenMP pools of 1), in a
    child process, for comparison with the paper's serial times."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-iteration-sample"],
                             env=env, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"skipped": "longer than %d s" % timeout_s}
    if res.returncode != 0:
        tail = res.stderr.strip().splitlines()
        return {"skipped": "child failed: " + (tail[-1] if tail else "exit %d" % res.returncode)}
    t_setup, t_iter, n = json.loads(res.stdout.strip().splitlines()[-1])
    solve_s = t_setup + iters * t_iter
    return {"value": n / solve_s, "unit": "DoF/s", "cores": 1, "solve_s_extrapolated": solve_s,
            "sample": "oracle setup (%.1f s) + one PCG iteration (%.1f s), one thread, extrapolated to "
                      "%d iterations" % (t_setup, t_iter, iters)}


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baseline_sample(F, iters, single_thread=True):
    """Oracle FP64 PCG on the same workload, on the host cores: setup + 1 iteration,
    extrapolated to `iters` iterations (and the same with one thread)."""
    t_setup, t_iter, n = oracle_iteration_times(F)
    solve_s = t_setup + iters * t_iter
    out = {"value": n / solve_s, "unit": "DoF/s", "cores": host_cores(), "kind": "oracle",
           "sample": "oracle setup (%.1f s) + one PCG iteration (%.1f s) on the full workload, "
                     "extrapolated to %d iterations" % (t_setup, t_iter, iters),
           "solve_s_extrapolated": solve_s}
    if single_thread:
        out["single_thread"] = single_thread_sample(iters)
    return out


def cpu_baseline_from_solve(n, t_tol, k_tol, t_setup, iters, single_thread=True):
    """The CPU baseline measured by the oracle's own solve of the workload: setup
    plus the iterations up to the first residual <= 1e-8."""
    out = {"value": n / t_tol, "unit": "DoF/s", "cores": host_cores(), "kind": "oracle",
           "sample": "the oracle's FP64 PCG solve of the full workload, timed from setup (%.1f s) to the "
                     "iterate with residual <= 1e-8 (%d iterations, %.1f s); the same run continued to "
                     "1e-12 for the error check" % (t_setup, k_tol, t_tol),
           "solve_s": t_tol}
    if single_thread:
        out["single_thread"] = single_thread_sample(iters)
    return out


def run_ours(args):
    import torch
    import paper_1809_10026_gb300 as stls
    from paper_1809_10026_gb300 import synth

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peaks["fp32_tflops"] = fp32_peak_tflops(sms, peaks["sm_max_mhz"])
    peaks["fp32_source"] = "FP32 FMA units x max SM clock (%d SMs x 128 x 2 x %.0f MHz)" % (sms, peaks["sm_max_mhz"])
    W = WORKLOAD
    head = args.precision + ("_ir" + ("64" if args.fp64_residuals else "")
                             if (args.precision != "fp64" and not args.no_refine) else
                             ("_fcg" if args.precision != "fp64" else "_pcg"))
    extra = [f for f in args.forms.split(",") if f and f != head] if args.forms else []
    for f in extra:
        if f not in FORMS:
            raise SystemExit("unknown form %r (known: %s)" % (f, ", ".join(FORMS)))
    F_host = synth.uniform(18125250, W["tag"])
    F = torch.from_numpy(F_host).to(device)
    main = run_form(stls, head, W, F, args, world, sampler=ClockSampler(local))
    S = main["S"]
    N = S.N
    p = W["p"]
    value = replica_rate(N, main["steps"], world, main["ms"])
    ph = main["phases"]
    entries = {k: roofline_entry(k, v[0], v[1], S, p, peaks, main["refine"]) for k, v in ph.items()}
    total_ph = sum(v[0] for v in ph.values())
    dominant = max((k for k in ph if entries.get(k)), key=lambda k: ph[k][0])
    # end to end through the host-pointer C entry point (pinned host buffers,
    # H2D of F and D2H of u inside the timed region)
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
        "vs_baseline": None,
        "dtype": {"bf16_ir": "bf16+f32+f64", "tf32_ir": "tf32+f32+f64", "bf16_ir64": "bf16+f32+f64",
                  "tf32_ir64": "tf32+f32+f64", "bf16_fcg": "bf16+f64", "tf32_fcg": "tf32+f64",
                  "fp64_pcg": "f64"}[head],
        "data": "synthetic",
        "config": {"workload": W["name"], "description": W["text"], "form": head,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (145 MB FP64 vectors, 129 MB L2)",
                   "iterations": it["iters"], "outer": it["outer"], "true_rel_res": it["true_rel_res"]},
        "roofline": dict(entries[dominant], phase=dominant,
                         phase_share=ph[dominant][0] / total_ph if total_ph else None),
        "precond_roofline": entries.get("precond"),
        "phase_ms_per_solve": {k: v[0] for k, v in ph.items()},
        "phase_calls_per_solve": {k: v[1] for k, v in ph.items()},
        # context creation (not in value): 1D matrices and eigendecompositions on
        # the host, uploads, workspace, tensor-core operand images
        "setup_ms": main["setup_ms"],
        "e2e": {"value": replica_rate(N, main["steps"], world, e2e_s * 1e3), "unit": "DoF/s",
                "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
        "paper_context": {"dofs_per_s": PAPER_DOFS,
                          "note": "Table 1, p=3, n_sub=64: 13 iterations / 227.93 s, serial Matlab FP64 "
                                  "on an i7-5820K incl. setup, manufactured right-hand side"},
    }
    forms = {}
    u_forms = {head: main["u_host"]}
    for name in extra:
        r = run_form(stls, name, W, F, args, world)
        u_forms[name] = r["u_host"]
        Sx, phx = r["S"], r["phases"]
        forms[name] = {"value": replica_rate(N, r["steps"], world, r["ms"]), "unit": "DoF/s",
                       "ms_per_step": r["ms"] / r["steps"], "steps": r["steps"],
                       "iterations": r["infos"][-1]["iters"], "outer": r["infos"][-1]["outer"],
                       "true_rel_res": r["infos"][-1]["true_rel_res"], "gpu_launches": r["launches"],
                       "setup_ms": r["setup_ms"],
                       "phase_ms_per_solve": {k: v[0] for k, v in phx.items()},
                       "rooflines": {k: roofline_entry(k, v[0], v[1], Sx, p, peaks, r["refine"])
                                     for k, v in phx.items() if v[1]}}
        Sx.close()
        del r
        torch.cuda.empty_cache()
    if forms:
        line["forms"] = forms
    if args.sweep:
        # degree sweep at fixed N: the FD cost 4N(d n_s + n_t) stays flat in p, A x grows with 2p + 1
        sweep = {}
        for pp in range(2, 7):
            for name in dict.fromkeys((head, "fp64_pcg")):
                sweep["p%d_%s" % (pp, name)] = sweep_entry(stls, pp, name, F, args, world)
                torch.cuda.empty_cache()
        line["sweep"] = sweep
    main["S"].close()
    del F
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_oracle_errors:
        # the oracle's own solution (FP64 PCG to 1e-12 on the host cores), after every GPU timing
        import numpy as np
        u_ref, t_tol, k_tol, k_ref, t_setup = oracle_reference_solve(F_host)
        nref = np.linalg.norm(u_ref)
        line["errors_vs_oracle"] = {
            "reference": "oracle FP64 PCG with the FD preconditioner to ||r|| / ||F|| <= 1e-12 "
                         "(%d iterations)" % k_ref,
            "rel_l2": {k: float(np.linalg.norm(v - u_ref) / nref) for k, v in u_forms.items()}}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_from_solve(u_ref.size, t_tol, k_tol, t_setup, FP64_ITERS)
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
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
        "vs_baseline": None,
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
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16"], default="tf32")
    ap.add_argument("--fp64-residuals", action="store_true",
                    help="headline refinement form with every outer residual in FP64")
    ap.add_argument("--no-refine", action="store_true",
                    help="headline mixed form without the FP64 outer residual (strict flexible CG)")
    ap.add_argument("--forms", default="tf32_ir64,bf16_ir,bf16_ir64,tf32_fcg,bf16_fcg,fp64_pcg",
                    help="other forms timed in the same run (comma separated; empty for none)")
    ap.add_argument("--form-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the degree sweep p = 2..6 at the workload's N")
    ap.add_argument("--no-oracle-errors", action="store_true",
                    help="skip the oracle's reference solve (errors of every form against it)")
    ap.add_argument("--oracle-iteration-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_iteration_sample:  # child of single_thread_sample
        from paper_1809_10026_gb300 import synth
        print(json.dumps(list(oracle_iteration_times(synth.uniform(18125250, WORKLOAD["tag"])))))
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
