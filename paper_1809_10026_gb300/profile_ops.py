"""Run one solver operation repeatedly (for timing and for ncu captures).

python -m paper_1809_10026_gb300.profile_ops --op precond --precision bf16 \
    --d 3 --p 3 --n-el 64 --reps 5

Prints the mean device time per application (CUDA events).  Inputs are
seeded U[-1,1] vectors from synth.
"""
import argparse
import json

import torch

import paper_1809_10026_gb300 as stls
from paper_1809_10026_gb300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["precond", "apply_A", "apply_A_df", "apply_A_f32", "solve"], default="precond")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16"], default="fp64")
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--n-el", type=int, default=64)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--refine", action="store_true", help="iterative-refinement form (mixed precisions)")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="inner tolerance of the refinement form (0: adaptive)")
    ap.add_argument("--no-phases", action="store_true",
                    help="solve: no per-phase timing (the refinement form then runs its inner loop as one graph)")
    a = ap.parse_args()
    S = stls.Solver(a.d, a.p, a.n_el, precision=a.precision, batch=a.batch, refine=a.refine,
                    inner_tol=a.inner_tol)
    x = torch.from_numpy(synth.uniform(S.N, 4, batch=a.batch)).cuda()
    y = torch.empty_like(x)
    x32, y32 = x.float(), torch.empty_like(x, dtype=torch.float32)

    def run():
        if a.op == "precond":
            S.apply_precond(x, out=y)
        elif a.op == "apply_A":
            S.apply_A(x, out=y)
        elif a.op == "apply_A_df":
            S.apply_A_df(x, out=y)
        elif a.op == "apply_A_f32":
            S.apply_A_f32(x32, out=y32)
        else:
            S.solve(x, a.tol, 500, out=y)

    info = None

    def run_solve():
        nonlocal info
        _, info = S.solve(x, a.tol, 1000, out=y)

    if a.op == "solve":
        run = run_solve  # noqa: F811
    for _ in range(a.warmup):
        run()
    if a.op == "solve" and not a.no_phases:
        S.enable_timing(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = S.launch_count()
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    out = {"op": a.op, "precision": a.precision, "refine": a.refine, "inner_tol": a.inner_tol, "N": S.N,
           "batch": a.batch, "ms": ms,
           "launches_per_rep": (S.launch_count() - l0) / a.reps}
    if info is not None:
        out["info"] = info[0]
    if info is not None and not a.no_phases:
        out["phases_ms_per_rep"] = {k: (v[0] / a.reps, v[1] / a.reps) for k, v in S.phase_times().items()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
