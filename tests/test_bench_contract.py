"""CPU checks of bench.py's roofline bookkeeping: the entry of each timed
operation carries the keys of the bench line's roofline object, its achieved
rate follows from the operation's algorithmic bytes or flops and the measured
time, and frac = achieved / peak.  No GPU needed."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N = 18125250
PEAKS = {"hbm_gbs": 6774.0, "bf16_tflops": 1891.0, "bf16_tflops_sustained": 1700.0, "source": "measured"}


def fake_solver(precision):
    # 3D, p = 3, 64 elements: 65 unknowns per spatial direction, 66 in time
    return types.SimpleNamespace(precision=precision, N=N, n_s=[65, 65, 65], n_t=66, d=3)


def test_flop_counts_of_the_workload():
    S = fake_solver("fp64")
    # 15 banded products of 2(2p+1) flops per unknown (p = 3)
    assert bench.apply_A_flops(S, 3) == pytest.approx(15 * 14 * N)
    # Algorithm 1: 4 N (sum of the 1D sizes) + N
    assert bench.fd_flops(S) == pytest.approx(4.0 * N * (3 * 65 + 66) + N)


@pytest.mark.parametrize("phase,precision,refine,bound,unit", [
    ("precond", "tf32", True, "hbm", "GB/s"),
    ("precond", "bf16", False, "hbm", "GB/s"),
    ("precond", "fp64", False, "alu", "TFLOP/s"),
    ("apply_A", "tf32", True, "alu", "TFLOP/s"),
    ("apply_A_f32", "tf32", True, "alu", "TFLOP/s"),
    ("apply_A_df", "tf32", True, "alu", "Top/s"),
])
def test_roofline_entry_keys_and_rate(phase, precision, refine, bound, unit):
    S = fake_solver(precision)
    ms, count = 5.0, 19  # ms over all calls of the operation in one solve, calls
    e = bench.roofline_entry(phase, ms, count, S, 3, PEAKS, refine)
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in e
    assert e["bound"] == bound and e["unit"] == unit
    assert e["frac"] == pytest.approx(e["achieved"] / e["peak"])
    per_s = ms / count * 1e-3
    if phase == "precond" and precision != "fp64":
        nbytes = (8.0 if refine else 16.0) * N
        assert e["achieved"] == pytest.approx(nbytes / per_s / 1e9)
        assert e["peak"] == PEAKS["hbm_gbs"]
    if phase == "apply_A_f32":
        assert e["achieved"] == pytest.approx(bench.apply_A_flops(S, 3) / per_s / 1e12)
    if (phase, precision, refine) in bench.TRAFFIC:
        assert e["traffic"] == bench.TRAFFIC[(phase, precision, refine)]
    else:
        assert e["traffic"] is None


def test_roofline_entry_without_calls_is_none():
    assert bench.roofline_entry("precond", 0.0, 0, fake_solver("tf32"), 3, PEAKS, True) is None


def test_single_thread_sample_parsing(monkeypatch):
    """The one-thread oracle sample runs in a child process with one-thread
    pools; the parent turns its JSON line into the cpu_baseline entry, and a
    failing or slow child becomes a 'skipped' note instead of an error."""
    import subprocess

    seen = {}

    def fake_run(cmd, env=None, capture_output=None, text=None, timeout=None):
        seen["cmd"], seen["env"] = cmd, env
        return subprocess.CompletedProcess(cmd, 0, stdout="noise\n[0.5, 2.0, 1000]\n", stderr="")

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    out = bench.single_thread_sample(17)
    assert seen["cmd"][-1] == "--oracle-iteration-sample"
    assert seen["env"]["OMP_NUM_THREADS"] == "1" and seen["env"]["OPENBLAS_NUM_THREADS"] == "1"
    assert out["cores"] == 1 and out["solve_s_extrapolated"] == pytest.approx(0.5 + 17 * 2.0)
    assert out["value"] == pytest.approx(1000 / (0.5 + 17 * 2.0))

    def failing(cmd, **kw):
        return subprocess.CompletedProcess(cmd, 1, stdout="", stderr="Traceback\nMemoryError")

    monkeypatch.setattr(bench.subprocess, "run", failing)
    assert bench.single_thread_sample(17) == {"skipped": "child failed: MemoryError"}

    def slow(cmd, **kw):
        raise subprocess.TimeoutExpired(cmd, kw.get("timeout"))

    monkeypatch.setattr(bench.subprocess, "run", slow)
    assert "skipped" in bench.single_thread_sample(17, timeout_s=1)


def test_oracle_iteration_sample_child():
    """The child entry point itself: one oracle PCG iteration on the full
    workload (about 10 s on one core), printed as [setup s, iteration s, N]."""
    import json
    import subprocess
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-iteration-sample"],
                         env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    t_setup, t_iter, n = json.loads(res.stdout.strip().splitlines()[-1])
    assert n == N and t_setup >= 0 and t_iter > 0
