"""Multi-rank logic of bench.py on CPU (gloo, world size 2): process-group set-up,
barrier, max over ranks of the timed interval, the whole-job replica rate, and
the reference arm running on rank 0 only.  No GPU needed."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    args = argparse.Namespace(impl="reference")
    w, r, local = bench.dist_setup(args)
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank r timed 10 * (r + 1) ms: every rank sees the slowest
    ms = bench.max_over_ranks(10.0 * (rank + 1), w, torch.device("cpu"))
    rate = bench.replica_rate(1000, 4, w, ms)
    out[rank] = (ms, rate)
    dist.destroy_process_group()


def test_two_ranks_gloo_max_and_rate():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == 20.0
        # 2 replicas x 1000 units x 4 steps in 20 ms
        assert rate == pytest.approx(2 * 1000 * 4 / 0.020)


def test_reference_arm_other_ranks_do_no_work(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def test_replica_rate_single_gpu():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(18125250, 5, 1, 1000.0) == pytest.approx(18125250 * 5)


def test_reference_arm_json_line(capsys, monkeypatch):
    """The reference arm (the oracle's FP64 PCG on the host) prints one JSON
    line with the keys of the bench contract; run here on a small cube."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "WORKLOAD", dict(bench.WORKLOAD, n_el=4, name="cube3d_p3_n4"))
    bench.run_reference(argparse.Namespace(steps=2, warmup=1))
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "DoF/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 2 and line["warmup"] == 1 and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "cube3d_p3_n4"
