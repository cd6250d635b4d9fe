"""The time-slab decomposition (paper_1809_10026_gb300.timeslab) on CPU: gloo
ranks in separate processes (world sizes 2 and 3) and, in one process, up to
four ranks exchanging through LoopbackComm, with the oracle's numpy local
operations.  The distributed A x, P^{-1} r and PCG solve equal the oracle's
global ones.  (The GPU local operations are checked in test_gpu_timeslab.py.)"""
import os
import socket

import numpy as np
import pytest
import torch

from oracle.system import STProblem
from oracle.fd import FD
from oracle.solve import direct_solve
from paper_1809_10026_gb300 import synth
from paper_1809_10026_gb300.timeslab import Partition, LoopbackComm, ProcessComm, TimeSlabPCG
from timeslab_oracle_local import OracleLocal



def _split(x, part, B):
    X = x.reshape(B, part.n_t, part.N_s)
    return {r: torch.from_numpy(np.ascontiguousarray(X[:, t0:t1])) for r, (t0, t1) in enumerate(part.t)}


def _join(parts, part, B):
    return np.concatenate([parts[r].numpy() for r in range(part.P)], axis=1).reshape(B, -1)


@pytest.mark.parametrize("P,d,p,n_el,T", [(1, 2, 3, 5, 1.0), (2, 2, 3, 5, 1.3), (3, 2, 2, 6, 1.0),
                                           (4, 1, 2, 9, 0.7), (2, 3, 2, 3, 1.0)])
def test_loopback_operators_equal_global(P, d, p, n_el, T):
    prob = STProblem(d, p, n_el, T)
    B = 2
    part = Partition(prob.n_t, prob.N_s, P, prob.p_t)
    local = {r: OracleLocal(prob, B) for r in range(P)}
    ts = TimeSlabPCG(part, local, LoopbackComm())
    x = synth.uniform(prob.N, 31, batch=B).reshape(B, prob.N)
    A = prob.assemble_A_kron()
    y = _join(ts.apply_A(_split(x, part, B)), part, B)
    z = _join(ts.apply_precond(_split(x, part, B)), part, B)
    fd = FD(prob)
    for b in range(B):
        ref = A @ x[b]
        assert np.abs(y[b] - ref).max() <= 1e-13 * np.abs(ref).max()
        refz = fd.apply(x[b])
        assert np.abs(z[b] - refz).max() <= 1e-12 * np.abs(refz).max()


def test_partition_rejects_thin_slabs():
    with pytest.raises(ValueError):
        Partition(7, 36, 3, 3)     # slabs of 2 or 3 slices with p_t = 3
    part = Partition(14, 36, 4, 3)
    assert [t1 - t0 for t0, t1 in part.t] == [3, 4, 3, 4] and part.ext(1) == (0, 10)


def test_loopback_solve_equals_direct_solve():
    prob = STProblem(2, 2, 6)      # n_t = 7, p_t = 2: three slabs
    B = 2
    part = Partition(prob.n_t, prob.N_s, 3, prob.p_t)
    local = {r: OracleLocal(prob, B) for r in range(3)}
    ts = TimeSlabPCG(part, local, LoopbackComm())
    F = synth.uniform(prob.N, 41, batch=B).reshape(B, prob.N)
    u, it, rel = ts.solve(_split(F, part, B), 1e-12, 200)
    u = _join(u, part, B)
    A = prob.assemble_A_kron()
    for b in range(B):
        ref = direct_solve(A, F[b])
        assert rel[b] <= 1e-12 and np.linalg.norm(u[b] - ref) <= 1e-10 * np.linalg.norm(ref)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = STProblem(2, 2, 6)
        B = 2
        part = Partition(prob.n_t, prob.N_s, world, prob.p_t)
        ts = TimeSlabPCG(part, {rank: OracleLocal(prob, B)}, ProcessComm(rank, world, "cpu"))
        x = synth.uniform(prob.N, 51, batch=B).reshape(B, prob.N)
        xs = {rank: _split(x, part, B)[rank]}
        t0, t1 = part.t[rank]
        A = prob.assemble_A_kron()
        fd = FD(prob)
        y = ts.apply_A(xs)[rank].numpy()
        z = ts.apply_precond(xs)[rank].numpy()
        F = synth.uniform(prob.N, 52, batch=B).reshape(B, prob.N)
        u, it, rel = ts.solve({rank: _split(F, part, B)[rank]}, 1e-12, 200)
        ok = True
        for b in range(B):
            refy = (A @ x[b]).reshape(prob.n_t, -1)[t0:t1]
            refz = fd.apply(x[b]).reshape(prob.n_t, -1)[t0:t1]
            refu = direct_solve(A, F[b]).reshape(prob.n_t, -1)
            ok &= np.abs(y[b] - refy).max() <= 1e-13 * np.abs(refy).max()
            ok &= np.abs(z[b] - refz).max() <= 1e-12 * np.abs(refz).max()
            ok &= np.linalg.norm(u[rank][b].numpy() - refu[t0:t1]) <= 1e-10 * np.linalg.norm(refu)
        with open(os.path.join(out_dir, "rank%d" % rank), "w") as f:
            f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_global(world, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        assert (tmp_path / ("rank%d" % r)).read_text() == "ok"
