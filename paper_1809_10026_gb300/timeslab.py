"""Time-slab decomposition of the FP64 solver over ranks (one GPU per rank).

The paper leaves parallel solvers to future work (Sec. 1 and Sec. 6).  Here
rank r owns the time slices [t0_r, t1_r) of every right-hand side; a local
vector has B x (t1_r - t0_r) x N_s entries.  The operators split as follows
(all arithmetic in the library's kernels, through the local-operation calls
of include/stls.h; this module only moves data):

* A x (Eq. A_kron) is local in space and banded in time with half-width p_t:
  each rank forms the spatial factors M_s x, J_s x of its slices
  (stls_slab_spatial), sends its first and last p_t slices of them to its
  neighbours, and applies the time band to its rows with those halos
  (stls_slab_time); L_s x of the last time slice stays with its owner.
* Algorithm 1 is local in space and dense in time: forward spatial mode
  products on the rank's slices (stls_fd_spatial), an all-to-all after which
  rank q holds all time slices of the spatial indices [s0_q, s1_q), the time
  products with the division on them (stls_fd_time_chunk), the reverse
  all-to-all and the backward spatial products.
* CG needs per-right-hand-side inner products summed over ranks
  (stls_vec_dot + a sum over ranks) and vector updates (stls_vec_axpby).

A ``Comm`` moves tensors between the ranks that the process holds:
``ProcessComm`` (torch.distributed point-to-point sends, one rank per
process; gloo on CPU, NCCL between GPUs) or ``LoopbackComm`` (all ranks in
one process: the exchange is a hand-over of tensors, so no kernel ever waits
for another).  ``TimeSlabPCG`` works on the list of ranks the process holds,
phase by phase.
"""
import numpy as np


class Partition:
    """Balanced time slabs [t0_r, t1_r) and spatial chunks [s0_r, s1_r) for P ranks.
    Every slab holds at least p_t slices (the halos come from direct neighbours)."""

    def __init__(self, n_t, N_s, P, p_t):
        if P < 1 or P > n_t or P > N_s:
            raise ValueError("need 1 <= P <= min(n_t, N_s)")
        self.n_t, self.N_s, self.P, self.p_t = n_t, N_s, P, p_t
        tb = [n_t * r // P for r in range(P + 1)]
        sb = [N_s * r // P for r in range(P + 1)]
        self.t = [(tb[r], tb[r + 1]) for r in range(P)]
        self.s = [(sb[r], sb[r + 1]) for r in range(P)]
        if P > 1 and min(t1 - t0 for t0, t1 in self.t) < p_t:
            raise ValueError("every time slab must hold at least p_t slices")

    def ext(self, r):
        """Rows [e0, e1) of rank r's time band: its slab and the halos."""
        t0, t1 = self.t[r]
        return max(0, t0 - self.p_t), min(self.n_t, t1 + self.p_t)


class LoopbackComm:
    """All ranks in this process: messages are handed over directly."""

    def exchange(self, msgs, expect):
        """msgs: (src, dst, tag, tensor) sent by the ranks this process holds;
        expect: (src, dst, tag, shape) they receive.  Returns {(src, dst, tag): tensor}."""
        return {(s, d, t): x for s, d, t, x in msgs}

    def sum_over_ranks(self, values):
        """values: {rank: numpy array}; the element-wise sum over all ranks."""
        return sum(values.values())


class ProcessComm:
    """One rank per process; torch.distributed point-to-point messages."""

    def __init__(self, rank, world, device):
        import torch.distributed as dist
        self.dist, self.rank, self.world, self.device = dist, rank, world, device

    def exchange(self, msgs, expect):
        import torch
        dist = self.dist
        reqs, out = [], {}
        local = {(s, d, t): x for s, d, t, x in msgs if d == self.rank}
        # messages between two ranks are posted in the order of (tag, src, dst)
        # on both sides, so that point-to-point order matches
        for s, d, t, shape in sorted(expect, key=lambda m: (m[2], m[0], m[1])):
            if s == self.rank:
                out[(s, d, t)] = local[(s, d, t)]
                continue
            buf = torch.empty(shape, dtype=torch.float64, device=self.device)
            out[(s, d, t)] = buf
            reqs.append(dist.irecv(buf, src=s, tag=_tag(t)))
        for s, d, t, x in sorted(msgs, key=lambda m: (m[2], m[0], m[1])):
            if d != self.rank:
                reqs.append(dist.isend(x.contiguous(), dst=d, tag=_tag(t)))
        for q in reqs:
            q.wait()
        return out

    def sum_over_ranks(self, values):
        import torch
        (v,) = values.values()
        t = torch.as_tensor(np.asarray(v, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()


_TAGS = {"loM": 1, "loJ": 2, "hiM": 3, "hiJ": 4, "fwd": 5, "bwd": 6}


def _tag(t):
    return _TAGS[t]


class GpuLocal:
    """Rank-local operations through the library (a context of the full problem
    sizes; its workspace serves every local call)."""

    def __init__(self, solver):
        import torch
        self.S, self.torch = solver, torch
        self.lib, self.ctx = solver.lib, solver.ctx
        self.B, self.N_s, self.n_t = solver.batch, solver.N_s, solver.n_t

    @staticmethod
    def _p(x):
        import ctypes
        return ctypes.c_void_p(x.data_ptr()) if x is not None else None

    def _chk(self, rc):
        from . import _check
        _check(rc, self.ctx)

    def empty(self, *shape):
        return self.torch.empty(shape, dtype=self.torch.float64, device=self.S.device)

    def spatial(self, x, want_ls):
        """M_s x and J_s x of the slices of x (B, nt, N_s); L_s x of its last slice."""
        B, nt, Ns = x.shape
        Ms, Js = self.empty(B, nt, Ns), self.empty(B, nt, Ns)
        self.S._stream()
        self._chk(self.lib.stls_slab_spatial(self.ctx, self._p(x), B * nt, self._p(Ms), self._p(Js), None))
        Ls = None
        if want_ls:
            last = x[:, -1, :].contiguous()
            Ls = self.empty(B, Ns)
            self._chk(self.lib.stls_slab_spatial(self.ctx, self._p(last), B, None, None, self._p(Ls)))
        return Ms, Js, Ls

    def time(self, Ms_ext, Js_ext, e0, e1, t0, t1, Ls_last):
        y = self.empty(self.B, t1 - t0, self.N_s)
        self._chk(self.lib.stls_slab_time(self.ctx, self._p(Ms_ext.contiguous()), self._p(Js_ext.contiguous()),
                                          e0, e1, t0, t1, self._p(Ls_last), self._p(y)))
        return y

    def fd_spatial(self, x, forward):
        B, nt, Ns = x.shape
        y = self.empty(B, nt, Ns)
        self._chk(self.lib.stls_fd_spatial(self.ctx, self._p(x.contiguous()), self._p(y), B * nt, int(forward)))
        return y

    def fd_time(self, x, s0, s1):
        y = self.empty(*x.shape)
        self._chk(self.lib.stls_fd_time_chunk(self.ctx, self._p(x.contiguous()), self._p(y), s0, s1))
        return y

    def dot(self, x, y):
        import ctypes
        out = np.zeros(self.B)
        n = x.numel() // self.B
        self._chk(self.lib.stls_vec_dot(self.ctx, self._p(x), self._p(y), n, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def axpby(self, a, x, b, y):
        import ctypes
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        n = x.numel() // self.B
        self._chk(self.lib.stls_vec_axpby(self.ctx, a.ctypes.data_as(ctypes.c_void_p), self._p(x),
                                          b.ctypes.data_as(ctypes.c_void_p), self._p(y), n))
        return y

    def zeros_like(self, x):
        return self.torch.zeros_like(x)

    def copy(self, x):
        return x.clone()


class TimeSlabPCG:
    """PCG (Sec. 4.2, x0 = 0, stop at ||r|| / ||F|| <= tol per right-hand side) on
    the time-slab decomposition.  ``local`` maps each rank held by this process
    to its local-operation object; ``comm`` moves data between ranks."""

    def __init__(self, part, local, comm):
        self.part, self.local, self.comm = part, local, comm
        self.ranks = sorted(local)

    # ---- A x ------------------------------------------------------------------------------
    def apply_A(self, xs):
        part, P = self.part, self.part.P
        fac = {r: self.local[r].spatial(xs[r], part.t[r][1] == part.n_t) for r in self.ranks}
        h = part.p_t
        B, Ns = self.local[self.ranks[0]].B, part.N_s
        msgs, expect = [], []
        for r in self.ranks:
            Ms, Js, _ = fac[r]
            if r > 0:  # my first p_t slices: the upper halo of rank r - 1
                msgs += [(r, r - 1, "hiM", Ms[:, :h].contiguous()), (r, r - 1, "hiJ", Js[:, :h].contiguous())]
                expect += [(r - 1, r, t, (B, h, Ns)) for t in ("loM", "loJ")]
            if r < P - 1:  # my last p_t slices: the lower halo of rank r + 1
                msgs += [(r, r + 1, "loM", Ms[:, -h:].contiguous()), (r, r + 1, "loJ", Js[:, -h:].contiguous())]
                expect += [(r + 1, r, t, (B, h, Ns)) for t in ("hiM", "hiJ")]
        got = self.comm.exchange(msgs, expect)
        ys = {}
        for r in self.ranks:
            Ms, Js, Ls = fac[r]
            e0, e1 = part.ext(r)
            t0, t1 = part.t[r]
            parts_M, parts_J = [], []
            if e0 < t0:
                parts_M.append(got[(r - 1, r, "loM")][:, -(t0 - e0):])
                parts_J.append(got[(r - 1, r, "loJ")][:, -(t0 - e0):])
            parts_M.append(Ms)
            parts_J.append(Js)
            if e1 > t1:
                parts_M.append(got[(r + 1, r, "hiM")][:, :e1 - t1])
                parts_J.append(got[(r + 1, r, "hiJ")][:, :e1 - t1])
            ys[r] = self.local[r].time(cat_time(parts_M), cat_time(parts_J), e0, e1, t0, t1, Ls)
        return ys

    # ---- P^{-1} r (Algorithm 1) --------------------------------------------------------------
    def apply_precond(self, rs):
        part, P = self.part, self.part.P
        B = self.local[self.ranks[0]].B
        Y = {r: self.local[r].fd_spatial(rs[r], True) for r in self.ranks}
        msgs, expect = [], []
        for r in self.ranks:
            for q in range(P):
                s0, s1 = part.s[q]
                msgs.append((r, q, "fwd", Y[r][:, :, s0:s1].contiguous()))
                t0, t1 = part.t[q]
                expect.append((q, r, "fwd", (B, t1 - t0, part.s[r][1] - part.s[r][0])))
        got = self.comm.exchange(msgs, expect)
        Z = {}
        for q in self.ranks:
            s0, s1 = part.s[q]
            block = cat_time([got[(r, q, "fwd")] for r in range(P)])
            Z[q] = self.local[q].fd_time(block, s0, s1)
        msgs, expect = [], []
        for q in self.ranks:
            for r in range(P):
                t0, t1 = part.t[r]
                msgs.append((q, r, "bwd", Z[q][:, t0:t1, :].contiguous()))
                s0, s1 = part.s[r]
                tq0, tq1 = part.t[q]
                expect.append((r, q, "bwd", (B, tq1 - tq0, s1 - s0)))
        got = self.comm.exchange(msgs, expect)
        out = {}
        for r in self.ranks:
            back = cat_space([got[(q, r, "bwd")] for q in range(P)])
            out[r] = self.local[r].fd_spatial(back, False)
        return out

    # ---- CG ---------------------------------------------------------------------------------
    def dot(self, xs, ys):
        return self.comm.sum_over_ranks({r: self.local[r].dot(xs[r], ys[r]) for r in self.ranks})

    def solve(self, Fs, tol, maxit):
        """Returns (u per rank, iterations, relative residual per right-hand side)."""
        loc = self.local
        B = loc[self.ranks[0]].B
        u = {r: loc[r].zeros_like(Fs[r]) for r in self.ranks}
        res = {r: loc[r].copy(Fs[r]) for r in self.ranks}
        nF = np.sqrt(self.dot(Fs, Fs))
        if not np.all(nF > 0):
            return u, 0, np.zeros(B)
        z = self.apply_precond(res)
        p = {r: loc[r].copy(z[r]) for r in self.ranks}
        rz = self.dot(res, z)
        ones, zeros = np.ones(B), np.zeros(B)
        active = np.ones(B, dtype=bool)
        rel = np.ones(B)
        it = 0
        for it in range(1, maxit + 1):
            q = self.apply_A(p)
            pq = self.dot(p, q)
            alpha = np.where(active, rz / pq, 0.0)
            for r in self.ranks:
                loc[r].axpby(alpha, p[r], ones, u[r])
                loc[r].axpby(-alpha, q[r], ones, res[r])
            rel = np.sqrt(self.dot(res, res)) / nF
            active &= rel > tol
            if not active.any():
                break
            z = self.apply_precond(res)
            rz_new = self.dot(res, z)
            beta = np.where(active, rz_new / rz, 0.0)
            rz = rz_new
            for r in self.ranks:
                loc[r].axpby(ones, z[r], beta, p[r])
        return u, it, rel


def cat_time(parts):
    """Concatenate (B, nt_i, ...) blocks along the time axis."""
    x = parts[0]
    if hasattr(x, "numpy"):
        import torch
        return torch.cat(list(parts), dim=1).contiguous()
    return np.concatenate(parts, axis=1)


def cat_space(parts):
    x = parts[0]
    if hasattr(x, "numpy"):
        import torch
        return torch.cat(list(parts), dim=2).contiguous()
    return np.concatenate(parts, axis=2)
