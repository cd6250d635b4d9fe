"""Rank-local operations of the time-slab decomposition computed by the
oracle (numpy, FP64), for CPU tests of the decomposition's data movement;
same interface as paper_1809_10026_gb300.timeslab.GpuLocal, on torch CPU
tensors.  Test infrastructure."""
import numpy as np
import torch

from oracle.fd import FD


class OracleLocal:
    def __init__(self, prob, B):
        self.prob, self.B = prob, B
        self.N_s, self.n_t = prob.N_s, prob.n_t
        self.fd = FD(prob)
        self.sshape = tuple(prob.n_s[::-1])   # C-order spatial shape (n_d, ..., n_1)

    def _space(self, x, mats):
        """Apply mats[k] in spatial direction k+1 to every slice of x (..., N_s)."""
        lead = x.shape[:-1]
        X = x.reshape((-1,) + self.sshape)
        d = self.prob.d
        for k, W in enumerate(mats):
            ax = X.ndim - 1 - k
            X = np.moveaxis(np.tensordot(W, X, axes=([1], [ax])), 0, ax)
        return X.reshape(lead + (self.N_s,))

    def _spatial_terms(self, x):
        sd, d = self.prob.space, self.prob.d
        M = [s.M for s in sd]
        Ms = self._space(x, M)
        Js = np.zeros_like(x)
        Ls = np.zeros_like(x)
        for k in range(d):
            for l in range(d):
                mats = list(M)
                if k == l:
                    mats[k] = sd[k].J
                else:
                    mats[k] = sd[k].D2
                    mats[l] = sd[l].D2.T
                Js += self._space(x, mats)
            mats = list(M)
            mats[k] = sd[k].K
            Ls += self._space(x, mats)
        return Ms, Js, Ls

    def spatial(self, x, want_ls):
        Ms, Js, _ = self._spatial_terms(x.numpy())
        Ls = None
        if want_ls:
            Ls = torch.from_numpy(self._spatial_terms(x.numpy()[:, -1, :])[2])
        return torch.from_numpy(Ms), torch.from_numpy(Js), Ls

    def time(self, Ms_ext, Js_ext, e0, e1, t0, t1, Ls_last):
        tm = self.prob.time
        K, M = tm.K[t0:t1, e0:e1], tm.M[t0:t1, e0:e1]
        y = np.einsum("te,bes->bts", K, Ms_ext.numpy()) + np.einsum("te,bes->bts", M, Js_ext.numpy())
        if t1 == self.n_t:
            y[:, -1, :] += tm.W[-1, -1] * Ls_last.numpy()
        return torch.from_numpy(y)

    def fd_spatial(self, x, forward):
        mats = [U.T if forward else U for U in self.fd.U]
        return torch.from_numpy(self._space(x.numpy(), mats))

    def fd_time(self, x, s0, s1):
        fd = self.fd
        X = np.einsum("mt,bts->bms", fd.U_t.T, x.numpy())
        lam_s = fd.eig_tensor()[0].reshape(-1) - fd.lam_t[0]   # sum_k lambda_k over the spatial index
        X = X / (fd.lam_t[None, :, None] + lam_s[None, None, s0:s1])
        return torch.from_numpy(np.einsum("tm,bms->bts", fd.U_t, X))

    def dot(self, x, y):
        return np.einsum("bi,bi->b", x.numpy().reshape(self.B, -1), y.numpy().reshape(self.B, -1))

    def axpby(self, a, x, b, y):
        yn = y.numpy().reshape(self.B, -1)
        yn[:] = np.asarray(a)[:, None] * x.numpy().reshape(self.B, -1) + np.asarray(b)[:, None] * yn
        return y

    def zeros_like(self, x):
        return torch.zeros_like(x)

    def copy(self, x):
        return x.clone()
