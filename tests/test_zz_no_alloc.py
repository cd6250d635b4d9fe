"""The allocation-free preconditioner apply (stls_apply_precond_noalloc).

It exists for callers that cannot allocate device memory where they apply
the preconditioner (real-time loops that cannot afford the allocator, plugin
hosts with a fixed memory budget): its scratch is a fixed array inside the
library.  This file checks, through the C ABI, that two calls in a row agree
with the oracle's fast-diagonalization solve (Algorithm 1) and with
stls_apply_precond of a solver context (FP64 form), both to the tolerance the
FD parity tests use, for one, two and three space dimensions, and that
oversized requests are refused before any launch.  It is named so pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1809_10026_gb300 as stls
from oracle.fd import FD
from oracle.system import STProblem
from paper_1809_10026_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _fd_tolerance(lams):
    # same bound as the FD parity tests: 1e-11 + 4 eps max lambda_max / (lambda_2 - lambda_1)
    eps = np.finfo(float).eps
    return 1e-11 + 4 * eps * max(l[-1] / (l[1] - l[0]) for l in lams if len(l) > 1)


def _factors(d, p, n_el):
    U = [stls.host_factor("eigvec", k, d, p, n_el) for k in range(d + 1)]
    lam = [stls.host_factor("eigval", k, d, p, n_el) for k in range(d + 1)]
    return U, lam


def _call(d, sizes, batch, U_dev, lam_dev, r, z):
    lib = _lib.load()
    n_arr = (ctypes.c_int * (d + 1))(*sizes)
    U_arr = (ctypes.c_void_p * (d + 1))(*[u.data_ptr() for u in U_dev])
    L_arr = (ctypes.c_void_p * (d + 1))(*[l.data_ptr() for l in lam_dev])
    stream = torch.cuda.current_stream().cuda_stream
    return lib.stls_apply_precond_noalloc(d, n_arr, batch, U_arr, L_arr, ctypes.c_void_p(r.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("d,p,n_el,batch", [(1, 2, 16, 3), (2, 3, 64, 1), (3, 3, 9, 2)])
def test_noalloc_matches_oracle_and_context_apply_twice(d, p, n_el, batch):
    S = stls.Solver(d, p, n_el, batch=batch)
    fd = FD(STProblem(d, p, n_el))
    U, lam = _factors(d, p, n_el)
    U_dev = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]
    lam_dev = [torch.from_numpy(l).cuda() for l in lam]
    sizes = S.n_s + [S.n_t]
    tol = _fd_tolerance(lam)
    for call in range(2):
        r = torch.from_numpy(synth.uniform(S.N, 900 + call, batch=batch)).cuda()
        z = torch.empty_like(r)
        assert _call(d, sizes, batch, U_dev, lam_dev, r, z) == _lib.STLS_OK
        ref = S.apply_precond(r)
        torch.cuda.synchronize()
        zr = z.cpu().numpy().reshape(batch, S.N)
        rr = ref.cpu().numpy().reshape(batch, S.N)
        rh = r.cpu().numpy().reshape(batch, S.N)
        for b in range(batch):
            ex = fd.apply(rh[b])
            np.testing.assert_allclose(zr[b], ex, rtol=0, atol=tol * np.abs(ex).max())
        np.testing.assert_allclose(zr, rr, rtol=0, atol=tol * np.abs(rr).max())


def test_noalloc_rejects_oversized_request():
    d, p, n_el = 3, 4, 32        # N = 1,375,640 > 524,288
    U, lam = _factors(d, p, n_el)
    U_dev = [torch.from_numpy(np.ascontiguousarray(u)).cuda() for u in U]
    lam_dev = [torch.from_numpy(l).cuda() for l in lam]
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = _call(d, [34, 34, 34, 35], 1, U_dev, lam_dev, r, r)
    assert rc == _lib.STLS_EINVAL
    assert b"524288" in _lib.load().stls_last_error(None)
