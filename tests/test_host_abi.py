"""CPU tests of the C-ABI library: it loads, exports every symbol of
include/stls.h, validates parameters, and its host setup (1D matrices and
generalized eigendecompositions) agrees with the oracle.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1809_10026_gb300 as stls
from paper_1809_10026_gb300 import _lib
from oracle.spaces import Direction1D
from oracle.fd import FD
from oracle.system import STProblem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_10026_gb300 import build
    build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "stls.h")).read()
    declared = set(re.findall(r"\b(stls_[A-Za-z_0-9]+)\s*\(", header))
    assert declared == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("bad", [dict(d=4), dict(p_s=1), dict(T=0.0), dict(T=float("nan")),
                                 dict(n_el_t=0), dict(batch=0), dict(precision=7), dict(fp64_residuals=2),
                                 dict(n_el_t=127, p_t=3), dict(n_el_s=(128, 4, 0))])
def test_invalid_parameters_rejected_on_host(lib, bad):
    prm = _lib.make_params(2, 3, 4)
    for k, v in bad.items():
        if k == "n_el_s":
            for i, e in enumerate(v):
                prm.n_el_s[i] = e
        else:
            setattr(prm, k, v)
    out = np.zeros(100000)
    rc = lib.stls_host_factor(ctypes.byref(prm), 0, 0, out.ctypes.data_as(ctypes.c_void_p))
    assert rc == _lib.STLS_EINVAL
    assert lib.stls_last_error(None).startswith(b"stls_host_factor: ")


def test_no_gpu_fails_loudly(lib):
    """Without a usable GPU the product path has no fallback: the binding's
    Solver raises, and stls_create returns an error with the CUDA reason and
    no context."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="CUDA"):
        stls.Solver(2, 3, 4)
    prm = _lib.make_params(2, 3, 4)
    ctx = ctypes.c_void_p()
    rc = lib.stls_create(ctypes.byref(ctx), ctypes.byref(prm), None)
    assert rc in (_lib.STLS_ENOMEM, _lib.STLS_ECUDA) and ctx.value is None
    assert lib.stls_last_error(None)


def test_largest_sizes_accepted(lib):
    """128 basis functions per direction (the dense 1D factors' limit): n_el + p - 2
    = 128 in space, n_el_t + p_t - 1 = 128 in time."""
    U = stls.host_factor("eigvec", 0, 2, 3, [127, 4], n_el_t=126)
    assert U.shape == (128, 128)
    Ut = stls.host_factor("eigvec", 2, 2, 3, [127, 4], n_el_t=126)
    assert Ut.shape == (128, 128)


def test_create_rejects_invalid_params_before_any_launch(lib):
    prm = _lib.make_params(2, 3, 4)
    prm.p_s = 1
    ctx = ctypes.c_void_p()
    assert lib.stls_create(ctypes.byref(ctx), ctypes.byref(prm), None) == _lib.STLS_EINVAL
    assert ctx.value is None
    assert b"p_s" in lib.stls_last_error(None)


@pytest.mark.parametrize("n_el,p,T", [(4, 2, 1.0), (16, 3, 0.7), (64, 3, 1.0), (32, 4, 1.0), (9, 6, 2.0)])
def test_host_matrices_match_oracle(lib, n_el, p, T):
    s = Direction1D(n_el, p, "space")
    t = Direction1D(n_el, p, "time", T)
    kw = dict(T=T)
    for name, ref in [("mass", s.M), ("stiff", s.K), ("bilap", s.J)]:
        got = stls.host_factor(name, 0, 1, p, n_el, **kw)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    for name, ref in [("mass", t.M), ("stiff", t.K), ("end", t.end_values), ("integral", t.integrals)]:
        got = stls.host_factor(name, 1, 1, p, n_el, **kw)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("n_el,p", [(16, 2), (64, 3), (32, 4), (61, 6), (125, 3)])
def test_host_eigendecomposition(lib, n_el, p):
    """Algorithm 1 step 1: U^T M U = I, U^T J U = Lambda, eigenvalues agree with scipy."""
    prob = STProblem(1, p, n_el)
    fd = FD(prob)
    U = stls.host_factor("eigvec", 0, 1, p, n_el)
    lam = stls.host_factor("eigval", 0, 1, p, n_el)
    s = prob.space[0]
    np.testing.assert_allclose(U.T @ s.M @ U, np.eye(s.n), atol=1e-13)
    np.testing.assert_allclose(U.T @ s.J @ U, np.diag(lam), atol=1e-12 * lam.max())
    np.testing.assert_allclose(lam, fd.lam[0], rtol=1e-9)
    Ut = stls.host_factor("eigvec", 1, 1, p, n_el)
    lt = stls.host_factor("eigval", 1, 1, p, n_el)
    np.testing.assert_allclose(Ut.T @ prob.time.M @ Ut, np.eye(prob.n_t), atol=1e-13)
    np.testing.assert_allclose(Ut.T @ prob.time.K @ Ut, np.diag(lt), atol=1e-12 * lt.max())
    np.testing.assert_allclose(lt, fd.lam_t, rtol=1e-9)


def test_hat_time_pencil(lib):
    lt_phys = stls.host_factor("eigval", 1, 1, 3, 8, T=2.5)
    lt_hat = stls.host_factor("eigval", 1, 1, 3, 8, T=2.5, time_pencil="hat")
    # (M_t, K_t) = (T M_hat, K_hat / T): eigenvalues scale by 1 / T^2
    np.testing.assert_allclose(lt_phys, lt_hat / 2.5 ** 2, rtol=1e-12)


@pytest.mark.parametrize("d,p,n_el,a", [(1, 3, 4, [0.5]), (2, 2, 3, [0.6, -0.4]), (3, 3, 2, [0.3, 0.5, -0.4])])
def test_geometry_host_factors_match_oracle(d, p, n_el, a):
    """Stretched parametrization (geometry = 1): the library's weighted 1D
    factors of A equal the oracle's (same Gauss rule), and the eigenvalues of
    the geometry-aware preconditioner's pencils (separation of variables in
    product form on the host) equal those of the oracle's full-tensor version."""
    from oracle.geometry import MappedProblem
    mp = MappedProblem(d, p, n_el, a)
    for k in range(d):
        for name, key in (("geo_mass", "M"), ("geo_stiff", "K"), ("geo_bilap", "J"), ("geo_e", "E")):
            A = stls.host_factor(name, k, d, p, n_el, geo_a=a)
            R = mp.weighted[k][key]
            assert np.abs(A - R).max() <= 1e-13 * np.abs(R).max(), (k, name)
    PG = mp.preconditioner()
    for k in range(d + 1):
        lam = stls.host_factor("eigval", k, d, p, n_el, geo_a=a)
        ref = PG.lam[k] if k < d else PG.lam_t
        assert np.abs(lam - ref).max() <= 1e-12 * np.abs(ref).max()


def test_geometry_parameters_are_validated():
    lib = _lib.load()
    out = np.zeros(256)
    for kw, msg in ((dict(precision="tf32", geo_a=[0.5, 0.5]), b"STLS_FP64"),
                    (dict(geo_a=[1.0, 0.5]), b"|geo_a[k]| < 1"),
                    (dict(geo_a=[0.2, 0.5], geo_precond="PG"), None)):
        prm = stls.make_params(2, 3, 4, **kw)
        rc = lib.stls_host_factor(ctypes.byref(prm), 0, 0, out.ctypes.data_as(ctypes.c_void_p))
        if msg is None:
            assert rc == _lib.STLS_OK
        else:
            assert rc == _lib.STLS_EINVAL and msg in lib.stls_last_error(None)
