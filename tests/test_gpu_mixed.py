"""GPU parity of the mixed-precision (tensor-core) preconditioner and solves.

The tensor-core FD apply is compared with oracle.mixed, which applies the
same BF16/TF32 operand roundings, FP32 accumulation and intermediate storage
formats.  The two differ in how the FP32 sums are rounded: the tensor core's
accumulator is not a correctly rounded FP32 sum of the K products, and the
products with the M-orthonormal eigenvector matrices cancel strongly (entries
of U grow like h^{-1/2}), so a few FP32 ulps per product become ~5e-5
normwise after 2(d+1) products.  A differently rounded BF16 intermediate
flips by one BF16 ulp now and then.  Normwise bounds: BF16 <= 2e-3, TF32 <=
2e-4 against the model, and against exact FP64 Algorithm 1 (the model's own
error is ~1e-2 / ~1e-3): BF16 <= 3e-2, TF32 <= 3e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from oracle.fd import FD
from oracle import mixed
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_MODEL = {"bf16": 2e-3, "tf32": 2e-4}
TOL_EXACT = {"bf16": 3e-2, "tf32": 3e-3}


def _solver(*a, **k):
    import paper_1809_10026_gb300 as stls
    return stls.Solver(*a, **k)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _bwd_order(form, d):
    # the fused BF16 kernels (d = 2, 3) run the backward products as t, d, ..., 1
    return "descending" if form == "bf16" and d >= 2 else "ascending"


@pytest.mark.parametrize("form", ["bf16", "tf32"])
@pytest.mark.parametrize("d,p,n_el,batch", [(1, 2, 7, 1), (2, 3, 6, 3), (2, 5, 9, 1), (3, 2, 4, 2),
                                            (3, 3, 9, 1), (3, 4, 12, 1), (2, 2, 70, 2), (3, 3, 20, 2),
                                            (3, 2, 1, 1)])
def test_tc_precond_matches_model(form, d, p, n_el, batch):
    """Several slab steps and streaming tiles with ragged tails, odd sizes (n = 2..71),
    batches, and the smallest mesh (one element)."""
    prob = STProblem(d, p, n_el)
    fd = FD(prob)
    S = _solver(d, p, n_el, precision=form, batch=batch)
    r = synth.uniform(prob.N, 500 + d + p, batch=batch).reshape(batch, prob.N)
    z = S.apply_precond(torch.from_numpy(r).cuda()).cpu().numpy().reshape(batch, prob.N)
    for b in range(batch):
        model = mixed.apply_mixed(fd, r[b], form, _bwd_order(form, d))
        exact = fd.apply(r[b])
        assert _rel(z[b], model) <= TOL_MODEL[form], (_rel(z[b], model), _rel(z[b], exact))
        assert _rel(z[b], exact) <= TOL_EXACT[form]


def test_operand_rounding_bit_exact():
    """FP64 -> FP32 -> BF16 rounding of the BF16 preconditioner's input (integer
    implementation on the GPU) equals numpy's IEEE rounding bit for bit: random
    values over the whole exponent range, exact FP64 -> FP32 and FP32 -> BF16 ties,
    the FP32 overflow threshold, FP32 subnormals, FP64 subnormals, signed zeros,
    infinities and NaN."""
    import paper_1809_10026_gb300 as stls
    rng = np.random.default_rng(1809)
    parts = [rng.standard_normal(100000) * np.exp2(rng.integers(-160, 140, 100000)).astype(np.float64)]
    # exact halfway points between neighbouring FP32 values (even and odd kept parts)
    f32 = rng.standard_normal(20000).astype(np.float32)
    f = f32.astype(np.float64)
    half32 = np.spacing(f32).astype(np.float64) / 2
    parts += [f + half32, f - half32 / 2, f + half32 * (1 - 2.0 ** -20)]
    # exact halfway points between neighbouring BF16 values
    b = mixed.round_bf16(rng.standard_normal(20000).astype(np.float32)).astype(np.float64)
    _, ex = np.frexp(b)
    half16 = np.ldexp(np.sign(b), ex - 9)
    parts += [b + half16, b - half16, b + half16 * 3]
    fmax = float(np.finfo(np.float32).max)
    parts.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2.0 ** -25),
                           fmax * (1 + 2.0 ** -24), 2.0 ** -126, 2.0 ** -130, 2.0 ** -149, 2.0 ** -150,
                           3 * 2.0 ** -151, 5e-324, -5e-324, 1e-310, 1.0, -1.0, 1 + 2.0 ** -24,
                           1 + 3 * 2.0 ** -24, 2.0 ** 128, 1e300, -1e300]))
    x = np.concatenate(parts)
    with np.errstate(over="ignore"):
        want = mixed.round_bf16(x.astype(np.float32)).astype(np.float64)
    got = stls.round_bf16(torch.from_numpy(x).cuda()).cpu().numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), want[~nan].view(np.uint64))


@pytest.mark.parametrize("form", ["bf16", "tf32"])
@pytest.mark.parametrize("d,p,n_el,kw,batch", [
    (3, 3, [4, 7, 5], dict(T=1.3, p_t=2, n_el_t=6), 2),
    (3, 2, [9, 3, 6], dict(T=0.7, p_t=4, n_el_t=3), 1),
    (2, 4, [11, 5], dict(T=2.0, p_t=1, n_el_t=9), 3),
    (2, 3, [40, 7], dict(T=1.0), 1)])
def test_tc_precond_anisotropic_matches_model(form, d, p, n_el, kw, batch):
    """Different sizes per direction (so the slab kernels' two directions and the
    streaming passes see different n), other time degrees and T != 1."""
    prob = STProblem(d, p, n_el, **kw)
    fd = FD(prob)
    S = _solver(d, p, n_el, precision=form, batch=batch, **kw)
    r = synth.uniform(prob.N, 700 + d + p, batch=batch).reshape(batch, prob.N)
    z = S.apply_precond(torch.from_numpy(r).cuda()).cpu().numpy().reshape(batch, prob.N)
    for b in range(batch):
        model = mixed.apply_mixed(fd, r[b], form, _bwd_order(form, d))
        assert _rel(z[b], model) <= TOL_MODEL[form], _rel(z[b], model)
        assert _rel(z[b], fd.apply(r[b])) <= TOL_EXACT[form]


@pytest.mark.parametrize("form", ["bf16", "tf32"])
def test_tc_precond_cube3d_p3_n64(form):
    prob = STProblem(3, 3, 64)
    fd = FD(prob)
    S = _solver(3, 3, 64, precision=form)
    r = synth.uniform(prob.N, 4)
    z = S.apply_precond(torch.from_numpy(r).cuda()).cpu().numpy()
    assert _rel(z, fd.apply(r)) <= TOL_EXACT[form]


@pytest.mark.parametrize("form", ["bf16", "tf32"])
def test_mixed_solve_cube3d_p4_n32(form):
    """3D, p = 4, 32 elements (1,375,640 DoF), manufactured load: flexible CG with the
    tensor-core preconditioner reaches the FP64 solution."""
    pi = np.pi
    prob = STProblem(3, 4, 32)
    s = lambda x: np.sin(pi * x)
    F = prob.load_separable([(1.0, np.cos, [s, s, s]), (3 * pi ** 2, np.sin, [s, s, s])])
    Fg = torch.from_numpy(F).cuda()
    S64 = _solver(3, 4, 32)
    u64, i64 = S64.solve(Fg, tol=1e-12, maxit=300)
    Sm = _solver(3, 4, 32, precision=form)
    u8, i8 = Sm.solve(Fg, tol=1e-8, maxit=300)
    assert i8[0]["status"] == "ok" and i8[0]["true_rel_res"] <= 1.5e-8
    assert i8[0]["iters"] <= 2 * 12 + 4
    u12, i12 = Sm.solve(Fg, tol=1e-12, maxit=300)
    assert i12[0]["status"] == "ok"
    assert _rel(u12.cpu().numpy(), u64.cpu().numpy()) <= 1e-8
    print(form, "iters@1e-8", i8[0]["iters"], "iters@1e-12", i12[0]["iters"], "fp64 iters@1e-12", i64[0]["iters"])


def test_mixed_solve_cube3d_p3_n64_bf16():
    prob_N = 18125250
    S = _solver(3, 3, 64, precision="bf16")
    F = torch.from_numpy(synth.uniform(prob_N, 4)).cuda()
    u, info = S.solve(F, tol=1e-8, maxit=200)
    assert info[0]["status"] == "ok" and info[0]["true_rel_res"] <= 1.5e-8
    assert info[0]["iters"] <= 40


@pytest.mark.parametrize("form", ["bf16", "tf32"])
def test_refinement_solve_cube3d_p4_n32(form):
    """Iterative refinement: FP64 residual F - A u, inner FP32 flexible CG with the
    tensor-core preconditioner; the stopping test is on the true FP64 residual."""
    pi = np.pi
    prob = STProblem(3, 4, 32)
    s = lambda x: np.sin(pi * x)
    F = prob.load_separable([(1.0, np.cos, [s, s, s]), (3 * pi ** 2, np.sin, [s, s, s])])
    Fg = torch.from_numpy(F).cuda()
    u64, _ = _solver(3, 4, 32).solve(Fg, tol=1e-12, maxit=300)
    S = _solver(3, 4, 32, precision=form, refine=True)
    u8, i8 = S.solve(Fg, tol=1e-8, maxit=400)
    assert i8[0]["status"] == "ok" and i8[0]["true_rel_res"] <= 1e-8 and i8[0]["outer"] >= 2
    # the first outer step's residual (predicted ~1e-3) is a provisional double-float one
    assert 1 <= i8[0]["outer_df"] < i8[0]["outer"]
    u12, i12 = S.solve(Fg, tol=1e-12, maxit=800)
    assert i12[0]["status"] == "ok" and i12[0]["true_rel_res"] <= 1e-12
    assert _rel(u12.cpu().numpy(), u64.cpu().numpy()) <= 1e-8
    assert i12[0]["outer_df"] < i12[0]["outer"]
    print(form, "refine: inner", i8[0]["iters"], "outer", i8[0]["outer"], "df", i8[0]["outer_df"],
          "| 1e-12:", i12[0]["iters"], i12[0]["outer"], i12[0]["outer_df"])


def test_refinement_batch_matches_direct_solve():
    from oracle.solve import direct_solve
    prob = STProblem(2, 3, 7)
    A = prob.assemble_A_kron()
    F = synth.uniform(prob.N, 77, batch=3)
    F[1] *= 1e-4
    S = _solver(2, 3, 7, precision="bf16", refine=True, batch=3)
    u, info = S.solve(torch.from_numpy(F).cuda(), tol=1e-12, maxit=500)
    u = u.cpu().numpy()
    for b in range(3):
        ref = direct_solve(A, F[b])
        assert info[b]["status"] == "ok"
        assert np.linalg.norm(u[b] - ref) / np.linalg.norm(ref) <= 1e-10


@pytest.mark.parametrize("form", ["bf16", "tf32"])
def test_contexts_of_different_sizes_coexist(form):
    """The tensor-core kernels' dynamic shared-memory limits are per kernel and
    per process: a small context created after a large one must leave the large
    one working, with the same result."""
    big = _solver(3, 3, 24, precision=form)
    r = _cuda_arr(synth.uniform(big.N, 21))
    z1 = big.apply_precond(r).cpu().numpy()
    small = _solver(2, 2, 3, precision=form)
    small.apply_precond(_cuda_arr(synth.uniform(small.N, 22)))
    z2 = big.apply_precond(r).cpu().numpy()
    assert np.array_equal(z1, z2)


def _cuda_arr(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()
