"""GPU parity of the FP32 A x, the operator of the refinement form's inner
flexible CG, through the C ABI (stls_apply_A_f32), against the oracle's FP64
Kronecker product (Eq. A_kron).

Every stage of the fused product (directions 1 and 2, direction 3, time) is
a fixed-order chain of FP32 fused multiply-adds over at most 3(2p+1) band
terms, and its output is rounded once.  With B = (sum of the absolute
Kronecker terms the product evaluates) |x|, the standard bound for such
chains gives |y - A x| <= (7 + 21 + 21 + 15 + 4) u B ~ 2^6.1 u B for p = 3
(u = 2^-24); the test bound is 2^-17 B = 2^7 u B.  A wrong band coefficient,
a dropped term or a misplaced halo row errs by O(B).

The cases cover the fused direction-3 and time kernel (n3 >= 8 and equal
space and time degrees <= 4): ragged column blocks (n1 n2 not a multiple of
32), n3 split into several row groups, time meshes shorter than a band, a
batch; and the two-pass path it falls back to (n3 < 8, p_t != p_s, p > 4).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.system import STProblem
from paper_1809_10026_gb300 import synth

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -17


def _solver(*a, **k):
    import paper_1809_10026_gb300 as stls
    return stls.Solver(*a, **k)


def abs_apply(prob, x):
    """B = (|K_t| x |M_s| + |M_t| x (sum_k |J_k| + 2 sum_{k<l} |K_k| |K_l|)
    + |W_t| x sum_k |K_k|) |x|, M in the other directions, by mode products."""
    X = np.abs(x).reshape(prob.shape)
    d, tm, sd = prob.d, prob.time, prob.space
    aM = [np.abs(s.M) for s in sd]
    aK = [np.abs(s.K) for s in sd]
    aJ = [np.abs(s.J) for s in sd]

    def spatial(mats):
        Z = X
        for k in range(d):
            Z = prob.mode_product(Z, mats[k], k + 1)
        return Z

    Y = prob.mode_product(spatial(aM), np.abs(tm.K), d + 1)
    Js = 0
    Ls = 0
    for k in range(d):
        m = list(aM)
        m[k] = aJ[k]
        Js = Js + spatial(m)
        m = list(aM)
        m[k] = aK[k]
        Ls = Ls + spatial(m)
        for l in range(k + 1, d):
            m = list(aM)
            m[k] = aK[k]
            m[l] = aK[l]
            Js = Js + 2 * spatial(m)
    Y = Y + prob.mode_product(Js, np.abs(tm.M), d + 1) + prob.mode_product(Ls, np.abs(tm.W), d + 1)
    return Y.reshape(-1)


CASES = [
    dict(d=3, p=2, n_el=8),                                   # n3 = 8: one row group of 8
    dict(d=3, p=2, n_el=[5, 7, 10]),                          # n3 = 10, n1 n2 = 35
    dict(d=3, p=3, n_el=13),                                  # n3 = 14, n1 n2 = 196 (ragged)
    dict(d=3, p=3, n_el=[6, 5, 30], T=0.7),                   # n3 = 31: two groups of 16 and 15
    dict(d=3, p=4, n_el=[9, 4, 20], T=1.2),                   # n3 = 22: two groups of 11
    dict(d=3, p=3, n_el=[7, 6, 12], n_el_t=2),                # n_t = 4 < 2p + 1
    dict(d=3, p=2, n_el=[3, 4, 40], n_el_t=1),                # n_t = 2, n3 = 41: three groups
    dict(d=3, p=3, n_el=[4, 3, 5]),                           # n3 = 6: two passes
    dict(d=3, p=3, n_el=[6, 5, 12], p_t=2, n_el_t=7),         # p_t != p_s: two passes
    dict(d=3, p=5, n_el=[3, 2, 6]),                           # p = 5: two passes
    dict(d=2, p=3, n_el=[11, 9]),                             # two spatial directions
]


def _id(c):
    return "-".join(f"{k}{v}" for k, v in c.items())


@pytest.mark.parametrize("batch", [1, 3])
@pytest.mark.parametrize("case", CASES, ids=_id)
def test_apply_A_f32_matches_oracle(case, batch):
    kw = {k: case[k] for k in ("T", "p_t", "n_el_t") if k in case}
    prob = STProblem(case["d"], case["p"], case["n_el"], **kw)
    S = _solver(case["d"], case["p"], case["n_el"], precision="tf32", refine=True, batch=batch, **kw)
    x = synth.uniform(prob.N, 61, batch=batch).reshape(batch, prob.N).astype(np.float32)
    if batch > 1:
        x[1] *= np.float32(2.0 ** 20)  # a second magnitude
        x[2] *= np.float32(2.0 ** -30)
    xg = torch.from_numpy(x.reshape(-1) if batch == 1 else x).cuda()
    y = S.apply_A_f32(xg).cpu().numpy().reshape(batch, prob.N).astype(np.float64)
    worst = 0.0
    for b in range(batch):
        xb = x[b].astype(np.float64)
        ref = prob.apply_A_kron(xb)
        B = abs_apply(prob, xb)
        err = np.abs(y[b] - ref)
        worst = max(worst, float(np.max(err / B)))
        assert np.all(err <= BOUND * B), (b, float(np.max(err / B)))
    print("%s batch %d: max |y - Ax| / B = 2^%.1f" % (_id(case), batch, np.log2(max(worst, 1e-300))))


def test_apply_A_f32_zero_and_linearity():
    """A 0 = 0 exactly, and scaling x by a power of two scales y exactly."""
    S = _solver(3, 3, 13, precision="tf32", refine=True)
    z = S.apply_A_f32(torch.zeros(S.N, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert not np.any(z)
    x = torch.from_numpy(synth.uniform(S.N, 5).astype(np.float32)).cuda()
    y1 = S.apply_A_f32(x).cpu().numpy()
    y2 = S.apply_A_f32(x * 8.0).cpu().numpy()
    assert np.array_equal(y2, y1 * 8.0)


def test_apply_A_f32_rejects_non_refinement_context():
    S = _solver(3, 2, 4)
    with pytest.raises(RuntimeError, match="apply_A_f32"):
        S.apply_A_f32(torch.zeros(S.N, dtype=torch.float32, device="cuda"))


def test_apply_A_f32_cube3d_p3_n64():
    """The benchmark's mesh (18,125,250 unknowns): every entry within the bound."""
    prob = STProblem(3, 3, 64)
    S = _solver(3, 3, 64, precision="tf32", refine=True)
    x = synth.uniform(prob.N, 4).astype(np.float32)
    y = S.apply_A_f32(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    xb = x.astype(np.float64)
    err = np.abs(y - prob.apply_A_kron(xb))
    B = abs_apply(prob, xb)
    ratio = float(np.max(err / B))
    print("cube3d_p3_n64: max |y - Ax| / B = 2^%.1f" % np.log2(ratio))
    assert ratio <= BOUND
