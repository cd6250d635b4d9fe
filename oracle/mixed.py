"""Reduced-precision model of the preconditioner solve (Algorithm 1 with the
mixed-precision form's roundings).

Oracle (test infrastructure).  The mixed form runs the mode products of
Algorithm 1 (steps 2 and 4) with BF16 or TF32 operands and FP32
accumulation; intermediate tensors are stored in BF16 (BF16 form) or FP32
(TF32 form); the division of step 3 is done in FP32 with the FP64
eigenvalues rounded to FP32; the input r is FP64 and is rounded to FP32 and
then to the operand format; the output is the FP32 accumulator widened to FP64.

Order of the products.  Algorithm 1 applies Kronecker products of the 1D
eigenvector matrices, i.e. d+1 mode products that act on different tensor
directions and commute in exact arithmetic, so the algorithm fixes no order;
with a rounding after every product the order matters at the level of the
rounding error.  The forward products always run in the order 1, ..., d, t
(the division needs the time product last).  ``bwd_order="ascending"``
applies the backward products in the order 1, ..., d, t;
``bwd_order="descending"`` in the order t, d, ..., 1 (the fused tensor-core
kernels of the BF16 form for d = 2, 3 run this order).

This model applies the same roundings with numpy: every operand is rounded
where the method rounds it, and every product is accumulated in FP64 and then
rounded to FP32.  It differs from any FP32 tensor-core accumulation only by
the accumulation order, i.e. by about one FP32 ulp per product before the
next rounding.  Pinned by tests/test_oracle_mixed.py: with identity rounding it
equals oracle.fd.FD.apply, and the rounding functions agree with numpy's own
float32 rounding and with hand-checked bit patterns.
"""
import numpy as np


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


def round_tf32(x):
    """Round to TF32 (10 explicit mantissa bits, ties away from zero), as float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32)


def apply_mixed(fd, r, form, bwd_order="ascending"):
    """z ~ P^{-1} r with the roundings of the mixed form ("bf16" or "tf32")."""
    prob = fd.prob
    d = prob.d
    if form == "fp64":   # no rounding at all: Algorithm 1 in FP64
        ident = lambda v: np.asarray(v, dtype=np.float64)
        q_op = q_store = f32 = ident
    else:
        q_op = round_bf16 if form == "bf16" else round_tf32
        f32 = lambda v: np.asarray(v, dtype=np.float32)
        q_store = round_bf16 if form == "bf16" else f32
    X = f32(np.asarray(r, dtype=np.float64)).reshape(prob.shape)
    modes_fwd = [(k + 1, fd.U[k].T) for k in range(d)] + [(d + 1, fd.U_t.T)]
    modes_bwd = [(k + 1, fd.U[k]) for k in range(d)] + [(d + 1, fd.U_t)]
    lam_t = f32(fd.lam_t)
    lam_s = [f32(l) for l in fd.lam]
    if bwd_order == "descending":
        modes_bwd = modes_bwd[::-1]
    elif bwd_order != "ascending":
        raise ValueError("bwd_order must be 'ascending' or 'descending'")
    steps = [(k, W, False) for k, W in modes_fwd] + [(k, W, True) for k, W in modes_bwd]
    for idx, (k, W, bwd) in enumerate(steps):
        Wq = q_op(W).astype(np.float64)
        Xq = q_op(X).astype(np.float64)
        Y = f32(prob.mode_product(Xq, Wq, k))
        if not bwd and k == d + 1:
            # eigenvalue sum in the order lambda_t + (sum of spatial lambdas)
            ls = f32(np.zeros(prob.shape[1:]))
            for kk in range(d):
                shape = [1] * d
                shape[d - 1 - kk] = -1
                ls = f32(ls + lam_s[kk].reshape(shape))
            E = f32(lam_t.reshape((-1,) + (1,) * d) + ls[None])
            Y = f32(Y / E)
        X = Y if idx == len(steps) - 1 else q_store(Y)
    return X.astype(np.float64).reshape(-1)
