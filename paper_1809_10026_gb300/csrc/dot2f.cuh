// Compensated FP32 inner-product accumulator shared by the CG kernels and the
// fused A x.
#pragma once

#include <cuda_runtime.h>

namespace stls {

// Inner products of FP32 vectors: compensated FP32 accumulation (TwoProd by
// FMA and TwoSum; the "Dot2" scheme of Ogita, Rump and Oishi, 2005), whose
// error is about eps_32 |x.y| + (n eps_32)^2 sum|x_i y_i| for the n terms of one
// thread, converted to FP64 once per thread.  On GB300 FP64 instructions
// issue at a small fraction of the FP32 rate, so converting and accumulating
// every term in FP64 would bound these kernels by the FP64 pipe.
struct Dot2f {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float h = __fmul_rn(a, b);
    const float l = __fmaf_rn(a, b, -h);  // a b = h + l exactly
    const float t = __fadd_rn(s, h);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(h, z));  // s + h = t + e exactly
    s = t;
    c = __fadd_rn(c, __fadd_rn(l, e));
  }
  __device__ __forceinline__ double value() const { return static_cast<double>(s) + static_cast<double>(c); }
};

}  // namespace stls
