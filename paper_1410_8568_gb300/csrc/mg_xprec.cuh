// mg_xprec.cuh -- extended precision from FP32 arithmetic for the outer
// iteration of the mixed-precision multigrid iteration (Sec. 2.3 of arXiv
// 1410.8568: the residual of the refinement step and the update p += e).
//
// On this GPU FP64 instructions issue at a small fraction of the FP32 rate,
// and the outer residual in FP64 was bound by the FP64 pipe.  Here the iterate
// is an unevaluated sum of three floats p = p0 + p1 + p2 (|p1| <= ulp(p0)/2,
// |p2| <= ulp(p1)/2: 72 significant bits, more than a double's 53), the
// level-0 faces and the right-hand side are float pairs (48 bits), and the
// residual b - A p is evaluated with error-free transformations in FP32:
//   two_sum: s + e = a + b exactly (Knuth, TAOCP vol. 2, 1969);
//   two_prod: p + e = a * b exactly, from one fused multiply-add
//     (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26, 2005).
// Every operation uses the explicitly rounded intrinsics, so the compiler can
// neither contract nor reassociate them.
//
// The face differences p_nb - p_c are formed exactly from the leading two
// components (as in the FP64 kernel, where the difference is taken before the
// product), so the residual keeps its accuracy when p carries a large
// constant or varies slowly.  Error: about 2^-48 of the sum of |w (p_nb - p_c)|
// and |b| per cell, against 2^-53 for FP64 arithmetic.
#pragma once

namespace gbmg {

__device__ __forceinline__ float two_sum(float a, float b, float &err)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ float two_diff(float a, float b, float &err) { return two_sum(a, -b, err); }

// Add an FP32 correction e to the triple (p0, p1, p2) and renormalise.  The
// sum is exact up to the rounding of the lowest component (2^-72 |p|).
__device__ __forceinline__ void triple_add(float &p0, float &p1, float &p2, float e)
{
    float t0, t1, r, q;
    const float s0 = two_sum(p0, e, t0);
    const float s1 = two_sum(p1, t0, t1);
    const float s2 = __fadd_rn(p2, t1);
    p0 = two_sum(s0, s1, r);
    p1 = two_sum(r, s2, q);
    p2 = q;
}

// (a0 + a1 + a2) - (b0 + b1 + b2) as a float pair (h, l): the differences of
// the leading two components are exact, the third is tiny.
__device__ __forceinline__ float triple_diff(float a0, float a1, float a2, float b0, float b1, float b2,
                                             float &l)
{
    float e0, e1, t;
    const float d0 = two_diff(a0, b0, e0);
    const float d1 = two_diff(a1, b1, e1);
    const float lo = __fadd_rn(__fadd_rn(e0, e1), __fsub_rn(a2, b2));
    const float h = two_sum(d0, d1, t);
    l = __fadd_rn(t, lo);
    return h;
}

// (F0, F1) += (h + l) * (w0 + w1), products exact to the dropped l * w1 term
__device__ __forceinline__ void pair_fma_acc(float &F0, float &F1, float h, float l, float w0, float w1)
{
    const float ph = __fmul_rn(h, w0);
    float pl = __fmaf_rn(h, w0, -ph);
    pl = __fmaf_rn(h, w1, pl);
    pl = __fmaf_rn(l, w0, pl);
    float t;
    F0 = two_sum(F0, ph, t);
    F1 = __fadd_rn(F1, __fadd_rn(t, pl));
}

}  // namespace gbmg
