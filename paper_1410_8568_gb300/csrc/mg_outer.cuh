// mg_outer.cuh -- device helpers of the FP64 outer kernels (residual, norms,
// conjugate gradients), shared by mg_kernels.cu and mg_pcg.cu.
//
// Outer kernels walk a grid's finest level in row tiles (fine_tile: 8 rows of
// 64 cells per block, 2 cells per lane) with a grid-stride over tiles, and
// reduce in a fixed order (block_sum4), so every sum is deterministic.
#pragma once

#include "mg_device.cuh"

namespace gbmg {

// Tiles of a block's grid-stride sequence whose loads the streaming outer
// kernels k_sum and k_center_rhs issue together before using them (a sum's
// order is unchanged: the additions run after the loads, in sequence order).
constexpr int kUnroll = 4;

// Deterministic block sum of up to 4 doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum4(double v[4], double *out)
{
    __shared__ double sh[kThreads / 32][4];
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; q++) sh[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; q++) {
            double s = 0.0;
            for (int t = 0; t < kThreads / 32; t++) s += sh[t][q];
            out[q] = s;
        }
    }
}

// The grid's iterate lives in the three-float form: an extended-precision
// solve that took at least one refinement step.
__device__ __forceinline__ bool xp_live(const OuterView &O) { return O.xp && O.st->steps > 0; }

// Row-tile coordinates of this thread for a fine launch (2 cells per lane).
struct Tile {
    int row, j, k, xbase;
    bool ok;
};

// (dxt divides by fine_xtiles(n[0]), dy by n[1]: multiply-shift divisions; an
// integer division by a run-time divisor goes through float conversions, which
// this GPU issues to its narrow FP64 pipe)
__device__ __forceinline__ Tile fine_tile(const int n[3], int lb, const FastDiv &dxt, const FastDiv &dy)
{
    Tile t;
    const int rb = fdiv(lb, dxt), xt = lb - rb * fine_xtiles(n[0]);
    t.row = rb * kRowsPerBlock + (threadIdx.x >> 5);
    t.ok = t.row < n[1] * n[2];
    t.k = t.ok ? fdiv(t.row, dy) : 0;
    t.j = t.ok ? t.row - t.k * n[1] : 0;
    t.xbase = xt * kSeg;
    return t;
}

// Sum over the 6 faces of w_f (x_nb - x_c), FP64: the face difference is taken
// before the product, which keeps the residual accurate to rounding of the
// differences when x is smooth or carries a large constant.
__device__ __forceinline__ double flux64(const OuterView &O, const double *__restrict__ x, int i,
                                         int j, int k, long long c)
{
    const int nx = O.n[0], ny = O.n[1], nz = O.n[2], per = O.per;
    const double *__restrict__ wx = O.w[0];
    const double *__restrict__ wy = O.w[1];
    const double *__restrict__ wz = O.w[2];
    const long long sy = nx, sz = (long long)nx * ny;
    const double xc = x[c];
    double f = wx[c] * (x[i > 0 ? c - 1 : ((per & 1) ? c + (nx - 1) : c)] - xc);
    if (i + 1 < nx) f += wx[c + 1] * (x[c + 1] - xc);
    else if (per & 1) f += wx[c + 1 - nx] * (x[c + 1 - nx] - xc);
    f += wy[c] * (x[j > 0 ? c - sy : ((per & 2) ? c + sy * (ny - 1) : c)] - xc);
    if (j + 1 < ny) f += wy[c + sy] * (x[c + sy] - xc);
    else if (per & 2) f += wy[c - sy * (ny - 1)] * (x[c - sy * (ny - 1)] - xc);
    f += wz[c] * (x[k > 0 ? c - sz : ((per & 4) ? c + sz * (nz - 1) : c)] - xc);
    if (k + 1 < nz) f += wz[c + sz] * (x[c + sz] - xc);
    else if (per & 4) f += wz[c - sz * (nz - 1)] * (x[c - sz * (nz - 1)] - xc);
    return f;
}

}  // namespace gbmg
