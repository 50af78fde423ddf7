// mg_gmres.cu -- restarted GMRES on the coarsest grid (Sec. 2.3 item 6 of
// arXiv 1410.8568: the error on the coarsest grid is solved by GMRES).
//
// Used for coarsest grids above the dense inverse's kMaxCoarse cells (sizes
// with a large odd factor) or on request.  One block of 1024 threads per grid
// solves A e = b - mean(b) in FP64 (the coarsest solve stays FP64 in every
// precision): Arnoldi with modified Gram-Schmidt, Givens rotations on the
// Hessenberg matrix (shared memory), the least-squares update at the end of
// each cycle of kGmresM steps or on convergence (Saad & Schultz 1986).  Stops
// when the recurrence's residual estimate is below gm_tol ||b - mean b|| or
// after gm_max Arnoldi steps; e is returned with zero mean.  Every dot product
// is a fixed-order block reduction, so the result is deterministic.
#include "mg_kernels.h"
#include "mg_stencil.cuh"

#include <math.h>

namespace gbmg {

namespace {

constexpr int kGmresThreads = 1024;

// Sum over the block of one double per thread, fixed order; every thread gets it.
__device__ __forceinline__ double block_all_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // red[] may still be read by the previous call
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += red[q];
    return s;
}

// (A x)_c on the coarsest grid, FP64, face differences first
__device__ __forceinline__ double apply_at(const CoarseView &C, const double *__restrict__ x, int c)
{
    const int nx = C.n[0], ny = C.n[1], nz = C.n[2], per = C.per;
    const int rest = c / nx;
    const int i = c - rest * nx, j = rest % ny, k = rest / ny;
    const int sy = nx, sz = nx * ny;
    const double *wx = C.w[0], *wy = C.w[1], *wz = C.w[2];
    const double xc = x[c];
    double f = 0.0;
    if (i > 0) f += wx[c] * (x[c - 1] - xc);
    else if (per & 1) f += wx[c] * (x[c + nx - 1] - xc);
    if (i + 1 < nx) f += wx[c + 1] * (x[c + 1] - xc);
    else if (per & 1) f += wx[c + 1 - nx] * (x[c + 1 - nx] - xc);
    if (j > 0) f += wy[c] * (x[c - sy] - xc);
    else if (per & 2) f += wy[c] * (x[c + sy * (ny - 1)] - xc);
    if (j + 1 < ny) f += wy[c + sy] * (x[c + sy] - xc);
    else if (per & 2) f += wy[c - sy * (ny - 1)] * (x[c - sy * (ny - 1)] - xc);
    if (k > 0) f += wz[c] * (x[c - sz] - xc);
    else if (per & 4) f += wz[c] * (x[c + sz * (nz - 1)] - xc);
    if (k + 1 < nz) f += wz[c + sz] * (x[c + sz] - xc);
    else if (per & 4) f += wz[c - sz * (nz - 1)] * (x[c - sz * (nz - 1)] - xc);
    return f;
}

}  // namespace

template <class T>
__global__ void __launch_bounds__(kGmresThreads) k_coarse_gmres(const CoarseView *__restrict__ cv, int cyc,
                                                                const OuterView *__restrict__ ov)
{
    dep_entry();
    const CoarseView &C = cv[blockIdx.x];
    if (!C.gmres || !in_cycle(C.st, cyc)) return;
    __shared__ double H[(kGmresM + 1) * kGmresM];
    __shared__ double cs[kGmresM], sn[kGmresM], g[kGmresM + 1], y[kGmresM];
    __shared__ double red[32];
    __shared__ int stop;
    const int n = C.nc, m = kGmresM, tid = threadIdx.x, nt = blockDim.x;
    double *b = C.gm, *e = b + n, *w = e + n, *V = w + n;
    const T *bt = (const T *)C.b;

    double s = 0.0;
    for (int c = tid; c < n; c += nt) s += (double)bt[c];
    const double mean = block_all_sum(s, red) / n;
    s = 0.0;
    for (int c = tid; c < n; c += nt) {
        const double v = (double)bt[c] - mean;
        b[c] = v;
        e[c] = 0.0;
        s += v * v;
    }
    const double bnorm = sqrt(block_all_sum(s, red));
    int it = 0;
    while (bnorm > 0.0 && it < C.gm_max) {
        __syncthreads();  // e complete
        s = 0.0;
        for (int c = tid; c < n; c += nt) {
            const double r = b[c] - apply_at(C, e, c);
            w[c] = r;
            s += r * r;
        }
        const double beta = sqrt(block_all_sum(s, red));
        if (!(beta > C.gm_tol * bnorm)) break;  // converged (or NaN: stop)
        for (int c = tid; c < n; c += nt) V[c] = w[c] / beta;
        if (tid == 0) {
            g[0] = beta;
            for (int i = 1; i <= m; i++) g[i] = 0.0;
            stop = 0;
        }
        int j = 0;
        while (j < m && it < C.gm_max) {
            const double *vj = V + (size_t)j * n;
            double *vn = V + (size_t)(j + 1) * n;
            __syncthreads();  // v_j complete
            for (int c = tid; c < n; c += nt) w[c] = apply_at(C, vj, c);
            for (int i = 0; i <= j; i++) {
                const double *vi = V + (size_t)i * n;
                __syncthreads();  // w complete
                s = 0.0;
                for (int c = tid; c < n; c += nt) s += w[c] * vi[c];
                const double h = block_all_sum(s, red);
                if (tid == 0) H[i * m + j] = h;
                for (int c = tid; c < n; c += nt) w[c] -= h * vi[c];
            }
            __syncthreads();
            s = 0.0;
            for (int c = tid; c < n; c += nt) s += w[c] * w[c];
            const double hn = sqrt(block_all_sum(s, red));
            for (int c = tid; c < n; c += nt) vn[c] = hn > 0.0 ? w[c] / hn : 0.0;
            if (tid == 0) {
                H[(j + 1) * m + j] = hn;
                for (int i = 0; i < j; i++) {
                    const double a = H[i * m + j], bb = H[(i + 1) * m + j];
                    H[i * m + j] = cs[i] * a + sn[i] * bb;
                    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
                }
                const double a = H[j * m + j], bb = H[(j + 1) * m + j];
                const double den = sqrt(a * a + bb * bb);
                cs[j] = den > 0.0 ? a / den : 1.0;
                sn[j] = den > 0.0 ? bb / den : 0.0;
                H[j * m + j] = den;
                H[(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                stop = (fabs(g[j + 1]) <= C.gm_tol * bnorm || hn == 0.0) ? 1 : 0;
            }
            __syncthreads();
            j++;
            it++;
            if (stop) break;
        }
        // y = H(0:j, 0:j)^-1 g, e += V y
        if (tid == 0) {
            for (int i = j - 1; i >= 0; i--) {
                double r = g[i];
                for (int k = i + 1; k < j; k++) r -= H[i * m + k] * y[k];
                y[i] = H[i * m + i] != 0.0 ? r / H[i * m + i] : 0.0;
            }
        }
        __syncthreads();
        for (int c = tid; c < n; c += nt) {
            double v = e[c];
            for (int i = 0; i < j; i++) v += y[i] * V[(size_t)i * n + c];
            e[c] = v;
        }
        if (stop) break;
    }
    __syncthreads();
    s = 0.0;
    for (int c = tid; c < n; c += nt) s += e[c];
    const double em = block_all_sum(s, red) / n;
    T *x = (T *)C.x;
    // single-level grid: the last cycle of a refinement step also updates p
    const bool out = ov != nullptr && C.outer && last_cycle(C.st, cyc);
    const OuterOut po = out ? outer_out(ov[C.g]) : OuterOut{};
    for (int c = tid; c < n; c += nt) {
        const T xn = (T)(e[c] - em);
        x[c] = xn;
        if (out) add_outer<T>(po, c, xn);
    }
}

template <class T>
void launch_coarse_gmres(const CoarseView *cv, int count, int cyc, const OuterView *ov, cudaStream_t s)
{
    launch_k(k_coarse_gmres<T>, count, kGmresThreads, 0, s, cv, cyc, ov);
}

template void launch_coarse_gmres<float>(const CoarseView *, int, int, const OuterView *, cudaStream_t);
template void launch_coarse_gmres<double>(const CoarseView *, int, int, const OuterView *, cudaStream_t);

}  // namespace gbmg
