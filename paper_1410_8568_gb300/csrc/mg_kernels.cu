// mg_kernels.cu -- CUDA kernels of the variable-density pressure multigrid.
//
// Shin, Chergui & Juric, arXiv 1410.8568, Sec. 2.3.  The kernels implement
//   (1) the cell-centred operator of Eq. 10 (divided by h^2), on every level;
//   (2) the harmonic face coefficient of Eqs. 11-12 (density -> faces);
//   (3) restriction of the residual (mean of the 8 fine children);
//   (4) prolongation of the coarse error (trilinear, 27/9/3/1 over 64);
//   (5) red-black SOR relaxation;
//   (6) the exact solve on the coarsest grid (dense inverse, FP64);
// plus the FP64 outer iteration (residual, correction update, norms of the
// stopping test and of Eq. 15) and the coarse-face coefficients (mean of the
// 4 fine faces that tile a coarse face).
//
// All cell kernels are bandwidth kernels: a warp owns a contiguous x segment
// of one grid row so every load and store is coalesced; neighbours in y and z
// come through L1/L2.  Reductions are deterministic: fixed per-thread order,
// fixed shuffle tree, per-block partials summed by one block in fixed order.
#include "mg_kernels.h"

#include <math.h>

namespace gbmg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_entry(const int *__restrict__ start, int count)
{
    if (count == 1) return 0;
    const int blk = blockIdx.x;
    int lo = 0, hi = count;  // start[lo] <= blk < start[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= blk) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Neighbour offsets of cell (i,j,k) with the boundary rules of the layout:
// low face of a cell is stored at the cell; at a Neumann low wall the stored
// coefficient is 0 and the neighbour index falls back to the cell itself; at a
// Neumann high wall the face is absent (coefficient 0).
template <class T, class Load>
__device__ __forceinline__ void stencil(const T *__restrict__ wx, const T *__restrict__ wy,
                                        const T *__restrict__ wz, const Load &ld, int nx, int ny,
                                        int nz, int per, int i, int j, int k, long long c, T xc,
                                        T &diag, T &flux)
{
    const long long sy = nx;
    const long long sz = (long long)nx * ny;
    T a, d, f;
    // x low / high
    a = wx[c];
    d = a;
    f = a * (ld(i > 0 ? c - 1 : ((per & 1) ? c + (nx - 1) : c)) - xc);
    if (i + 1 < nx) {
        a = wx[c + 1];
        d += a;
        f += a * (ld(c + 1) - xc);
    } else if (per & 1) {
        a = wx[c + 1 - nx];
        d += a;
        f += a * (ld(c + 1 - nx) - xc);
    }
    // y low / high
    a = wy[c];
    d += a;
    f += a * (ld(j > 0 ? c - sy : ((per & 2) ? c + sy * (ny - 1) : c)) - xc);
    if (j + 1 < ny) {
        a = wy[c + sy];
        d += a;
        f += a * (ld(c + sy) - xc);
    } else if (per & 2) {
        a = wy[c - sy * (ny - 1)];
        d += a;
        f += a * (ld(c - sy * (ny - 1)) - xc);
    }
    // z low / high
    a = wz[c];
    d += a;
    f += a * (ld(k > 0 ? c - sz : ((per & 4) ? c + sz * (nz - 1) : c)) - xc);
    if (k + 1 < nz) {
        a = wz[c + sz];
        d += a;
        f += a * (ld(c + sz) - xc);
    } else if (per & 4) {
        a = wz[c - sz * (nz - 1)];
        d += a;
        f += a * (ld(c - sz * (nz - 1)) - xc);
    }
    diag = d;
    flux = f;
}

// Sum of the coefficients of the faces of cell c (the diagonal of -A).
template <class T>
__device__ __forceinline__ T diag_of(const T *__restrict__ wx, const T *__restrict__ wy,
                                     const T *__restrict__ wz, int nx, int ny, int nz, int per,
                                     int i, int j, int k, long long c)
{
    const long long sy = nx;
    const long long sz = (long long)nx * ny;
    T d = wx[c];
    if (i + 1 < nx) d += wx[c + 1];
    else if (per & 1) d += wx[c + 1 - nx];
    d += wy[c];
    if (j + 1 < ny) d += wy[c + sy];
    else if (per & 2) d += wy[c - sy * (ny - 1)];
    d += wz[c];
    if (k + 1 < nz) d += wz[c + sz];
    else if (per & 4) d += wz[c - sz * (nz - 1)];
    return d;
}

template <class T>
struct LoadPlain {
    const T *x;
    __device__ __forceinline__ T operator()(long long q) const { return x[q]; }
};

template <class Te>
struct LoadSum {  // FP64 iterate plus the V-cycle correction
    const double *x;
    const Te *e;
    __device__ __forceinline__ double operator()(long long q) const { return x[q] + (double)e[q]; }
};

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

// Row-tile coordinates of this thread for a fine launch (2 cells per lane).
struct Tile {
    int row, j, k, xbase;
    bool ok;
};

__device__ __forceinline__ Tile fine_tile(const int n[3], int lb)
{
    Tile t;
    const int xt_n = fine_xtiles(n[0]);
    const int xt = lb % xt_n, rb = lb / xt_n;
    t.row = rb * kRowsPerBlock + (threadIdx.x >> 5);
    t.ok = t.row < n[1] * n[2];
    t.j = t.ok ? t.row % n[1] : 0;
    t.k = t.ok ? t.row / n[1] : 0;
    t.xbase = xt * kSeg;
    return t;
}

// ---------------------------------------------------------------------------
// (5) red-black relaxation: one half-sweep over the cells of one colour
// ---------------------------------------------------------------------------

// zero_guess: x is taken as 0 on entry (first pre-smoothing half-sweep of a
// level): the relaxed colour gets omega * (-b / diag), the other colour 0, so
// no separate clearing pass is needed.
template <class T>
__global__ void __launch_bounds__(kThreads) k_smooth(const LevelView *__restrict__ lv,
                                                     const int *__restrict__ start, int count,
                                                     int colour, T omega, int zero_guess)
{
    const int e = find_entry(start, count);
    const LevelView L = lv[e];
    if (!L.st->active) return;
    const Tile t = fine_tile(L.n, blockIdx.x - start[e]);
    if (!t.ok) return;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int i0 = t.xbase + ((threadIdx.x & 31) << 1);
    if (i0 >= nx) return;
    const int par = (colour + t.j + t.k) & 1;
    const int i = i0 + par;
    T *x = (T *)L.x;
    const T *b = (const T *)L.b;
    const T *wx = (const T *)L.w[0], *wy = (const T *)L.w[1], *wz = (const T *)L.w[2];
    const long long rowoff = (long long)nx * t.row;
    if (i < nx) {
        const long long c = rowoff + i;
        if (zero_guess) {
            const T d = diag_of(wx, wy, wz, nx, ny, nz, L.per, i, t.j, t.k, c);
            x[c] = d > T(0) ? omega * (-b[c] / d) : T(0);
        } else {
            const T xc = x[c];
            T d, f;
            stencil(wx, wy, wz, LoadPlain<T>{x}, nx, ny, nz, L.per, i, t.j, t.k, c, xc, d, f);
            if (d > T(0)) x[c] = xc + omega * ((f - b[c]) / d);
        }
    }
    if (zero_guess) {
        const int io = i0 + 1 - par;
        if (io < nx) x[rowoff + io] = T(0);
    }
}

// ---------------------------------------------------------------------------
// (3) residual and restriction: coarse b = mean of (b - A x) over 8 children
// ---------------------------------------------------------------------------

template <class T>
__global__ void __launch_bounds__(kThreads) k_restrict(const LevelView *__restrict__ lv,
                                                       const int *__restrict__ start, int count)
{
    const int e = find_entry(start, count);
    const LevelView L = lv[e];
    if (!L.st->active) return;
    const int ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2];
    const int lb = blockIdx.x - start[e];
    const int xt_n = coarse_xtiles(ncx);
    const int xt = lb % xt_n, rb = lb / xt_n;
    const int crow = rb * kRowsPerBlock + (threadIdx.x >> 5);
    if (crow >= ncy * ncz) return;
    const int I = xt * kCSeg + (threadIdx.x & 31);
    if (I >= ncx) return;
    const int J = crow % ncy, K = crow / ncy;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const T *x = (const T *)L.x;
    const T *b = (const T *)L.b;
    const T *wx = (const T *)L.w[0], *wy = (const T *)L.w[1], *wz = (const T *)L.w[2];
    T s = T(0);
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
                const long long c = i + (long long)nx * (j + (long long)ny * k);
                T d, f;
                stencil(wx, wy, wz, LoadPlain<T>{x}, nx, ny, nz, L.per, i, j, k, c, x[c], d, f);
                s += b[c] - f;
            }
    ((T *)L.bc)[I + (long long)ncx * crow] = s * T(0.125);
}

// ---------------------------------------------------------------------------
// (4) prolongation and correction: x += trilinear(e_coarse)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int partner(int i, int nc, int periodic)
{
    const int I = i >> 1;
    int J = (i & 1) ? I + 1 : I - 1;
    if (J < 0 || J >= nc) J = periodic ? (J + nc) % nc : I;  // wrap, or mirror at a wall
    return J;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_prolong(const LevelView *__restrict__ lv,
                                                      const int *__restrict__ start, int count)
{
    const int e = find_entry(start, count);
    const LevelView L = lv[e];
    if (!L.st->active) return;
    const Tile t = fine_tile(L.n, blockIdx.x - start[e]);
    if (!t.ok) return;
    const int nx = L.n[0];
    const int ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2];
    const T *ec = (const T *)L.xc;
    T *x = (T *)L.x;
    const int J0 = t.j >> 1, J1 = partner(t.j, ncy, L.per & 2);
    const int K0 = t.k >> 1, K1 = partner(t.k, ncz, L.per & 4);
    const long long r00 = (long long)ncx * (J0 + (long long)ncy * K0);
    const long long r10 = (long long)ncx * (J1 + (long long)ncy * K0);
    const long long r01 = (long long)ncx * (J0 + (long long)ncy * K1);
    const long long r11 = (long long)ncx * (J1 + (long long)ncy * K1);
    const T w0 = T(0.75), w1 = T(0.25);
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
        if (i >= nx) continue;
        const int I0 = i >> 1, I1 = partner(i, ncx, L.per & 1);
        // order: z outer, y, x inner; weight product (wx * wy) * wz
        T s = T(0);
        s += w0 * w0 * w0 * ec[r00 + I0];
        s += w1 * w0 * w0 * ec[r00 + I1];
        s += w0 * w1 * w0 * ec[r10 + I0];
        s += w1 * w1 * w0 * ec[r10 + I1];
        s += w0 * w0 * w1 * ec[r01 + I0];
        s += w1 * w0 * w1 * ec[r01 + I1];
        s += w0 * w1 * w1 * ec[r11 + I0];
        s += w1 * w1 * w1 * ec[r11 + I1];
        x[(long long)nx * t.row + i] += s;
    }
}

// ---------------------------------------------------------------------------
// y = A x on one level (unit checks)
// ---------------------------------------------------------------------------

template <class T>
__global__ void __launch_bounds__(kThreads) k_apply(const LevelView *__restrict__ lv,
                                                    const int *__restrict__ start, int count)
{
    const int e = find_entry(start, count);
    const LevelView L = lv[e];
    const Tile t = fine_tile(L.n, blockIdx.x - start[e]);
    if (!t.ok) return;
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const T *x = (const T *)L.x;
    T *y = (T *)L.b;
    const T *wx = (const T *)L.w[0], *wy = (const T *)L.w[1], *wz = (const T *)L.w[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
        if (i >= nx) continue;
        const long long c = (long long)nx * t.row + i;
        T d, f;
        stencil(wx, wy, wz, LoadPlain<T>{x}, nx, ny, nz, L.per, i, t.j, t.k, c, x[c], d, f);
        y[c] = f;
    }
}

// ---------------------------------------------------------------------------
// (6) coarsest grid: exact solve e = -G b with G = (-A + c 1 1^T)^{-1}
// ---------------------------------------------------------------------------

// For sum(b) = 0 this is the zero-mean solution of A e = b; for sum(b) != 0 it
// solves A e = b - mean(b) and adds a constant, which the cycle ignores
// (A 1 = 0) and the final mean removal takes out.
template <class T>
__global__ void __launch_bounds__(kThreads) k_coarse_solve(const CoarseView *__restrict__ cv)
{
    const CoarseView &C = cv[blockIdx.x];
    if (!C.st->active) return;
    __shared__ double rb[kMaxCoarse];
    const int n = C.nc;
    const T *b = (const T *)C.b;
    for (int t = threadIdx.x; t < n; t += blockDim.x) rb[t] = (double)b[t];
    __syncthreads();
    T *x = (T *)C.x;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double s = 0.0;
        for (int u = 0; u < n; u++) s += C.G[(long long)u * n + t] * rb[u];
        x[t] = (T)(-s);
    }
}

// Assemble S = -A + c 1 1^T of the coarsest level (c = mean diagonal / n, so the
// constant vector becomes an eigenvector with a mid-spectrum eigenvalue) and
// invert it in place by Gauss-Jordan elimination.  S is symmetric positive
// definite, so no pivoting is needed; a non-positive pivot means the grid is
// cut into pieces by zero coefficients and raises *err.
__global__ void __launch_bounds__(1024) k_coarse_setup(const CoarseView *__restrict__ cv)
{
    const CoarseView &C = cv[blockIdx.x];
    const int n = C.nc;
    const int nx = C.n[0], ny = C.n[1], nz = C.n[2];
    double *S = C.G;
    __shared__ double col[kMaxCoarse];
    __shared__ double red[32];
    __shared__ double c0;
    __shared__ int bad;
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) S[q] = 0.0;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double dsum = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
        const int q[3] = {i, j, k};
        const int nn[3] = {nx, ny, nz};
        const long long stride[3] = {1, nx, (long long)nx * ny};
        double diag = 0.0;
        for (int d = 0; d < 3; d++) {
            // low face
            if (q[d] > 0 || (C.per >> d & 1)) {
                const double a = C.w[d][c];
                const long long nb = q[d] > 0 ? c - stride[d] : c + stride[d] * (nn[d] - 1);
                if (nb != c) {
                    diag += a;
                    S[(long long)c * n + nb] -= a;
                }
            }
            // high face
            if (q[d] + 1 < nn[d] || (C.per >> d & 1)) {
                const long long fc = q[d] + 1 < nn[d] ? c + stride[d] : c - stride[d] * (nn[d] - 1);
                const double a = C.w[d][fc];
                if (fc != c) {
                    diag += a;
                    S[(long long)c * n + fc] -= a;
                }
            }
        }
        S[(long long)c * n + c] += diag;
        dsum += diag;
    }
    // deterministic block sum of the diagonal
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        c0 = s / n / n;
    }
    __syncthreads();
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) S[q] += c0;
    __syncthreads();
    const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 0; k < n; k++) {
        for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = S[(long long)r * n + k];
        __syncthreads();
        const double piv = col[k];
        if (!(piv > 0.0)) {
            if (threadIdx.x == 0) bad = 1;
            __syncthreads();
            break;
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            S[(long long)k * n + j] = (j == k ? 1.0 : S[(long long)k * n + j]) / piv;
        __syncthreads();
        for (int r = wid; r < n; r += warps) {
            if (r == k) continue;
            const double f = col[r];
            double *Sr = S + (long long)r * n;
            const double *Sk = S + (long long)k * n;
            for (int j = lane; j < n; j += 32) Sr[j] = (j == k ? 0.0 : Sr[j]) - f * Sk[j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) *C.err = 1;
}

// ---------------------------------------------------------------------------
// coefficients: density -> faces (2), caller faces -> scaled level-0 faces,
// and coarse faces
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) k_faces_from_density(FaceArgs a)
{
    const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % a.n[0]);
        const long long rest = c / a.n[0];
        const int j = (int)(rest % a.n[1]);
        const int k = (int)(rest / a.n[1]);
        const int q[3] = {i, j, k};
        const long long stride[3] = {1, a.n[0], (long long)a.n[0] * a.n[1]};
        const double rho_c = a.rho[c];
        bool ok = rho_c > 0.0 && isfinite(rho_c);
        for (int d = 0; d < 3; d++) {
            double v;
            if (q[d] == 0 && !(a.per >> d & 1)) {
                v = 0.0;  // Neumann wall
            } else {
                const long long l = q[d] > 0 ? c - stride[d] : c + stride[d] * (a.n[d] - 1);
                const double rho_l = a.rho[l];
                // Eqs. 11-12 with alpha = 1/rho: 2 a_l a_c / (a_l + a_c) = 2 / (rho_l + rho_c)
                v = a.mode == 0 ? 2.0 / (rho_l + rho_c) : 0.5 * (1.0 / rho_l + 1.0 / rho_c);
            }
            v *= a.scale[d];
            if (a.out64[d]) a.out64[d][c] = v;
            if (a.out32[d]) a.out32[d][c] = (float)v;
        }
        if (!ok && a.err) *a.err = 1;
    }
}

__global__ void __launch_bounds__(kThreads) k_scale_faces(FaceArgs a)
{
    const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % a.n[0]);
        const long long rest = c / a.n[0];
        const int j = (int)(rest % a.n[1]);
        const int k = (int)(rest / a.n[1]);
        const int q[3] = {i, j, k};
        for (int d = 0; d < 3; d++) {
            double v = 0.0;
            if (!(q[d] == 0 && !(a.per >> d & 1))) {
                const double alpha = a.in[d][c];
                if (!(alpha > 0.0 && isfinite(alpha)) && a.err) *a.err = 1;
                v = alpha * a.scale[d];
            }
            a.out64[d][c] = v;
            if (a.out32[d]) a.out32[d][c] = (float)v;
        }
    }
}

// coarse w_d(I,J,K) = (1/16) * sum of the 4 fine w_d that tile the coarse face:
// alpha_c = mean of the 4 fine alpha, and 1/(2h)^2 = (1/4)(1/h^2).
__global__ void __launch_bounds__(kThreads) k_coarsen_faces(CoarsenArgs a)
{
    const long long NC = (long long)a.nc[0] * a.nc[1] * a.nc[2];
    const int nx = a.nf[0], ny = a.nf[1];
    for (long long C = blockIdx.x * (long long)blockDim.x + threadIdx.x; C < NC;
         C += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(C % a.nc[0]);
        const long long rest = C / a.nc[0];
        const int J = (int)(rest % a.nc[1]);
        const int K = (int)(rest / a.nc[1]);
        const int base[3] = {2 * I, 2 * J, 2 * K};
        for (int d = 0; d < 3; d++) {
            const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
            double s = 0.0;
            for (int u = 0; u < 2; u++)
                for (int v = 0; v < 2; v++) {
                    int f[3];
                    f[d] = base[d];
                    f[e1] = base[e1] + u;
                    f[e2] = base[e2] + v;
                    s += a.wf[d][f[0] + (long long)nx * (f[1] + (long long)ny * f[2])];
                }
            const double w = s * 0.0625;
            a.wc[d][C] = w;
            if (a.wc32[d]) a.wc32[d][C] = (float)w;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 outer iteration
// ---------------------------------------------------------------------------

// Start of a solve: reset the state of every grid.
__global__ void k_begin(const OuterView *__restrict__ ov)
{
    if (threadIdx.x != 0) return;
    const OuterView &O = ov[blockIdx.x];
    GridState *s = O.st;
    s->tol = O.tol;
    s->max_iters = O.max_iters;
    s->iters = 0;
    s->status = 8;  // MG_EAGAIN while running
    s->active = 1;
    s->bmean = 0.0;
    s->bnorm = 0.0;
    s->r0 = 0.0;
    s->rnorm = 0.0;
    s->xmean = 0.0;
}

// Partial sums of the right-hand side (slot 3 of each block's partials).
__global__ void __launch_bounds__(kThreads) k_bsum(const OuterView *__restrict__ ov,
                                                   const int *__restrict__ start, int count)
{
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const int lb = blockIdx.x - start[e];
    const Tile t = fine_tile(O.n, lb);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (t.ok) {
        const long long rowoff = (long long)O.n[0] * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i < O.n[0]) v[3] += O.b[rowoff + i];
        }
    }
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) O.part[kPart * lb + 3] = out[3];
}

// Residual of the outer iteration.  update = 0: r = (b - bmean) - A x for the
// starting iterate x = p.  update = 1: x' = x + e (x in the buffer selected by
// the iteration parity, x' written to the other one) and r = (b - bmean) - A x'.
// r is handed to the V-cycle in its precision Te; ||r||^2, sum x', and (first
// call) ||b - bmean||^2 go to the block partials.  All arithmetic FP64, with the
// face differences taken before the products for accuracy near convergence.
template <class Te>
__global__ void __launch_bounds__(kThreads) k_residual(const OuterView *__restrict__ ov,
                                                       const int *__restrict__ start, int count,
                                                       int update)
{
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    if (!s->active) return;
    const int lb = blockIdx.x - start[e];
    const Tile t = fine_tile(O.n, lb);
    const int nx = O.n[0], ny = O.n[1], nz = O.n[2];
    const bool odd = s->iters & 1;
    const double *xin = odd ? O.xbuf : O.p;
    double *xout = odd ? O.p : O.xbuf;
    const Te *ec = (const Te *)O.e;
    Te *r = (Te *)O.r;
    const double m = s->bmean;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (t.ok) {
        const long long rowoff = (long long)nx * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i >= nx) continue;
            const long long c = rowoff + i;
            double d, f, xc;
            if (update) {
                xc = xin[c] + (double)ec[c];
                stencil(O.w[0], O.w[1], O.w[2], LoadSum<Te>{xin, ec}, nx, ny, nz, O.per, i, t.j,
                        t.k, c, xc, d, f);
                xout[c] = xc;
            } else {
                xc = xin[c];
                stencil(O.w[0], O.w[1], O.w[2], LoadPlain<double>{xin}, nx, ny, nz, O.per, i, t.j,
                        t.k, c, xc, d, f);
            }
            const double bc = O.b[c] - m;
            const double rc = bc - f;
            r[c] = (Te)rc;
            v[0] += rc * rc;
            v[1] += xc;
            v[2] += bc * bc;
        }
    }
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) {
        O.part[kPart * lb + 0] = out[0];
        O.part[kPart * lb + 1] = out[1];
        O.part[kPart * lb + 2] = out[2];
    }
}

// One block per grid: sum the block partials in a fixed order and update the
// state.  mode 0: mean of b.  mode 1: after the starting residual.  mode 2:
// after a cycle (counts it).  Stopping test: ||r|| <= tol ||b||; NaN/Inf
// residual = diverged; max_iters reached = not converged.
__global__ void __launch_bounds__(kThreads) k_finalize(const OuterView *__restrict__ ov, int mode)
{
    const OuterView &O = ov[blockIdx.x];
    GridState *s = O.st;
    if (!s->active) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < O.nblk; q += blockDim.x)
        for (int f = 0; f < 4; f++) v[f] += O.part[kPart * q + f];
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x != 0) return;
    const double N = (double)O.n[0] * O.n[1] * O.n[2];
    if (mode == 0) {
        s->bmean = out[3] / N;
        return;
    }
    const double rn = sqrt(out[0]);
    if (mode == 1) {
        s->bnorm = sqrt(out[2]);
        s->r0 = rn;
    } else {
        s->iters += 1;
    }
    s->rnorm = rn;
    s->xmean = out[1] / N;
    if (!isfinite(rn)) {
        s->status = 5;  // MG_EDIVERGED
        s->active = 0;
    } else if (s->bnorm == 0.0 || rn <= s->tol * s->bnorm) {
        s->status = 0;
        s->active = 0;
    } else if (s->iters >= s->max_iters) {
        s->status = 4;  // MG_ENOTCONV
        s->active = 0;
    }
}

// End of a solve: p = x - mean(x) from whichever buffer holds the iterate (a
// zero right-hand side gives p = 0).
__global__ void __launch_bounds__(kThreads) k_final(const OuterView *__restrict__ ov,
                                                    const int *__restrict__ start, int count)
{
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    const Tile t = fine_tile(O.n, blockIdx.x - start[e]);
    if (!t.ok) return;
    const double *x = (s->iters & 1) ? O.xbuf : O.p;
    const double m = s->xmean;
    const bool zero = s->bnorm == 0.0;
    const long long rowoff = (long long)O.n[0] * t.row;
    for (int h = 0; h < 2; h++) {
        const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
        if (i < O.n[0]) O.p[rowoff + i] = zero ? 0.0 : x[rowoff + i] - m;
    }
}

// Loop control of a graph-driven solve: keep iterating while any grid of the
// plan is still active.  Every grid stops after at most max_iters cycles, so
// the loop is bounded.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, const OuterView *__restrict__ ov, int count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned int any = 0;
    for (int g = 0; g < count; g++) any |= (unsigned int)(ov[g].st->active != 0);
    cudaGraphSetConditional(h, any);
}

// Copy the state of every grid of a plan into one contiguous array (one
// device-to-host copy then serves the whole batch).
__global__ void k_gather_states(const OuterView *__restrict__ ov, int count, GridState *out)
{
    for (int g = threadIdx.x; g < count; g += blockDim.x) out[g] = *ov[g].st;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

void launch_gather_states(const OuterTable &ot, GridState *out, cudaStream_t s)
{
    k_gather_states<<<1, 128, 0, s>>>(ot.ov, ot.count, out);
}

void launch_loop_ctl(cudaGraphConditionalHandle h, const OuterTable &ot, cudaStream_t s)
{
    k_loop_ctl<<<1, 32, 0, s>>>(h, ot.ov, ot.count);
}

template <class T>
void launch_smooth(const Table &tb, int colour, double omega, int zero_guess, cudaStream_t s)
{
    k_smooth<T><<<tb.blocks, kThreads, 0, s>>>(tb.lv, tb.start, tb.count, colour, (T)omega,
                                               zero_guess);
}
template <class T>
void launch_restrict(const Table &tb, cudaStream_t s)
{
    k_restrict<T><<<tb.blocks, kThreads, 0, s>>>(tb.lv, tb.start, tb.count);
}
template <class T>
void launch_prolong(const Table &tb, cudaStream_t s)
{
    k_prolong<T><<<tb.blocks, kThreads, 0, s>>>(tb.lv, tb.start, tb.count);
}
template <class T>
void launch_apply(const Table &tb, cudaStream_t s)
{
    k_apply<T><<<tb.blocks, kThreads, 0, s>>>(tb.lv, tb.start, tb.count);
}
template <class T>
void launch_coarse_solve(const CoarseView *cv, int count, cudaStream_t s)
{
    k_coarse_solve<T><<<count, kThreads, 0, s>>>(cv);
}
void launch_coarse_setup(const CoarseView *cv, int count, cudaStream_t s)
{
    k_coarse_setup<<<count, 1024, 0, s>>>(cv);
}
static int cells_grid(long long N)
{
    long long b = (N + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}
void launch_faces_from_density(const FaceArgs &a, cudaStream_t s)
{
    k_faces_from_density<<<cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s>>>(a);
}
void launch_scale_faces(const FaceArgs &a, cudaStream_t s)
{
    k_scale_faces<<<cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s>>>(a);
}
void launch_coarsen_faces(const CoarsenArgs &a, cudaStream_t s)
{
    k_coarsen_faces<<<cells_grid((long long)a.nc[0] * a.nc[1] * a.nc[2]), kThreads, 0, s>>>(a);
}
void launch_begin(const OuterView *ov, int count, cudaStream_t s) { k_begin<<<count, 32, 0, s>>>(ov); }
void launch_bsum(const OuterTable &ot, cudaStream_t s)
{
    k_bsum<<<ot.blocks, kThreads, 0, s>>>(ot.ov, ot.start, ot.count);
}
template <class Te>
void launch_residual(const OuterTable &ot, int update, cudaStream_t s)
{
    k_residual<Te><<<ot.blocks, kThreads, 0, s>>>(ot.ov, ot.start, ot.count, update);
}
void launch_finalize(const OuterTable &ot, int mode, cudaStream_t s)
{
    k_finalize<<<ot.count, kThreads, 0, s>>>(ot.ov, mode);
}
void launch_final(const OuterTable &ot, cudaStream_t s)
{
    k_final<<<ot.blocks, kThreads, 0, s>>>(ot.ov, ot.start, ot.count);
}

template void launch_smooth<float>(const Table &, int, double, int, cudaStream_t);
template void launch_smooth<double>(const Table &, int, double, int, cudaStream_t);
template void launch_restrict<float>(const Table &, cudaStream_t);
template void launch_restrict<double>(const Table &, cudaStream_t);
template void launch_prolong<float>(const Table &, cudaStream_t);
template void launch_prolong<double>(const Table &, cudaStream_t);
template void launch_apply<float>(const Table &, cudaStream_t);
template void launch_apply<double>(const Table &, cudaStream_t);
template void launch_coarse_solve<float>(const CoarseView *, int, cudaStream_t);
template void launch_coarse_solve<double>(const CoarseView *, int, cudaStream_t);
template void launch_residual<float>(const OuterTable &, int, cudaStream_t);
template void launch_residual<double>(const OuterTable &, int, cudaStream_t);

}  // namespace gbmg
