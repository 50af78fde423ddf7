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
#include "mg_stencil.cuh"
#include "mg_outer.cuh"
#include "mg_bulk.cuh"

#include <math.h>
#include <stdlib.h>

namespace gbmg {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

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

// ---------------------------------------------------------------------------
// (5) red-black relaxation, one colour per launch
// ---------------------------------------------------------------------------
//
// Cells of one colour only read cells of the other colour, so updating them in
// place equals the textbook half-sweep whatever the order of the threads.  When
// the row length is a multiple of 4 a thread owns an aligned quad of 4 cells of
// a row (one 16-byte vector per operand for FP32, two for FP64), relaxes the 2
// cells of the launch's colour and writes the other two back unchanged;
// otherwise (small coarse levels) one cell per thread.  The FP32 cycle uses the
// 2-ulp division (__fdividef): the inner cycle is a preconditioner and only
// steers convergence; the FP64 path divides exactly.
//
// flags: kZeroGuess  (red launch) the iterate is zero on entry: red cells get
//                    omega * (-b / d), black cells 0, so no clearing pass;
//        kOuter      (finest level, last black half-sweep of a cycle) a grid
//                    whose refinement step ends with this cycle also adds the
//                    final values of every cell (both colours) to its outer
//                    iterate.
// cyc: index of the V-cycle within its refinement step (in_cycle).
template <class T, bool OUT>
__device__ __forceinline__ void half_body(const LevelView &L, int lb, int colour, T omega, bool zero,
                                          const OuterOut &po, bool go = true)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], per = L.per;
    T *__restrict__ x = (T *)L.x;
    const T *__restrict__ b = (const T *)L.b;
    const T *__restrict__ wx = (const T *)L.w[0];
    const T *__restrict__ wy = (const T *)L.w[1];
    const T *__restrict__ wz = (const T *)L.w[2];
    const long long sy = nx, sz = (long long)nx * ny;

    if ((nx & 3) != 0) {
        // one cell per thread (row tiles of 64 cells per warp, 2 per lane)
        const Tile t = fine_tile(L.n, lb, L.dxt, L.dy);
        if (!t.ok) return;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (!go) return;
            if (i >= nx || ((i + t.j + t.k) & 1) != colour) {
                if (zero && i < nx) x[(long long)nx * t.row + i] = T(0);
                // the other colour's final value (the launch leaves it as it is)
                if constexpr (OUT)
                    if (i < nx) add_outer<T>(po, (int)((long long)nx * t.row + i), x[(long long)nx * t.row + i]);
                continue;
            }
            const long long c = (long long)nx * t.row + i;
            const T *di = (sizeof(T) == 8) ? (const T *)L.dinv : nullptr;
            T v;
            if (zero) {
                if (di) {
                    v = di[c] > T(0) ? omega * ((-b[c]) * di[c]) : T(0);
                } else {
                    const T d = diag_of(wx, wy, wz, nx, ny, nz, per, i, t.j, t.k, c);
                    v = d > T(0) ? omega * relax_div(-b[c], d) : T(0);
                }
            } else {
                const T xc = x[c];
                T d, f;
                stencil(wx, wy, wz, LoadPlain<T>{x}, nx, ny, nz, per, i, t.j, t.k, c, xc, d, f);
                if (di) v = di[c] > T(0) ? xc + omega * ((f - b[c]) * di[c]) : xc;  // (rows of other than whole quads)
                else v = d > T(0) ? xc + omega * relax_div(f - b[c], d) : xc;
            }
            x[c] = v;
            if constexpr (OUT) add_outer<T>(po, (int)c, v);
        }
        return;
    }

    // an aligned quad of 4 cells per thread: a warp covers 32 quads of one row,
    // a block 8 rows
    const int nq = nx >> 2;
    const int xt_n = (nq + 31) >> 5;
    const int rb = fdiv(lb, L.dxq), tq = lb - rb * xt_n;
    const int row = rb * kRowsPerBlock + (threadIdx.x >> 5);
    if (row >= ny * nz) return;
    const int qx = (tq << 5) + (threadIdx.x & 31);
    if (qx >= nq) return;
    const int k = fdiv(row, L.dy);
    half_quad<T, OUT>(x, b, wx, wy, wz, nx, ny, nz, per, row, row - k * ny, k, qx, colour, omega, zero, po, go,
                      (const T *)L.dinv);
}

// MAYOUT: the launch carries kOuter; the test of the step's last cycle is
// per grid, so uniform over a block, and picks one of two instances of the body.
// defer (one-grid tables, whose launches the graph limits to the grid's own
// cycles): the state's load overlaps the data's and only the stores wait for
// it; with several grids a grid that sits the cycle out returns at once.
template <class T, bool MAYOUT>
__device__ __forceinline__ void half_entry(const LevelView &L, int lb, int colour, T omega, int flags, int cyc,
                                           const OuterView *__restrict__ ov, bool defer)
{
    const bool zero = flags & kZeroGuess;
    if (!MAYOUT && defer) {
        half_body<T, false>(L, lb, colour, omega, zero, OuterOut{}, in_cycle(L.st, cyc));
        return;
    }
    if (!in_cycle(L.st, cyc)) return;
    if constexpr (MAYOUT) {
        if (last_cycle(L.st, cyc)) {
            half_body<T, true>(L, lb, colour, omega, zero, outer_out(ov[L.g]));
            return;
        }
    }
    half_body<T, false>(L, lb, colour, omega, zero, OuterOut{});
}

// single: a one-grid table, its view passed by value (`one`, parameter space):
// no dependent load of the view before the grid's state and data.
template <class T, bool MAYOUT>
__global__ void __launch_bounds__(kThreads) k_half(const LevelView *__restrict__ lv,
                                                   const int *__restrict__ start, int count,
                                                   int colour, T omega, int flags, int cyc,
                                                   const OuterView *__restrict__ ov,
                                                   const __grid_constant__ LevelView one, int single)
{
    dep_entry();
    if (single) {
        half_entry<T, MAYOUT>(one, blockIdx.x, colour, omega, flags, cyc, ov, true);
        return;
    }
    const int e = find_entry(start, count);
    half_entry<T, MAYOUT>(lv[e], blockIdx.x - start[e], colour, omega, flags, cyc, ov, false);
}

// Blocks of a half-sweep launch over a level: row tiles of 32 quads (or 64
// cells) per warp, 8 rows per block.
__host__ __device__ inline int half_blocks(const int n[3])
{
    if ((n[0] & 3) != 0) return fine_blocks(n);
    const int nq = n[0] >> 2;
    return ((nq + 31) >> 5) * ((n[1] * n[2] + kRowsPerBlock - 1) / kRowsPerBlock);
}
int half_sweep_blocks(const int n[3]) { return half_blocks(n); }
int prolong_blocks(const int n[3]) { return half_blocks(n); }

// ---------------------------------------------------------------------------
// (3) residual and restriction: coarse b = mean of (b - A x) over 8 children
// ---------------------------------------------------------------------------

// defer: see half_entry
template <class T>
__device__ __forceinline__ void restrict_entry(const LevelView &L, int lb, int cyc, T omega, bool defer)
{
    const bool go = in_cycle(L.st, cyc);
    if (!defer && !go) return;
    const int ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2];
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const T *x = (const T *)L.x;
    const T *b = (const T *)L.b;
    const T *wx = (const T *)L.w[0], *wy = (const T *)L.w[1], *wz = (const T *)L.w[2];
    if ((nx & 3) == 0) {
        // a thread owns the coarse pair (2P, 2P+1) of a coarse row: one fine quad
        // in each of the 2 x 2 fine rows below it
        const int np = ncx >> 1;
        const int xt_n = (np + 31) >> 5;
        const int rb = fdiv(lb, L.dxp), xt = lb - rb * xt_n;
        const int crow = rb * kRowsPerBlock + (threadIdx.x >> 5);
        if (crow >= ncy * ncz) return;
        const int P = (xt << 5) + (threadIdx.x & 31);
        if (P >= np) return;
        const int K = fdiv(crow, L.dcy);
        restrict_pair<T>(L, crow, crow - K * ncy, K, P, omega, go);
        return;
    }
    if (!go) return;
    const int xt_n = coarse_xtiles(ncx);
    const int rb = fdiv(lb, L.dxc), xt = lb - rb * xt_n;
    const int crow = rb * kRowsPerBlock + (threadIdx.x >> 5);
    if (crow >= ncy * ncz) return;
    const int I = xt * kCSeg + (threadIdx.x & 31);
    if (I >= ncx) return;
    const int K = fdiv(crow, L.dcy), J = crow - K * ncy;
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
    const T bcv = s * T(0.125);
    ((T *)L.bc)[I + (long long)ncx * crow] = bcv;
    if (L.zr) ((T *)L.xc)[I + (long long)ncx * crow] = zero_start_red<T>(L, I, J, K, bcv, omega);
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_restrict(const LevelView *__restrict__ lv,
                                                       const int *__restrict__ start, int count, int cyc,
                                                       T omega, const __grid_constant__ LevelView one,
                                                       int single)
{
    dep_entry();
    if (single) {
        restrict_entry<T>(one, blockIdx.x, cyc, omega, true);
        return;
    }
    const int e = find_entry(start, count);
    restrict_entry<T>(lv[e], blockIdx.x - start[e], cyc, omega, false);
}

// Blocks of a restriction launch over the coarse level of `n`.
int restrict_blocks(const int n[3], const int nc[3])
{
    if ((n[0] & 3) != 0) return coarse_blocks(nc);
    const int np = nc[0] >> 1;
    return ((np + 31) >> 5) * ((nc[1] * nc[2] + kRowsPerBlock - 1) / kRowsPerBlock);
}

// ---------------------------------------------------------------------------
// (4) prolongation and correction: x += P e_c.  With no post-smoothing the
// finest level's prolongation ends the cycle, so a launch with MAYOUT adds the
// result to the FP64 iterate of the grids whose step ends with this cycle
// (row tiles only: a configuration without post-smoothing is not tuned for).
// ---------------------------------------------------------------------------

template <class T, bool FLUX, bool OUT>
__device__ __forceinline__ void prolong_body(const LevelView &L, int lb, const OuterOut &po, bool go = true)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const T *ec = (const T *)L.xc;
    T *x = (T *)L.x;
    if ((nx & 3) == 0) {
        const int nq = nx >> 2;
        const int xt_n = (nq + 31) >> 5;
        const int rb = fdiv(lb, L.dxq), xt = lb - rb * xt_n;
        const int row = rb * kRowsPerBlock + (threadIdx.x >> 5);
        if (row >= ny * nz) return;
        const int qx = (xt << 5) + (threadIdx.x & 31);
        if (qx >= nq) return;
        const int k = fdiv(row, L.dy);
        if constexpr (FLUX) {
            if (!go) return;
            prolong_quad_flux<T, OUT>(L, row, row - k * ny, k, qx, po);
        } else {
            prolong_quad<T, OUT>(L, row, row - k * ny, k, qx, po, go);
        }
        return;
    }
    if (!go) return;
    const Tile t = fine_tile(L.n, lb, L.dxt, L.dy);
    if (!t.ok) return;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
        if (i >= nx) continue;
        const long long c = (long long)nx * t.row + i;
        const T xn = x[c] + (FLUX ? prolong_at_flux(ec, (const T *)L.ac, L.nc, L.per, i, t.j, t.k)
                                  : prolong_at(ec, L.nc, L.per, i, t.j, t.k));
        x[c] = xn;
        if constexpr (OUT) add_outer<T>(po, (int)c, xn);
    }
}

// defer: see half_entry
template <class T, bool FLUX, bool MAYOUT>
__device__ __forceinline__ void prolong_entry(const LevelView &L, int lb, int cyc, const OuterView *__restrict__ ov,
                                              bool defer)
{
    if (!MAYOUT && defer) {
        prolong_body<T, FLUX, false>(L, lb, OuterOut{}, in_cycle(L.st, cyc));
        return;
    }
    if (!in_cycle(L.st, cyc)) return;
    if constexpr (MAYOUT) {
        if (last_cycle(L.st, cyc)) {
            prolong_body<T, FLUX, true>(L, lb, outer_out(ov[L.g]));
            return;
        }
    }
    prolong_body<T, FLUX, false>(L, lb, OuterOut{});
}

template <class T, bool FLUX, bool MAYOUT>
__global__ void __launch_bounds__(kThreads) k_prolong(const LevelView *__restrict__ lv,
                                                      const int *__restrict__ start, int count, int cyc,
                                                      const OuterView *__restrict__ ov,
                                                      const __grid_constant__ LevelView one, int single)
{
    dep_entry();
    if (single) {
        prolong_entry<T, FLUX, MAYOUT>(one, blockIdx.x, cyc, ov, true);
        return;
    }
    const int e = find_entry(start, count);
    prolong_entry<T, FLUX, MAYOUT>(lv[e], blockIdx.x - start[e], cyc, ov, false);
}

// ---------------------------------------------------------------------------
// The bottom of the V-cycle in one launch: every level of a grid with at most
// kTailCells cells (and the coarsest solve) is processed by one block of kTailThreads
// threads, all operands in shared memory, phases separated by block barriers.
// These levels are too small to fill the GPU; as separate launches they cost
// a launch latency each (10 per level per cycle) while doing almost no work.
// The arithmetic is the same as the per-level kernels: red-black half-sweeps
// (red first, zero initial correction), 8-child restriction of the residual,
// trilinear prolongation, and the exact coarsest solve e = -G b in FP64.
// ---------------------------------------------------------------------------

// n elements (n % 4 == 0, both pointers 16-byte aligned) from global to shared memory
template <class T>
__device__ __forceinline__ void stage(T *__restrict__ dst, const T *__restrict__ src, int n)
{
    if constexpr (sizeof(T) == 4) {
        for (int c = threadIdx.x; c < (n >> 2); c += blockDim.x)
            reinterpret_cast<float4 *>(dst)[c] = reinterpret_cast<const float4 *>(src)[c];
    } else {
        for (int c = threadIdx.x; c < (n >> 1); c += blockDim.x)
            reinterpret_cast<double2 *>(dst)[c] = reinterpret_cast<const double2 *>(src)[c];
    }
}

template <class T>
__device__ __forceinline__ T smem_flux(const T *x, const T *wx, const T *wy, const T *wz, int nx,
                                       int ny, int nz, int per, int i, int j, int k, int c, T xc,
                                       T &diag)
{
    const int sy = nx, sz = nx * ny;
    T a, d, f;
    a = wx[c];
    d = a;
    f = a * (x[i > 0 ? c - 1 : ((per & 1) ? c + nx - 1 : c)] - xc);
    if (i + 1 < nx) {
        a = wx[c + 1];
        d += a;
        f += a * (x[c + 1] - xc);
    } else if (per & 1) {
        a = wx[c + 1 - nx];
        d += a;
        f += a * (x[c + 1 - nx] - xc);
    }
    a = wy[c];
    d += a;
    f += a * (x[j > 0 ? c - sy : ((per & 2) ? c + sy * (ny - 1) : c)] - xc);
    if (j + 1 < ny) {
        a = wy[c + sy];
        d += a;
        f += a * (x[c + sy] - xc);
    } else if (per & 2) {
        a = wy[c - sy * (ny - 1)];
        d += a;
        f += a * (x[c - sy * (ny - 1)] - xc);
    }
    a = wz[c];
    d += a;
    f += a * (x[k > 0 ? c - sz : ((per & 4) ? c + sz * (nz - 1) : c)] - xc);
    if (k + 1 < nz) {
        a = wz[c + sz];
        d += a;
        f += a * (x[c + sz] - xc);
    } else if (per & 4) {
        a = wz[c - sz * (nz - 1)];
        d += a;
        f += a * (x[c - sz * (nz - 1)] - xc);
    }
    diag = d;
    return f;
}

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailView *__restrict__ tv, T omega,
                                                       int nu1, int nu2, int cyc)
{
    dep_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = (T *)smem_raw;
    const TailView &V = tv[blockIdx.x];
    if (!in_cycle(V.st, cyc)) return;
    const int nt = V.nt, per = V.per;
    // stage the faces of every tail level but the coarsest (solved with G) and
    // the right-hand side of the first by bulk asynchronous copies, issued by
    // one thread and completed on one mbarrier; levels above the coarsest have
    // even sizes, so N % 8 == 0: sizes are multiples of 32 bytes and the slab
    // offsets keep 16-byte alignment
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        const int N0 = V.n[0][0] * V.n[0][1] * V.n[0][2];
        unsigned bytes = (unsigned)(N0 * sizeof(T));
        for (int t = 0; t + 1 < nt; t++) bytes += 3u * (unsigned)(V.n[t][0] * V.n[t][1] * V.n[t][2] * sizeof(T));
        mbar_arrive_expect_tx(&bar, bytes);
        for (int t = 0; t + 1 < nt; t++) {
            const int N = V.n[t][0] * V.n[t][1] * V.n[t][2];
            T *base = sm + V.off[t];
            for (int d = 0; d < 3; d++) bulk_g2s(base + (2 + d) * N, V.w[t][d], (unsigned)(N * sizeof(T)), &bar);
        }
        bulk_g2s(sm + V.off[0] + N0, V.b0, (unsigned)(N0 * sizeof(T)), &bar);
    }
    if (V.flux) {
        // cell coefficients of the tail's coarse levels (a small odd-sized
        // coarsest level rules out the vector copy)
        for (int t = 1; t < nt; t++) {
            const int N = V.n[t][0] * V.n[t][1] * V.n[t][2];
            const T *g = (const T *)V.a[t];
            T *d = sm + V.off[t] + 5 * N;
            for (int c = threadIdx.x; c < N; c += blockDim.x) d[c] = g[c];
        }
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
    // every thread waits (bounded); the outcome is made uniform over the block
    const int staged = __syncthreads_and(mbar_wait(&bar, 0, V.wait_polls) ? 1 : 0);
    if (!staged) {
        // give up on this grid (reported as MG_ETIMEOUT), but let the copies
        // land before the block's shared memory is released
        if (threadIdx.x == 0 && V.err) *V.err = 1;
        mbar_wait(&bar, 0, kBulkWaitPolls);
        return;
    }

    // A tail level as a LevelView on shared memory, so that the per-quad
    // functions of the per-level kernels (half_quad, restrict_pair,
    // prolong_quad) run here unchanged on levels whose rows are a multiple of 4
    // cells: one quad per thread at 16^3, 16-byte shared-memory loads, and the
    // zero-start red half-sweep writes both colours (no clearing pass).  Other
    // levels take one cell per thread.
    auto view = [&](int t) {
        LevelView L;
        const int N = V.n[t][0] * V.n[t][1] * V.n[t][2];
        for (int d = 0; d < 3; d++) {
            L.n[d] = V.n[t][d];
            L.w[d] = sm + V.off[t] + (2 + d) * N;
            L.nc[d] = t + 1 < nt ? V.n[t + 1][d] : 1;
        }
        L.per = per;
        L.x = sm + V.off[t];
        L.b = sm + V.off[t] + N;
        if (t + 1 < nt) {
            const int NC = V.n[t + 1][0] * V.n[t + 1][1] * V.n[t + 1][2];
            L.xc = sm + V.off[t + 1];
            L.bc = sm + V.off[t + 1] + NC;
            L.ac = sm + V.off[t + 1] + 5 * NC;
        }
        L.zr = 0;
        return L;
    };

    // zero: the correction is zero on entry (first red half-sweep of a cycle)
    auto half = [&](int t, int colour, bool zero) {
        const int nx = V.n[t][0], ny = V.n[t][1], nz = V.n[t][2], N = nx * ny * nz;
        T *x = sm + V.off[t];
        const T *b = x + N, *wx = x + 2 * N, *wy = x + 3 * N, *wz = x + 4 * N;
        if ((nx & 3) == 0) {
            const int nq = nx >> 2;
            for (int q = threadIdx.x; q < (N >> 2); q += blockDim.x) {
                const int row = fdiv(q, V.dq[t]);
                const int k = fdiv(row, V.dy[t]);
                half_quad_sm<T>(x, b, wx, wy, wz, nx, ny, nz, per, row, row - k * ny, k, q - row * nq, colour,
                                omega, zero);
            }
            __syncthreads();
            return;
        }
        if (zero) {
            // no cell of the level may be read before it is set
            for (int c = threadIdx.x; c < N; c += blockDim.x) x[c] = T(0);
            __syncthreads();
        }
        const int hx = nx >> 1;
        for (int m = threadIdx.x; m < (N >> 1); m += blockDim.x) {
            // m-th cell of the colour: rows of hx cells, the colour's cells at
            // every other i starting from (colour + j + k) & 1
            const int row = fdiv(m, V.dhx[t]);
            const int k = fdiv(row, V.dy[t]);
            const int j = row - k * ny;
            const int i = 2 * (m - row * hx) + ((colour + j + k) & 1);
            const int c = i + nx * row;
            const T xc = x[c];
            T d;
            const T f = smem_flux(x, wx, wy, wz, nx, ny, nz, per, i, j, k, c, xc, d);
            x[c] = d > T(0) ? xc + omega * relax_div(f - b[c], d) : xc;
        }
        __syncthreads();
    };

    for (int t = 0; t + 1 < nt; t++) {
        for (int it = 0; it < nu1; it++) {
            half(t, 0, it == 0);
            half(t, 1, false);
        }
        // restriction of the residual to level t + 1
        const int nx = V.n[t][0], ny = V.n[t][1], nz = V.n[t][2], N = nx * ny * nz;
        const int ncx = V.n[t + 1][0], ncy = V.n[t + 1][1], NC = ncx * ncy * V.n[t + 1][2];
        if ((nx & 3) == 0) {
            const LevelView L = view(t);
            const int np = ncx >> 1;
            for (int g = threadIdx.x; g < (NC >> 1); g += blockDim.x) {
                const int crow = fdiv(g, V.dq[t]);  // np = nx / 4
                const int K = fdiv(crow, V.dy[t + 1]);
                restrict_pair<T>(L, crow, crow - K * ncy, K, g - crow * np, omega);
            }
        } else {
            const T *x = sm + V.off[t];
            const T *b = x + N, *wx = x + 2 * N, *wy = x + 3 * N, *wz = x + 4 * N;
            T *bc = sm + V.off[t + 1] + NC;
            for (int C = threadIdx.x; C < NC; C += blockDim.x) {
                const int crow = fdiv(C, V.dx[t + 1]);
                const int K = fdiv(crow, V.dy[t + 1]);
                const int I = C - crow * ncx, J = crow - K * ncy;
                T s = T(0);
                for (int dz = 0; dz < 2; dz++)
                    for (int dy = 0; dy < 2; dy++)
                        for (int dx = 0; dx < 2; dx++) {
                            const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
                            const int c = i + nx * (j + ny * k);
                            T d;
                            s += b[c] - smem_flux(x, wx, wy, wz, nx, ny, nz, per, i, j, k, c, x[c], d);
                        }
                bc[C] = s * T(0.125);
            }
        }
        __syncthreads();
    }
    {
        // exact solve on the coarsest level: e = -G b, FP64, one warp per row
        const int t = nt - 1;
        const int n = V.n[t][0] * V.n[t][1] * V.n[t][2];
        T *x = sm + V.off[t];
        const T *b = x + n;
        const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
        for (int r = threadIdx.x >> 5; r < n; r += warps) {
            const double *Gr = V.G + (long long)r * n;
            double s = 0.0;
            for (int u = lane; u < n; u += 32) s += Gr[u] * (double)b[u];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) x[r] = (T)(-s);
        }
        __syncthreads();
    }
    for (int t = nt - 2; t >= 0; t--) {
        const int nx = V.n[t][0], ny = V.n[t][1], N = nx * ny * V.n[t][2];
        if ((nx & 3) == 0) {
            const LevelView L = view(t);
            const int nq = nx >> 2;
            for (int q = threadIdx.x; q < (N >> 2); q += blockDim.x) {
                const int row = fdiv(q, V.dq[t]);
                const int k = fdiv(row, V.dy[t]);
                if (V.flux) prolong_quad_flux<T, false>(L, row, row - k * ny, k, q - row * nq, OuterOut{});
                else prolong_quad<T, false>(L, row, row - k * ny, k, q - row * nq, OuterOut{});
            }
        } else {
            const int nc[3] = {V.n[t + 1][0], V.n[t + 1][1], V.n[t + 1][2]};
            T *x = sm + V.off[t];
            const T *ec = sm + V.off[t + 1];
            const T *ac = ec + 5 * (nc[0] * nc[1] * nc[2]);
            for (int c = threadIdx.x; c < N; c += blockDim.x) {
                const int row = fdiv(c, V.dx[t]);
                const int k = fdiv(row, V.dy[t]);
                x[c] += V.flux ? prolong_at_flux(ec, ac, nc, per, c - row * nx, row - k * ny, k)
                               : prolong_at(ec, nc, per, c - row * nx, row - k * ny, k);
            }
        }
        __syncthreads();
        for (int it = 0; it < nu2; it++) {
            half(t, 0, false);
            half(t, 1, false);
        }
    }
    stage((T *)V.x0, sm + V.off[0], V.n[0][0] * V.n[0][1] * V.n[0][2]);
}

// ---------------------------------------------------------------------------
// y = A x on one level (unit checks): x in x, y in b
// ---------------------------------------------------------------------------

template <class T>
__global__ void __launch_bounds__(kThreads) k_apply(const LevelView *__restrict__ lv,
                                                    const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const LevelView L = lv[e];
    const Tile t = fine_tile(L.n, blockIdx.x - start[e], L.dxt, L.dy);
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
// (A 1 = 0) and the final mean removal takes out.  One warp per row of G
// (rows are contiguous, G is symmetric), lanes split the dot product, fixed
// shuffle tree.  A grid whose finest level is its coarsest (C.outer) adds e
// to its FP64 iterate in the last cycle of a refinement step (ov non-null).
template <class T>
__global__ void __launch_bounds__(kThreads) k_coarse_solve(const CoarseView *__restrict__ cv, int cyc,
                                                           const OuterView *__restrict__ ov)
{
    dep_entry();
    const CoarseView &C = cv[blockIdx.x];
    if (C.gmres || !in_cycle(C.st, cyc)) return;  // GMRES grids: k_coarse_gmres
    __shared__ double rb[kMaxCoarse];
    const int n = C.nc;
    const T *b = (const T *)C.b;
    for (int t = threadIdx.x; t < n; t += blockDim.x) rb[t] = (double)b[t];
    __syncthreads();
    T *x = (T *)C.x;
    const bool out = ov != nullptr && C.outer && last_cycle(C.st, cyc);
    const OuterOut po = out ? outer_out(ov[C.g]) : OuterOut{};
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int t = threadIdx.x >> 5; t < n; t += warps) {
        const double *Gt = C.G + (long long)t * n;
        double s = 0.0;
        for (int u = lane; u < n; u += 32) s += Gt[u] * rb[u];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const T xn = (T)(-s);
            x[t] = xn;
            if (out) add_outer<T>(po, t, xn);
        }
    }
}

// Assemble S = -A + c 1 1^T of the coarsest level (c = mean diagonal / n, so the
// constant vector becomes an eigenvector with a mid-spectrum eigenvalue) and
// invert it in place by Gauss-Jordan elimination.  S is symmetric positive
// definite, so no pivoting is needed; a non-positive pivot means the grid is
// cut into pieces by zero coefficients and raises *err.
__global__ void __launch_bounds__(1024) k_coarse_setup(const CoarseView *__restrict__ cv)
{
    dep_entry();
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

// Conversions between FP32 and FP64 by their IEEE 754 bit fields, for positive
// values whose exponent fits the FP32 normal range (the face set-up's case):
// this GPU issues the F2F conversion instructions to its narrow FP64 pipe, the
// integer forms run on the ALU.  Exponent bias 1023 (double) vs 127 (float):
// 896 between them; double mantissa 52 bits, float 23: 29 bits dropped.
//   widen_pos:   exact float -> double (normal positive f).
//   trunc_pos:   double -> float, low 29 mantissa bits dropped (a seed).
//   narrow_rn:   double -> float, round to nearest, ties to even; values
//                outside the fast range take the hardware conversion.
__device__ __forceinline__ double widen_pos(float f)
{
    const unsigned b = __float_as_uint(f);
    return __hiloint2double((int)((b >> 3) + (896u << 20)), (int)(b << 29));
}
__device__ __forceinline__ float trunc_pos(unsigned hi, unsigned lo)
{
    return __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}
__device__ __forceinline__ float narrow_rn(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    // positive, biased exponent 897 .. 1150: a normal float (or, rounding up
    // from the largest, the overflow to infinity that the rounding rule gives)
    if ((hi >> 20) - 897u > 253u) return (float)d;
    unsigned b = __float_as_uint(trunc_pos(hi, lo));
    const unsigned rem = lo & 0x1FFFFFFFu, half = 0x10000000u;
    b += (rem > half || (rem == half && (b & 1u))) ? 1u : 0u;  // a carry steps the exponent
    return __uint_as_float(b);
}

// 1 / x in FP64 by Newton-Raphson iteration on f(y) = 1/y - x, y <- y + y (1 - x y),
// from the FP32 reciprocal of x truncated to FP32 (relative error below
// 2^-22).  Each step squares the relative error and the last one rounds once,
// so two steps end within about one ulp of the quotient (Markstein, IBM J.
// Res. Dev. 34, 1990).  FP64 division is a long instruction sequence on this
// GPU's slow FP64 pipe; the Newton form is 4 fused multiply-adds.  Arguments
// that are not positive or lie outside [2^-125, 2^126) divide exactly.
__device__ __forceinline__ double recip_nr(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    if ((hi >> 20) - 898u > 250u) return 1.0 / x;  // biased exponent 898 .. 1148
    double y = widen_pos(__frcp_rn(trunc_pos(hi, lo)));
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__global__ void __launch_bounds__(kThreads) k_faces_from_density(FaceArgs a)
{
    dep_entry();
    const int N = a.n[0] * a.n[1] * a.n[2];  // grids have fewer than 2^31 cells
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int rest = fdiv(c, a.dx);
        const int i = c - rest * a.n[0];
        const int k = fdiv(rest, a.dy);
        const int j = rest - k * a.n[1];
        const int q[3] = {i, j, k};
        const int stride[3] = {1, a.n[0], a.n[0] * a.n[1]};
        const double rho_c = a.rho[c];
        bool ok = rho_c > 0.0 && isfinite(rho_c);
        const double inv_c = a.mode == 0 ? 0.0 : recip_nr(rho_c);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            double v;
            if (q[d] == 0 && !(a.per >> d & 1)) {
                v = 0.0;  // Neumann wall
            } else {
                const int l = q[d] > 0 ? c - stride[d] : c + stride[d] * (a.n[d] - 1);
                const double rho_l = a.rho[l];
                // Eqs. 11-12 with alpha = 1/rho: 2 a_l a_c / (a_l + a_c) = 2 / (rho_l + rho_c)
                v = a.mode == 0 ? (2.0 * a.scale[d]) * recip_nr(rho_l + rho_c)
                                : (0.5 * a.scale[d]) * (recip_nr(rho_l) + inv_c);
            }
            if (a.out64[d]) a.out64[d][c] = v;
            if (a.out32[d]) a.out32[d][c] = narrow_rn(v);
            if (a.out32lo[d]) a.out32lo[d][c] = (float)(v - (double)(float)v);
        }
        if (!ok && a.err) *a.err = 1;
    }
}

__global__ void __launch_bounds__(kThreads) k_scale_faces(FaceArgs a)
{
    dep_entry();
    const int N = a.n[0] * a.n[1] * a.n[2];  // grids have fewer than 2^31 cells
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int i = c % a.n[0];
        const int rest = c / a.n[0];
        const int j = rest % a.n[1];
        const int k = rest / a.n[1];
        const int q[3] = {i, j, k};
        for (int d = 0; d < 3; d++) {
            double v = 0.0;
            if (!(q[d] == 0 && !(a.per >> d & 1))) {
                const double alpha = a.in[d][c];
                if (!(alpha > 0.0 && isfinite(alpha)) && a.err) *a.err = 1;
                v = alpha * a.scale[d];
            }
            a.out64[d][c] = v;
            if (a.out32[d]) a.out32[d][c] = narrow_rn(v);
            if (a.out32lo[d]) a.out32lo[d][c] = (float)(v - (double)(float)v);
        }
    }
}

// coarse w_d(I,J,K) = (1/16) * sum of the 4 fine w_d that tile the coarse face:
// alpha_c = mean of the 4 fine alpha, and 1/(2h)^2 = (1/4)(1/h^2).
// Cell coefficient of the flux-conserving prolongation: mean over the cell's
// non-wall faces of alpha = w h_d^2 (1 for a cell without any).
__global__ void __launch_bounds__(kThreads) k_cell_alpha(AlphaArgs a)
{
    dep_entry();
    const int N = a.n[0] * a.n[1] * a.n[2];  // grids have fewer than 2^31 cells
    const int stride[3] = {1, a.n[0], a.n[0] * a.n[1]};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int rest = c / a.n[0];
        const int q[3] = {c - rest * a.n[0], rest % a.n[1], rest / a.n[1]};
        double s = 0.0;
        int m = 0;
        for (int d = 0; d < 3; d++) {
            const bool periodic = (a.per >> d) & 1;
            if (q[d] > 0 || periodic) {
                s += a.w[d][c] * a.h2[d];
                m++;
            }
            if (q[d] + 1 < a.n[d]) {
                s += a.w[d][c + stride[d]] * a.h2[d];
                m++;
            } else if (periodic) {
                s += a.w[d][c - stride[d] * (a.n[d] - 1)] * a.h2[d];
                m++;
            }
        }
        const double v = m ? s / m : 1.0;
        if (a.out64) a.out64[c] = v;
        if (a.out32) a.out32[c] = narrow_rn(v);
    }
}

// ---------------------------------------------------------------------------
// Projection step around the solve (Chorin's projection on the MAC grid).
// u[d][c] is the normal velocity on the LOW face of cell c along d; on a
// Neumann axis the low face of the first cell is a wall (zero) and the high
// wall of the last cell carries no velocity.
// ---------------------------------------------------------------------------

// S = D u / dt: sum over axes of (high face - low face) / h_d, divided by dt
__global__ void __launch_bounds__(kThreads) k_divergence(ProjArgs a)
{
    dep_entry();
    const int N = a.n[0] * a.n[1] * a.n[2];  // grids have fewer than 2^31 cells
    const int stride[3] = {1, a.n[0], a.n[0] * a.n[1]};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int rest = c / a.n[0];
        const int q[3] = {c - rest * a.n[0], rest % a.n[1], rest / a.n[1]};
        double div = 0.0;
        for (int d = 0; d < 3; d++) {
            const bool periodic = (a.per >> d) & 1;
            const double lo = (q[d] > 0 || periodic) ? a.u[d][c] : 0.0;
            const double hi = q[d] + 1 < a.n[d] ? a.u[d][c + stride[d]]
                              : periodic       ? a.u[d][c - stride[d] * (a.n[d] - 1)]
                                               : 0.0;
            div += (hi - lo) / a.h[d];
        }
        a.S[c] = div / a.dt;
    }
}

// u_f -= dt alpha_f (p_c - p_low) / h_d on every face that is not a wall;
// alpha_f / h_d = w h_d with the scaled coefficient w = alpha / h_d^2.  With
// the operator of Eq. 10, D(alpha G p) = A p, so D u = dt (S - A p).
__global__ void __launch_bounds__(kThreads) k_project(ProjArgs a)
{
    dep_entry();
    const int N = a.n[0] * a.n[1] * a.n[2];
    const int stride[3] = {1, a.n[0], a.n[0] * a.n[1]};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int rest = c / a.n[0];
        const int q[3] = {c - rest * a.n[0], rest % a.n[1], rest / a.n[1]};
        const double pc = a.p[c];
        for (int d = 0; d < 3; d++) {
            const bool periodic = (a.per >> d) & 1;
            if (q[d] == 0 && !periodic) continue;  // wall face
            const int m = q[d] > 0 ? c - stride[d] : c + stride[d] * (a.n[d] - 1);
            a.u[d][c] -= a.dt * (a.w[d][c] * a.h[d]) * (pc - a.p[m]);
        }
    }
}

// 1 / (sum of the cell's 6 face coefficients), summed in relax_cell's order
// (x low, x high, y low, y high, z low, z high; a wall's face is 0), so that
// relax_cell_inv relaxes against the same diagonal; 0 for a cell without faces.
__global__ void __launch_bounds__(kThreads) k_diag_inv(DiagArgs a)
{
    dep_entry();
    const int nx = a.n[0], ny = a.n[1], nz = a.n[2], per = a.per;
    const int N = nx * ny * nz, sy = nx, sz = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int rest = fdiv(c, a.dx);
        const int i = c - rest * nx;
        const int k = fdiv(rest, a.dy);
        const int j = rest - k * ny;
        double d = a.w[0][c];
        d += i + 1 < nx ? a.w[0][c + 1] : ((per & 1) ? a.w[0][c + 1 - nx] : 0.0);
        d += a.w[1][c];
        d += j + 1 < ny ? a.w[1][c + sy] : ((per & 2) ? a.w[1][c - sy * (ny - 1)] : 0.0);
        d += a.w[2][c];
        d += k + 1 < nz ? a.w[2][c + sz] : ((per & 4) ? a.w[2][c - sz * (nz - 1)] : 0.0);
        a.out[c] = d > 0.0 ? 1.0 / d : 0.0;
    }
}

__global__ void __launch_bounds__(kThreads) k_coarsen_faces(CoarsenArgs a)
{
    dep_entry();
    const int NC = a.nc[0] * a.nc[1] * a.nc[2];
    const int nx = a.nf[0], ny = a.nf[1];
    for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < NC; C += gridDim.x * blockDim.x) {
        const int rest = fdiv(C, a.dx);
        const int I = C - rest * a.nc[0];
        const int K = fdiv(rest, a.dy);
        const int J = rest - K * a.nc[1];
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
            if (a.wc32[d]) a.wc32[d][C] = narrow_rn(w);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 outer iteration
// ---------------------------------------------------------------------------

// Start of a solve: reset the state of every grid.
__global__ void k_begin(const OuterView *__restrict__ ov)
{
    dep_entry();
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
    s->cycles_next = O.inner < O.max_iters ? O.inner : O.max_iters;
    s->steps = 0;
    s->xscale = 1.0;
    s->xinv = 1.0;
    s->rprev = 0.0;
    s->pnz = 0;
}

// Partial sums of the caller's right-hand side (which = 0, partial slot 3) or
// of the iterate p (which = 1, slot 1), FP64.
__global__ void __launch_bounds__(kThreads) k_sum(const OuterView *__restrict__ ov,
                                                  const int *__restrict__ start, int count, int which)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const int lb = blockIdx.x - start[e];
    const int ntiles = fine_blocks(O.n);
    const double *src = which == 0 ? O.b : O.p;
    // end of an extended-precision solve that took a step: the iterate is the
    // three-float one (summed in its internal scale)
    const bool conv = which == 1 && xp_live(O);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    // kUnroll tiles of the block's grid-stride sequence per pass: every load of
    // the pass is issued before the additions, which then run in the order of
    // the sequence (one tile after the other, two cells per tile)
    for (int tile = lb; tile < ntiles; tile += kUnroll * O.nblk) {
        double val[kUnroll][2];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int tu = tile + u * O.nblk;
            const Tile t = fine_tile(O.n, tu < ntiles ? tu : tile, O.dxt, O.xy);
            const long long rowoff = (long long)O.n[0] * t.row;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
                const bool in = tu < ntiles && t.ok && i < O.n[0];
                const long long c = rowoff + i;
                double x = 0.0;
                if (in) x = conv ? ((double)O.xp3[0][c] + (double)O.xp3[1][c]) + (double)O.xp3[2][c] : src[c];
                val[u][h] = in ? x : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int tu = tile + u * O.nblk;
            if (tu >= ntiles) break;
            const Tile t = fine_tile(O.n, tu, O.dxt, O.xy);
            if (!t.ok) continue;
#pragma unroll
            for (int h = 0; h < 2; h++)
                if (t.xbase + (threadIdx.x & 31) + 32 * h < O.n[0]) v[0] += val[u][h];
        }
    }
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) O.part[kPart * lb + (which == 0 ? 3 : 1)] = out[0];
}

// ---- extended-precision outer iteration (mixed-precision multigrid) --------
//
// The FP64 prologue reduces the right-hand side; the refinement loop itself
// runs in FP32 arithmetic on the three-float iterate (mg_xprec.cuh); the
// epilogue converts back.  Internal quantities are scaled by xscale = 2^-k,
// k chosen from the right-hand side's rms, so that the float components stay
// far from the FP32 exponent limits whatever the scale of the problem.

// Split an FP64 value into floats: v = h + m (+ z): exact for z (the 53-bit
// significand fits 72 bits), to 2^-48 |v| for the pair.
__device__ __forceinline__ void split3(double v, float &h, float &m, float &z)
{
    h = (float)v;
    const double r = v - (double)h;
    m = (float)r;
    z = (float)(r - (double)m);
}

// b0 = b - mean(b) in FP64 and the partial sums of ||b0||^2 (slot 2).  Also
// notes whether the caller's starting iterate p has a cell that is not zero
// (GridState::pnz; a NaN counts as nonzero): a cold start (p = 0) then takes
// its starting residual as b0 itself (k_residual, mode 2).
__global__ void __launch_bounds__(kThreads) k_center_rhs(const OuterView *__restrict__ ov,
                                                    const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    if (!O.st->active) return;
    const int lb = blockIdx.x - start[e];
    const int ntiles = fine_blocks(O.n);
    const double m = O.st->bmean;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    int nz = 0;
    // loads of kUnroll tiles first, then the sequence's arithmetic in order (see k_sum)
    for (int tile = lb; tile < ntiles; tile += kUnroll * O.nblk) {
        double bv[kUnroll][2], pv[kUnroll][2];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int tu = tile + u * O.nblk;
            const Tile t = fine_tile(O.n, tu < ntiles ? tu : tile, O.dxt, O.xy);
            const long long rowoff = (long long)O.n[0] * t.row;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
                const bool in = tu < ntiles && t.ok && i < O.n[0];
                bv[u][h] = in ? O.b[rowoff + i] : 0.0;
                pv[u][h] = in ? O.p[rowoff + i] : 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int tu = tile + u * O.nblk;
            if (tu >= ntiles) break;
            const Tile t = fine_tile(O.n, tu, O.dxt, O.xy);
            if (!t.ok) continue;
            const long long rowoff = (long long)O.n[0] * t.row;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
                if (i >= O.n[0]) continue;
                const double bc = bv[u][h] - m;
                O.b0[rowoff + i] = bc;
                v[2] += bc * bc;
                nz |= !(pv[u][h] == 0.0);
            }
        }
    }
    double out[4];
    block_sum4(v, out);
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&O.st->pnz, 1);
    if (threadIdx.x == 0) O.part[kPart * lb + 2] = out[2];
}

// Scaled right-hand side and iterate in their float forms.
__global__ void __launch_bounds__(kThreads) k_xp_prepare(const OuterView *__restrict__ ov,
                                                         const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    if (!O.st->active) return;
    const int lb = blockIdx.x - start[e];
    const int ntiles = fine_blocks(O.n);
    const double sc = O.st->xscale;
    for (int tile = lb; tile < ntiles; tile += O.nblk) {
        const Tile t = fine_tile(O.n, tile, O.dxt, O.xy);
        if (!t.ok) continue;
        const long long rowoff = (long long)O.n[0] * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i >= O.n[0]) continue;
            const long long c = rowoff + i;
            float z;
            split3(O.b0[c] * sc, O.xb[0][c], O.xb[1][c], z);
            split3(O.p[c] * sc, O.xp3[0][c], O.xp3[1][c], O.xp3[2][c]);
        }
    }
}

// One face of the residual: (F0, F1) += w (p_nb - p_c), w = w0 + w1
#define XP_FACE(NB, W0, W1)                                                                    \
    do {                                                                                       \
        const int nb_ = (NB);                                                                  \
        float l_;                                                                              \
        const float h_ = triple_diff(P0[nb_], P1[nb_], P2[nb_], a0, a1, a2, l_);               \
        pair_fma_acc(F0, F1, h_, l_, (W0), (W1));                                              \
    } while (0)

// r = (b - mean b) - A p in the three-float arithmetic, scaled: the V-cycle's
// FP32 right-hand side, and the partial sums of ||r||^2 (slot 0, accumulated
// from the rounded r as in the FP64 kernel).  Every cell sums its faces in the
// order of flux64 (x low, x high, y low, y high, z low, z high).  Rows of a
// multiple of 4 cells: a thread takes an aligned quad, loads every operand as
// 16-byte vectors and treats wall faces as faces of zero weight (the stored
// low wall face is 0; its neighbour index is the cell itself), so the loads
// carry no branches; the zero terms leave the sums unchanged.  Other rows: one
// cell at a time, wall faces skipped.
__global__ void __launch_bounds__(kThreads) k_residual_xp(const OuterView *__restrict__ ov,
                                                          const int *__restrict__ start, int count,
                                                          int first)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView &O = ov[e];
    if (!O.st->active) return;
    // first: the starting residual, r = b0 where the starting iterate is zero
    const bool cold = first && !O.st->pnz;
    const int lb = blockIdx.x - start[e];
    const int nx = O.n[0], ny = O.n[1], nz = O.n[2], per = O.per, nblk = O.nblk;
    const int sy = nx, sz = nx * ny;  // grids have fewer than 2^31 cells
    const float *__restrict__ P0 = O.xp3[0];
    const float *__restrict__ P1 = O.xp3[1];
    const float *__restrict__ P2 = O.xp3[2];
    const float *__restrict__ wx = O.w32[0];
    const float *__restrict__ wy = O.w32[1];
    const float *__restrict__ wz = O.w32[2];
    const float *__restrict__ lx = O.wlo[0];
    const float *__restrict__ ly = O.wlo[1];
    const float *__restrict__ lz = O.wlo[2];
    const float *__restrict__ B0 = O.xb[0];
    const float *__restrict__ B1 = O.xb[1];
    float *__restrict__ r = (float *)O.r;
    float racc = 0.f;
    if ((nx & 3) == 0) {
        const int nq = nx >> 2, items = nq * ny * nz;
        const FastDiv dq = O.xq, dy = O.xy;
        for (int g = lb * kThreads + (int)threadIdx.x; g < items; g += nblk * kThreads) {
            const int row = fdiv(g, dq);
            const int k = fdiv(row, dy), j = row - k * ny;
            const int i0 = (g - row * nq) << 2;
            const int c = row * nx + i0;
            const bool has_e = i0 + 4 < nx || (per & 1);
            const int cw = i0 > 0 ? c - 1 : ((per & 1) ? c + nx - 1 : c);
            const int ce = i0 + 4 < nx ? c + 4 : ((per & 1) ? c + 4 - nx : c + 3);
            const bool has_n = j + 1 < ny || (per & 2), has_t = k + 1 < nz || (per & 4);
            const int ds = j > 0 ? -sy : ((per & 2) ? sy * (ny - 1) : 0);
            const int dn = j + 1 < ny ? sy : ((per & 2) ? -sy * (ny - 1) : 0);
            const int db = k > 0 ? -sz : ((per & 4) ? sz * (nz - 1) : 0);
            const int dt = k + 1 < nz ? sz : ((per & 4) ? -sz * (nz - 1) : 0);
            float F0[4] = {0.f, 0.f, 0.f, 0.f}, F1[4] = {0.f, 0.f, 0.f, 0.f};
            if (!cold) {  // A p is zero: no terms
                const float4 A0 = *(const float4 *)(P0 + c), A1 = *(const float4 *)(P1 + c),
                             A2 = *(const float4 *)(P2 + c);
                const float a0[4] = {A0.x, A0.y, A0.z, A0.w}, a1[4] = {A1.x, A1.y, A1.z, A1.w},
                            a2[4] = {A2.x, A2.y, A2.z, A2.w};
                auto term = [&](int u, float n0, float n1, float n2, float w0, float w1) {
                    float l;
                    const float h = triple_diff(n0, n1, n2, a0[u], a1[u], a2[u], l);
                    pair_fma_acc(F0[u], F1[u], h, l, w0, w1);
                };
                {
                    const float4 X0 = *(const float4 *)(wx + c), X1 = *(const float4 *)(lx + c);
                    const float x0[5] = {X0.x, X0.y, X0.z, X0.w, has_e ? wx[ce] : 0.f};
                    const float x1[5] = {X1.x, X1.y, X1.z, X1.w, has_e ? lx[ce] : 0.f};
                    const float w0v = P0[cw], w1v = P1[cw], w2v = P2[cw];
                    const float e0v = P0[ce], e1v = P1[ce], e2v = P2[ce];
    #pragma unroll
                    for (int u = 0; u < 4; u++) {
                        if (u == 0) term(0, w0v, w1v, w2v, x0[0], x1[0]);
                        else term(u, a0[u - 1], a1[u - 1], a2[u - 1], x0[u], x1[u]);
                        if (u == 3) term(3, e0v, e1v, e2v, x0[4], x1[4]);
                        else term(u, a0[u + 1], a1[u + 1], a2[u + 1], x0[u + 1], x1[u + 1]);
                    }
                }
                auto axis = [&](int dlo, int dhi, bool has_hi, const float *w, const float *wl) {
                    const float4 L0 = *(const float4 *)(P0 + c + dlo), L1 = *(const float4 *)(P1 + c + dlo),
                                 L2 = *(const float4 *)(P2 + c + dlo);
                    const float4 H0 = *(const float4 *)(P0 + c + dhi), H1 = *(const float4 *)(P1 + c + dhi),
                                 H2 = *(const float4 *)(P2 + c + dhi);
                    const float4 WL0 = *(const float4 *)(w + c), WL1 = *(const float4 *)(wl + c);
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 WH0 = has_hi ? *(const float4 *)(w + c + dhi) : z4;
                    const float4 WH1 = has_hi ? *(const float4 *)(wl + c + dhi) : z4;
                    const float l0[4] = {L0.x, L0.y, L0.z, L0.w}, l1[4] = {L1.x, L1.y, L1.z, L1.w},
                                l2[4] = {L2.x, L2.y, L2.z, L2.w};
                    const float h0[4] = {H0.x, H0.y, H0.z, H0.w}, h1[4] = {H1.x, H1.y, H1.z, H1.w},
                                h2[4] = {H2.x, H2.y, H2.z, H2.w};
                    const float wl0[4] = {WL0.x, WL0.y, WL0.z, WL0.w}, wl1[4] = {WL1.x, WL1.y, WL1.z, WL1.w};
                    const float wh0[4] = {WH0.x, WH0.y, WH0.z, WH0.w}, wh1[4] = {WH1.x, WH1.y, WH1.z, WH1.w};
    #pragma unroll
                    for (int u = 0; u < 4; u++) {
                        term(u, l0[u], l1[u], l2[u], wl0[u], wl1[u]);
                        term(u, h0[u], h1[u], h2[u], wh0[u], wh1[u]);
                    }
                };
                axis(ds, dn, has_n, wy, ly);
                axis(db, dt, has_t, wz, lz);
            }
            const float4 Q0 = *(const float4 *)(B0 + c), Q1 = *(const float4 *)(B1 + c);
            const float q0[4] = {Q0.x, Q0.y, Q0.z, Q0.w}, q1[4] = {Q1.x, Q1.y, Q1.z, Q1.w};
            float rq[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                float tt;
                const float hh = two_diff(q0[u], F0[u], tt);
                rq[u] = __fadd_rn(hh, __fadd_rn(tt, __fsub_rn(q1[u], F1[u])));
                racc = __fmaf_rn(rq[u], rq[u], racc);
            }
            *(float4 *)(r + c) = make_float4(rq[0], rq[1], rq[2], rq[3]);
        }
    } else {
        const int n3[3] = {nx, ny, nz};
        const int ntiles = fine_blocks(n3);
        for (int tile = lb; tile < ntiles; tile += nblk) {
            const Tile t = fine_tile(n3, tile, O.dxt, O.xy);
            if (!t.ok) continue;
            const int rowoff = nx * t.row;
            const int j = t.j, k = t.k;
            for (int h = 0; h < 2; h++) {
                const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
                if (i >= nx) continue;
                const int c = rowoff + i;
                const float a0 = P0[c], a1 = P1[c], a2 = P2[c];
                float F0 = 0.f, F1 = 0.f;
                if (!cold) {
                    if (i > 0) XP_FACE(c - 1, wx[c], lx[c]);
                    else if (per & 1) XP_FACE(c + nx - 1, wx[c], lx[c]);
                    if (i + 1 < nx) XP_FACE(c + 1, wx[c + 1], lx[c + 1]);
                    else if (per & 1) XP_FACE(c + 1 - nx, wx[c + 1 - nx], lx[c + 1 - nx]);
                    if (j > 0) XP_FACE(c - sy, wy[c], ly[c]);
                    else if (per & 2) XP_FACE(c + sy * (ny - 1), wy[c], ly[c]);
                    if (j + 1 < ny) XP_FACE(c + sy, wy[c + sy], ly[c + sy]);
                    else if (per & 2) XP_FACE(c - sy * (ny - 1), wy[c - sy * (ny - 1)], ly[c - sy * (ny - 1)]);
                    if (k > 0) XP_FACE(c - sz, wz[c], lz[c]);
                    else if (per & 4) XP_FACE(c + sz * (nz - 1), wz[c], lz[c]);
                    if (k + 1 < nz) XP_FACE(c + sz, wz[c + sz], lz[c + sz]);
                    else if (per & 4) XP_FACE(c - sz * (nz - 1), wz[c - sz * (nz - 1)], lz[c - sz * (nz - 1)]);
                }
                float tt;
                const float hh = two_diff(B0[c], F0, tt);
                const float rc = __fadd_rn(hh, __fadd_rn(tt, __fsub_rn(B1[c], F1)));
                r[c] = rc;
                racc = __fmaf_rn(rc, rc, racc);
            }
        }
    }
    double v[4] = {(double)racc, 0.0, 0.0, 0.0};
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) O.part[kPart * lb + 0] = out[0];
}
#undef XP_FACE

// Outer residual r = (b - mean b) - A p in FP64, handed to the V-cycle in its
// precision Te, scaled by xscale (a power of 2; 1 for CG).  init = 1 (start of
// a CG solve): also stores b0 = b - mean(b) and the partial sums of ||b0||^2
// (slot 2), all FP64.  init = 2 (start of a multigrid iteration): as 0, but a
// grid whose starting iterate is zero everywhere (GridState::pnz clear) takes
// r = b0 without evaluating A p, which is exactly zero there.  ||r||^2 goes to
// slot 0; after the first CG residual it is accumulated from the rounded,
// scaled r handed to the cycle (a norm only steers the stopping test, so its
// own rounding at 1e-7 relative is immaterial, and the scale keeps FP32
// squares inside the FP32 range).
template <class Te>
__global__ void __launch_bounds__(kThreads) k_residual(const OuterView *__restrict__ ov,
                                                       const int *__restrict__ start, int count,
                                                       int init)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    if (!s->active) return;
    const int lb = blockIdx.x - start[e];
    const int ntiles = fine_blocks(O.n);
    const int nx = O.n[0];
    Te *r = (Te *)O.r;
    const double m = s->bmean, sc = s->xscale;
    const bool cold = init == 2 && !s->pnz;
    if (init == 2) init = 0;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    Te racc = Te(0);
    for (int tile = lb; tile < ntiles; tile += O.nblk) {
        const Tile t = fine_tile(O.n, tile, O.dxt, O.xy);
        if (!t.ok) continue;
        const long long rowoff = (long long)nx * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i >= nx) continue;
            const long long c = rowoff + i;
            const double f = cold ? 0.0 : flux64(O, O.p, i, t.j, t.k, c);
            double bc;
            if (init) {
                bc = O.b[c] - m;
                O.b0[c] = bc;
                v[2] += bc * bc;
            } else {
                bc = O.b0[c];
            }
            const double rc = bc - f;
            const Te rt = (Te)(rc * sc);
            r[c] = rt;
            if (O.r64) O.r64[c] = rc;  // conjugate gradients keep the FP64 residual
            if (init) v[0] += rc * rc;
            else racc += rt * rt;
        }
    }
    if (!init) v[0] = (double)racc;
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) {
        O.part[kPart * lb + 0] = out[0];
        if (init) O.part[kPart * lb + 2] = out[2];
    }
}

// One block per grid: sum the block partials in a fixed order and update the
// state.  mode 0: mean of b.  mode 1: after the starting residual.  mode 2:
// after a cycle (counts it).  mode 3: mean of the final iterate.  mode 4
// (multigrid iteration): ||b - mean b|| and the scale of the cycles.  Stopping
// test: ||r|| <= tol ||b||; NaN/Inf residual = diverged; max_iters reached =
// not converged.
__global__ void __launch_bounds__(kThreads) k_finalize(const OuterView *__restrict__ ov, int mode)
{
    dep_entry();
    const OuterView &O = ov[blockIdx.x];
    GridState *s = O.st;
    if (mode != 3 && !s->active) return;
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
    if (mode == 3) {
        s->xmean = out[1] / N;
        return;
    }
    if (mode == 4) {
        // extended precision: ||b - mean b|| and the internal scale 2^-k,
        // 2^k near the rms of b - mean b (k kept inside the FP32 exponent range)
        s->bnorm = sqrt(out[2]);
        const double rms = s->bnorm / sqrt(N);
        int k = (rms > 0.0 && isfinite(rms)) ? ilogb(rms) : 0;
        k = k < -100 ? -100 : (k > 100 ? 100 : k);
        s->xscale = ldexp(1.0, -k);
        s->xinv = ldexp(1.0, k);
        return;
    }
    // the partials are of the scaled residual (xscale = 1 for CG)
    const double rn = sqrt(out[0]) * s->xinv;
    int done = 0;
    if (mode == 1) {
        if (O.r64) s->bnorm = sqrt(out[2]);  // CG: the starting residual kernel also reduced b
        s->r0 = rn;
    } else {
        done = s->cycles_next;
        s->iters += done;
        s->steps += 1;
    }
    s->rnorm = rn;
    if (!isfinite(rn)) stop_grid(s, 5);                                      // MG_EDIVERGED
    else if (s->bnorm == 0.0 || rn <= s->tol * s->bnorm) stop_grid(s, 0);   // converged
    else if (s->iters >= s->max_iters) stop_grid(s, 4);                      // MG_ENOTCONV
    if (s->active) {
        // V-cycles of the next refinement step: inner, or (adaptive, multigrid
        // iteration) the number the last step's per-cycle reduction rate g
        // needs to reach the tolerance, taken with a 10% margin on g
        // (FP32 logarithms: the estimate only picks a cycle count, and one
        // thread's FP64 transcendentals are a long chain on the FP64 pipe)
        int c = O.inner;
        if (mode == 2 && O.adaptive && !O.r64 && s->rprev > 0.0) {
            const float lr = logf((float)(rn / s->rprev)) / (float)done;  // log g
            if (lr < 0.0f && isfinite(lr)) {
                const float lge = fminf(logf(0.95f), logf(1.1f) + lr);      // log min(0.95, 1.1 g)
                const float need = ceilf(logf((float)(s->tol * s->bnorm / rn)) / lge);
                c = need < 1.0f ? 1 : (need < (float)O.inner ? (int)need : O.inner);
            }
        }
        const int left = s->max_iters - s->iters;  // >= 1 here
        s->cycles_next = c < left ? c : left;
    }
    s->rprev = rn;
}

// End of a solve: p = p - mean(p) (a zero right-hand side gives p = 0).  After
// an extended-precision solve p = ((p0 - mean) + p1 + p2) / xscale from the
// three-float iterate: the mean leaves the leading component first, so a
// constant carried by the iterate costs no accuracy in the FP64 result.
__global__ void __launch_bounds__(kThreads) k_final(const OuterView *__restrict__ ov,
                                                    const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    const int lb = blockIdx.x - start[e];
    const int ntiles = fine_blocks(O.n);
    const double m = s->xmean;
    const bool zero = s->bnorm == 0.0;
    const bool conv = xp_live(O);
    const double inv = conv ? 1.0 / s->xscale : 1.0;  // a power of 2: exact
    for (int tile = lb; tile < ntiles; tile += O.nblk) {
        const Tile t = fine_tile(O.n, tile, O.dxt, O.xy);
        if (!t.ok) continue;
        const long long rowoff = (long long)O.n[0] * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i >= O.n[0]) continue;
            const long long c = rowoff + i;
            double v;
            if (zero) v = 0.0;
            else if (conv) v = ((((double)O.xp3[0][c] - m) + (double)O.xp3[1][c]) + (double)O.xp3[2][c]) * inv;
            else v = O.p[c] - m;
            O.p[c] = v;
        }
    }
}

// Loop control of a graph-driven solve: keep iterating while any grid of the
// plan is still active.  Every grid stops after at most max_iters cycles, so
// the loop is bounded.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, const OuterView *__restrict__ ov, int count)
{
    dep_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned int any = 0;
    for (int g = 0; g < count; g++) any |= (unsigned int)(ov[g].st->active != 0);
    cudaGraphSetConditional(h, any);
}

// Start of a refinement step of a graph-driven solve: the step's V-cycles are
// the most any active grid of the plan asks for (switch branch c - 1).
__global__ void k_step_ctl(cudaGraphConditionalHandle h, const OuterView *__restrict__ ov, int count)
{
    dep_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 1;
    for (int g = 0; g < count; g++) {
        const GridState *s = ov[g].st;
        if (s->active && s->cycles_next > c) c = s->cycles_next;
    }
    cudaGraphSetConditional(h, (unsigned int)(c - 1));
}

// Copy the state of every grid of a plan into one contiguous array (one
// device-to-host copy then serves the whole batch).
__global__ void k_gather_states(const OuterView *__restrict__ ov, int count, GridState *out)
{
    dep_entry();
    for (int g = threadIdx.x; g < count; g += blockDim.x) out[g] = *ov[g].st;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

thread_local int tl_dep_launch = 0;

int dep_launch_default()
{
    static const int on = [] {
        const char *e = getenv("MG_DEP_LAUNCH");
        return (e && e[0] == '0') ? 0 : 1;
    }();
    return on;
}

void launch_gather_states(const OuterTable &ot, GridState *out, cudaStream_t s)
{
    launch_k(k_gather_states, 1, 128, 0, s, ot.ov, ot.count, out);
}

void launch_step_ctl(cudaGraphConditionalHandle h, const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_step_ctl, 1, 32, 0, s, h, ot.ov, ot.count);
}
void launch_loop_ctl(cudaGraphConditionalHandle h, const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_loop_ctl, 1, 32, 0, s, h, ot.ov, ot.count);
}

template <class T>
void launch_half_rows(const Table &tb, int colour, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    if (flags & kOuter)
        launch_k(k_half<T, true>, tb.blocks, kThreads, 0, s, tb.lv, tb.start, tb.count, colour, (T)omega, flags,
                 tb.cyc, ov, table_view(tb), table_single(tb));
    else
        launch_k(k_half<T, false>, tb.blocks, kThreads, 0, s, tb.lv, tb.start, tb.count, colour, (T)omega, flags,
                 tb.cyc, nullptr, table_view(tb), table_single(tb));
}
template <class T>
void launch_restrict_rows(const Table &tb, double omega, cudaStream_t s)
{
    launch_k(k_restrict<T>, tb.blocks, kThreads, 0, s, tb.lv, tb.start, tb.count, tb.cyc, (T)omega,
             table_view(tb), table_single(tb));
}
template <class T>
void launch_prolong_rows(const Table &tb, const OuterView *ov, cudaStream_t s)
{
    const int c = tb.cyc;
    const LevelView one = table_view(tb);
    const int single = table_single(tb);
    const dim3 g(tb.blocks), b(kThreads);
    if (tb.flux) {
        if (ov) launch_k(k_prolong<T, true, true>, g, b, 0, s, tb.lv, tb.start, tb.count, c, ov, one, single);
        else launch_k(k_prolong<T, true, false>, g, b, 0, s, tb.lv, tb.start, tb.count, c, nullptr, one, single);
    } else {
        if (ov) launch_k(k_prolong<T, false, true>, g, b, 0, s, tb.lv, tb.start, tb.count, c, ov, one, single);
        else launch_k(k_prolong<T, false, false>, g, b, 0, s, tb.lv, tb.start, tb.count, c, nullptr, one, single);
    }
}
template <class T>
void launch_tail(const TailView *tv, int count, size_t smem, double omega, int nu1, int nu2, int cyc,
                 cudaStream_t s)
{
    static size_t attr = 0;  // opt in to more than 48 KB of shared memory when needed
    if (smem > attr) {
        cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    launch_k(k_tail<T>, count, kTailThreads, smem, s, tv, (T)omega, nu1, nu2, cyc);
}
template <class T>
void launch_apply(const Table &tb, cudaStream_t s)
{
    launch_k(k_apply<T>, tb.blocks, kThreads, 0, s, tb.lv, tb.start, tb.count);
}
template <class T>
void launch_coarse_solve(const CoarseView *cv, int count, int cyc, const OuterView *ov, cudaStream_t s)
{
    launch_k(k_coarse_solve<T>, count, kThreads, 0, s, cv, cyc, ov);
}
void launch_coarse_setup(const CoarseView *cv, int count, cudaStream_t s)
{
    launch_k(k_coarse_setup, count, 1024, 0, s, cv);
}
static int cells_grid(long long N)
{
    long long b = (N + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}
void launch_faces_from_density(const FaceArgs &a, cudaStream_t s)
{
    FaceArgs b = a;
    b.dx = make_fastdiv((unsigned)a.n[0]);
    b.dy = make_fastdiv((unsigned)a.n[1]);
    launch_k(k_faces_from_density, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, b);
}
void launch_scale_faces(const FaceArgs &a, cudaStream_t s)
{
    launch_k(k_scale_faces, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, a);
}
void launch_cell_alpha(const AlphaArgs &a, cudaStream_t s)
{
    launch_k(k_cell_alpha, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, a);
}
void launch_divergence(const ProjArgs &a, cudaStream_t s)
{
    launch_k(k_divergence, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, a);
}
void launch_project(const ProjArgs &a, cudaStream_t s)
{
    launch_k(k_project, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, a);
}
void launch_diag_inv(const DiagArgs &a, cudaStream_t s)
{
    launch_k(k_diag_inv, cells_grid((long long)a.n[0] * a.n[1] * a.n[2]), kThreads, 0, s, a);
}
void launch_coarsen_faces(const CoarsenArgs &a, cudaStream_t s)
{
    launch_k(k_coarsen_faces, cells_grid((long long)a.nc[0] * a.nc[1] * a.nc[2]), kThreads, 0, s, a);
}
void launch_begin(const OuterView *ov, int count, cudaStream_t s) { launch_k(k_begin, count, 32, 0, s, ov); }
void launch_sum(const OuterTable &ot, int which, cudaStream_t s)
{
    launch_k(k_sum, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count, which);
}
template <class Te>
void launch_residual(const OuterTable &ot, int init, cudaStream_t s)
{
    launch_k(k_residual<Te>, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count, init);
}
void launch_center_rhs(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_center_rhs, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}
void launch_xp_prepare(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_xp_prepare, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}
void launch_residual_xp(const OuterTable &ot, int first, cudaStream_t s)
{
    launch_k(k_residual_xp, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count, first);
}
void launch_finalize(const OuterTable &ot, int mode, cudaStream_t s)
{
    launch_k(k_finalize, ot.count, kThreads, 0, s, ot.ov, mode);
}
void launch_final(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_final, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}

template void launch_half_rows<float>(const Table &, int, double, int, const OuterView *, cudaStream_t);
template void launch_half_rows<double>(const Table &, int, double, int, const OuterView *, cudaStream_t);
template void launch_restrict_rows<float>(const Table &, double, cudaStream_t);
template void launch_restrict_rows<double>(const Table &, double, cudaStream_t);
template void launch_prolong_rows<float>(const Table &, const OuterView *, cudaStream_t);
template void launch_prolong_rows<double>(const Table &, const OuterView *, cudaStream_t);
template void launch_tail<float>(const TailView *, int, size_t, double, int, int, int, cudaStream_t);
template void launch_tail<double>(const TailView *, int, size_t, double, int, int, int, cudaStream_t);
template void launch_apply<float>(const Table &, cudaStream_t);
template void launch_apply<double>(const Table &, cudaStream_t);
template void launch_coarse_solve<float>(const CoarseView *, int, int, const OuterView *, cudaStream_t);
template void launch_coarse_solve<double>(const CoarseView *, int, int, const OuterView *, cudaStream_t);
template void launch_residual<float>(const OuterTable &, int, cudaStream_t);
template void launch_residual<double>(const OuterTable &, int, cudaStream_t);

}  // namespace gbmg
