// mg_pcg.cu -- conjugate gradients preconditioned by V-cycles (MG_SOLVER_PCG).
//
// The pressure operator A of Eq. 10 (arXiv 1410.8568) is symmetric negative
// semidefinite with the constants as its null space; CG runs on the SPD
// operator -A on the zero-mean subspace.  The residual keeps the sign of the
// multigrid iteration, r = b0 - A p, and q = A d, so that
//   alpha = (r.z) / (d.q),  p += alpha d,  r -= alpha q,
//   beta = -alpha (z_new.q) / (r.z)_old  (Polak-Ribiere form: equal to the
//   classical one for a fixed symmetric preconditioner, and tolerant of the
//   FP32 V-cycle being a slightly variable one),
//   d = (z_new - mean z_new) + beta d,
// with z = M r the correction of inner_cycles V-cycles from zero.  Every
// vector of the outer iteration is FP64; the V-cycle runs in its own
// precision.  All sums are block partials reduced in a fixed order by one
// block per grid (deterministic, the same alone and in a batch).
#include "mg_kernels.h"
#include "mg_outer.cuh"
#include "mg_stencil.cuh"

#include <math.h>

namespace gbmg {

// Iterate over the finest-level cells owned by this block (row tiles, grid
// stride over tiles); f(c, i, j, k).
template <class F>
__device__ __forceinline__ void for_cells(const OuterView &O, int lb, F &&f)
{
    const int ntiles = fine_blocks(O.n);
    for (int tile = lb; tile < ntiles; tile += O.nblk) {
        const Tile t = fine_tile(O.n, tile, O.dxt, O.xy);
        if (!t.ok) continue;
        const long long rowoff = (long long)O.n[0] * t.row;
        for (int h = 0; h < 2; h++) {
            const int i = t.xbase + (threadIdx.x & 31) + 32 * h;
            if (i < O.n[0]) f(rowoff + i, i, t.j, t.k);
        }
    }
}

// q = A d (FP64, face differences first) and partial d.q (slot 0)
__global__ void __launch_bounds__(kThreads) k_pcg_matvec(const OuterView *__restrict__ ov,
                                                         const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    if (!O.st->active) return;
    const int lb = blockIdx.x - start[e];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for_cells(O, lb, [&](long long c, int i, int j, int k) {
        const double qc = flux64(O, O.d, i, j, k, c);
        O.q[c] = qc;
        v[0] += O.d[c] * qc;
    });
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) O.part[kPart * lb + 0] = out[0];
}

// p += alpha d, r -= alpha q, the V-cycle's right-hand side = r in its
// precision Te, partial ||r||^2 (slot 0, FP64)
template <class Te>
__global__ void __launch_bounds__(kThreads) k_pcg_update(const OuterView *__restrict__ ov,
                                                         const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    if (!s->active) return;
    const int lb = blockIdx.x - start[e];
    const double a = s->alpha;
    Te *rv = (Te *)O.r;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for_cells(O, lb, [&](long long c, int, int, int) {
        O.p[c] += a * O.d[c];
        const double r = O.r64[c] - a * O.q[c];
        O.r64[c] = r;
        rv[c] = (Te)r;
        v[0] += r * r;
    });
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0) O.part[kPart * lb + 0] = out[0];
}

// z = the V-cycle correction (FP64); partials z.q (slot 0), r.z (slot 1),
// sum z (slot 2)
template <class Te>
__global__ void __launch_bounds__(kThreads) k_pcg_z(const OuterView *__restrict__ ov,
                                                    const int *__restrict__ start, int count)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    if (!O.st->active) return;
    const int lb = blockIdx.x - start[e];
    const Te *ev = (const Te *)O.e;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for_cells(O, lb, [&](long long c, int, int, int) {
        const double z = (double)ev[c];
        O.z[c] = z;
        v[0] += z * O.q[c];
        v[1] += O.r64[c] * z;
        v[2] += z;
    });
    double out[4];
    block_sum4(v, out);
    if (threadIdx.x == 0)
        for (int f = 0; f < 3; f++) O.part[kPart * lb + f] = out[f];
}

// d = (z - mean z) + beta d (first: d = z - mean z)
__global__ void __launch_bounds__(kThreads) k_pcg_dir(const OuterView *__restrict__ ov,
                                                      const int *__restrict__ start, int count, int first)
{
    dep_entry();
    const int e = find_entry(start, count);
    const OuterView O = ov[e];
    const GridState *s = O.st;
    if (!s->active) return;
    const int lb = blockIdx.x - start[e];
    const double m = s->zmean, b = s->beta;
    for_cells(O, lb, [&](long long c, int, int, int) {
        const double z = O.z[c] - m;
        O.d[c] = first ? z : z + b * O.d[c];
    });
}

// One block per grid: reduce the partials in a fixed order and update the
// scalars.  mode 0: after the first preconditioning (rz, mean z, beta = 0);
// mode 1: after the product A d (alpha; d.q must be negative, else the
// iteration broke down and the grid stops as diverged); mode 2: after a
// later preconditioning (beta, rz, mean z).
__global__ void __launch_bounds__(kThreads) k_pcg_finalize(const OuterView *__restrict__ ov, int mode)
{
    dep_entry();
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
    if (mode == 1) {
        const double dq = out[0];
        const double a = s->rz / dq;
        if (!(dq < 0.0) || !isfinite(a)) {
            stop_grid(s, 5);  // MG_EDIVERGED
            return;
        }
        s->alpha = a;
        return;
    }
    s->beta = mode == 0 ? 0.0 : -s->alpha * out[0] / s->rz;
    s->rz = out[1];
    s->zmean = out[2] / N;
    if (!isfinite(s->beta) || !isfinite(s->rz)) stop_grid(s, 5);
}

void launch_pcg_matvec(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_pcg_matvec, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}
template <class Te>
void launch_pcg_update(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_pcg_update<Te>, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}
template <class Te>
void launch_pcg_z(const OuterTable &ot, cudaStream_t s)
{
    launch_k(k_pcg_z<Te>, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count);
}
void launch_pcg_dir(const OuterTable &ot, int first, cudaStream_t s)
{
    launch_k(k_pcg_dir, ot.blocks, kThreads, 0, s, ot.ov, ot.start, ot.count, first);
}
void launch_pcg_finalize(const OuterTable &ot, int mode, cudaStream_t s)
{
    launch_k(k_pcg_finalize, ot.count, kThreads, 0, s, ot.ov, mode);
}

template void launch_pcg_update<float>(const OuterTable &, cudaStream_t);
template void launch_pcg_update<double>(const OuterTable &, cudaStream_t);
template void launch_pcg_z<float>(const OuterTable &, cudaStream_t);
template void launch_pcg_z<double>(const OuterTable &, cudaStream_t);

}  // namespace gbmg
