// mg_device.cuh -- data structures shared by the host driver and the kernels of
// the variable-density pressure multigrid (arXiv 1410.8568, Sec. 2.3).
//
// Every V-cycle kernel works on a TABLE of level views: one entry per grid of
// a batch.  A launch covers the blocks of all entries back to back; a block
// finds its entry by binary search in the prefix array `start`.  A single
// solve is a table of one entry, so a grid's arithmetic does not depend on
// what else is in the launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_launch.cuh"

namespace gbmg {

constexpr int kThreads = 256;     // threads per block of every cell kernel
constexpr int kRowsPerBlock = 8;  // one grid row (fixed j, k) per warp
constexpr int kSeg = 64;          // x extent of a warp's row segment (2 cells per lane)
constexpr int kCSeg = 32;         // x extent of a warp's coarse row segment (restriction)
constexpr int kMaxCoarse = 512;   // most cells of the coarsest grid (dense inverse)
constexpr int kMaxCoarseGmres = 32768;  // most cells of a coarsest grid solved by GMRES
constexpr int kGmresM = 30;       // Krylov vectors per GMRES cycle
constexpr int kPart = 4;          // doubles of reduction partials per block
constexpr int kOuterCap = 608;    // most blocks of one grid in an outer (FP64) launch: 4 per SM


// Per-grid solve state, in device memory, written only by kernels.
struct GridState {
    double tol;
    double bmean;   // mean of the right-hand side (removed)
    double bnorm;   // ||b - bmean||_2
    double r0;      // R_0 of Eq. 15
    double rnorm;   // current ||r||_2
    double xmean;   // mean of the current iterate
    int max_iters;
    int iters;      // completed V-cycles
    int status;     // gbmg status code
    int active;     // 1 while the grid is being iterated
    int cycles_next;  // V-cycles of the next refinement step (1 .. inner)
    int steps;        // refinement steps done
    int pnz;          // the caller's starting iterate has a nonzero cell (multigrid iteration)
    double rprev;     // ||r|| before the last refinement step
    double rz;      // conjugate gradients: r . z of the current step
    double alpha;   //   step length
    double beta;    //   direction update
    double zmean;   //   mean of the preconditioned residual
    double xscale;  // multigrid iteration: the cycles see r * xscale, a power of 2 near 1 / rms(b - mean b)
    double xinv;    //   1 / xscale
};

// A grid takes part in V-cycle `cyc` (0-based) of the current refinement step
// while its step asks for more than cyc cycles.  A batch runs as many cycles as
// its most demanding grid and the others sit the extra ones out, so every grid
// gets exactly its own arithmetic, alone or batched.  A grid that stopped has
// cycles_next = 0 (every kernel that clears `active` also clears it), so the
// test is one load at the head of every V-cycle kernel.
__device__ __forceinline__ bool in_cycle(const GridState *s, int cyc) { return cyc < s->cycles_next; }

// Stop a grid's iteration with the given status.
__device__ __forceinline__ void stop_grid(GridState *s, int status)
{
    s->status = status;
    s->active = 0;
    s->cycles_next = 0;
}
// V-cycle `cyc` is the last of the grid's current refinement step.
__device__ __forceinline__ bool last_cycle(const GridState *s, int cyc) { return cyc + 1 == s->cycles_next; }

// Division by a fixed divisor d >= 1 of numerators n < 2^31 by one multiply
// and a shift (Granlund & Montgomery, PLDI 1994, round-up variant): with
// l = ceil(log2 d), m = floor(2^(32+l) / d) + 1, floor(n / d) = (n m) >> (32+l).
// m overestimates 2^(32+l)/d by at most 1, so the error term n / 2^(32+l) is
// below 1/(2d) for n < 2^31 and never carries the quotient past an integer.
struct FastDiv {
    unsigned long long m;
    int s;
};

inline FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while ((1ull << l) < d) l++;
    FastDiv f;
    f.s = 32 + l;
    f.m = ((1ull << f.s) / d) + 1;
    return f;
}

__host__ __device__ __forceinline__ int fdiv(int n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    // 32 x 33-bit product: m = 2^32 mh + ml, mh in {0, 1}
    const unsigned ml = (unsigned)f.m, mh = (unsigned)(f.m >> 32);
    const unsigned long long p = (unsigned long long)(unsigned)n * ml + ((unsigned long long)(mh * (unsigned)n) << 32);
    return (int)(p >> f.s);
#else
    return (int)(((unsigned __int128)(unsigned)n * f.m) >> f.s);
#endif
}

// Launch shapes of the half-sweep, restriction and prolongation kernels
// (chosen per level by the autotuner).  Variant 0 is the row tiling: a warp
// owns one grid row of up to 32 quads (or 64 cells), 8 rows per 256-thread
// block.  Variants 1.. are flat tilings for rows of a multiple of 4 cells: the
// level's quads (restriction and prolongation: coarse cell pairs, a pair
// covering one quad in each of the 2 x 2 fine rows above it) are numbered row
// by row and a block of B threads owns Q * B consecutive ones, thread t the items t, t + B,
// ...; short rows then fill whole warps, and B and Q set the blocks per SM and
// the loads each thread has in flight.
constexpr int kTileVariants = 7;
struct TileShape {
    int B, Q;
};
__host__ __device__ constexpr TileShape tile_shape(int v)
{
    return v == 1 ? TileShape{64, 1}
         : v == 2 ? TileShape{128, 1}
         : v == 3 ? TileShape{128, 2}
         : v == 4 ? TileShape{256, 1}
         : v == 5 ? TileShape{256, 2}
         : v == 6 ? TileShape{512, 1}
                  : TileShape{kThreads, 1};
}

// Launch shapes of the one-pass red-black sweep: B threads per block and Kc
// planes per block (a chunk of the z march).  Variants 1 .. 6 (mg_fused.cu):
// a block owns a strip of full rows, a thread per quad of each row of the
// strip (2 halo rows included).  Variants 7 .. 10 (mg_staged.cu, FP32 cycles):
// a block owns a tile of tile_x = 128 cells of up to 14 rows and stages its
// operands in shared memory.  Variant 0 is no one-pass sweep (two half-sweep
// launches per sweep).
constexpr int kSweepVariants = 11;
struct SweepShape {
    int B, Kc, tile_x;  // tile_x: cells of a block's tile along x, 0 for whole rows
};
__host__ __device__ constexpr SweepShape sweep_shape(int v)
{
    return v == 1  ? SweepShape{1024, 16, 0}
         : v == 2  ? SweepShape{1024, 32, 0}
         : v == 3  ? SweepShape{1024, 64, 0}
         : v == 4  ? SweepShape{512, 16, 0}
         : v == 5  ? SweepShape{512, 32, 0}
         : v == 6  ? SweepShape{512, 64, 0}
         : v == 7  ? SweepShape{544, 64, 128}
         : v == 8  ? SweepShape{544, 128, 128}
         : v == 9  ? SweepShape{544, 512, 128}
         : v == 10 ? SweepShape{544, 1024, 128}
                   : SweepShape{0, 0, 0};
}

// One level of one grid as seen by the V-cycle kernels (precision T is fixed
// by the kernel instantiation; pointers are typeless here).
struct LevelView {
    int n[3];
    int per;        // bit d set: axis d periodic
    void *w[3];     // scaled face coefficients alpha / h^2 (low face of each cell)
    void *x;        // iterate / correction
    void *b;        // right-hand side
    void *xc;       // next coarser level: its final correction (null at the coarsest)
    void *bc;       // next coarser level: right-hand side
    int nc[3];
    int g;          // index of the grid in its plan (selects its OuterView)
    const GridState *st;
    // flat tilings: quads per fine row n[0]/4, fine rows per plane n[1],
    // coarse cell pairs per coarse row nc[0]/2, coarse rows per plane nc[1]
    FastDiv dq, dy, dp, dcy;
    // row-tiled kernels: division by the block columns of a row, for quad rows
    // ((n[0]/4 + 31) / 32), coarse pair rows ((nc[0]/2 + 31) / 32), coarse cell
    // rows (coarse_xtiles(nc[0])) and fine cell rows (fine_xtiles(n[0]))
    FastDiv dxq, dxp, dxc, dxt;
    const void *ac;  // cell coefficients of the next coarser level (flux-conserving prolongation)
    // restriction: also give the next coarser level its first (zero-start) red
    // half-sweep, from the restricted right-hand side and that level's faces wc
    int zr;
    const void *wc[3];
    // one-pass red-black sweep (finest level): the second iterate buffer (a
    // sweep reads one and writes the other), rows per strip, planes per chunk,
    // strips per plane, and division by the strips and by the quads per row
    void *x2;
    int fR, fKc, fS;
    FastDiv dfS, dfq;
    // FP64 cycles: inverse diagonals (1 / sum of the cell's face coefficients,
    // 0 for a cell without faces) of this level and of the next coarser one;
    // null in FP32 cycles (and for FP64 unit calls on a mixed-precision handle)
    const void *dinv;
    const void *dinvc;
};

// The finest level of one grid for the FP64 outer iteration.
struct OuterView {
    int n[3];
    int per;
    const double *w[3];  // FP64 scaled faces of level 0
    const double *b;     // caller's right-hand side
    double *p;           // caller's iterate / solution
    double *b0;          // right-hand side minus its mean, FP64 (library buffer)
    void *r;             // level-0 right-hand side of the V-cycle (V-cycle precision)
    double *part;        // kPart doubles per block of this grid's outer launches
    int nblk;            // blocks of this grid in an outer launch
    GridState *st;
    double tol;
    int max_iters;
    int inner;           // V-cycles per refinement step
    // conjugate gradients (null otherwise): FP64 residual, preconditioned
    // residual, direction, A times direction; e = the V-cycle's level-0
    // correction (V-cycle precision)
    double *r64, *z, *d, *q;
    const void *e;
    int adaptive;        // choose the V-cycles of each refinement step from the measured rate
    // extended-precision outer iteration (mixed-precision multigrid iteration,
    // mg_xprec.cuh): iterate p * xscale = xp[0] + xp[1] + xp[2], right-hand
    // side (b - mean b) * xscale = xb[0] + xb[1], level-0 faces w32[d] + wlo[d]
    int xp;
    FastDiv xq, xy;      // division by the quads per row n[0] / 4 and by n[1]
    FastDiv dxt;         // division by the row tiles of a row, fine_xtiles(n[0])
    float *xp3[3];
    float *xb[2];
    const float *w32[3];
    const float *wlo[3];
};

// Where a kernel adds the final correction of a refinement step: the FP64
// iterate (FP64 cycles) or the three-float iterate (FP32 cycles).
struct OuterOut {
    double *p;
    float *t[3];
    double inv;  // FP64 iterate: p += e * inv (the cycles work in the scaled units)
};
__device__ __forceinline__ OuterOut outer_out(const OuterView &O)
{
    OuterOut o;
    o.p = O.p;
    for (int q = 0; q < 3; q++) o.t[q] = O.xp3[q];
    o.inv = O.st->xinv;
    return o;
}

// The coarsest level of one grid.
struct CoarseView {
    int n[3];
    int per;
    int nc;              // cells
    double *G;           // nc x nc inverse of (-A + c 1 1^T), FP64
    const double *w[3];  // FP64 scaled faces of the coarsest level (set-up only)
    void *x;             // solution (V-cycle precision)
    const void *b;       // right-hand side (V-cycle precision)
    const GridState *st;
    int *err;            // set-up error flag (non-positive pivot)
    int g;               // index of the grid in its plan
    int outer;           // 1 if this is also the finest level (p += e happens here)
    int gmres;           // 1: solved by restarted GMRES (G unused)
    double *gm;          // GMRES scratch: b, e, w, then kGmresM + 1 Krylov vectors (FP64, nc each)
    int gm_max;          // most Arnoldi steps
    double gm_tol;       // relative residual
};

// Bottom of the V-cycle in one block per grid (levels of at most kTailCells
// cells, shared memory resident).
constexpr int kTailCells = 4096;
constexpr int kTailThreads = 512;
constexpr int kMaxTail = 8;

struct TailView {
    int nt;                  // tail levels: the first one down to the coarsest
    int per;
    int n[kMaxTail][3];
    int off[kMaxTail];       // element offset of level t's x, b, wx, wy, wz (N each) in shared memory
    void *w[kMaxTail][3];    // scaled faces of each tail level (V-cycle precision)
    void *x0;                // first tail level: correction (out)
    void *b0;                // first tail level: right-hand side (in)
    const double *G;         // coarsest-level inverse
    const GridState *st;
    FastDiv dx[kMaxTail], dhx[kMaxTail], dy[kMaxTail];  // division by n[t][0], n[t][0] / 2, n[t][1]
    FastDiv dq[kMaxTail];    // division by n[t][0] / 4 (quads per row)
    int *err;                // set to 1 when the staging copies did not complete in time
    long long wait_polls;    // polls of the staging wait before it gives up (kBulkWaitPolls by default)
    int flux;                // flux-conserving prolongation: level t >= 1 also holds its cell
    const void *a[kMaxTail]; //   coefficients (6th array of the level in shared memory)
};

// Blocks of a launch over the cells of an n[0] x n[1] x n[2] level: a block is
// 8 rows, each row split in segments of 64 cells along x.
__host__ __device__ inline int fine_xtiles(int nx) { return (nx + kSeg - 1) / kSeg; }
__host__ __device__ inline int fine_blocks(const int n[3])
{
    return fine_xtiles(n[0]) * ((n[1] * n[2] + kRowsPerBlock - 1) / kRowsPerBlock);
}
// Outer (FP64) launches: at most kOuterCap blocks per grid, grid-stride over tiles.
__host__ __device__ inline int outer_blocks(const int n[3])
{
    const int t = fine_blocks(n);
    return t < kOuterCap ? t : kOuterCap;
}
// Blocks of a launch over the cells of a coarse level (32 coarse cells per warp row).
__host__ __device__ inline int coarse_xtiles(int nx) { return (nx + kCSeg - 1) / kCSeg; }
__host__ __device__ inline int coarse_blocks(const int n[3])
{
    return coarse_xtiles(n[0]) * ((n[1] * n[2] + kRowsPerBlock - 1) / kRowsPerBlock);
}

}  // namespace gbmg
