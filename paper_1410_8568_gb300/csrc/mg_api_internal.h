// mg_api_internal.h -- host-side structures of the multigrid library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gbmg.h"
#include "mg_kernels.h"
#include "mg_bulk.cuh"

namespace gbmg {

void note_cuda_error(cudaError_t e);
cudaError_t last_cuda_error();

// Bump allocator of offsets inside one device slab (256-byte aligned pieces).
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes);
};

int make_levels(const mg_grid &g, int n[][3], int *L);
int check_grid(const mg_grid *g);
int check_params(const mg_params *p);

// One level of a handle's hierarchy.
struct HLevel {
    int n[3];
    long long N;
    double h[3];
    double *w64[3];  // alpha / h^2, FP64
    float *w32[3];   // FP32 copy (mixed precision only)
    void *x;         // V-cycle iterate / correction (V-cycle precision)
    void *x2;        // finest level: second iterate buffer of the one-pass sweep (or null)
    void *b;         // V-cycle right-hand side (V-cycle precision)
    double *dinv;    // FP64 cycles: inverse diagonal 1 / (sum of the cell's faces), levels below the coarsest
    double *alpha64; // cell coefficients (flux-conserving prolongation, levels >= 1), FP64
    float *alpha32;  // FP32 copy (mixed precision only)
};

// CUDA-event timing of kernel classes (host-driven solves only).
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    int cur_kind = 0, cur_level = 0;
    struct Pending {
        int kind, level, ev;
    };
    std::vector<Pending> pending;
    double total_ms[MG_K_KINDS][MG_MAX_LEVELS] = {};
    int64_t launches[MG_K_KINDS][MG_MAX_LEVELS] = {};
    void begin(cudaStream_t s, int kind, int level);
    void end(cudaStream_t s);
    void collect();
    void reset();
    ~Prof();
};

struct Plan;

}  // namespace gbmg

struct mg_handle {
    mg_grid g;
    mg_params prm;
    cudaStream_t stream = nullptr;
    int device = 0;
    int per = 0;
    bool mixed = true;
    int L = 0;
    gbmg::HLevel lev[MG_MAX_LEVELS];
    double *G = nullptr;       // coarsest-grid inverse
    double *b0 = nullptr;      // right-hand side minus its mean (FP64)
    double *part = nullptr;    // reduction partials of the outer launches
    int nblk0 = 0;
    int *err = nullptr;        // [0] bad coefficient, [1] singular coarsest grid, [2] device wait gave up
    gbmg::GridState *state = nullptr;    // solve state of this grid (kept across plans)
    gbmg::GridState *dstate = nullptr;   // always-active state of the unit calls
    gbmg::LevelView *dview = nullptr;    // view slot of the unit calls
    int *dstart = nullptr;
    gbmg::CoarseView *dcview = nullptr;
    gbmg::CoarseView *setup_cv = nullptr;  // coarsest level, for building its inverse
    char *slab = nullptr;
    size_t bytes = 0;
    gbmg::Plan *plan = nullptr;          // single-grid launch plan
    gbmg::Prof prof;
    double *io_rhs = nullptr, *io_p = nullptr, *io_rho = nullptr;  // host-call staging
    cudaStream_t io_stream = nullptr;  // host-call input copies that overlap the face set-up
    cudaEvent_t io_ready = nullptr;
    signed char tile[4][MG_MAX_LEVELS] = {};  // launch shape per kernel (MG_TILE_*) and level
    double *pcg[4] = {nullptr, nullptr, nullptr, nullptr};  // CG: r, z, d, q (FP64, finest level)
    bool gmres = false;        // coarsest grid solved by GMRES (no dense inverse)
    double *gm = nullptr;      // GMRES scratch
    // extended-precision outer iteration (mixed precision, multigrid iteration):
    // three-float iterate, float-pair right-hand side, low parts of the level-0 faces
    bool xp = false;
    float *xp3[3] = {nullptr, nullptr, nullptr};
    float *xb[2] = {nullptr, nullptr};
    float *wlo[3] = {nullptr, nullptr, nullptr};
    long long wait_polls = gbmg::kBulkWaitPolls;  // first staging wait of the tail kernel (mg_set_wait_limit)
};

namespace gbmg {

// Launch tables over one or more handles plus the per-solve state.
struct Plan {
    std::vector<mg_handle *> hs;
    int G = 0;
    int Lmax = 0;
    bool mixed = true;
    bool xp = false;  // extended-precision outer iteration (every handle of a plan shares its params)
    // optional device-to-host copy enqueued after the solve and before its final
    // synchronisation (the host-buffer calls: one round trip instead of two)
    void *post_dst = nullptr;
    const void *post_src = nullptr;
    size_t post_bytes = 0;
    mg_params prm;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    char *mem = nullptr;
    Table down[MG_MAX_LEVELS];  // prolongation (fine tiles of level l)
    Table rest[MG_MAX_LEVELS];  // restriction (coarse tiles of level l+1)
    Table half[MG_MAX_LEVELS];  // red-black half-sweeps of level l
    Table sweep0;               // one-pass sweeps of the finest level (count 0: half-sweeps)
    CoarseView *cv = nullptr;   // coarsest solves of the grids without a tail
    int ncv = 0;
    bool cv_dense = false, cv_gmres = false;  // which coarse kernels the cv table needs
    TailView *tv = nullptr;     // bottom-of-cycle blocks of the grids with a tail
    int ntv = 0;
    size_t tail_smem = 0;
    OuterView *ov = nullptr;
    OuterTable ot;
    GridState *st = nullptr;    // gathered copy of the grids' states (device)
    OuterView *ov_h = nullptr;  // pinned host mirror of ov
    GridState *st_h = nullptr;  // pinned host mirror of st
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEvent_t staged = nullptr;  // the last table copy out of stage_h has run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // launches of this plan may be scheduled while the previous kernel runs
    // (programmatic dependent launch, mg_launch.cuh); cleared if a graph with
    // such edges is not accepted
    int dep = dep_launch_default();
    int capacity = 0;              // most grids the tables can hold
    char *stage_h = nullptr;       // pinned host copy of the table region of mem
    size_t tables_bytes = 0, o_lv = 0, o_starts = 0, o_cv = 0, o_tv = 0;
    int alloc(int cap);                                  // allocate once for up to cap grids
    int fill(mg_handle *const *handles, int count);      // rewrite the tables (async, no allocation)
    int build(mg_handle *const *handles, int count);     // alloc(count) + fill + wait
    void release();
};

int run_plan(Plan &P, Prof &pf, const double *const *rhs, double *const *p, const double *tol,
             mg_stats *out);

// Pieces of a solve, for the serving loop (host-driven, no graph):
// set the caller pointers of grid g of the plan (host mirror only)
void plan_bind(Plan &P, int g, const double *rhs, double *p, double tol, int max_iters);
// upload the host mirror of the outer views
int plan_upload(Plan &P);
// start of a solve for every grid of the plan (state reset, mean of b, R_0)
int plan_prologue(Plan &P);
// one V-cycle + FP64 update for every active grid of the plan
int plan_body(Plan &P);
// p = x - mean(x) for every grid of the plan
int plan_final(Plan &P);
// states of all grids of the plan into P.st_h (synchronises the stream)
int plan_sync_states(Plan &P);
// the same, enqueued on the plan's stream only (valid once the stream reaches it)
int plan_gather_states(Plan &P);
// autotuner (mg_tune.cu): launch shapes of h's levels into h->tile
int tune_handle(mg_handle *h);
void tune_cache_clear();
int first_tail_level(const mg_handle *h);
void fill_fastdiv(LevelView &v);
int kernel_blocks(int kind, const int n[3], const int nc[3], int v);
// allocate a handle (no coefficients yet) / set its coefficients (async)
int handle_alloc(const mg_grid *grid, const mg_params *params, void *stream, mg_handle **out);
int set_faces_impl(mg_handle *h, const double *ax, const double *ay, const double *az);
void fill_stats(const GridState &s, const int herr[3], double ms, mg_stats *o, int *status);

}  // namespace gbmg
