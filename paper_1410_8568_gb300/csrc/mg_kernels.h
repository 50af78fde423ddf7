// mg_kernels.h -- host-side launchers of the multigrid kernels (mg_kernels.cu).
#pragma once

#include "mg_device.cuh"

namespace gbmg {

// A launch table: `count` views in device memory and the prefix `start`
// (count + 1 entries) of their block ranges; `blocks` = start[count].
struct Table {
    const LevelView *lv;
    const int *start;
    int count;
    int blocks;
    int variant = 0;  // launch shape (tile_shape); 0 = row tiles
    int flux = 0;     // prolongation tables: flux-conserving (row tiles only)
    int cyc = 0;      // V-cycle of the refinement step: grids asking fewer cycles skip the launch
    const LevelView *hv = nullptr;  // host copy of the view of a one-grid table: passed by value
};

// the by-value view of a one-grid table (kernel parameter space), else zeros
inline int table_single(const Table &tb) { return (tb.hv != nullptr && tb.count == 1) ? 1 : 0; }
inline LevelView table_view(const Table &tb) { return table_single(tb) ? *tb.hv : LevelView{}; }

struct OuterTable {
    const OuterView *ov;
    const int *start;
    int count;
    int blocks;
};

// density -> faces, or caller faces -> scaled faces: out_d = scale_d * face_d
struct FaceArgs {
    int n[3];
    int per;
    int mode;                // 0 harmonic (Eqs. 11-12), 1 arithmetic
    const double *rho;       // density (faces_from_density)
    const double *in[3];     // caller faces (scale_faces)
    double scale[3];         // 1 for raw alpha, 1/h_d^2 for level-0 coefficients
    double *out64[3];
    float *out32[3];         // optional FP32 copy (round to nearest)
    float *out32lo[3];       // optional: out64 - out32 rounded to FP32 (float-pair faces)
    FastDiv dx, dy;          // division by n[0], n[1] (set by the launcher)
    int *err;                // set to 1 on a non-positive / non-finite value
};

// cell coefficient of the flux-conserving prolongation: mean over the cell's
// non-wall faces of alpha = w h_d^2 (w the scaled FP64 face coefficients)
struct AlphaArgs {
    int n[3];
    int per;
    double h2[3];
    const double *w[3];
    float *out32;   // optional
    double *out64;  // optional
};

// projection step around the solve (MAC grid, low-face layout of the velocity)
struct ProjArgs {
    int n[3];
    int per;
    double h[3];
    double dt;
    const double *w[3];   // scaled FP64 faces alpha / h^2 of level 0 (project)
    const double *p;      // pressure (project)
    double *u[3];         // face velocities (divergence: read; project: updated)
    double *S;            // divergence / dt (divergence: written)
};

// inverse diagonal of a level for the FP64 relaxation: out = 1 / d, d the sum
// of the cell's face coefficients (relax_cell's order), 0 where d <= 0
struct DiagArgs {
    int n[3];
    int per;
    const double *w[3];  // scaled FP64 faces of the level
    double *out;
    FastDiv dx, dy;      // division by n[0] and by n[1]
};

struct CoarsenArgs {
    int nf[3];
    int nc[3];
    const double *wf[3];
    double *wc[3];
    float *wc32[3];
    FastDiv dx, dy;  // division by nc[0] and by nc[1]
};

// red-black half-sweep of one colour; flags: 1 zero initial iterate (red
// launch), 4 the grids whose refinement step ends with this cycle add the
// relaxed values to their FP64 iterate (finest level, last post-sweep)
constexpr int kHalfZero = 1, kHalfOuter = 4;
int half_sweep_blocks(const int n[3]);
int restrict_blocks(const int n[3], const int nc[3]);
int prolong_blocks(const int n[3]);
// the same for launch shape v (mg_tiles.cu); v > 0 needs n[0] % 4 == 0
bool tile_fits(const int n[3], int v);
int half_sweep_blocks_v(const int n[3], int v);
int restrict_blocks_v(const int n[3], const int nc[3], int v);
int prolong_blocks_v(const int n[3], const int nc[3], int v);
// launchers that dispatch on Table::variant (mg_tiles.cu) ...
// ov: the plan's outer views where the launch may update the FP64 iterate
// (kHalfOuter; prolongation and coarse solve of the finest level), else null
template <class T> void launch_half(const Table &, int colour, double omega, int flags,
                                    const OuterView *ov, cudaStream_t);
// restriction; omega: the coarse level's zero-start red half-sweep where the view asks (zr)
template <class T> void launch_restrict(const Table &, double omega, cudaStream_t);
template <class T> void launch_prolong(const Table &, const OuterView *ov, cudaStream_t);
// ... and the row-tiled kernels they fall back to (mg_kernels.cu)
template <class T> void launch_half_rows(const Table &, int colour, double omega, int flags,
                                         const OuterView *ov, cudaStream_t);
template <class T> void launch_restrict_rows(const Table &, double omega, cudaStream_t);
template <class T> void launch_prolong_rows(const Table &, const OuterView *ov, cudaStream_t);
// one-pass red-black sweep (mg_fused.cu, and mg_staged.cu for the staged
// shapes): shape v fits a level with n cells per axis and periodic bits per in
// FP32 (fp32) or FP64 cycles; sweep_layout fills the view's strip and chunk
// fields for shape v and returns the blocks of the grid; a launch reads the
// iterate from x (dir 0) or x2 (dir 1) and writes the other buffer; flags as
// for the half-sweep (kHalfZero, kHalfOuter)
bool sweep_fits(const int n[3], int per, int v, bool fp32);
bool staged_fits(const int n[3], int per);
int staged_layout(LevelView &v, int kc);
void launch_sweep_staged(const Table &, int dir, double omega, int flags, const OuterView *ov, cudaStream_t);
int sweep_layout(LevelView &v, int variant);
int sweep_blocks(const int n[3], int variant);
template <class T> void launch_sweep(const Table &, int dir, double omega, int flags, const OuterView *ov,
                                     cudaStream_t);
// V-cycle stages below the row-tiled levels; cyc as Table::cyc
template <class T> void launch_tail(const TailView *, int count, size_t smem, double omega, int nu1,
                                    int nu2, int cyc, cudaStream_t);
template <class T> void launch_apply(const Table &, cudaStream_t);
template <class T> void launch_coarse_solve(const CoarseView *, int count, int cyc, const OuterView *ov,
                                            cudaStream_t);
template <class T> void launch_coarse_gmres(const CoarseView *, int count, int cyc, const OuterView *ov,
                                            cudaStream_t);
void launch_coarse_setup(const CoarseView *, int count, cudaStream_t);
void launch_faces_from_density(const FaceArgs &, cudaStream_t);
void launch_scale_faces(const FaceArgs &, cudaStream_t);
void launch_coarsen_faces(const CoarsenArgs &, cudaStream_t);
void launch_diag_inv(const DiagArgs &, cudaStream_t);
void launch_cell_alpha(const AlphaArgs &, cudaStream_t);
void launch_divergence(const ProjArgs &, cudaStream_t);
void launch_project(const ProjArgs &, cudaStream_t);
void launch_begin(const OuterView *, int count, cudaStream_t);
void launch_sum(const OuterTable &, int which, cudaStream_t);
// init: 0 after a refinement step, 1 start of a CG solve, 2 start of a multigrid
// iteration (a zero starting iterate gives r = b - mean b without A p)
template <class Te> void launch_residual(const OuterTable &, int init, cudaStream_t);
// multigrid iteration: b - mean b and its norm (sets the cycles' scale);
// extended-precision outer iteration: the scaled float forms of b and p, the residual
void launch_center_rhs(const OuterTable &, cudaStream_t);
void launch_xp_prepare(const OuterTable &, cudaStream_t);
void launch_residual_xp(const OuterTable &, int first, cudaStream_t);
void launch_finalize(const OuterTable &, int mode, cudaStream_t);
void launch_final(const OuterTable &, cudaStream_t);
void launch_gather_states(const OuterTable &, GridState *out, cudaStream_t);
// conjugate gradients (mg_pcg.cu)
void launch_pcg_matvec(const OuterTable &, cudaStream_t);
template <class Te> void launch_pcg_update(const OuterTable &, cudaStream_t);
template <class Te> void launch_pcg_z(const OuterTable &, cudaStream_t);
void launch_pcg_dir(const OuterTable &, int first, cudaStream_t);
void launch_pcg_finalize(const OuterTable &, int mode, cudaStream_t);
void launch_loop_ctl(cudaGraphConditionalHandle, const OuterTable &, cudaStream_t);
void launch_step_ctl(cudaGraphConditionalHandle, const OuterTable &, cudaStream_t);

}  // namespace gbmg
