// mg_api.cu -- C ABI of the GB300 pressure multigrid (include/gbmg.h).
//
// A handle owns the hierarchy of one grid; a Plan holds the launch tables of
// one or more handles (a single solve is a plan of one grid, a batch a plan of
// many) and runs the FP64 outer iteration of Sec. 2.3 of arXiv 1410.8568 with
// the V-cycle either as a host-driven loop or as one CUDA-graph launch whose
// loop is a device-side conditional `while` node.
#include "gbmg.h"
#include "mg_api_internal.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

using namespace gbmg;

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) {                      \
            gbmg::note_cuda_error(e_);                \
            return MG_ECUDA;                          \
        }                                             \
    } while (0)

namespace gbmg {

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void note_cuda_error(cudaError_t e) { g_last_cuda = e; }
cudaError_t last_cuda_error() { return g_last_cuda; }

size_t Carve::take(size_t bytes)
{
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
}

int make_levels(const mg_grid &g, int n[][3], int *L)
{
    n[0][0] = g.nx;
    n[0][1] = g.ny;
    n[0][2] = g.nz;
    int l = 1;
    while (l < MG_MAX_LEVELS) {
        const int *p = n[l - 1];
        bool ok = true;
        for (int d = 0; d < 3; d++)
            if (p[d] % 2 != 0 || p[d] <= 2) ok = false;
        if (!ok) break;
        for (int d = 0; d < 3; d++) n[l][d] = p[d] / 2;
        l++;
    }
    *L = l;
    const long long nc = (long long)n[l - 1][0] * n[l - 1][1] * n[l - 1][2];
    return nc <= kMaxCoarseGmres ? MG_OK : MG_EINVAL;
}

int check_grid(const mg_grid *g)
{
    if (!g) return MG_EINVAL;
    const int n[3] = {g->nx, g->ny, g->nz};
    const double l[3] = {g->lx, g->ly, g->lz};
    for (int d = 0; d < 3; d++) {
        if (n[d] < 2 || n[d] > (1 << 16)) return MG_EINVAL;
        if (!(l[d] > 0.0) || !isfinite(l[d])) return MG_EINVAL;
        if (g->bc[d] != MG_BC_NEUMANN && g->bc[d] != MG_BC_PERIODIC) return MG_EINVAL;
    }
    if ((long long)n[0] * n[1] * n[2] >= (1LL << 31)) return MG_EINVAL;
    int lv[MG_MAX_LEVELS][3], L;
    return make_levels(*g, lv, &L);
}

int check_params(const mg_params *p)
{
    if (p->nu1 < 1 || p->nu1 > 16 || p->nu2 < 0 || p->nu2 > 16) return MG_EINVAL;
    if (!(p->omega > 0.0 && p->omega < 2.0)) return MG_EINVAL;
    if (p->max_iters < 1 || p->max_iters > 100000) return MG_EINVAL;
    if (p->precision != MG_PREC_FP64 && p->precision != MG_PREC_MIXED) return MG_EINVAL;
    if (p->inner_cycles < 0 || p->inner_cycles > 16) return MG_EINVAL;
    if (p->tiles < MG_TILES_AUTO || p->tiles >= MG_TILE_VARIANTS) return MG_EINVAL;
    if (p->prolongation != MG_PROLONG_TRILINEAR && p->prolongation != MG_PROLONG_FLUX) return MG_EINVAL;
    if (p->solver != MG_SOLVER_MG && p->solver != MG_SOLVER_PCG) return MG_EINVAL;
    if (p->coarse_solver != MG_COARSE_AUTO && p->coarse_solver != MG_COARSE_GMRES) return MG_EINVAL;
    if (p->coarse_max_iters < 1 || p->coarse_max_iters > 100000) return MG_EINVAL;
    if (!(p->coarse_tol > 0.0 && p->coarse_tol < 1.0)) return MG_EINVAL;
    if (p->adaptive_cycles != 0 && p->adaptive_cycles != 1) return MG_EINVAL;
    if (p->outer != MG_OUTER_FP64 && p->outer != MG_OUTER_XP) return MG_EINVAL;
    if (p->sweep < MG_SWEEP_AUTO || p->sweep >= MG_SWEEP_VARIANTS) return MG_EINVAL;
    return MG_OK;
}

// Byte layout of a handle's device slab (also used for the memory estimate).
struct Layout {
    int L;
    int n[MG_MAX_LEVELS][3];
    size_t w64[MG_MAX_LEVELS][3], w32[MG_MAX_LEVELS][3], x[MG_MAX_LEVELS], b[MG_MAX_LEVELS];
    size_t x2;  // second iterate buffer of the finest level (one-pass sweep), 0 if none
    size_t dinv[MG_MAX_LEVELS];  // FP64 cycles: inverse diagonals of the relaxed levels (0 if none)
    size_t alpha64[MG_MAX_LEVELS], alpha32[MG_MAX_LEVELS];
    size_t G, b0, part, err, state, dstate, dview, dstart, dcview, setup_cv, total;
    size_t pcg[4];
    size_t xp3[3], xb[2], wlo[3];  // extended-precision outer iteration
    bool xp;
    bool gmres;
    size_t gm;
    int nblk0;
};

// the finest level can run one-pass sweeps (mg_fused.cu): even nu1 and nu2
// (the sweeps alternate between two buffers and must end in the first) and
// some one-pass shape fits it
static bool onepass_possible(const mg_grid &g, const mg_params &p, const int n[3])
{
    if (p.sweep == MG_SWEEP_HALF || (p.nu1 & 1) || (p.nu2 & 1)) return false;
    const int per = (g.bc[0] == MG_BC_PERIODIC ? 1 : 0) | (g.bc[1] == MG_BC_PERIODIC ? 2 : 0) |
                    (g.bc[2] == MG_BC_PERIODIC ? 4 : 0);
    for (int v = 1; v < kSweepVariants; v++)
        if (sweep_fits(n, per, v, p.precision == MG_PREC_MIXED)) return true;
    return false;
}

static int plan_layout(const mg_grid &g, const mg_params &p, Layout &lay)
{
    int rc = make_levels(g, lay.n, &lay.L);
    if (rc) return rc;
    const bool mixed = p.precision == MG_PREC_MIXED;
    const size_t vs = mixed ? 4 : 8;
    Carve c;
    for (int l = 0; l < lay.L; l++) {
        const size_t N = (size_t)lay.n[l][0] * lay.n[l][1] * lay.n[l][2];
        for (int d = 0; d < 3; d++) lay.w64[l][d] = c.take(N * 8);
        for (int d = 0; d < 3; d++) lay.w32[l][d] = mixed ? c.take(N * 4) : 0;
        lay.x[l] = c.take(N * vs);
        lay.b[l] = c.take(N * vs);
        if (l == 0) lay.x2 = (lay.L > 1 && onepass_possible(g, p, lay.n[0])) ? c.take(N * vs) : 0;
        // FP64 cycles relax every level but the coarsest with its inverse diagonal
        lay.dinv[l] = (!mixed && l + 1 < lay.L) ? c.take(N * 8) : 0;
        const bool flux = l > 0 && p.prolongation == MG_PROLONG_FLUX;
        lay.alpha64[l] = flux ? c.take(N * 8) : 0;
        lay.alpha32[l] = (flux && mixed) ? c.take(N * 4) : 0;
    }
    const int *nc = lay.n[lay.L - 1];
    const size_t ncells = (size_t)nc[0] * nc[1] * nc[2];
    // dense inverse for small coarsest grids, GMRES scratch otherwise
    lay.gmres = p.coarse_solver == MG_COARSE_GMRES || ncells > (size_t)kMaxCoarse;
    lay.G = lay.gmres ? 0 : c.take(ncells * ncells * 8);
    lay.gm = lay.gmres ? c.take((size_t)(kGmresM + 4) * ncells * 8) : 0;
    const size_t N0 = (size_t)g.nx * g.ny * g.nz;
    lay.b0 = c.take(N0 * 8);
    for (int v = 0; v < 4; v++) lay.pcg[v] = p.solver == MG_SOLVER_PCG ? c.take(N0 * 8) : 0;
    lay.xp = mixed && p.solver == MG_SOLVER_MG && p.outer == MG_OUTER_XP;
    for (int v = 0; v < 3; v++) lay.xp3[v] = lay.xp ? c.take(N0 * 4) : 0;
    for (int v = 0; v < 2; v++) lay.xb[v] = lay.xp ? c.take(N0 * 4) : 0;
    for (int v = 0; v < 3; v++) lay.wlo[v] = lay.xp ? c.take(N0 * 4) : 0;
    const int n0[3] = {g.nx, g.ny, g.nz};
    lay.nblk0 = outer_blocks(n0);
    lay.part = c.take((size_t)lay.nblk0 * kPart * 8);
    lay.err = c.take(16 * sizeof(int));
    lay.state = c.take(sizeof(GridState));
    lay.dstate = c.take(sizeof(GridState));
    lay.dview = c.take(sizeof(LevelView));
    lay.dstart = c.take(2 * sizeof(int));
    lay.dcview = c.take(sizeof(CoarseView));
    lay.setup_cv = c.take(sizeof(CoarseView));
    lay.total = c.off;
    return MG_OK;
}

}  // namespace gbmg

// ---------------------------------------------------------------------------
// Plan: launch tables over one or more handles
// ---------------------------------------------------------------------------

namespace gbmg {

static int per_bits(const mg_grid &g)
{
    return (g.bc[0] == MG_BC_PERIODIC ? 1 : 0) | (g.bc[1] == MG_BC_PERIODIC ? 2 : 0) |
           (g.bc[2] == MG_BC_PERIODIC ? 4 : 0);
}

void Plan::release()
{
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    if (mem) cudaFree(mem);
    mem = nullptr;
    if (ov_h) cudaFreeHost(ov_h);
    if (st_h) cudaFreeHost(st_h);
    if (stage_h) cudaFreeHost(stage_h);
    ov_h = nullptr;
    st_h = nullptr;
    stage_h = nullptr;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (staged) cudaEventDestroy(staged);
    e0 = e1 = staged = nullptr;
}

// Device memory for the tables of up to `cap` grids (worst case of every
// table), a pinned host copy of the same layout, and the per-solve mirrors.
// Allocated once; fill() rewrites the tables without allocating.
int Plan::alloc(int cap)
{
    capacity = cap;
    const int LV = cap * (MG_MAX_LEVELS - 1);
    const int ST = 3 * (cap + 1) * (MG_MAX_LEVELS - 1) + 2 * (cap + 1);
    Carve c;
    o_lv = c.take((size_t)LV * sizeof(LevelView));
    o_starts = c.take((size_t)ST * sizeof(int));
    o_cv = c.take((size_t)cap * sizeof(CoarseView));
    o_tv = c.take((size_t)cap * sizeof(TailView));
    tables_bytes = c.off;
    const size_t o_ov = c.take((size_t)cap * sizeof(OuterView));
    const size_t o_gs = c.take((size_t)cap * sizeof(GridState));
    CK(cudaMalloc((void **)&mem, c.off));
    CK(cudaMallocHost((void **)&stage_h, tables_bytes));
    cv = (CoarseView *)(mem + o_cv);
    tv = (TailView *)(mem + o_tv);
    ov = (OuterView *)(mem + o_ov);
    st = (GridState *)(mem + o_gs);
    CK(cudaMallocHost((void **)&ov_h, (size_t)cap * sizeof(OuterView)));
    CK(cudaMallocHost((void **)&st_h, (size_t)cap * sizeof(GridState)));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreateWithFlags(&staged, cudaEventDisableTiming));
    return MG_OK;
}

int Plan::build(mg_handle *const *handles, int count)
{
    int rc = alloc(count);
    if (rc) return rc;
    stream = handles[0]->stream;
    rc = fill(handles, count);
    if (rc) return rc;
    CK(cudaStreamSynchronize(stream));
    return MG_OK;
}

// (Re)write the launch tables for `handles` (count <= capacity) into the
// plan's memory: host tables in the pinned staging copy, one asynchronous
// copy on the plan's stream.  No allocation, no device synchronisation.
int Plan::fill(mg_handle *const *handles, int count)
{
    if (count < 1 || count > capacity) return MG_EINVAL;
    CK(cudaEventSynchronize(staged));  // the previous copy out of the staging buffer is done
    hs.assign(handles, handles + count);
    G = count;
    mixed = hs[0]->mixed;
    xp = hs[0]->xp;
    stream = hs[0]->stream;
    prm = hs[0]->prm;
    Lmax = 0;
    for (auto *h : hs) Lmax = std::max(Lmax, h->L);
    std::vector<int> lt(G);
    for (int g = 0; g < G; g++) lt[g] = first_tail_level(hs[g]);
    const bool flux = prm.prolongation == MG_PROLONG_FLUX;
    LevelView *lv = (LevelView *)(stage_h + o_lv);
    int *starts = (int *)(stage_h + o_starts);
    CoarseView *cvh = (CoarseView *)(stage_h + o_cv);
    TailView *tvh = (TailView *)(stage_h + o_tv);
    LevelView *d_lv = (LevelView *)(mem + o_lv);
    int *d_starts = (int *)(mem + o_starts);
    int nlv = 0, nst = 0;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        down[l] = Table{d_lv, d_starts, 0, 0};
        rest[l] = down[l];
        half[l] = down[l];
    }
    sweep0 = Table{d_lv, d_starts, 0, 0};
    for (int l = 0; l + 1 < Lmax; l++) {
        const int lv0 = nlv;
        int sf0 = nst, sc0, sh0, cnt = 0;
        // launch shape of each table: that of the grid with the most cells on
        // this level, if it fits every grid of the table, else the row shape
        int var[3] = {0, 0, 0};
        long long most = -1;
        // flux-conserving prolongation runs in the row-tiled kernel only
        for (int g = 0; g < G; g++) {
            mg_handle *h = hs[g];
            if (l + 1 >= h->L || l >= lt[g] || h->lev[l].N <= most) continue;
            most = h->lev[l].N;
            for (int k = 0; k < 3; k++) var[k] = h->tile[k][l];
        }
        for (int g = 0; g < G; g++) {
            mg_handle *h = hs[g];
            if (l + 1 >= h->L || l >= lt[g]) continue;
            for (int k = 0; k < 3; k++)
                if (!tile_fits(h->lev[l].n, var[k])) var[k] = 0;
        }
        if (flux) var[MG_TILE_PROLONG] = 0;
        // finest level: one-pass sweep shape of the largest grid if it fits
        // every grid of the table (each with its second iterate buffer)
        int sv = 0;
        if (l == 0) {
            long long big = -1;
            for (int g = 0; g < G; g++) {
                mg_handle *h = hs[g];
                if (l + 1 >= h->L || l >= lt[g] || h->lev[0].N <= big) continue;
                big = h->lev[0].N;
                sv = h->tile[MG_TILE_SWEEP][0];
            }
            for (int g = 0; g < G && sv > 0; g++) {
                mg_handle *h = hs[g];
                if (l + 1 >= h->L || l >= lt[g]) continue;
                if (!h->lev[0].x2 || !sweep_fits(h->lev[0].n, h->per, sv, h->mixed)) sv = 0;
            }
        }
        // three prefix arrays (four on the finest level), each count + 1 long,
        // laid out one after the other
        std::vector<int> sf{0}, sc{0}, sh{0}, sw{0};
        for (int g = 0; g < G; g++) {
            mg_handle *h = hs[g];
            if (l + 1 >= h->L || l >= lt[g]) continue;
            const HLevel &F = h->lev[l], &C = h->lev[l + 1];
            LevelView &v = lv[nlv++];
            memset(&v, 0, sizeof(v));
            for (int d = 0; d < 3; d++) {
                v.n[d] = F.n[d];
                v.nc[d] = C.n[d];
                v.w[d] = mixed ? (void *)F.w32[d] : (void *)F.w64[d];
            }
            v.per = h->per;
            v.x = F.x;
            v.b = F.b;
            v.xc = C.x;
            v.bc = C.b;
            v.g = g;
            v.st = h->state;
            v.ac = mixed ? (const void *)C.alpha32 : (const void *)C.alpha64;
            // the next level has its own half-sweeps (neither a tail level nor
            // the coarsest): its zero-start red half-sweep rides on this restriction
            v.zr = (l + 1 < lt[g] && l + 2 < h->L) ? 1 : 0;
            for (int d = 0; d < 3; d++) v.wc[d] = mixed ? (const void *)C.w32[d] : (const void *)C.w64[d];
            fill_fastdiv(v);
            v.x2 = F.x2;
            v.dinv = mixed ? nullptr : F.dinv;
            v.dinvc = mixed ? nullptr : C.dinv;
            if (sv > 0) sw.push_back(sw.back() + sweep_layout(v, sv));
            sf.push_back(sf.back() + prolong_blocks_v(F.n, C.n, var[MG_TILE_PROLONG]));
            sc.push_back(sc.back() + restrict_blocks_v(F.n, C.n, var[MG_TILE_RESTRICT]));
            sh.push_back(sh.back() + half_sweep_blocks_v(F.n, var[MG_TILE_HALF]));
            cnt++;
        }
        for (int v : sf) starts[nst++] = v;
        sc0 = nst;
        for (int v : sc) starts[nst++] = v;
        sh0 = nst;
        for (int v : sh) starts[nst++] = v;
        down[l] = Table{d_lv + lv0, d_starts + sf0, cnt, sf.back(), var[MG_TILE_PROLONG], flux ? 1 : 0};
        rest[l] = Table{d_lv + lv0, d_starts + sc0, cnt, sc.back(), var[MG_TILE_RESTRICT]};
        half[l] = Table{d_lv + lv0, d_starts + sh0, cnt, sh.back(), var[MG_TILE_HALF]};
        if (sv > 0) {
            const int sw0 = nst;
            for (int v : sw) starts[nst++] = v;
            sweep0 = Table{d_lv + lv0, d_starts + sw0, cnt, sw.back(), sv};
        }
        // a one-grid table also hands its view to the kernels by value (the
        // host copy stays in the staging buffer, rewritten only by fill)
        if (cnt == 1) down[l].hv = rest[l].hv = half[l].hv = lv + lv0;
        if (cnt == 1 && sv > 0) sweep0.hv = lv + lv0;
    }
    const int so0 = nst;
    starts[nst++] = 0;
    for (int g = 0; g < G; g++) {
        starts[nst] = starts[nst - 1] + hs[g]->nblk0;
        nst++;
    }
    ot = OuterTable{ov, d_starts + so0, G, starts[nst - 1]};
    const size_t esz = mixed ? sizeof(float) : sizeof(double);
    tail_smem = 0;
    ntv = 0;
    ncv = 0;
    cv_dense = cv_gmres = false;
    for (int g = 0; g < G; g++) {
        mg_handle *h = hs[g];
        if (lt[g] >= h->L) continue;
        TailView &v = tvh[ntv++];
        memset(&v, 0, sizeof(v));
        v.nt = h->L - lt[g];
        v.per = h->per;
        v.flux = flux ? 1 : 0;
        int off = 0;
        for (int t = 0; t < v.nt; t++) {
            const HLevel &Lv = h->lev[lt[g] + t];
            for (int d = 0; d < 3; d++) {
                v.n[t][d] = Lv.n[d];
                v.w[t][d] = mixed ? (void *)Lv.w32[d] : (void *)Lv.w64[d];
            }
            v.off[t] = off;
            v.dx[t] = make_fastdiv((unsigned)Lv.n[0]);
            v.dhx[t] = make_fastdiv(Lv.n[0] >= 2 ? (unsigned)(Lv.n[0] >> 1) : 1u);
            v.dy[t] = make_fastdiv((unsigned)Lv.n[1]);
            v.dq[t] = make_fastdiv(Lv.n[0] >= 4 ? (unsigned)(Lv.n[0] >> 2) : 1u);
            v.a[t] = mixed ? (const void *)Lv.alpha32 : (const void *)Lv.alpha64;
            off += (flux ? 6 : 5) * (int)Lv.N;
            off = (off + 3) & ~3;
        }
        v.x0 = h->lev[lt[g]].x;
        v.b0 = h->lev[lt[g]].b;
        v.G = h->G;
        v.st = h->state;
        v.err = h->err + 2;
        v.wait_polls = h->wait_polls;
        tail_smem = std::max(tail_smem, (size_t)off * esz);
    }
    for (int g = 0; g < G; g++) {
        mg_handle *h = hs[g];
        if (lt[g] < h->L) continue;
        const HLevel &Cl = h->lev[h->L - 1];
        CoarseView &v = cvh[ncv++];
        memset(&v, 0, sizeof(v));
        for (int d = 0; d < 3; d++) {
            v.n[d] = Cl.n[d];
            v.w[d] = Cl.w64[d];
        }
        v.per = h->per;
        v.nc = (int)Cl.N;
        v.G = h->G;
        v.x = Cl.x;
        v.b = Cl.b;
        v.st = h->state;
        v.err = h->err + 1;
        v.g = g;
        v.outer = h->L == 1 ? 1 : 0;
        v.gmres = h->gmres ? 1 : 0;
        v.gm = h->gm;
        v.gm_max = h->prm.coarse_max_iters;
        v.gm_tol = h->prm.coarse_tol;
        if (h->gmres) cv_gmres = true;
        else cv_dense = true;
    }
    for (int g = 0; g < G; g++) {
        mg_handle *h = hs[g];
        OuterView &v = ov_h[g];
        memset(&v, 0, sizeof(v));
        for (int d = 0; d < 3; d++) {
            v.n[d] = h->lev[0].n[d];
            v.w[d] = h->lev[0].w64[d];
        }
        v.per = h->per;
        v.b0 = h->b0;
        v.r = h->lev[0].b;
        v.part = h->part;
        v.nblk = h->nblk0;
        v.st = h->state;
        v.tol = 1e-10;
        v.max_iters = h->prm.max_iters;
        v.inner = prm.inner_cycles;
        v.r64 = h->pcg[0];
        v.z = h->pcg[1];
        v.d = h->pcg[2];
        v.q = h->pcg[3];
        v.e = h->lev[0].x;
        v.adaptive = prm.adaptive_cycles;
        v.xp = h->xp ? 1 : 0;
        v.xq = make_fastdiv(v.n[0] >= 4 ? (unsigned)(v.n[0] >> 2) : 1u);
        v.xy = make_fastdiv((unsigned)v.n[1]);
        v.dxt = make_fastdiv((unsigned)fine_xtiles(v.n[0]));
        for (int q = 0; q < 3; q++) {
            v.xp3[q] = h->xp3[q];
            v.w32[q] = h->xp ? h->lev[0].w32[q] : nullptr;
            v.wlo[q] = h->wlo[q];
        }
        for (int q = 0; q < 2; q++) v.xb[q] = h->xb[q];
    }
    CK(cudaMemcpyAsync(mem, stage_h, tables_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaEventRecord(staged, stream));
    return MG_OK;
}

// ---- profiling: events around launches -------------------------------------

void Prof::begin(cudaStream_t s, int kind, int level)
{
    if (!on) return;
    if (used + 2 > pool.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        pool.push_back(a);
        pool.push_back(b);
    }
    cur_kind = kind;
    cur_level = std::min(level, MG_MAX_LEVELS - 1);
    cudaEventRecord(pool[used], s);
}

void Prof::end(cudaStream_t s)
{
    if (!on) return;
    cudaEventRecord(pool[used + 1], s);
    pending.push_back({cur_kind, cur_level, (int)used});
    used += 2;
}

void Prof::collect()
{
    for (auto &p : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pool[p.ev], pool[p.ev + 1]) == cudaSuccess) {
            total_ms[p.kind][p.level] += ms;
            launches[p.kind][p.level] += 1;
        }
    }
    pending.clear();
    used = 0;
}

void Prof::reset()
{
    memset(total_ms, 0, sizeof(total_ms));
    memset(launches, 0, sizeof(launches));
}

Prof::~Prof()
{
    for (auto e : pool) cudaEventDestroy(e);
}

// ---- the V-cycle and the outer iteration -----------------------------------

// V-cycle `cyc` (0-based) of a refinement step over every grid of the plan,
// red-black half-sweeps in place; a grid whose step asks for at most cyc
// cycles skips every launch of it (in_cycle).  Coarse levels start every cycle
// from a zero correction: their first red half-sweep, which reads only b and
// the faces, is done by the restriction that produces b.  The finest
// level starts from zero in the first cycle of a step and from the previous
// cycle's correction in the next ones.  outer: this cycle may end a grid's
// step (the caller passes it for every cycle of a plan of several grids, for
// the last cycle only of a lone grid's); in the grid's last cycle of the step,
// the last black half-sweep on the finest level then also adds the correction
// (both colours) to the outer iterate (the prolongation does if nu2 = 0, the
// coarse solve if the grid has one level).
template <class T>
static void vcycle(Plan &P, Prof &pf, int cyc, bool outer)
{
    const cudaStream_t s = P.stream;
    const mg_params &q = P.prm;
    auto at = [cyc](Table t) {
        t.cyc = cyc;
        return t;
    };
    for (int l = 0; l + 1 < P.Lmax; l++) {
        const Table H = at(P.half[l]);
        if (H.count == 0) continue;
        const bool zero = !(l == 0 && cyc > 0);
        if (l == 0 && P.sweep0.count > 0) {
            // one-pass sweeps, alternating between the two iterate buffers
            // (nu1 even: the last one writes x)
            const Table W = at(P.sweep0);
            for (int it = 0; it < q.nu1; it++) {
                pf.begin(s, MG_K_SMOOTH, l);
                launch_sweep<T>(W, it & 1, q.omega, (it == 0 && zero) ? kHalfZero : 0, nullptr, s);
                pf.end(s);
            }
        }
        for (int it = 0; it < q.nu1 && !(l == 0 && P.sweep0.count > 0); it++) {
            // below the finest level the restriction into this level already
            // did the zero-start red half-sweep of every grid in this table
            if (!(it == 0 && l > 0)) {
                pf.begin(s, MG_K_SMOOTH, l);
                launch_half<T>(H, 0, q.omega, (it == 0 && zero) ? kHalfZero : 0, nullptr, s);
                pf.end(s);
            }
            pf.begin(s, MG_K_SMOOTH, l);
            launch_half<T>(H, 1, q.omega, 0, nullptr, s);
            pf.end(s);
        }
        pf.begin(s, MG_K_RESTRICT, l);
        launch_restrict<T>(at(P.rest[l]), q.omega, s);
        pf.end(s);
    }
    if (P.ntv) {
        pf.begin(s, MG_K_TAIL, 0);
        launch_tail<T>(P.tv, P.ntv, P.tail_smem, q.omega, q.nu1, q.nu2, cyc, s);
        pf.end(s);
    }
    if (P.ncv) {
        pf.begin(s, MG_K_COARSE, P.Lmax - 1);
        if (P.cv_dense) launch_coarse_solve<T>(P.cv, P.ncv, cyc, outer ? P.ov : nullptr, s);
        if (P.cv_gmres) launch_coarse_gmres<T>(P.cv, P.ncv, cyc, outer ? P.ov : nullptr, s);
        pf.end(s);
    }
    for (int l = P.Lmax - 2; l >= 0; l--) {
        const Table H = at(P.half[l]);
        if (H.count == 0) continue;
        const bool top = outer && l == 0;
        pf.begin(s, MG_K_PROLONG, l);
        launch_prolong<T>(at(P.down[l]), (top && q.nu2 == 0) ? P.ov : nullptr, s);
        pf.end(s);
        // the post-sweeps that end a refinement step also add the final values
        // to the outer iterate: as half-sweep launches where the one-pass shape
        // is a staged one (bitwise the same; the staged kernel's instance with
        // that update runs out of registers and takes twice as long)
        if (l == 0 && P.sweep0.count > 0 && !(top && sweep_shape(P.sweep0.variant).tile_x)) {
            const Table W = at(P.sweep0);
            for (int it = 0; it < q.nu2; it++) {
                // the last sweep adds both colours' final values
                const int fl = (top && it == q.nu2 - 1) ? kHalfOuter : 0;
                pf.begin(s, MG_K_SMOOTH, l);
                launch_sweep<T>(W, it & 1, q.omega, fl, fl ? P.ov : nullptr, s);
                pf.end(s);
            }
            continue;
        }
        for (int it = 0; it < q.nu2; it++) {
            // the last black half-sweep adds both colours' final values
            const int fl = (top && it == q.nu2 - 1) ? kHalfOuter : 0;
            pf.begin(s, MG_K_SMOOTH, l);
            launch_half<T>(H, 0, q.omega, 0, nullptr, s);
            pf.end(s);
            pf.begin(s, MG_K_SMOOTH, l);
            launch_half<T>(H, 1, q.omega, fl, P.ov, s);
            pf.end(s);
        }
    }
}

// Conjugate gradients: z = M r (the step's V-cycles from zero, no update of
// the FP64 iterate), the dot products of z, the new direction.
template <class T>
static void pcg_precondition(Plan &P, Prof &pf, int first)
{
    const cudaStream_t s = P.stream;
    for (int c = 0; c < P.prm.inner_cycles; c++) vcycle<T>(P, pf, c, false);
    pf.begin(s, MG_K_OTHER, 0);
    launch_pcg_z<T>(P.ot, s);
    launch_pcg_finalize(P.ot, first ? 0 : 2, s);
    launch_pcg_dir(P.ot, first, s);
    pf.end(s);
}

template <class T>
static void prologue(Plan &P, Prof &pf)
{
    const cudaStream_t s = P.stream;
    pf.begin(s, MG_K_OTHER, 0);
    launch_begin(P.ov, P.G, s);
    launch_sum(P.ot, 0, s);
    launch_finalize(P.ot, 0, s);
    pf.end(s);
    if (P.prm.solver == MG_SOLVER_PCG) {
        pf.begin(s, MG_K_RESIDUAL0, 0);
        launch_residual<T>(P.ot, 1, s);
        pf.end(s);
    } else {
        // multigrid iteration: b - mean b and its norm (FP64) set the power-of-2
        // scale the cycles work in; then the starting residual, FP64 or (extended
        // precision) from the float forms of b and p
        pf.begin(s, MG_K_OTHER, 0);
        launch_center_rhs(P.ot, s);
        launch_finalize(P.ot, 4, s);
        if (P.xp) launch_xp_prepare(P.ot, s);
        pf.end(s);
        pf.begin(s, MG_K_RESIDUAL0, 0);
        if (P.xp) launch_residual_xp(P.ot, 1, s);
        else launch_residual<T>(P.ot, 2, s);
        pf.end(s);
    }
    pf.begin(s, MG_K_OTHER, 0);
    launch_finalize(P.ot, 1, s);
    pf.end(s);
    if (P.prm.solver == MG_SOLVER_PCG) pcg_precondition<T>(P, pf, 1);
}

template <class T> static void body_cycles(Plan &P, Prof &pf, int cycles);
template <class T> static void body_residual(Plan &P, Prof &pf);

// One step of the outer iteration.  Multigrid iteration: up to `cycles`
// V-cycles on A e = r (the first from e = 0, the next ones continuing from the
// current e; each grid runs the number its state asks for, the last one adding
// e to the FP64 iterate), then the FP64 residual and the stopping test.
template <class T>
static void body(Plan &P, Prof &pf, int cycles)
{
    const cudaStream_t s = P.stream;
    if (P.prm.solver == MG_SOLVER_PCG) {
        // one CG step: q = A d, alpha, p and r updated, stopping test, z = M r, d
        pf.begin(s, MG_K_RESIDUAL, 0);
        launch_pcg_matvec(P.ot, s);
        pf.end(s);
        pf.begin(s, MG_K_OTHER, 0);
        launch_pcg_finalize(P.ot, 1, s);
        launch_pcg_update<T>(P.ot, s);
        launch_finalize(P.ot, 2, s);
        pf.end(s);
        pcg_precondition<T>(P, pf, 0);
        return;
    }
    body_cycles<T>(P, pf, cycles);
    body_residual<T>(P, pf);
}

template <class T>
static void body_cycles(Plan &P, Prof &pf, int cycles)
{
    // a lone grid's step runs exactly `cycles` cycles (the graph branch and the
    // host loop both take its own count), so only the last one can end it: the
    // others launch the half-sweep without the update of the outer iterate
    for (int c = 0; c < cycles; c++) vcycle<T>(P, pf, c, P.G > 1 || c + 1 == cycles);
}

template <class T>
static void body_residual(Plan &P, Prof &pf)
{
    const cudaStream_t s = P.stream;
    pf.begin(s, MG_K_RESIDUAL, 0);
    if (P.xp) launch_residual_xp(P.ot, 0, s);
    else launch_residual<T>(P.ot, 0, s);
    pf.end(s);
    pf.begin(s, MG_K_OTHER, 0);
    launch_finalize(P.ot, 2, s);
    pf.end(s);
}

static void epilogue(Plan &P, Prof &pf)
{
    const cudaStream_t s = P.stream;
    pf.begin(s, MG_K_OTHER, 0);
    launch_sum(P.ot, 1, s);
    launch_finalize(P.ot, 3, s);
    launch_final(P.ot, s);
    pf.end(s);
}

template <class T>
static int build_graph(Plan &P)
{
    Prof off;  // no events inside graphs
    cudaStream_t cs = P.capture_stream;
    if (!cs) {
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        P.capture_stream = cs;
    }
    Plan Q = P;  // same tables, launches go to the capture stream
    Q.stream = cs;
    Q.mem = nullptr;
    Q.ov_h = nullptr;
    Q.st_h = nullptr;
    Q.e0 = Q.e1 = nullptr;
    Q.graph = nullptr;
    Q.gexec = nullptr;
    cudaGraph_t main_g = nullptr, pro_g = nullptr, body_g = nullptr, epi_g = nullptr;
    CK(cudaGraphCreate(&main_g, 0));
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, main_g, 0, cudaGraphCondAssignDefault));
    // prologue
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    prologue<T>(Q, off);
    launch_loop_ctl(cond, Q.ot, cs);
    CK(cudaStreamEndCapture(cs, &pro_g));
    // loop body: with a variable number of V-cycles per step (multigrid
    // iteration, inner_cycles > 1) the body is [step control] -> [switch over
    // 1 .. inner V-cycles] -> [residual, test, loop control]; else one piece
    const bool switched = P.prm.solver != MG_SOLVER_PCG && P.prm.inner_cycles > 1;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (switched) body_residual<T>(Q, off);
    else body<T>(Q, off, P.prm.inner_cycles);
    launch_loop_ctl(cond, Q.ot, cs);
    CK(cudaStreamEndCapture(cs, &body_g));
    // epilogue
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    epilogue(Q, off);
    CK(cudaStreamEndCapture(cs, &epi_g));
    cudaGraphNode_t n_pro, n_loop, n_epi, n_inner;
    CK(cudaGraphAddChildGraphNode(&n_pro, main_g, nullptr, 0, pro_g));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    CK(cudaGraphAddNode(&n_loop, main_g, &n_pro, nullptr, 1, &cp));
    cudaGraph_t loop_body = cp.conditional.phGraph_out[0];
    if (switched) {
        cudaGraphConditionalHandle sw;
        CK(cudaGraphConditionalHandleCreate(&sw, loop_body, 0, cudaGraphCondAssignDefault));
        cudaGraph_t ctl_g = nullptr;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        launch_step_ctl(sw, Q.ot, cs);
        CK(cudaStreamEndCapture(cs, &ctl_g));
        cudaGraphNode_t n_ctl, n_sw;
        CK(cudaGraphAddChildGraphNode(&n_ctl, loop_body, nullptr, 0, ctl_g));
        cudaGraphDestroy(ctl_g);
        cudaGraphNodeParams sp = {};
        sp.type = cudaGraphNodeTypeConditional;
        sp.conditional.handle = sw;
        sp.conditional.type = cudaGraphCondTypeSwitch;
        sp.conditional.size = (unsigned int)P.prm.inner_cycles;
        CK(cudaGraphAddNode(&n_sw, loop_body, &n_ctl, nullptr, 1, &sp));
        for (int c = 1; c <= P.prm.inner_cycles; c++) {
            cudaGraph_t cyc_g = nullptr;
            CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            body_cycles<T>(Q, off, c);
            CK(cudaStreamEndCapture(cs, &cyc_g));
            cudaGraphNode_t n_c;
            CK(cudaGraphAddChildGraphNode(&n_c, sp.conditional.phGraph_out[c - 1], nullptr, 0, cyc_g));
            cudaGraphDestroy(cyc_g);
        }
        CK(cudaGraphAddChildGraphNode(&n_inner, loop_body, &n_sw, 1, body_g));
    } else {
        CK(cudaGraphAddChildGraphNode(&n_inner, loop_body, nullptr, 0, body_g));
    }
    CK(cudaGraphAddChildGraphNode(&n_epi, main_g, &n_loop, 1, epi_g));
    cudaGraphDestroy(pro_g);
    cudaGraphDestroy(body_g);
    cudaGraphDestroy(epi_g);
    CK(cudaGraphInstantiate(&P.gexec, main_g, 0));
    P.graph = main_g;
    return MG_OK;
}

// V-cycles of the next refinement step (host-driven loops, from the states
// just read back): the most any active grid asks for, as k_step_ctl decides
static int step_cycles(const Plan &P)
{
    int c = 1;
    for (int g = 0; g < P.G; g++)
        if (P.st_h[g].active && P.st_h[g].cycles_next > c) c = P.st_h[g].cycles_next;
    return c;
}

template <class T>
static int run_plan_t(Plan &P, Prof &pf, bool use_graph)
{
    const cudaStream_t s = P.stream;
    // per-launch event profiling times each kernel alone: plain launches there
    DepScope dep(P.dep && !pf.on);
    CK(cudaMemcpyAsync(P.ov, P.ov_h, P.G * sizeof(OuterView), cudaMemcpyHostToDevice, s));
    if (use_graph && !pf.on) {
        if (!P.gexec) {
            int rc = build_graph<T>(P);
            if (rc && P.dep) {
                // the graph was not accepted with programmatic edges: rebuild it
                // with plain launches
                cudaGetLastError();
                P.dep = 0;
                DepScope plain(0);
                rc = build_graph<T>(P);
            }
            if (rc) return rc;
        }
        CK(cudaEventRecord(P.e0, s));
        CK(cudaGraphLaunch(P.gexec, s));
        CK(cudaEventRecord(P.e1, s));
    } else {
        CK(cudaEventRecord(P.e0, s));
        prologue<T>(P, pf);
        int max_it = 0;
        for (auto *h : P.hs) max_it = std::max(max_it, h->prm.max_iters);
        for (int it = 0; it <= max_it; it++) {
            launch_gather_states(P.ot, P.st, s);
            CK(cudaMemcpyAsync(P.st_h, P.st, P.G * sizeof(GridState), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            bool any = false;
            for (int g = 0; g < P.G; g++) any |= P.st_h[g].active != 0;
            if (!any) break;
            body<T>(P, pf, step_cycles(P));
        }
        epilogue(P, pf);
        CK(cudaEventRecord(P.e1, s));
    }
    CK(cudaGetLastError());
    if (P.post_bytes) CK(cudaMemcpyAsync(P.post_dst, P.post_src, P.post_bytes, cudaMemcpyDeviceToHost, s));
    launch_gather_states(P.ot, P.st, s);
    CK(cudaMemcpyAsync(P.st_h, P.st, P.G * sizeof(GridState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    pf.collect();
    return MG_OK;
}

void plan_bind(Plan &P, int g, const double *rhs, double *p, double tol, int max_iters)
{
    P.ov_h[g].b = rhs;
    P.ov_h[g].p = p;
    P.ov_h[g].tol = tol;
    P.ov_h[g].max_iters = max_iters;
}

int plan_upload(Plan &P)
{
    CK(cudaMemcpyAsync(P.ov, P.ov_h, P.G * sizeof(OuterView), cudaMemcpyHostToDevice, P.stream));
    return MG_OK;
}

static Prof g_no_prof;

int plan_prologue(Plan &P)
{
    DepScope dep(P.dep);
    if (P.mixed) prologue<float>(P, g_no_prof);
    else prologue<double>(P, g_no_prof);
    CK(cudaGetLastError());
    return MG_OK;
}

int plan_body(Plan &P)
{
    DepScope dep(P.dep);
    const int c = step_cycles(P);
    if (P.mixed) body<float>(P, g_no_prof, c);
    else body<double>(P, g_no_prof, c);
    CK(cudaGetLastError());
    return MG_OK;
}

int plan_final(Plan &P)
{
    DepScope dep(P.dep);
    epilogue(P, g_no_prof);
    CK(cudaGetLastError());
    return MG_OK;
}

int plan_gather_states(Plan &P)
{
    launch_gather_states(P.ot, P.st, P.stream);
    CK(cudaMemcpyAsync(P.st_h, P.st, P.G * sizeof(GridState), cudaMemcpyDeviceToHost, P.stream));
    return MG_OK;
}

int plan_sync_states(Plan &P)
{
    launch_gather_states(P.ot, P.st, P.stream);
    CK(cudaMemcpyAsync(P.st_h, P.st, P.G * sizeof(GridState), cudaMemcpyDeviceToHost, P.stream));
    CK(cudaStreamSynchronize(P.stream));
    return MG_OK;
}

void fill_stats(const GridState &s, const int herr[3], double ms, mg_stats *o, int *status_out)
{
    int status = s.status;
    if (herr[0]) status = MG_EINVAL;
    else if (herr[1]) status = MG_ESINGULAR;
    else if (herr[2]) status = MG_ETIMEOUT;  // a staging wait on the device gave up
    if (o) {
        o->iters = s.iters;
        o->status = status;
        o->res0 = s.r0;
        o->res = s.rnorm;
        o->bnorm = s.bnorm;
        o->rel_res = s.bnorm > 0.0 ? s.rnorm / s.bnorm : 0.0;
        o->gamma = (s.iters > 0 && s.r0 > 0.0) ? pow(s.rnorm / s.r0, 1.0 / s.iters) : 0.0;
        o->rhs_mean = s.bmean;
        o->ms = ms;
        o->steps = s.steps;
        o->admit_tick = o->finish_tick = 0;
        o->inflight_at_admit = o->lane = 0;
    }
    *status_out = status;
}

int run_plan(Plan &P, Prof &pf, const double *const *rhs, double *const *p, const double *tol,
             mg_stats *out)
{
    for (int g = 0; g < P.G; g++) {
        if (!rhs[g] || !p[g] || !(tol[g] >= 0.0)) return MG_EINVAL;
        if (((uintptr_t)p[g] & 15) != 0) return MG_EINVAL;  // p is staged in 16-byte pieces
        P.ov_h[g].b = rhs[g];
        P.ov_h[g].p = p[g];
        P.ov_h[g].tol = tol[g];
        P.ov_h[g].max_iters = P.hs[g]->prm.max_iters;
    }
    const bool use_graph = P.prm.use_graph != 0;
    int rc = P.mixed ? run_plan_t<float>(P, pf, use_graph) : run_plan_t<double>(P, pf, use_graph);
    if (rc) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.e0, P.e1);
    int first_bad = MG_OK;
    for (int g = 0; g < P.G; g++) {
        // coefficient problems found on the device by mg_set_faces / mg_set_density
        int herr[3] = {0, 0, 0};
        cudaMemcpy(herr, P.hs[g]->err, sizeof(herr), cudaMemcpyDeviceToHost);
        int status;
        fill_stats(P.st_h[g], herr, ms, out ? &out[g] : nullptr, &status);
        if (status != MG_OK && first_bad == MG_OK) first_bad = status;
    }
    return first_bad;
}

}  // namespace gbmg

// ---------------------------------------------------------------------------
// handle life cycle
// ---------------------------------------------------------------------------

static int upload_faces(mg_handle *h)
{
    // coarse levels: mean of the 4 fine faces tiling each coarse face
    for (int l = 1; l < h->L; l++) {
        CoarsenArgs a;
        memset(&a, 0, sizeof(a));
        for (int d = 0; d < 3; d++) {
            a.nf[d] = h->lev[l - 1].n[d];
            a.nc[d] = h->lev[l].n[d];
            a.wf[d] = h->lev[l - 1].w64[d];
            a.wc[d] = h->lev[l].w64[d];
            a.wc32[d] = h->mixed ? h->lev[l].w32[d] : nullptr;
        }
        a.dx = make_fastdiv((unsigned)a.nc[0]);
        a.dy = make_fastdiv((unsigned)a.nc[1]);
        launch_coarsen_faces(a, h->stream);
        if (h->lev[l].alpha64) {
            // cell coefficients for the flux-conserving prolongation into level l - 1
            AlphaArgs c;
            memset(&c, 0, sizeof(c));
            for (int d = 0; d < 3; d++) {
                c.n[d] = h->lev[l].n[d];
                c.h2[d] = h->lev[l].h[d] * h->lev[l].h[d];
                c.w[d] = h->lev[l].w64[d];
            }
            c.per = h->per;
            c.out64 = h->lev[l].alpha64;
            c.out32 = h->lev[l].alpha32;
            launch_cell_alpha(c, h->stream);
        }
    }
    // FP64 cycles: inverse diagonals of the levels that are relaxed
    for (int l = 0; l < h->L; l++) {
        if (!h->lev[l].dinv) continue;
        DiagArgs a;
        memset(&a, 0, sizeof(a));
        for (int d = 0; d < 3; d++) {
            a.n[d] = h->lev[l].n[d];
            a.w[d] = h->lev[l].w64[d];
        }
        a.per = h->per;
        a.out = h->lev[l].dinv;
        a.dx = make_fastdiv((unsigned)a.n[0]);
        a.dy = make_fastdiv((unsigned)a.n[1]);
        launch_diag_inv(a, h->stream);
    }
    if (!h->gmres) launch_coarse_setup(h->setup_cv, 1, h->stream);
    CK(cudaGetLastError());
    return MG_OK;
}

int gbmg::set_faces_impl(mg_handle *h, const double *ax, const double *ay, const double *az)
{
    DepScope dep(dep_launch_default());
    if (!ax || !ay || !az) return MG_EINVAL;
    CK(cudaMemsetAsync(h->err, 0, 3 * sizeof(int), h->stream));
    FaceArgs a;
    memset(&a, 0, sizeof(a));
    const double *in[3] = {ax, ay, az};
    for (int d = 0; d < 3; d++) {
        a.n[d] = h->lev[0].n[d];
        a.in[d] = in[d];
        a.scale[d] = 1.0 / (h->lev[0].h[d] * h->lev[0].h[d]);
        a.out64[d] = h->lev[0].w64[d];
        a.out32[d] = h->mixed ? h->lev[0].w32[d] : nullptr;
        a.out32lo[d] = h->wlo[d];
    }
    a.per = h->per;
    a.err = h->err;
    launch_scale_faces(a, h->stream);
    return upload_faces(h);
}

static int set_density_impl(mg_handle *h, const double *rho, int mode)
{
    DepScope dep(dep_launch_default());
    if (!rho || (mode != MG_FACE_HARMONIC && mode != MG_FACE_ARITHMETIC)) return MG_EINVAL;
    CK(cudaMemsetAsync(h->err, 0, 3 * sizeof(int), h->stream));
    FaceArgs a;
    memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; d++) {
        a.n[d] = h->lev[0].n[d];
        a.scale[d] = 1.0 / (h->lev[0].h[d] * h->lev[0].h[d]);
        a.out64[d] = h->lev[0].w64[d];
        a.out32[d] = h->mixed ? h->lev[0].w32[d] : nullptr;
        a.out32lo[d] = h->wlo[d];
    }
    a.per = h->per;
    a.mode = mode;
    a.rho = rho;
    a.err = h->err;
    launch_faces_from_density(a, h->stream);
    return upload_faces(h);
}

int gbmg::handle_alloc(const mg_grid *grid, const mg_params *params, void *stream, mg_handle **out)
{
    if (!out) return MG_EINVAL;
    *out = nullptr;
    int rc = check_grid(grid);
    if (rc) return rc;
    mg_params prm;
    mg_params_default(&prm);
    if (params) prm = *params;
    rc = check_params(&prm);
    if (rc) return rc;
    // most V-cycles per FP64 residual: the residual pass is bound by the FP64
    // pipe, slow on this GPU, so fewer passes pay; the adaptive step length
    // trims the steps that need fewer cycles.  FP32 cycles stop gaining within a
    // step near a 1e-5 reduction (their rounding), about 6 cycles at the rates
    // of the drop/film fields; FP64 cycles have no such limit
    if (prm.inner_cycles == 0)
        prm.inner_cycles = prm.solver == MG_SOLVER_PCG ? 1 : prm.precision == MG_PREC_MIXED ? 6 : 8;
    Layout lay;
    rc = plan_layout(*grid, prm, lay);
    if (rc) return rc;
    mg_handle *h = new (std::nothrow) mg_handle();
    if (!h) return MG_ENOMEM;
    h->g = *grid;
    h->prm = prm;
    h->stream = (cudaStream_t)stream;
    h->per = per_bits(*grid);
    h->mixed = prm.precision == MG_PREC_MIXED;
    CK(cudaGetDevice(&h->device));
    cudaError_t e = cudaMalloc((void **)&h->slab, lay.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MG_ENOMEM;
    }
    h->bytes = lay.total;
    h->L = lay.L;
    const double len[3] = {grid->lx, grid->ly, grid->lz};
    for (int l = 0; l < lay.L; l++) {
        HLevel &L = h->lev[l];
        for (int d = 0; d < 3; d++) {
            L.n[d] = lay.n[l][d];
            L.h[d] = len[d] / lay.n[l][d];
            L.w64[d] = (double *)(h->slab + lay.w64[l][d]);
            L.w32[d] = h->mixed ? (float *)(h->slab + lay.w32[l][d]) : nullptr;
        }
        L.N = (long long)L.n[0] * L.n[1] * L.n[2];
        L.x = h->slab + lay.x[l];
        L.x2 = (l == 0 && lay.x2) ? (void *)(h->slab + lay.x2) : nullptr;
        L.dinv = lay.dinv[l] ? (double *)(h->slab + lay.dinv[l]) : nullptr;
        L.alpha64 = lay.alpha64[l] ? (double *)(h->slab + lay.alpha64[l]) : nullptr;
        L.alpha32 = lay.alpha32[l] ? (float *)(h->slab + lay.alpha32[l]) : nullptr;
        L.b = h->slab + lay.b[l];
    }
    h->gmres = lay.gmres;
    h->G = lay.gmres ? nullptr : (double *)(h->slab + lay.G);
    h->gm = lay.gmres ? (double *)(h->slab + lay.gm) : nullptr;
    h->b0 = (double *)(h->slab + lay.b0);
    for (int v = 0; v < 4; v++) h->pcg[v] = lay.pcg[v] ? (double *)(h->slab + lay.pcg[v]) : nullptr;
    h->xp = lay.xp;
    for (int v = 0; v < 3; v++) h->xp3[v] = lay.xp ? (float *)(h->slab + lay.xp3[v]) : nullptr;
    for (int v = 0; v < 2; v++) h->xb[v] = lay.xp ? (float *)(h->slab + lay.xb[v]) : nullptr;
    for (int v = 0; v < 3; v++) h->wlo[v] = lay.xp ? (float *)(h->slab + lay.wlo[v]) : nullptr;
    h->part = (double *)(h->slab + lay.part);
    h->nblk0 = lay.nblk0;
    h->err = (int *)(h->slab + lay.err);
    h->state = (GridState *)(h->slab + lay.state);
    h->dstate = (GridState *)(h->slab + lay.dstate);
    h->dview = (LevelView *)(h->slab + lay.dview);
    h->dstart = (int *)(h->slab + lay.dstart);
    h->dcview = (CoarseView *)(h->slab + lay.dcview);
    h->setup_cv = (CoarseView *)(h->slab + lay.setup_cv);
    GridState ds;
    memset(&ds, 0, sizeof(ds));
    ds.active = 1;
    ds.cycles_next = 1 << 30;  // unit calls run whatever cycle index they are given
    CK(cudaMemcpy(h->dstate, &ds, sizeof(ds), cudaMemcpyHostToDevice));
    CK(cudaMemset(h->state, 0, sizeof(GridState)));
    CK(cudaMemset(h->err, 0, 16 * sizeof(int)));
    {
        // view of the coarsest level for building its inverse (mg_create / mg_set_faces)
        const HLevel &Cl = h->lev[h->L - 1];
        CoarseView v;
        memset(&v, 0, sizeof(v));
        for (int d = 0; d < 3; d++) {
            v.n[d] = Cl.n[d];
            v.w[d] = Cl.w64[d];
        }
        v.per = h->per;
        v.nc = (int)Cl.N;
        v.G = h->G;
        v.err = h->err + 1;
        CK(cudaMemcpy(h->setup_cv, &v, sizeof(v), cudaMemcpyHostToDevice));
    }
    rc = tune_handle(h);
    if (rc) {
        mg_destroy(h);
        return rc;
    }
    h->plan = new (std::nothrow) Plan();
    if (!h->plan) {
        mg_destroy(h);
        return MG_ENOMEM;
    }
    rc = h->plan->build(&h, 1);
    if (rc) {
        mg_destroy(h);
        return rc;
    }
    *out = h;
    return MG_OK;
}

extern "C" {

const char *mg_strerror(int s)
{
    switch (s) {
    case MG_OK: return "ok";
    case MG_EINVAL: return "invalid argument";
    case MG_ENOMEM: return "out of device memory";
    case MG_ECUDA: return "CUDA error";
    case MG_ENOTCONV: return "not converged within max_iters";
    case MG_EDIVERGED: return "residual became NaN or Inf";
    case MG_ETIMEOUT: return "bounded device wait expired";
    case MG_EBUSY: return "busy: requests outstanding";
    case MG_EAGAIN: return "pending";
    case MG_EBUDGET: return "request exceeds the device-memory budget";
    case MG_ESINGULAR: return "coarsest-grid matrix is singular (grid cut by zero coefficients)";
    case MG_ENOTFOUND: return "unknown ticket";
    case MG_ETOOBIG: return "grid larger than the static scratch area (MG_STATIC_MAX_CELLS cells)";
    default: return "unknown status";
    }
}

int mg_last_cuda_error(void) { return (int)gbmg::last_cuda_error(); }

int mg_params_default(mg_params *p)
{
    if (!p) return MG_EINVAL;
    p->nu1 = 2;
    p->nu2 = 2;
    p->omega = 1.0;
    p->max_iters = 100;
    p->precision = MG_PREC_MIXED;
    p->use_graph = 1;
    p->inner_cycles = 0;
    p->tiles = MG_TILES_AUTO;
    p->prolongation = MG_PROLONG_TRILINEAR;
    p->solver = MG_SOLVER_MG;
    p->coarse_solver = MG_COARSE_AUTO;
    p->coarse_max_iters = 300;
    p->coarse_tol = 1e-8;
    p->adaptive_cycles = 1;
    p->outer = MG_OUTER_FP64;
    p->sweep = MG_SWEEP_AUTO;
    return MG_OK;
}

int mg_faces_from_density(const mg_grid *grid, const double *rho, int mode, double *ax, double *ay,
                          double *az, void *stream)
{
    int rc = check_grid(grid);
    if (rc) return rc;
    if (!rho || !ax || !ay || !az) return MG_EINVAL;
    if (mode != MG_FACE_HARMONIC && mode != MG_FACE_ARITHMETIC) return MG_EINVAL;
    FaceArgs a;
    memset(&a, 0, sizeof(a));
    a.n[0] = grid->nx;
    a.n[1] = grid->ny;
    a.n[2] = grid->nz;
    a.per = per_bits(*grid);
    a.mode = mode;
    a.rho = rho;
    a.scale[0] = a.scale[1] = a.scale[2] = 1.0;
    a.out64[0] = ax;
    a.out64[1] = ay;
    a.out64[2] = az;
    launch_faces_from_density(a, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return MG_OK;
}

int mg_create(const mg_grid *grid, const double *ax, const double *ay, const double *az,
              const mg_params *params, void *stream, mg_handle **out)
{
    if (!ax || !ay || !az) return MG_EINVAL;
    mg_handle *h = nullptr;
    int rc = handle_alloc(grid, params, stream, &h);
    if (rc) return rc;
    rc = set_faces_impl(h, ax, ay, az);
    if (rc == MG_OK) {
        int herr[3] = {0, 0, 0};
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = cudaMemcpy(herr, h->err, sizeof(herr), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            note_cuda_error(e);
            rc = MG_ECUDA;
        } else if (herr[0]) {
            rc = MG_EINVAL;
        } else if (herr[1]) {
            rc = MG_ESINGULAR;
        }
    }
    if (rc) {
        mg_destroy(h);
        return rc;
    }
    *out = h;
    return MG_OK;
}

int mg_set_faces(mg_handle *h, const double *ax, const double *ay, const double *az)
{
    if (!h) return MG_EINVAL;
    return set_faces_impl(h, ax, ay, az);
}

int mg_set_density(mg_handle *h, const double *rho, int mode)
{
    if (!h) return MG_EINVAL;
    return set_density_impl(h, rho, mode);
}

int mg_solve(mg_handle *h, const double *rhs, double *p, double tol, mg_stats *st)
{
    if (!h || !rhs || !p) return MG_EINVAL;
    mg_stats tmp;
    return run_plan(*h->plan, h->prof, &rhs, &p, &tol, st ? st : &tmp);
}

static ProjArgs proj_args(const mg_handle *h, double dt)
{
    ProjArgs a;
    memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; d++) {
        a.n[d] = h->lev[0].n[d];
        a.h[d] = h->lev[0].h[d];
        a.w[d] = h->lev[0].w64[d];
    }
    a.per = h->per;
    a.dt = dt;
    return a;
}

int mg_divergence(mg_handle *h, const double *ux, const double *uy, const double *uz, double dt, double *S)
{
    if (!h || !ux || !uy || !uz || !S || !(dt > 0.0) || !std::isfinite(dt)) return MG_EINVAL;
    ProjArgs a = proj_args(h, dt);
    a.u[0] = (double *)ux;
    a.u[1] = (double *)uy;
    a.u[2] = (double *)uz;
    a.S = S;
    launch_divergence(a, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_project(mg_handle *h, const double *p, double dt, double *ux, double *uy, double *uz)
{
    if (!h || !p || !ux || !uy || !uz || !(dt > 0.0) || !std::isfinite(dt)) return MG_EINVAL;
    ProjArgs a = proj_args(h, dt);
    a.p = p;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    launch_project(a, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_projection_step(mg_handle *h, double *ux, double *uy, double *uz, double dt, double *p, double *S,
                       double tol, mg_stats *st)
{
    if (!h || !ux || !uy || !uz || !p || !S || !(dt > 0.0) || !std::isfinite(dt)) return MG_EINVAL;
    ProjArgs a = proj_args(h, dt);
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.S = S;
    a.p = p;
    launch_divergence(a, h->stream);
    CK(cudaGetLastError());
    mg_stats tmp;
    const double *rhs = S;
    const int rc = run_plan(*h->plan, h->prof, &rhs, &p, &tol, st ? st : &tmp);
    if (rc != MG_OK && rc != MG_ENOTCONV) return rc;
    launch_project(a, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return rc;
}

static int ensure_host_buffers(mg_handle *h, bool rho)
{
    const size_t n = (size_t)h->lev[0].N * sizeof(double);
    if (!h->io_rhs) CK(cudaMalloc((void **)&h->io_rhs, n));
    if (!h->io_p) CK(cudaMalloc((void **)&h->io_p, n));
    if (rho && !h->io_rho) CK(cudaMalloc((void **)&h->io_rho, n));
    if (rho && !h->io_stream) CK(cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking));
    if (rho && !h->io_ready) CK(cudaEventCreateWithFlags(&h->io_ready, cudaEventDisableTiming));
    return MG_OK;
}

// Solve on the staged io_rhs / io_p; the result goes back to p_host before the
// solve's own synchronisation.
static int solve_staged(mg_handle *h, double *p_host, double tol, mg_stats *st)
{
    Plan &P = *h->plan;
    P.post_dst = p_host;
    P.post_src = h->io_p;
    P.post_bytes = (size_t)h->lev[0].N * sizeof(double);
    const int rc = mg_solve(h, h->io_rhs, h->io_p, tol, st);
    P.post_dst = nullptr;
    P.post_src = nullptr;
    P.post_bytes = 0;
    return rc;
}

int mg_solve_host(mg_handle *h, const double *rhs_host, double *p_host, double tol, mg_stats *st)
{
    if (!h || !rhs_host || !p_host) return MG_EINVAL;
    int rc = ensure_host_buffers(h, false);
    if (rc) return rc;
    const size_t n = (size_t)h->lev[0].N * sizeof(double);
    CK(cudaMemcpyAsync(h->io_rhs, rhs_host, n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->io_p, p_host, n, cudaMemcpyHostToDevice, h->stream));
    return solve_staged(h, p_host, tol, st);
}

int mg_step_host(mg_handle *h, const double *rho_host, int mode, const double *rhs_host,
                 double *p_host, double tol, mg_stats *st)
{
    if (!h || !rho_host || !rhs_host || !p_host) return MG_EINVAL;
    int rc = ensure_host_buffers(h, true);
    if (rc) return rc;
    const size_t n = (size_t)h->lev[0].N * sizeof(double);
    // the density first; the right-hand side and the initial p on a side
    // stream while the faces, coarse faces and coarsest inverse are built
    CK(cudaMemcpyAsync(h->io_rho, rho_host, n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->io_rhs, rhs_host, n, cudaMemcpyHostToDevice, h->io_stream));
    CK(cudaMemcpyAsync(h->io_p, p_host, n, cudaMemcpyHostToDevice, h->io_stream));
    CK(cudaEventRecord(h->io_ready, h->io_stream));
    rc = set_density_impl(h, h->io_rho, mode);
    if (rc) {
        cudaStreamSynchronize(h->io_stream);
        return rc;
    }
    CK(cudaStreamWaitEvent(h->stream, h->io_ready, 0));
    return solve_staged(h, p_host, tol, st);
}

int mg_destroy(mg_handle *h)
{
    if (!h) return MG_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->plan) {
        if (h->plan->capture_stream) cudaStreamDestroy(h->plan->capture_stream);
        h->plan->release();
        delete h->plan;
    }
    if (h->io_stream) cudaStreamSynchronize(h->io_stream);
    if (h->io_rhs) cudaFree(h->io_rhs);
    if (h->io_p) cudaFree(h->io_p);
    if (h->io_rho) cudaFree(h->io_rho);
    if (h->io_ready) cudaEventDestroy(h->io_ready);
    if (h->io_stream) cudaStreamDestroy(h->io_stream);
    if (h->slab) cudaFree(h->slab);
    delete h;
    return MG_OK;
}

// ---- batches ----------------------------------------------------------------

struct mg_batch {
    Plan plan;
    Prof prof;
};

int mg_batch_create(mg_handle *const *handles, int count, mg_batch **out)
{
    if (!handles || count < 1 || !out) return MG_EINVAL;
    for (int g = 0; g < count; g++) {
        if (!handles[g]) return MG_EINVAL;
        if (handles[g]->mixed != handles[0]->mixed || handles[g]->stream != handles[0]->stream)
            return MG_EINVAL;
        if (handles[g]->prm.nu1 != handles[0]->prm.nu1 || handles[g]->prm.nu2 != handles[0]->prm.nu2 ||
            handles[g]->prm.omega != handles[0]->prm.omega ||
            handles[g]->prm.inner_cycles != handles[0]->prm.inner_cycles ||
            handles[g]->prm.prolongation != handles[0]->prm.prolongation ||
            handles[g]->prm.solver != handles[0]->prm.solver)
            return MG_EINVAL;
        for (int q = 0; q < g; q++)
            if (handles[q] == handles[g]) return MG_EINVAL;
    }
    mg_batch *b = new (std::nothrow) mg_batch();
    if (!b) return MG_ENOMEM;
    int rc = b->plan.build(handles, count);
    if (rc) {
        b->plan.release();
        delete b;
        return rc;
    }
    *out = b;
    return MG_OK;
}

int mg_batch_solve(mg_batch *b, const double *const *rhs, double *const *p, const double *tol,
                   mg_stats *st)
{
    if (!b || !rhs || !p || !tol) return MG_EINVAL;
    std::vector<mg_stats> tmp;
    if (!st) {
        tmp.resize(b->plan.G);
        st = tmp.data();
    }
    return run_plan(b->plan, b->prof, rhs, p, tol, st);
}

int mg_batch_destroy(mg_batch *b)
{
    if (!b) return MG_EINVAL;
    if (b->plan.stream) cudaStreamSynchronize(b->plan.stream);
    if (b->plan.capture_stream) cudaStreamDestroy(b->plan.capture_stream);
    b->plan.release();
    delete b;
    return MG_OK;
}

// ---- single steps -------------------------------------------------------------

int mg_num_levels(const mg_handle *h, int *levels)
{
    if (!h || !levels) return MG_EINVAL;
    *levels = h->L;
    return MG_OK;
}

int mg_level_shape(const mg_handle *h, int level, int *nx, int *ny, int *nz)
{
    if (!h || level < 0 || level >= h->L || !nx || !ny || !nz) return MG_EINVAL;
    *nx = h->lev[level].n[0];
    *ny = h->lev[level].n[1];
    *nz = h->lev[level].n[2];
    return MG_OK;
}

int mg_level_cell_alpha(const mg_handle *h, int level, double *alpha)
{
    if (!h || !alpha || level < 0 || level >= h->L) return MG_EINVAL;
    AlphaArgs c;
    memset(&c, 0, sizeof(c));
    for (int d = 0; d < 3; d++) {
        c.n[d] = h->lev[level].n[d];
        c.h2[d] = h->lev[level].h[d] * h->lev[level].h[d];
        c.w[d] = h->lev[level].w64[d];
    }
    c.per = h->per;
    c.out64 = alpha;
    launch_cell_alpha(c, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_level_faces(const mg_handle *h, int level, double *wx, double *wy, double *wz)
{
    if (!h || level < 0 || level >= h->L || !wx || !wy || !wz) return MG_EINVAL;
    const size_t n = (size_t)h->lev[level].N * sizeof(double);
    double *o[3] = {wx, wy, wz};
    for (int d = 0; d < 3; d++)
        CK(cudaMemcpyAsync(o[d], h->lev[level].w64[d], n, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_level_faces32(const mg_handle *h, int level, float *wx, float *wy, float *wz)
{
    if (!h || level < 0 || level >= h->L || !wx || !wy || !wz || !h->mixed) return MG_EINVAL;
    const size_t n = (size_t)h->lev[level].N * sizeof(float);
    float *o[3] = {wx, wy, wz};
    for (int d = 0; d < 3; d++)
        CK(cudaMemcpyAsync(o[d], h->lev[level].w32[d], n, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

enum UnitTiles { kFineTiles, kCoarseTiles, kHalfTiles, kProlongTiles };

static int unit_view(mg_handle *h, int level, int prec, const void *x, void *b,
                     const void *xc, void *bc, Table *tb, UnitTiles tiles)
{
    if (!h || level < 0 || level >= h->L) return MG_EINVAL;
    if (prec != MG_PREC_FP64 && prec != MG_PREC_MIXED) return MG_EINVAL;
    if (prec == MG_PREC_MIXED && !h->mixed) return MG_EINVAL;
    LevelView v;
    memset(&v, 0, sizeof(v));
    const HLevel &L = h->lev[level];
    for (int d = 0; d < 3; d++) {
        v.n[d] = L.n[d];
        v.w[d] = prec == MG_PREC_MIXED ? (void *)L.w32[d] : (void *)L.w64[d];
        v.nc[d] = level + 1 < h->L ? h->lev[level + 1].n[d] : 0;
    }
    v.per = h->per;
    v.x = (void *)x;
    v.b = b;
    v.xc = (void *)xc;
    v.bc = bc;
    v.st = h->dstate;
    v.ac = level + 1 >= h->L ? nullptr
           : prec == MG_PREC_MIXED ? (const void *)h->lev[level + 1].alpha32
                                   : (const void *)h->lev[level + 1].alpha64;
    // FP64 unit calls on an FP64 handle relax as its solves do (inverse diagonals)
    v.dinv = prec == MG_PREC_FP64 ? L.dinv : nullptr;
    v.dinvc = (prec == MG_PREC_FP64 && level + 1 < h->L) ? h->lev[level + 1].dinv : nullptr;
    fill_fastdiv(v);
    // the shape the handle's solves use on this level (not on the coarsest)
    const int kind = tiles == kCoarseTiles ? MG_TILE_RESTRICT : tiles == kProlongTiles ? MG_TILE_PROLONG
                                                                                       : MG_TILE_HALF;
    const int var = (tiles != kFineTiles && level + 1 < h->L) ? h->tile[kind][level] : 0;
    const int blocks = tiles == kFineTiles ? fine_blocks(v.n) : kernel_blocks(kind, v.n, v.nc, var);
    const int starts[2] = {0, blocks};
    CK(cudaMemcpyAsync(h->dview, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->dstart, starts, sizeof(starts), cudaMemcpyHostToDevice, h->stream));
    *tb = Table{h->dview, h->dstart, 1, blocks, var,
                (tiles == kProlongTiles && h->prm.prolongation == MG_PROLONG_FLUX) ? 1 : 0};
    return MG_OK;
}

int mg_apply(mg_handle *h, int level, int prec, const void *x, void *y)
{
    if (!x || !y) return MG_EINVAL;
    Table tb;
    int rc = unit_view(h, level, prec, x, y, nullptr, nullptr, &tb, kFineTiles);
    if (rc) return rc;
    if (prec == MG_PREC_MIXED) launch_apply<float>(tb, h->stream);
    else launch_apply<double>(tb, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_smooth(mg_handle *h, int level, int prec, const void *b, void *x, int sweeps)
{
    if (!h || !x || !b || sweeps < 0) return MG_EINVAL;
    Table tb;
    int rc = unit_view(h, level, prec, x, (void *)b, nullptr, nullptr, &tb, kHalfTiles);
    if (rc) return rc;
    for (int s = 0; s < sweeps; s++) {
        for (int colour = 0; colour < 2; colour++) {
            if (prec == MG_PREC_MIXED) launch_half<float>(tb, colour, h->prm.omega, 0, nullptr, h->stream);
            else launch_half<double>(tb, colour, h->prm.omega, 0, nullptr, h->stream);
        }
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_smooth_onepass(mg_handle *h, int level, int prec, const void *b, void *x, void *work, int sweeps,
                      int variant)
{
    if (!h || !x || !b || !work || sweeps < 0 || level < 0 || level >= h->L) return MG_EINVAL;
    if (variant < 0 || variant >= kSweepVariants) return MG_EINVAL;
    if (prec != MG_PREC_FP64 && prec != MG_PREC_MIXED) return MG_EINVAL;
    if (prec == MG_PREC_MIXED && !h->mixed) return MG_EINVAL;
    if (variant == 0) variant = level == 0 ? h->tile[MG_TILE_SWEEP][0] : 0;
    const HLevel &L = h->lev[level];
    if (!sweep_fits(L.n, h->per, variant, prec == MG_PREC_MIXED)) return MG_EINVAL;
    LevelView v;
    memset(&v, 0, sizeof(v));
    for (int d = 0; d < 3; d++) {
        v.n[d] = L.n[d];
        v.w[d] = prec == MG_PREC_MIXED ? (void *)L.w32[d] : (void *)L.w64[d];
    }
    v.per = h->per;
    v.x = x;
    v.x2 = work;
    v.b = (void *)b;
    v.st = h->dstate;
    v.dinv = prec == MG_PREC_FP64 ? L.dinv : nullptr;
    fill_fastdiv(v);
    const int blocks = sweep_layout(v, variant);
    const int starts[2] = {0, blocks};
    CK(cudaMemcpyAsync(h->dview, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->dstart, starts, sizeof(starts), cudaMemcpyHostToDevice, h->stream));
    Table tb{h->dview, h->dstart, 1, blocks, variant};
    tb.hv = &v;
    for (int it = 0; it < sweeps; it++) {
        if (prec == MG_PREC_MIXED) launch_sweep<float>(tb, it & 1, h->prm.omega, 0, nullptr, h->stream);
        else launch_sweep<double>(tb, it & 1, h->prm.omega, 0, nullptr, h->stream);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_restrict_residual(mg_handle *h, int level, int prec, const void *b, const void *x,
                         void *coarse_b)
{
    if (!x || !b || !coarse_b || !h || level + 1 >= h->L) return MG_EINVAL;
    Table tb;
    int rc = unit_view(h, level, prec, x, (void *)b, nullptr, coarse_b, &tb, kCoarseTiles);
    if (rc) return rc;
    if (prec == MG_PREC_MIXED) launch_restrict<float>(tb, h->prm.omega, h->stream);
    else launch_restrict<double>(tb, h->prm.omega, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_prolong(mg_handle *h, int level, int prec, const void *coarse_e, void *x)
{
    if (!x || !coarse_e || !h || level + 1 >= h->L) return MG_EINVAL;
    Table tb;
    int rc = unit_view(h, level, prec, x, nullptr, coarse_e, nullptr, &tb, kProlongTiles);
    if (rc) return rc;
    if (prec == MG_PREC_MIXED) launch_prolong<float>(tb, nullptr, h->stream);
    else launch_prolong<double>(tb, nullptr, h->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

int mg_coarse_solve(mg_handle *h, int prec, const void *r, void *e)
{
    if (!h || !r || !e) return MG_EINVAL;
    if (prec != MG_PREC_FP64 && prec != MG_PREC_MIXED) return MG_EINVAL;
    if (prec == MG_PREC_MIXED && !h->mixed) return MG_EINVAL;
    const HLevel &C = h->lev[h->L - 1];
    CoarseView v;
    memset(&v, 0, sizeof(v));
    for (int d = 0; d < 3; d++) {
        v.n[d] = C.n[d];
        v.w[d] = C.w64[d];
    }
    v.per = h->per;
    v.nc = (int)C.N;
    v.G = h->G;
    v.x = e;
    v.b = r;
    v.st = h->dstate;
    v.err = h->err + 1;
    v.gmres = h->gmres ? 1 : 0;
    v.gm = h->gm;
    v.gm_max = h->prm.coarse_max_iters;
    v.gm_tol = h->prm.coarse_tol;
    CK(cudaMemcpyAsync(h->dcview, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    if (h->gmres) {
        if (prec == MG_PREC_MIXED) launch_coarse_gmres<float>(h->dcview, 1, 0, nullptr, h->stream);
        else launch_coarse_gmres<double>(h->dcview, 1, 0, nullptr, h->stream);
    } else {
        if (prec == MG_PREC_MIXED) launch_coarse_solve<float>(h->dcview, 1, 0, nullptr, h->stream);
        else launch_coarse_solve<double>(h->dcview, 1, 0, nullptr, h->stream);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

// ---- profiling / memory ---------------------------------------------------------

int mg_profile_enable(mg_handle *h, int enable)
{
    if (!h) return MG_EINVAL;
    h->prof.on = enable != 0;
    h->prof.reset();
    return MG_OK;
}

int mg_profile_read(mg_handle *h, int kind, int level, int64_t *launches, double *total_ms)
{
    if (!h || kind < 0 || kind >= MG_K_KINDS || level < 0 || level >= MG_MAX_LEVELS) return MG_EINVAL;
    if (launches) *launches = h->prof.launches[kind][level];
    if (total_ms) *total_ms = h->prof.total_ms[kind][level];
    return MG_OK;
}

int mg_set_wait_limit(mg_handle *h, long long polls)
{
    if (!h || polls < 0) return MG_EINVAL;
    h->wait_polls = polls;
    // the tail views live in the plan's device tables (read by the kernels at
    // run time, also from a captured graph): rewrite them
    if (h->plan) {
        mg_handle *one = h;
        int rc = h->plan->fill(&one, 1);
        if (rc) return rc;
        CK(cudaStreamSynchronize(h->stream));
    }
    return MG_OK;
}

int mg_handle_params(const mg_handle *h, mg_params *params)
{
    if (!h || !params) return MG_EINVAL;
    *params = h->prm;
    return MG_OK;
}

int mg_memory_bytes(const mg_handle *h, size_t *bytes)
{
    if (!h || !bytes) return MG_EINVAL;
    *bytes = h->bytes;
    return MG_OK;
}

int mg_memory_estimate(const mg_grid *grid, const mg_params *params, size_t *bytes)
{
    if (!bytes) return MG_EINVAL;
    int rc = check_grid(grid);
    if (rc) return rc;
    mg_params prm;
    mg_params_default(&prm);
    if (params) prm = *params;
    rc = check_params(&prm);
    if (rc) return rc;
    Layout lay;
    rc = plan_layout(*grid, prm, lay);
    if (rc) return rc;
    *bytes = lay.total;
    return MG_OK;
}

}  // extern "C"
