// mg_tune.cu -- autotuner of the launch shapes of the V-cycle kernels.
//
// The half-sweep, restriction and prolongation kernels each come in
// kTileVariants launch shapes (tile_shape in mg_device.cuh): the row tiling and
// six flat tilings that differ in threads per block and items per thread.  The
// best shape depends on the level size: large levels are bound by HBM
// bandwidth and want enough loads in flight per SM, small levels are bound by
// latency and want their few quads spread over as many SMs and warps as
// possible.  The tuner times every shape that fits a level on the handle's own
// buffers and keeps the fastest; choices are cached per process by (kernel,
// precision, periodic axes, level size), so each level size is timed once.
//
// Timing runs on the handle's V-cycle work arrays (x, b of each level), which
// hold no caller data between solves; coefficients need not be set yet.  The
// kernels have no data-dependent control flow, so the values in those arrays
// do not change the timings.  A shape never changes a result: the per-cell
// arithmetic is shared by all shapes, and the tests check solves bitwise equal
// across shapes.
//
// The choices can outlive the process: mg_tune_cache_save / _load write and
// read them as text, one line per choice ("kind mixed per nx ny nz variant"),
// and when the environment variable MG_TUNE_CACHE names a file, the first
// tuning of the process loads it and every new choice is appended to it.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>

#include "mg_api_internal.h"

#define TK(call)                          \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess) {          \
            gbmg::note_cuda_error(e_);    \
            return MG_ECUDA;              \
        }                                 \
    } while (0)

namespace gbmg {

// First level of a grid handled by the bottom-of-cycle kernel: the first level
// below the finest with at most kTailCells cells, if at least one level above
// the coarsest qualifies (else the grid has no tail: L).  FP32 cycles only: one
// block per grid runs at one SM's FP64 rate, which on this GPU is far below
// that of the per-level FP64 kernels spread over all SMs.
int first_tail_level(const mg_handle *h)
{
    if (!h->mixed || h->gmres) return h->L;  // the tail solves the coarsest grid with its inverse
    for (int l = 1; l + 1 < h->L && l < MG_MAX_LEVELS; l++)
        if (h->lev[l].N <= kTailCells && h->L - l <= kMaxTail) return l;
    return h->L;
}

void fill_fastdiv(LevelView &v)
{
    v.dq = make_fastdiv(v.n[0] >= 4 ? (unsigned)(v.n[0] >> 2) : 1u);
    v.dy = make_fastdiv(v.n[1] >= 1 ? (unsigned)v.n[1] : 1u);
    v.dp = make_fastdiv(v.nc[0] >= 2 ? (unsigned)(v.nc[0] >> 1) : 1u);
    v.dcy = make_fastdiv(v.nc[1] >= 1 ? (unsigned)v.nc[1] : 1u);
    v.dxq = make_fastdiv((unsigned)(((v.n[0] >> 2) + 31) >> 5 > 0 ? ((v.n[0] >> 2) + 31) >> 5 : 1));
    v.dxp = make_fastdiv((unsigned)(((v.nc[0] >> 1) + 31) >> 5 > 0 ? ((v.nc[0] >> 1) + 31) >> 5 : 1));
    v.dxc = make_fastdiv((unsigned)(coarse_xtiles(v.nc[0]) > 0 ? coarse_xtiles(v.nc[0]) : 1));
    v.dxt = make_fastdiv((unsigned)(fine_xtiles(v.n[0]) > 0 ? fine_xtiles(v.n[0]) : 1));
}

int kernel_blocks(int kind, const int n[3], const int nc[3], int v)
{
    return kind == MG_TILE_RESTRICT ? restrict_blocks_v(n, nc, v)
         : kind == MG_TILE_PROLONG  ? prolong_blocks_v(n, nc, v)
                                    : half_sweep_blocks_v(n, v);
}

namespace {

struct TuneKey {
    int kind, mixed, per, n[3];
    bool operator<(const TuneKey &o) const { return memcmp(this, &o, sizeof(TuneKey)) < 0; }
};

std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
bool g_env_loaded = false;

// read choices from `path` into the cache (caller holds g_tune_mu); lines that
// do not parse or name an unknown shape are skipped
int load_locked(const char *path, int *loaded)
{
    FILE *f = fopen(path, "r");
    if (!f) return MG_ENOTFOUND;
    char line[256];
    int n = 0;
    while (fgets(line, sizeof(line), f)) {
        TuneKey k;
        memset(&k, 0, sizeof(k));
        int v;
        if (sscanf(line, "%d %d %d %d %d %d %d", &k.kind, &k.mixed, &k.per, &k.n[0], &k.n[1], &k.n[2], &v) != 7)
            continue;
        if (k.kind < 0 || k.kind > MG_TILE_SWEEP || (k.mixed != 0 && k.mixed != 1) || k.per < 0 || k.per > 7 ||
            v < 0)
            continue;
        if (k.kind == MG_TILE_SWEEP ? (v >= kSweepVariants || (v > 0 && !sweep_fits(k.n, k.per, v, k.mixed == 1)))
                                    : (v >= kTileVariants || !tile_fits(k.n, v)))
            continue;
        g_tune[k] = v;
        n++;
    }
    fclose(f);
    if (loaded) *loaded = n;
    return MG_OK;
}

void write_line(FILE *f, const TuneKey &k, int v)
{
    fprintf(f, "%d %d %d %d %d %d %d\n", k.kind, k.mixed, k.per, k.n[0], k.n[1], k.n[2], v);
}

// the environment's cache file, read once per process (caller holds g_tune_mu)
const char *env_cache_locked()
{
    const char *path = getenv("MG_TUNE_CACHE");
    if (!path || !*path) return nullptr;
    if (!g_env_loaded) {
        g_env_loaded = true;
        load_locked(path, nullptr);
    }
    return path;
}

template <class T>
int time_shape(mg_handle *h, int kind, int l, int v, float *ms)
{
    const HLevel &F = h->lev[l], &C = h->lev[l + 1];
    LevelView lv;
    memset(&lv, 0, sizeof(lv));
    for (int d = 0; d < 3; d++) {
        lv.n[d] = F.n[d];
        lv.nc[d] = C.n[d];
        lv.w[d] = h->mixed ? (void *)F.w32[d] : (void *)F.w64[d];
    }
    lv.per = h->per;
    lv.x = F.x;
    lv.b = F.b;
    lv.xc = C.x;
    lv.bc = C.b;
    lv.st = h->dstate;
    lv.dinv = h->mixed ? nullptr : F.dinv;
    lv.dinvc = h->mixed ? nullptr : C.dinv;
    fill_fastdiv(lv);
    const int blocks = kernel_blocks(kind, lv.n, lv.nc, v);
    const int starts[2] = {0, blocks};
    cudaStream_t s = h->stream;
    TK(cudaMemcpyAsync(h->dview, &lv, sizeof(lv), cudaMemcpyHostToDevice, s));
    TK(cudaMemcpyAsync(h->dstart, starts, sizeof(starts), cudaMemcpyHostToDevice, s));
    Table tb{h->dview, h->dstart, 1, blocks, v};
    tb.hv = &lv;  // as the solves launch one-grid tables
    auto run = [&](int i) {
        if (kind == MG_TILE_RESTRICT) launch_restrict<T>(tb, 1.0, s);
        else if (kind == MG_TILE_PROLONG) launch_prolong<T>(tb, nullptr, s);
        else launch_half<T>(tb, i & 1, 1.0, 0, nullptr, s);
    };
    cudaEvent_t e0, e1;
    TK(cudaEventCreate(&e0));
    TK(cudaEventCreate(&e1));
    // one launch to estimate, then enough launches for about half a millisecond
    run(0);
    run(1);
    cudaEventRecord(e0, s);
    run(0);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float one = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&one, e0, e1);
    int reps = one > 0.f ? (int)(0.5f / one) : 64;
    reps = reps < 4 ? 4 : (reps > 64 ? 64 : reps);
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; i++) run(i);
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float tot = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&tot, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    TK(err);
    *ms = tot / reps;
    return MG_OK;
}

// One full red-black sweep of the finest level: two half-sweep launches in
// the level's tuned half-sweep shape (v = 0) or one one-pass launch of shape v
// (alternating between the two iterate buffers).
template <class T>
int time_sweep(mg_handle *h, int v, float *ms)
{
    const HLevel &F = h->lev[0], &C = h->lev[1];
    LevelView lv;
    memset(&lv, 0, sizeof(lv));
    for (int d = 0; d < 3; d++) {
        lv.n[d] = F.n[d];
        lv.nc[d] = C.n[d];
        lv.w[d] = h->mixed ? (void *)F.w32[d] : (void *)F.w64[d];
    }
    lv.per = h->per;
    lv.x = F.x;
    lv.x2 = F.x2;
    lv.b = F.b;
    lv.xc = C.x;
    lv.bc = C.b;
    lv.st = h->dstate;
    lv.dinv = h->mixed ? nullptr : F.dinv;
    lv.dinvc = h->mixed ? nullptr : C.dinv;
    fill_fastdiv(lv);
    const int hv = h->tile[MG_TILE_HALF][0];
    const int blocks = v > 0 ? sweep_layout(lv, v) : half_sweep_blocks_v(lv.n, hv);
    const int starts[2] = {0, blocks};
    cudaStream_t s = h->stream;
    TK(cudaMemcpyAsync(h->dview, &lv, sizeof(lv), cudaMemcpyHostToDevice, s));
    TK(cudaMemcpyAsync(h->dstart, starts, sizeof(starts), cudaMemcpyHostToDevice, s));
    Table tb{h->dview, h->dstart, 1, blocks, v > 0 ? v : hv};
    tb.hv = &lv;
    auto run = [&](int i) {
        if (v > 0) {
            launch_sweep<T>(tb, i & 1, 1.0, 0, nullptr, s);
        } else {
            launch_half<T>(tb, 0, 1.0, 0, nullptr, s);
            launch_half<T>(tb, 1, 1.0, 0, nullptr, s);
        }
    };
    cudaEvent_t e0, e1;
    TK(cudaEventCreate(&e0));
    TK(cudaEventCreate(&e1));
    run(0);
    run(1);
    cudaEventRecord(e0, s);
    run(0);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float one = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&one, e0, e1);
    int reps = one > 0.f ? (int)(0.5f / one) : 64;
    reps = reps < 4 ? 4 : (reps > 64 ? 64 : reps);
    reps &= ~1;  // an even number: the one-pass sweeps end in the first buffer
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; i++) run(i);
    cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float tot = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&tot, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    TK(err);
    *ms = tot / reps;
    return MG_OK;
}

// Finest-level sweep: MG_SWEEP_HALF, a forced one-pass shape, or the fastest
// of the half-sweep pair and every one-pass shape that fits (cached like the
// launch shapes).
int tune_sweep(mg_handle *h)
{
    h->tile[MG_TILE_SWEEP][0] = 0;
    if (!h->lev[0].x2 || h->L < 2 || first_tail_level(h) < 1) return MG_OK;
    const int *n = h->lev[0].n;
    const int forced = h->prm.sweep;
    if (forced >= 0) {
        h->tile[MG_TILE_SWEEP][0] = (signed char)((forced > 0 && sweep_fits(n, h->per, forced, h->mixed)) ? forced : 0);
        return MG_OK;
    }
    TuneKey key;
    memset(&key, 0, sizeof(key));
    key.kind = MG_TILE_SWEEP;
    key.mixed = h->mixed;
    key.per = h->per;
    for (int d = 0; d < 3; d++) key.n[d] = n[d];
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        env_cache_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            h->tile[MG_TILE_SWEEP][0] = (signed char)it->second;
            return MG_OK;
        }
    }
    float t[kSweepVariants];
    for (int v = 0; v < kSweepVariants; v++) t[v] = -1.f;
    for (int round = 0; round < 3; round++)
        for (int v = 0; v < kSweepVariants; v++) {
            if (v > 0 && !sweep_fits(n, h->per, v, h->mixed)) continue;
            float ms = 0.f;
            const int rc = h->mixed ? time_sweep<float>(h, v, &ms) : time_sweep<double>(h, v, &ms);
            if (rc) return rc;
            t[v] = (t[v] < 0.f || ms < t[v]) ? ms : t[v];
        }
    int best = 0;
    for (int v = 1; v < kSweepVariants; v++)
        if (t[v] >= 0.f && t[v] < t[best]) best = v;
    h->tile[MG_TILE_SWEEP][0] = (signed char)best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
    if (const char *path = env_cache_locked()) {
        if (FILE *f = fopen(path, "a")) {
            write_line(f, key, best);
            fclose(f);
        }
    }
    return MG_OK;
}

}  // namespace

int tune_handle(mg_handle *h)
{
    memset(h->tile, 0, sizeof(h->tile));
    const int forced = h->prm.tiles;
    const int lt = first_tail_level(h);
    for (int l = 0; l + 1 < h->L; l++) {
        const int *n = h->lev[l].n;
        for (int kind = 0; kind < 3; kind++) {
            if (kind == MG_TILE_PROLONG && h->prm.prolongation == MG_PROLONG_FLUX) continue;  // row tiles
            if (forced >= 0) {
                h->tile[kind][l] = (signed char)(tile_fits(n, forced) ? forced : 0);
                continue;
            }
            if (l >= lt || !tile_fits(n, 1)) continue;  // row tiles only
            TuneKey key;
            memset(&key, 0, sizeof(key));
            key.kind = kind;
            key.mixed = h->mixed;
            key.per = h->per;
            for (int d = 0; d < 3; d++) key.n[d] = n[d];
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                env_cache_locked();
                auto it = g_tune.find(key);
                if (it != g_tune.end()) {
                    h->tile[kind][l] = (signed char)it->second;
                    continue;
                }
            }
            // three interleaved rounds over the shapes, best time of each: drift
            // of clocks or of other work on the GPU hits every shape alike
            float t[kTileVariants];
            for (int round = 0; round < 3; round++)
                for (int v = 0; v < kTileVariants; v++) {
                    float ms = 0.f;
                    const int rc = h->mixed ? time_shape<float>(h, kind, l, v, &ms)
                                            : time_shape<double>(h, kind, l, v, &ms);
                    if (rc) return rc;
                    t[v] = round == 0 || ms < t[v] ? ms : t[v];
                }
            int best = 0;
            for (int v = 1; v < kTileVariants; v++)
                if (t[v] < t[best]) best = v;
            h->tile[kind][l] = (signed char)best;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = best;
            if (const char *path = env_cache_locked()) {
                if (FILE *f = fopen(path, "a")) {
                    write_line(f, key, best);
                    fclose(f);
                }
            }
        }
    }
    return tune_sweep(h);
}

void tune_cache_clear()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // namespace gbmg

extern "C" {

int mg_tile_choice(const mg_handle *h, int kind, int level, int *variant)
{
    if (!h || !variant || kind < 0 || kind > MG_TILE_SWEEP || level < 0 || level >= h->L) return MG_EINVAL;
    *variant = level + 1 < h->L ? h->tile[kind][level] : 0;
    return MG_OK;
}

int mg_sweep_shape(int variant, int *threads, int *planes, int *tile_x)
{
    if (variant < 0 || variant >= gbmg::kSweepVariants || !threads || !planes || !tile_x) return MG_EINVAL;
    const gbmg::SweepShape sh = gbmg::sweep_shape(variant);
    *threads = sh.B;
    *planes = sh.Kc;
    *tile_x = sh.tile_x;
    return MG_OK;
}

int mg_tile_shape(int variant, int *threads, int *items_per_thread)
{
    if (variant < 0 || variant >= gbmg::kTileVariants || !threads || !items_per_thread) return MG_EINVAL;
    const gbmg::TileShape ts = gbmg::tile_shape(variant);
    *threads = ts.B;
    *items_per_thread = ts.Q;
    return MG_OK;
}

int mg_tune_cache_clear(void)
{
    gbmg::tune_cache_clear();
    return MG_OK;
}

int mg_tune_cache_save(const char *path)
{
    if (!path) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(gbmg::g_tune_mu);
    FILE *f = fopen(path, "w");
    if (!f) return MG_EINVAL;
    for (const auto &kv : gbmg::g_tune) gbmg::write_line(f, kv.first, kv.second);
    return fclose(f) == 0 ? MG_OK : MG_EINVAL;
}

int mg_tune_cache_load(const char *path, int *loaded)
{
    if (!path) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(gbmg::g_tune_mu);
    return gbmg::load_locked(path, loaded);
}

int mg_tune_cache_size(int *entries)
{
    if (!entries) return MG_EINVAL;
    std::lock_guard<std::mutex> lk(gbmg::g_tune_mu);
    *entries = (int)gbmg::g_tune.size();
    return MG_OK;
}

}  // extern "C"
