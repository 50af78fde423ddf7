// mg_tiles.cu -- flat-tiled variants of the half-sweep, restriction and
// prolongation kernels, and the launchers that run a table with the launch
// shape chosen for it (Table::variant, see tile_shape in mg_device.cuh).
//
// The per-quad arithmetic is the same code as the row-tiled kernels
// (mg_stencil.cuh), and every cell's result depends only on its own operands,
// so a solve gives bitwise the same result whatever shapes are chosen.
#include <type_traits>

#include "mg_kernels.h"
#include "mg_stencil.cuh"

namespace gbmg {

// Block lb of a table entry owns items [lb Q B, (lb + 1) Q B); thread t handles
// lb Q B + q B + t for q < Q.  Items are numbered row by row, so consecutive
// threads touch consecutive 16-byte vectors.
template <class T, int B, int Q, bool OUT>
__device__ __forceinline__ void half_flat_body(const LevelView &L, int lb, int colour, T omega, bool zero,
                                               const OuterOut &po, bool go = true)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], nq = nx >> 2;
    const int items = nq * ny * nz;
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int g = (lb * Q + q) * B + (int)threadIdx.x;
        if (g >= items) return;
        const int row = fdiv(g, L.dq);
        const int k = fdiv(row, L.dy);
        half_quad<T, OUT>((T *)L.x, (const T *)L.b, (const T *)L.w[0], (const T *)L.w[1],
                          (const T *)L.w[2], nx, ny, nz, L.per, row, row - k * ny, k, g - row * nq, colour,
                          omega, zero, po, go, (const T *)L.dinv);
    }
}

// MAYOUT: the launch carries kOuter (see k_half)
// defer: see half_entry
template <class T, int B, int Q, bool MAYOUT>
__device__ __forceinline__ void half_flat_entry(const LevelView &L, int lb, int colour, T omega, int flags,
                                                int cyc, const OuterView *__restrict__ ov, bool defer)
{
    const bool zero = flags & kZeroGuess;
    if (!MAYOUT && defer) {
        half_flat_body<T, B, Q, false>(L, lb, colour, omega, zero, OuterOut{}, in_cycle(L.st, cyc));
        return;
    }
    if (!in_cycle(L.st, cyc)) return;
    if constexpr (MAYOUT) {
        if (last_cycle(L.st, cyc)) {
            half_flat_body<T, B, Q, true>(L, lb, colour, omega, zero, outer_out(ov[L.g]));
            return;
        }
    }
    half_flat_body<T, B, Q, false>(L, lb, colour, omega, zero, OuterOut{});
}

// single: a one-grid table, its view passed by value (see k_half)
template <class T, int B, int Q, bool MAYOUT>
__global__ void __launch_bounds__(B) k_half_flat(const LevelView *__restrict__ lv,
                                                 const int *__restrict__ start, int count,
                                                 int colour, T omega, int flags, int cyc,
                                                 const OuterView *__restrict__ ov,
                                                 const __grid_constant__ LevelView one, int single)
{
    dep_entry();
    if (single) {
        half_flat_entry<T, B, Q, MAYOUT>(one, blockIdx.x, colour, omega, flags, cyc, ov, true);
        return;
    }
    const int e = find_entry(start, count);
    half_flat_entry<T, B, Q, MAYOUT>(lv[e], blockIdx.x - start[e], colour, omega, flags, cyc, ov, false);
}

// defer: see half_entry
template <class T, int B, int Q>
__device__ __forceinline__ void restrict_flat_entry(const LevelView &L, int lb, int cyc, T omega, bool defer)
{
    const bool go = in_cycle(L.st, cyc);
    if (!defer && !go) return;
    const int np = L.nc[0] >> 1, ncy = L.nc[1];
    const int items = np * ncy * L.nc[2];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int g = (lb * Q + q) * B + (int)threadIdx.x;
        if (g >= items) return;
        const int crow = fdiv(g, L.dp);
        const int K = fdiv(crow, L.dcy);
        restrict_pair<T>(L, crow, crow - K * ncy, K, g - crow * np, omega, go);
    }
}

template <class T, int B, int Q>
// at least 1024 threads per SM (64 registers a thread): the residuals of the
// 4 fine rows hold many operands in flight, and unbounded the kernel took 86
// registers and left DRAM 67 % busy at 29 % of the SM's warps
__global__ void __launch_bounds__(B, 1024 / B) k_restrict_flat(const LevelView *__restrict__ lv,
                                                     const int *__restrict__ start, int count, int cyc,
                                                     T omega, const __grid_constant__ LevelView one,
                                                     int single)
{
    dep_entry();
    if (single) {
        restrict_flat_entry<T, B, Q>(one, blockIdx.x, cyc, omega, true);
        return;
    }
    const int e = find_entry(start, count);
    restrict_flat_entry<T, B, Q>(lv[e], blockIdx.x - start[e], cyc, omega, false);
}

// defer: see half_entry
template <class T, int B, int Q>
__device__ __forceinline__ void prolong_flat_entry(const LevelView &L, int lb, int cyc, bool defer)
{
    // items: coarse cell pairs; each covers a quad of the 2 x 2 fine rows above it
    const bool go = in_cycle(L.st, cyc);
    if (!defer && !go) return;
    const int np = L.nc[0] >> 1, ncy = L.nc[1];
    const int items = np * ncy * L.nc[2];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int g = (lb * Q + q) * B + (int)threadIdx.x;
        if (g >= items) return;
        const int crow = fdiv(g, L.dp);
        const int K = fdiv(crow, L.dcy);
        prolong_block<T>(L, crow - K * ncy, K, g - crow * np, go);
    }
}

template <class T, int B, int Q>
__global__ void __launch_bounds__(B) k_prolong_flat(const LevelView *__restrict__ lv,
                                                    const int *__restrict__ start, int count, int cyc,
                                                    const __grid_constant__ LevelView one, int single)
{
    dep_entry();
    if (single) {
        prolong_flat_entry<T, B, Q>(one, blockIdx.x, cyc, true);
        return;
    }
    const int e = find_entry(start, count);
    prolong_flat_entry<T, B, Q>(lv[e], blockIdx.x - start[e], cyc, false);
}

namespace {

// call f(std::integral_constant<int, v>) for a flat variant v (1 .. kTileVariants - 1)
template <class F>
bool with_variant(int v, F &&f)
{
    switch (v) {
    case 1: f(std::integral_constant<int, 1>{}); return true;
    case 2: f(std::integral_constant<int, 2>{}); return true;
    case 3: f(std::integral_constant<int, 3>{}); return true;
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 5: f(std::integral_constant<int, 5>{}); return true;
    case 6: f(std::integral_constant<int, 6>{}); return true;
    default: return false;
    }
}
static_assert(kTileVariants == 7, "with_variant lists every flat variant");

int flat_blocks(long long items, int v)
{
    const TileShape ts = tile_shape(v);
    const long long per = (long long)ts.B * ts.Q;
    return (int)((items + per - 1) / per);
}

}  // namespace

bool tile_fits(const int n[3], int v) { return v == 0 || (v > 0 && v < kTileVariants && (n[0] & 3) == 0); }

int half_sweep_blocks_v(const int n[3], int v)
{
    if (v == 0) return half_sweep_blocks(n);
    return flat_blocks((long long)(n[0] >> 2) * n[1] * n[2], v);
}

int prolong_blocks_v(const int n[3], const int nc[3], int v)
{
    if (v == 0) return prolong_blocks(n);
    return flat_blocks((long long)(nc[0] >> 1) * nc[1] * nc[2], v);
}

int restrict_blocks_v(const int n[3], const int nc[3], int v)
{
    if (v == 0) return restrict_blocks(n, nc);
    return flat_blocks((long long)(nc[0] >> 1) * nc[1] * nc[2], v);
}

template <class T>
void launch_half(const Table &tb, int colour, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    if (tb.blocks == 0) return;
    const bool flat = with_variant(tb.variant, [&](auto V) {
        constexpr TileShape ts = tile_shape(decltype(V)::value);
        if (flags & kOuter)
            launch_k(k_half_flat<T, ts.B, ts.Q, true>, tb.blocks, ts.B, 0, s, tb.lv, tb.start, tb.count, colour,
                     (T)omega, flags, tb.cyc, ov, table_view(tb), table_single(tb));
        else
            launch_k(k_half_flat<T, ts.B, ts.Q, false>, tb.blocks, ts.B, 0, s, tb.lv, tb.start, tb.count, colour,
                     (T)omega, flags, tb.cyc, nullptr, table_view(tb), table_single(tb));
    });
    if (!flat) launch_half_rows<T>(tb, colour, omega, flags, ov, s);
}

template <class T>
void launch_restrict(const Table &tb, double omega, cudaStream_t s)
{
    if (tb.blocks == 0) return;
    const bool flat = with_variant(tb.variant, [&](auto V) {
        constexpr TileShape ts = tile_shape(decltype(V)::value);
        launch_k(k_restrict_flat<T, ts.B, ts.Q>, tb.blocks, ts.B, 0, s, tb.lv, tb.start, tb.count, tb.cyc,
                 (T)omega, table_view(tb), table_single(tb));
    });
    if (!flat) launch_restrict_rows<T>(tb, omega, s);
}

template <class T>
void launch_prolong(const Table &tb, const OuterView *ov, cudaStream_t s)
{
    if (tb.blocks == 0) return;
    if (tb.flux || ov) {  // flux-conserving prolongation, or the FP64 update: row tiles only
        launch_prolong_rows<T>(tb, ov, s);
        return;
    }
    const bool flat = with_variant(tb.variant, [&](auto V) {
        constexpr TileShape ts = tile_shape(decltype(V)::value);
        launch_k(k_prolong_flat<T, ts.B, ts.Q>, tb.blocks, ts.B, 0, s, tb.lv, tb.start, tb.count, tb.cyc,
                 table_view(tb), table_single(tb));
    });
    if (!flat) launch_prolong_rows<T>(tb, nullptr, s);
}

template void launch_half<float>(const Table &, int, double, int, const OuterView *, cudaStream_t);
template void launch_half<double>(const Table &, int, double, int, const OuterView *, cudaStream_t);
template void launch_restrict<float>(const Table &, double, cudaStream_t);
template void launch_restrict<double>(const Table &, double, cudaStream_t);
template void launch_prolong<float>(const Table &, const OuterView *, cudaStream_t);
template void launch_prolong<double>(const Table &, const OuterView *, cudaStream_t);

}  // namespace gbmg
