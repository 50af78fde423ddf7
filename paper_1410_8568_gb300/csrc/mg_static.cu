// mg_static.cu -- exact small-grid solve that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: real-time loops whose device memory is budgeted up front, or host
// programs whose own allocator has reserved the device memory (cudaMalloc may
// then fail, and it can synchronise the device).  For them
// mg_coarse_solve_static solves a grid of at most MG_STATIC_MAX_CELLS cells
// exactly, using only a scratch area that lives for the whole process in this
// file's static device array.  The first call on a device looks up the
// array's device address (and, with lazy module loading, loads this file's
// device code): make it at start-up, before any stream capture begins; later
// calls allocate nothing.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; the kernel rewrites everything it reads before reading it.
// Two calls whose kernels overlap on the GPU (different streams, no ordering)
// race on the scratch array and give wrong results: order them.
#include <mutex>

#include "gbmg.h"
#include "mg_device.cuh"

namespace {

constexpr int kMaxCells = MG_STATIC_MAX_CELLS;
constexpr int kThreadsStatic = 1024;

// dense matrix of the bordered-free regularised system (kMaxCells^2 doubles,
// 2 MiB) followed by an error flag
static __device__ __align__(256) double g_static_scratch[kMaxCells * kMaxCells + 32];

struct StaticArgs {
    int n[3];
    int per;
    double scale[3];  // 1 / h_d^2
    const double *a[3];
    const double *r;
    double *e;
    double *S;        // device address of g_static_scratch
};

// One block: assemble S = -A + c 1 1^T (A the operator of the cell-centred
// scheme with face coefficients alpha / h^2, c = mean diagonal / n), invert it
// in place by Gauss-Jordan elimination (S is symmetric positive definite, no
// pivoting), and apply e = -S^{-1} r.  A non-positive pivot (a grid cut into
// pieces by zero coefficients) sets the flag after the matrix to 1, a
// non-positive or non-finite coefficient off the walls sets it to 2.
__global__ void __launch_bounds__(kThreadsStatic) k_coarse_static(StaticArgs A)
{
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int n = nx * ny * nz;
    double *S = A.S;
    double *flag = S + (long long)kMaxCells * kMaxCells;
    __shared__ double col[kMaxCells];
    __shared__ double rr[kMaxCells];
    __shared__ double red[32];
    __shared__ double c0;
    __shared__ int bad;
    if (threadIdx.x == 0) {
        bad = 0;
        flag[0] = 0.0;
    }
    for (long long q = threadIdx.x; q < (long long)n * n; q += blockDim.x) S[q] = 0.0;
    __syncthreads();
    double dsum = 0.0;
    int badc = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int q[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
        const int nn[3] = {nx, ny, nz};
        const long long stride[3] = {1, nx, (long long)nx * ny};
        double diag = 0.0;
        for (int d = 0; d < 3; d++) {
            const bool periodic = (A.per >> d) & 1;
            if (q[d] > 0 || periodic) {  // low face: stored at the cell itself
                const double alpha = A.a[d][c];
                if (!(alpha > 0.0) || !isfinite(alpha)) badc = 1;
                const long long nb = q[d] > 0 ? c - stride[d] : c + stride[d] * (nn[d] - 1);
                if (nb != c) {
                    const double w = alpha * A.scale[d];
                    diag += w;
                    S[(long long)c * n + nb] -= w;
                }
            }
            if (q[d] + 1 < nn[d] || periodic) {  // high face: the low face of the next cell
                const long long nb = q[d] + 1 < nn[d] ? c + stride[d] : c - stride[d] * (nn[d] - 1);
                if (nb != c) {
                    const double w = A.a[d][nb] * A.scale[d];
                    diag += w;
                    S[(long long)c * n + nb] -= w;
                }
            }
        }
        S[(long long)c * n + c] += diag;
        dsum += diag;
        rr[c] = A.r[c];
    }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dsum;
    if (badc) bad = 2;
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
    for (int k = 0; k < n && !bad; k++) {
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
    if (bad) {
        if (threadIdx.x == 0) flag[0] = (double)bad;
        return;
    }
    // e = -S^{-1} r, one warp per row, fixed shuffle tree
    for (int t = wid; t < n; t += warps) {
        const double *St = S + (long long)t * n;
        double s = 0.0;
        for (int u = lane; u < n; u += 32) s += St[u] * rr[u];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) A.e[t] = -s;
    }
}

// device address of the scratch array, looked up once per device
std::mutex g_static_mu;
double *g_static_ptr[256] = {};

}  // namespace

extern "C" int mg_coarse_solve_static(const mg_grid *grid, const double *ax, const double *ay,
                                      const double *az, const double *r, double *e, void *stream)
{
    if (!grid || !ax || !ay || !az || !r || !e) return MG_EINVAL;
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    const double len[3] = {grid->lx, grid->ly, grid->lz};
    for (int d = 0; d < 3; d++) {
        if (n[d] < 1 || !(len[d] > 0.0) || !isfinite(len[d])) return MG_EINVAL;
        if (grid->bc[d] != MG_BC_NEUMANN && grid->bc[d] != MG_BC_PERIODIC) return MG_EINVAL;
    }
    if ((long long)n[0] * n[1] * n[2] > kMaxCells) return MG_ETOOBIG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return MG_ECUDA;
    double *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            // host code only holds a stand-in for the array: ask for its device address
            double *p = nullptr;
            if (cudaGetSymbolAddress((void **)&p, g_static_scratch) != cudaSuccess || !p) return MG_ECUDA;
            g_static_ptr[dev] = p;
        }
        S = g_static_ptr[dev];
    }
    StaticArgs A;
    for (int d = 0; d < 3; d++) {
        A.n[d] = n[d];
        A.scale[d] = 1.0 / ((len[d] / n[d]) * (len[d] / n[d]));
    }
    A.per = (grid->bc[0] == MG_BC_PERIODIC ? 1 : 0) | (grid->bc[1] == MG_BC_PERIODIC ? 2 : 0) |
            (grid->bc[2] == MG_BC_PERIODIC ? 4 : 0);
    A.a[0] = ax;
    A.a[1] = ay;
    A.a[2] = az;
    A.r = r;
    A.e = e;
    A.S = S;
    cudaStream_t s = (cudaStream_t)stream;
    k_coarse_static<<<1, kThreadsStatic, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
    double flag = 0.0;
    if (cudaMemcpyAsync(&flag, S + (long long)kMaxCells * kMaxCells, sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MG_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MG_ECUDA;
    if (flag == 2.0) return MG_EINVAL;
    return flag != 0.0 ? MG_ESINGULAR : MG_OK;
}
