// mg_stencil.cuh -- per-quad device code of the V-cycle kernels, shared by the
// row-tiled kernels (mg_kernels.cu) and the flat-tiled variants (mg_tiles.cu).
//
// Shin, Chergui & Juric, arXiv 1410.8568, Sec. 2.3: the cell-centred operator
// of Eq. 10 (divided by h^2), red-black relaxation, restriction of the residual
// (mean of the 8 fine children) and trilinear prolongation of the coarse error.
// A quad is 4 consecutive cells of one grid row starting at a multiple of 4;
// every operand of a quad is one 16-byte vector (FP32) or two (FP64).
#pragma once

#include "mg_device.cuh"

namespace gbmg {

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

template <class T>
struct Quad {
    T v[4];
};

template <class T>
__device__ __forceinline__ Quad<T> ldq(const T *__restrict__ p)
{
    Quad<T> q;
    if constexpr (sizeof(T) == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = a.z;
        q.v[3] = a.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        q.v[0] = a.x;
        q.v[1] = a.y;
        q.v[2] = b.x;
        q.v[3] = b.y;
    }
    return q;
}

template <class T>
__device__ __forceinline__ void stq(T *p, const Quad<T> &q)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(q.v[0], q.v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(q.v[2], q.v[3]);
    }
}

template <class T>
__device__ __forceinline__ T relax_div(T num, T den)
{
    if constexpr (sizeof(T) == 4) return __fdividef(num, den);  // inner cycle: 2-ulp division
    else return num / den;
}

// outer_update / zero flags
constexpr int kZeroGuess = 1, kOuter = 4;

// Relaxation of the cells of colour `colour` in the aligned quad (4 qx .. 4 qx + 3,
// j, k) of row `row` = j + ny k: all operands as 16-byte vectors, the two cells
// of the other colour written back unchanged.
template <class T>
__device__ __forceinline__ void half_quad(T *x, const T *b, const T *wx, const T *wy, const T *wz,
                                          int nx, int ny, int nz, int per, int row, int j, int k,
                                          int qx, int colour, T omega, bool zero, double *pout)
{
    const long long sy = nx, sz = (long long)nx * ny;
    const int i0 = qx << 2;
    const long long c = (long long)row * nx + i0;
    const int par = (colour + j + k) & 1;  // first cell of the colour in the quad
    const Quad<T> Z{{T(0), T(0), T(0), T(0)}};
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const long long cw = i0 > 0 ? c - 1 : c + nx - 1;
    const long long ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_s = j > 0 || (per & 2), has_n = j + 1 < ny || (per & 2);
    const long long cs = j > 0 ? c - sy : c + sy * (ny - 1);
    const long long cn = j + 1 < ny ? c + sy : c - sy * (ny - 1);
    const bool has_b = k > 0 || (per & 4), has_t = k + 1 < nz || (per & 4);
    const long long cb = k > 0 ? c - sz : c + sz * (nz - 1);
    const long long ct = k + 1 < nz ? c + sz : c - sz * (nz - 1);
    const Quad<T> bq = ldq(b + c);
    const Quad<T> fx = ldq(wx + c);
    const T fxe = has_e ? wx[ce] : T(0);  // high x face of the last cell
    const Quad<T> fy = ldq(wy + c);
    const Quad<T> fyn = has_n ? ldq(wy + cn) : Z;
    const Quad<T> fz = ldq(wz + c);
    const Quad<T> fzt = has_t ? ldq(wz + ct) : Z;
    Quad<T> xq = Z, xs = Z, xn = Z, xb = Z, xt = Z;
    T xw = T(0), xe = T(0);
    if (!zero) {
        xq = ldq(x + c);
        if (has_s) xs = ldq(x + cs);
        if (has_n) xn = ldq(x + cn);
        if (has_b) xb = ldq(x + cb);
        if (has_t) xt = ldq(x + ct);
        if (has_w) xw = x[cw];
        if (has_e) xe = x[ce];
    }
    Quad<T> out = xq;
#pragma unroll
    for (int u = 0; u < 4; u++) {
        // static indices; par is uniform over a warp when the warp holds one row
        if ((u & 1) != par) continue;
        const T xc = xq.v[u];
        const T xl = u > 0 ? xq.v[u - 1] : xw;
        const T xr = u < 3 ? xq.v[u + 1] : xe;
        T a, d, f;
        a = fx.v[u];
        d = a;
        f = a * (xl - xc);
        a = u < 3 ? fx.v[u + 1] : fxe;
        d += a;
        f += a * (xr - xc);
        a = fy.v[u];
        d += a;
        f += a * (xs.v[u] - xc);
        a = fyn.v[u];
        d += a;
        f += a * (xn.v[u] - xc);
        a = fz.v[u];
        d += a;
        f += a * (xb.v[u] - xc);
        a = fzt.v[u];
        d += a;
        f += a * (xt.v[u] - xc);
        const T v = d > T(0) ? xc + omega * relax_div(f - bq.v[u], d) : xc;
        out.v[u] = v;
        if (pout) pout[c + u] += (double)v;
    }
    stq(x + c, out);
}

__device__ __forceinline__ int partner(int i, int nc, int periodic)
{
    const int I = i >> 1;
    int J = (i & 1) ? I + 1 : I - 1;
    if (J < 0 || J >= nc) J = periodic ? (J + nc) % nc : I;  // wrap, or mirror at a wall
    return J;
}

// (4) trilinear prolongation at fine cell (i,j,k): weights 3/4 on the coarse
// cell containing the fine centre and 1/4 on its partner, per axis.
template <class T>
__device__ __forceinline__ T prolong_at(const T *__restrict__ ec, const int nc[3], int per, int i,
                                        int j, int k)
{
    const int I0 = i >> 1, I1 = partner(i, nc[0], per & 1);
    const int J0 = j >> 1, J1 = partner(j, nc[1], per & 2);
    const int K0 = k >> 1, K1 = partner(k, nc[2], per & 4);
    const long long r00 = (long long)nc[0] * (J0 + (long long)nc[1] * K0);
    const long long r10 = (long long)nc[0] * (J1 + (long long)nc[1] * K0);
    const long long r01 = (long long)nc[0] * (J0 + (long long)nc[1] * K1);
    const long long r11 = (long long)nc[0] * (J1 + (long long)nc[1] * K1);
    const T w0 = T(0.75), w1 = T(0.25);
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
    return s;
}

// Residual of the 4 cells of the quad at (i0, j, k): b - A x, faces in the
// order of stencil() (x-, x+, y-, y+, z-, z+).
template <class T>
__device__ __forceinline__ Quad<T> residual_quad(const T *__restrict__ x, const T *__restrict__ b,
                                                 const T *__restrict__ wx, const T *__restrict__ wy,
                                                 const T *__restrict__ wz, int nx, int ny, int nz,
                                                 int per, int i0, int j, int k)
{
    const long long sy = nx, sz = (long long)nx * ny;
    const long long c = i0 + sy * j + sz * k;
    const Quad<T> Z{{T(0), T(0), T(0), T(0)}};
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const long long cw = i0 > 0 ? c - 1 : c + nx - 1;
    const long long ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_s = j > 0 || (per & 2), has_n = j + 1 < ny || (per & 2);
    const long long cs = j > 0 ? c - sy : c + sy * (ny - 1);
    const long long cn = j + 1 < ny ? c + sy : c - sy * (ny - 1);
    const bool has_b = k > 0 || (per & 4), has_t = k + 1 < nz || (per & 4);
    const long long cb = k > 0 ? c - sz : c + sz * (nz - 1);
    const long long ct = k + 1 < nz ? c + sz : c - sz * (nz - 1);
    const Quad<T> xq = ldq(x + c), bq = ldq(b + c);
    const Quad<T> fx = ldq(wx + c), fy = ldq(wy + c), fz = ldq(wz + c);
    const Quad<T> fyn = has_n ? ldq(wy + cn) : Z, fzt = has_t ? ldq(wz + ct) : Z;
    const Quad<T> xs = has_s ? ldq(x + cs) : Z, xn = has_n ? ldq(x + cn) : Z;
    const Quad<T> xb = has_b ? ldq(x + cb) : Z, xt = has_t ? ldq(x + ct) : Z;
    const T xw = has_w ? x[cw] : T(0), xe = has_e ? x[ce] : T(0);
    const T fxe = has_e ? wx[ce] : T(0);
    Quad<T> r;
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const T xc = xq.v[u];
        T f = fx.v[u] * ((u > 0 ? xq.v[u - 1] : xw) - xc);
        f += (u < 3 ? fx.v[u + 1] : fxe) * ((u < 3 ? xq.v[u + 1] : xe) - xc);
        f += fy.v[u] * (xs.v[u] - xc);
        f += fyn.v[u] * (xn.v[u] - xc);
        f += fz.v[u] * (xb.v[u] - xc);
        f += fzt.v[u] * (xt.v[u] - xc);
        r.v[u] = bq.v[u] - f;
    }
    return r;
}

// Restriction for the coarse cell pair (2P, 2P+1) of coarse row `crow` = J + ncy K:
// the residuals of the fine quad below it in each of the 4 fine rows
// (2J + dy, 2K + dz), summed per coarse cell in a fixed order, times 1/8.
template <class T>
__device__ __forceinline__ void restrict_pair(const LevelView &L, int crow, int J, int K, int P)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], ncx = L.nc[0];
    const T *x = (const T *)L.x;
    const T *b = (const T *)L.b;
    const T *wx = (const T *)L.w[0], *wy = (const T *)L.w[1], *wz = (const T *)L.w[2];
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const Quad<T> r = residual_quad(x, b, wx, wy, wz, nx, ny, nz, L.per, 4 * P, 2 * J + dy,
                                            2 * K + dz);
            s0 += r.v[0];
            s0 += r.v[1];
            s1 += r.v[2];
            s1 += r.v[3];
        }
    T *bc = (T *)L.bc + (long long)ncx * crow + 2 * P;
    bc[0] = s0 * T(0.125);
    bc[1] = s1 * T(0.125);
}

// x += P e_c on the aligned quad (4 qx .. 4 qx + 3, j, k) of row `row`.
template <class T>
__device__ __forceinline__ void prolong_quad(const LevelView &L, int row, int j, int k, int qx,
                                             double *__restrict__ pout)
{
    const int nx = L.n[0];
    const T *ec = (const T *)L.xc;
    T *x = (T *)L.x;
    const long long c = (long long)row * nx + 4 * qx;
    Quad<T> xq = ldq(x + c);
#pragma unroll
    for (int u = 0; u < 4; u++) {
        xq.v[u] += prolong_at(ec, L.nc, L.per, 4 * qx + u, j, k);
        if (pout) pout[c + u] += (double)xq.v[u];
    }
    stq(x + c, xq);
}

}  // namespace gbmg
