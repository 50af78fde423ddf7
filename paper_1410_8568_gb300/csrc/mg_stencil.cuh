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
#include "mg_xprec.cuh"

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

// half-sweep flags: the iterate is zero on entry (first red launch); the
// launch may add its relaxed values to the FP64 iterate (level 0, last
// post-smoothing sweep, done by the grids whose step ends with this cycle)
constexpr int kZeroGuess = 1, kOuter = 4;

// Relaxation of the cells of colour `colour` in the aligned quad (4 qx .. 4 qx + 3,
// j, k) of row `row` = j + ny k.  The two cells of the colour are p0 = 4 qx + par
// and p0 + 2 (par = 0 or 1).  The quad of x and its x-faces are loaded as
// 16-byte vectors (each colour cell needs its in-row neighbours, which are
// the other colour); b and the y/z neighbours and faces only at the two colour
// cells.  The quad is written back whole, the other colour unchanged.  Per
// cell, the terms are summed in the order x-, x+, y-, y+, z-, z+ as in every
// other kernel.  The rounding steps are written out (a product rounded on its
// own, then fused multiply-adds, and a fused multiply-add for the update):
// left to the compiler, the first two products of the sum could be contracted
// either way, differently in different kernels, and the kernels that relax the
// same cell (half-sweep tilings, one-pass sweeps, the tail) would then differ in
// the last bits.
template <class T>
__device__ __forceinline__ T mul_rn(T a, T b)
{
    if constexpr (sizeof(T) == 4) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}

template <class T>
__device__ __forceinline__ T relax_cell(T xc, T xl, T xr, T fl, T fr, T fs, T fn, T fb, T ft, T xs,
                                        T xn, T xb, T xt, T bc, T omega)
{
    const T d = ((((fl + fr) + fs) + fn) + fb) + ft;
    T f = mul_rn(fl, xl - xc);
    f = fma(fr, xr - xc, f);
    f = fma(fs, xs - xc, f);
    f = fma(fn, xn - xc, f);
    f = fma(fb, xb - xc, f);
    f = fma(ft, xt - xc, f);
    return d > T(0) ? fma(omega, relax_div(f - bc, d), xc) : xc;
}

// The relaxation of FP64 cycles, with the cell's diagonal given by its inverse
// di = 1 / d (d summed as relax_cell sums it; 0 for a cell without faces),
// computed once per coefficient set: the Gauss-Seidel value
// g = (sum of w_f x_nb - b) di, then x = g (omega = 1) or xc + omega (g - xc).
// Eight FP64 operations per cell at omega = 1 (six fused multiply-adds, a
// subtraction, a multiply) where the difference form with a division takes
// about thirty; this GPU issues FP64 on a narrow pipe, which bounds the FP64
// half-sweep.  The neighbours are summed in relax_cell's order.
template <class T>
__device__ __forceinline__ T relax_cell_inv(T xc, T xl, T xr, T fl, T fr, T fs, T fn, T fb, T ft, T xs,
                                            T xn, T xb, T xt, T bc, T omega, T di)
{
    T s = fl * xl;
    s = fma(fr, xr, s);
    s = fma(fs, xs, s);
    s = fma(fn, xn, s);
    s = fma(fb, xb, s);
    s = fma(ft, xt, s);
    const T g = (s - bc) * di;
    if (!(di > T(0))) return xc;
    return omega == T(1) ? g : fma(omega, g - xc, xc);
}

// Add the final correction v of cell c of a refinement step to the outer
// iterate: p += v / xscale in FP64 (the scale a power of 2, so exact), or the
// exact three-float update in the scaled units (FP32 cycles with the
// extended-precision outer iteration, mg_xprec.cuh; o.t set).
template <class T>
__device__ __forceinline__ void add_outer(const OuterOut &o, int c, T v)
{
    if constexpr (sizeof(T) == 4) {
        if (o.t[0] != nullptr) {
            float a = o.t[0][c], m = o.t[1][c], z = o.t[2][c];
            triple_add(a, m, z, v);
            o.t[0][c] = a;
            o.t[1][c] = m;
            o.t[2][c] = z;
            return;
        }
    }
    o.p[c] += (double)v * o.inv;
}

// The same for the cells of an aligned quad at c (4 | c) selected by `sel`
// (bit u: cell c + u), with the three-float components moved as 16-byte vectors.
template <class T>
__device__ __forceinline__ void add_outer_quad(const OuterOut &o, int c, const T v[4], int sel)
{
    if (sizeof(T) == 8 || o.t[0] == nullptr) {
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (sel >> u & 1) o.p[c + u] += (double)v[u] * o.inv;
    } else {
        float4 a = *(const float4 *)(o.t[0] + c), m = *(const float4 *)(o.t[1] + c),
               z = *(const float4 *)(o.t[2] + c);
        float *pa = &a.x, *pm = &m.x, *pz = &z.x;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            float a1 = pa[u], m1 = pm[u], z1 = pz[u];
            triple_add(a1, m1, z1, v[u]);
            const bool on = sel >> u & 1;
            pa[u] = on ? a1 : pa[u];
            pm[u] = on ? m1 : pm[u];
            pz[u] = on ? z1 : pz[u];
        }
        *(float4 *)(o.t[0] + c) = a;
        *(float4 *)(o.t[1] + c) = m;
        *(float4 *)(o.t[2] + c) = z;
    }
}

// OUT (the last black half-sweep of a cycle): also add the quad's final
// values to the outer iterate, the relaxed cells and the other colour's cells,
// which that half-sweep does not change (add_outer; a compile-time choice: a
// per-thread run-time test would leave predicated update instructions in every
// launch, FP64 ones in the FP64 case, whose throughput on this GPU is a small
// fraction of FP32's; kernels that may update pick one of the two instances
// per block).
// go: store the result (false: a grid that sits this cycle out; the loads are
// issued before its state is known, so they overlap that load's latency).
// dinv: FP64 cycles, the level's inverse diagonals (relax_cell_inv), or null.
template <class T, bool OUT>
__device__ __forceinline__ void half_quad(T *x, const T *b, const T *wx, const T *wy, const T *wz,
                                          int nx, int ny, int nz, int per, int row, int j, int k,
                                          int qx, int colour, T omega, bool zero, const OuterOut &po,
                                          bool go = true, const T *dinv = nullptr)
{
    // cell indices fit in 32 bits: a grid has fewer than 2^31 cells
    const int sy = nx, sz = nx * ny;
    const int i0 = qx << 2;
    const int c = row * nx + i0;
    const int par = (colour + j + k) & 1;
    const int c0 = c + par;  // first cell of the colour; the second is c0 + 2
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const int cw = i0 > 0 ? c - 1 : c + nx - 1;
    const int ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_n = j + 1 < ny || (per & 2), has_t = k + 1 < nz || (per & 4);
    const bool has_s = j > 0 || (per & 2), has_b = k > 0 || (per & 4);
    const int ds = j > 0 ? -sy : sy * (ny - 1);  // offset of the y- neighbour
    const int dn = j + 1 < ny ? sy : -sy * (ny - 1);
    const int db = k > 0 ? -sz : sz * (nz - 1);
    const int dt = k + 1 < nz ? sz : -sz * (nz - 1);
    const Quad<T> fx = ldq(wx + c);
    const T fxe = has_e ? wx[ce] : T(0);  // high x face of the last cell of the quad
    const T b0 = b[c0], b1 = b[c0 + 2];
    const T fs0 = wy[c0], fs1 = wy[c0 + 2];
    const T fn0 = has_n ? wy[c0 + dn] : T(0), fn1 = has_n ? wy[c0 + 2 + dn] : T(0);
    const T fb0 = wz[c0], fb1 = wz[c0 + 2];
    const T ft0 = has_t ? wz[c0 + dt] : T(0), ft1 = has_t ? wz[c0 + 2 + dt] : T(0);
    Quad<T> xq{{T(0), T(0), T(0), T(0)}};
    T xw = T(0), xe = T(0);
    T xs0 = T(0), xs1 = T(0), xn0 = T(0), xn1 = T(0), xb0 = T(0), xb1 = T(0), xt0 = T(0), xt1 = T(0);
    if (!zero) {
        xq = ldq(x + c);
        if (has_w) xw = x[cw];
        if (has_e) xe = x[ce];
        if (has_s) {
            xs0 = x[c0 + ds];
            xs1 = x[c0 + 2 + ds];
        }
        if (has_n) {
            xn0 = x[c0 + dn];
            xn1 = x[c0 + 2 + dn];
        }
        if (has_b) {
            xb0 = x[c0 + db];
            xb1 = x[c0 + 2 + db];
        }
        if (has_t) {
            xt0 = x[c0 + dt];
            xt1 = x[c0 + 2 + dt];
        }
    }
    // cell p0 (u = par) and cell p0 + 2 (u = par + 2): centre, x neighbours, x faces
    const T xc0 = par ? xq.v[1] : xq.v[0], xc1 = par ? xq.v[3] : xq.v[2];
    const T xl0 = par ? xq.v[0] : xw, xr0 = par ? xq.v[2] : xq.v[1];
    const T xl1 = par ? xq.v[2] : xq.v[1], xr1 = par ? xe : xq.v[3];
    const T fl0 = par ? fx.v[1] : fx.v[0], fr0 = par ? fx.v[2] : fx.v[1];
    const T fl1 = par ? fx.v[3] : fx.v[2], fr1 = par ? fxe : fx.v[3];
    T v0, v1;
    if (sizeof(T) == 8 && dinv != nullptr) {
        const T di0 = dinv[c0], di1 = dinv[c0 + 2];
        v0 = relax_cell_inv(xc0, xl0, xr0, fl0, fr0, fs0, fn0, fb0, ft0, xs0, xn0, xb0, xt0, b0, omega, di0);
        v1 = relax_cell_inv(xc1, xl1, xr1, fl1, fr1, fs1, fn1, fb1, ft1, xs1, xn1, xb1, xt1, b1, omega, di1);
    } else {
        v0 = relax_cell(xc0, xl0, xr0, fl0, fr0, fs0, fn0, fb0, ft0, xs0, xn0, xb0, xt0, b0, omega);
        v1 = relax_cell(xc1, xl1, xr1, fl1, fr1, fs1, fn1, fb1, ft1, xs1, xn1, xb1, xt1, b1, omega);
    }
    Quad<T> out = xq;
    out.v[0] = par ? xq.v[0] : v0;
    out.v[1] = par ? v0 : xq.v[1];
    out.v[2] = par ? xq.v[2] : v1;
    out.v[3] = par ? v1 : xq.v[3];
    if (!go) return;
    stq(x + c, out);
    if constexpr (OUT) add_outer_quad<T>(po, c, out.v, 0xF);
}

// half_quad for operands in shared memory (the tail kernel): the same
// relaxation with the same relax_cell inputs, so the same results, but every
// operand of the two colour cells comes from a 16-byte quad load.  A warp's
// scalar loads at a stride of one quad (4 words) hit 8 of the 32 banks: 4
// wavefronts for 128 useful bytes, where a quad load carries 512.
template <class T>
__device__ __forceinline__ T colour_cell(const Quad<T> &q, int par, int second)
{
    return second ? (par ? q.v[3] : q.v[2]) : (par ? q.v[1] : q.v[0]);
}

template <class T>
__device__ __forceinline__ void half_quad_sm(T *x, const T *b, const T *wx, const T *wy, const T *wz, int nx,
                                             int ny, int nz, int per, int row, int j, int k, int qx, int colour,
                                             T omega, bool zero)
{
    const int sy = nx, sz = nx * ny;
    const int i0 = qx << 2;
    const int c = row * nx + i0;
    const int par = (colour + j + k) & 1;
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const int cw = i0 > 0 ? c - 1 : c + nx - 1;
    const int ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_n = j + 1 < ny || (per & 2), has_t = k + 1 < nz || (per & 4);
    const bool has_s = j > 0 || (per & 2), has_b = k > 0 || (per & 4);
    const int ds = j > 0 ? -sy : sy * (ny - 1);
    const int dn = j + 1 < ny ? sy : -sy * (ny - 1);
    const int db = k > 0 ? -sz : sz * (nz - 1);
    const int dt = k + 1 < nz ? sz : -sz * (nz - 1);
    const Quad<T> z4{{T(0), T(0), T(0), T(0)}};
    const Quad<T> fx = ldq(wx + c);
    const T fxe = has_e ? wx[ce] : T(0);
    const Quad<T> bq = ldq(b + c);
    const Quad<T> fsq = ldq(wy + c), fnq = has_n ? ldq(wy + c + dn) : z4;
    const Quad<T> fbq = ldq(wz + c), ftq = has_t ? ldq(wz + c + dt) : z4;
    Quad<T> xq = z4, xsq = z4, xnq = z4, xbq = z4, xtq = z4;
    T xw = T(0), xe = T(0);
    if (!zero) {
        xq = ldq(x + c);
        if (has_w) xw = x[cw];
        if (has_e) xe = x[ce];
        if (has_s) xsq = ldq(x + c + ds);
        if (has_n) xnq = ldq(x + c + dn);
        if (has_b) xbq = ldq(x + c + db);
        if (has_t) xtq = ldq(x + c + dt);
    }
    const T xc0 = par ? xq.v[1] : xq.v[0], xc1 = par ? xq.v[3] : xq.v[2];
    const T xl0 = par ? xq.v[0] : xw, xr0 = par ? xq.v[2] : xq.v[1];
    const T xl1 = par ? xq.v[2] : xq.v[1], xr1 = par ? xe : xq.v[3];
    const T fl0 = par ? fx.v[1] : fx.v[0], fr0 = par ? fx.v[2] : fx.v[1];
    const T fl1 = par ? fx.v[3] : fx.v[2], fr1 = par ? fxe : fx.v[3];
    const T v0 = relax_cell(xc0, xl0, xr0, fl0, fr0, colour_cell(fsq, par, 0), colour_cell(fnq, par, 0),
                            colour_cell(fbq, par, 0), colour_cell(ftq, par, 0), colour_cell(xsq, par, 0),
                            colour_cell(xnq, par, 0), colour_cell(xbq, par, 0), colour_cell(xtq, par, 0),
                            colour_cell(bq, par, 0), omega);
    const T v1 = relax_cell(xc1, xl1, xr1, fl1, fr1, colour_cell(fsq, par, 1), colour_cell(fnq, par, 1),
                            colour_cell(fbq, par, 1), colour_cell(ftq, par, 1), colour_cell(xsq, par, 1),
                            colour_cell(xnq, par, 1), colour_cell(xbq, par, 1), colour_cell(xtq, par, 1),
                            colour_cell(bq, par, 1), omega);
    Quad<T> out;
    out.v[0] = par ? xq.v[0] : v0;
    out.v[1] = par ? v0 : xq.v[1];
    out.v[2] = par ? xq.v[2] : v1;
    out.v[3] = par ? v1 : xq.v[3];
    stq(x + c, out);
}

// Coarse partner of fine index i along an axis of nc coarse cells: the coarse
// cell across the coarse face nearer to the fine centre.  It lies one step
// outside [0, nc) at most: wrap on a periodic axis, else (wall) the cell itself.
__device__ __forceinline__ int partner(int i, int nc, int periodic)
{
    const int I = i >> 1;
    const int J = (i & 1) ? I + 1 : I - 1;
    if (J < 0) return periodic ? nc - 1 : I;
    if (J >= nc) return periodic ? 0 : I;
    return J;
}

// Linear interpolation to a fine centre between the coarse value it lies over
// (weight 3/4) and its partner across the nearer coarse face (1/4), with one
// explicit rounding order so that every kernel that prolongs gets bitwise the
// same value for a cell.
template <class T>
__device__ __forceinline__ T lin(T own, T par)
{
    return fma(T(0.25), par, T(0.75) * own);
}

// (4) trilinear prolongation at fine cell (i,j,k): lin along x on the 4 coarse
// rows (own/partner in y and z), then along y, then along z; the weights
// multiply out to 27/9/3/1 over 64.
template <class T>
__device__ __forceinline__ T prolong_at(const T *__restrict__ ec, const int nc[3], int per, int i,
                                        int j, int k)
{
    const int I0 = i >> 1, I1 = partner(i, nc[0], per & 1);
    const int J0 = j >> 1, J1 = partner(j, nc[1], per & 2);
    const int K0 = k >> 1, K1 = partner(k, nc[2], per & 4);
    const T *r00 = ec + nc[0] * (J0 + nc[1] * K0), *r10 = ec + nc[0] * (J1 + nc[1] * K0);
    const T *r01 = ec + nc[0] * (J0 + nc[1] * K1), *r11 = ec + nc[0] * (J1 + nc[1] * K1);
    const T y0 = lin(lin(r00[I0], r00[I1]), lin(r10[I0], r10[I1]));
    const T y1 = lin(lin(r01[I0], r01[I1]), lin(r11[I0], r11[I1]));
    return lin(y0, y1);
}

// Flux-conserving prolongation (Sec. 2.3 item 4, Eqs. 13-14) at one fine cell.
// e[q], a[q]: coarse error and cell coefficient of the 8 coarse cells around
// the fine centre, q = bit 0 (x partner) | bit 1 (y partner) | bit 2 (z partner),
// q = 0 the coarse cell holding the fine cell.  The corners of the fine cell's
// octant are the coarse centre, 3 face centres, 3 edge midpoints and a node;
// the value at each is the a-weighted mean of the coarse cells meeting there
// (flux continuity across the face, Eq. 13, and its analogue at edges and
// nodes), and the fine value is the mean of the 8 corners.  For constant a
// this is the trilinear 27/9/3/1 rule.  Fixed summation order.
template <class T>
__device__ __forceinline__ T flux_corner_mean(const T e[8], const T a[8])
{
    T ae[8];
#pragma unroll
    for (int q = 0; q < 8; q++) ae[q] = a[q] * e[q];
    const T s01 = ae[0] + ae[1], s02 = ae[0] + ae[2], s04 = ae[0] + ae[4];
    const T d01 = a[0] + a[1], d02 = a[0] + a[2], d04 = a[0] + a[4];
    const T s0123 = s01 + (ae[2] + ae[3]), d0123 = d01 + (a[2] + a[3]);
    const T s0145 = s01 + (ae[4] + ae[5]), d0145 = d01 + (a[4] + a[5]);
    const T s0246 = s02 + (ae[4] + ae[6]), d0246 = d02 + (a[4] + a[6]);
    const T s_all = s0123 + ((ae[4] + ae[5]) + (ae[6] + ae[7]));
    const T d_all = d0123 + ((a[4] + a[5]) + (a[6] + a[7]));
    const T fx = relax_div(s01, d01), fy = relax_div(s02, d02), fz = relax_div(s04, d04);
    const T exy = relax_div(s0123, d0123), exz = relax_div(s0145, d0145), eyz = relax_div(s0246, d0246);
    const T node = relax_div(s_all, d_all);
    return T(0.125) * (((e[0] + fx) + (fy + fz)) + ((exy + exz) + (eyz + node)));
}

// flux-conserving counterpart of prolong_at; ac = coarse cell coefficients
template <class T>
__device__ __forceinline__ T prolong_at_flux(const T *__restrict__ ec, const T *__restrict__ ac,
                                             const int nc[3], int per, int i, int j, int k)
{
    const int I[2] = {i >> 1, partner(i, nc[0], per & 1)};
    const int J[2] = {j >> 1, partner(j, nc[1], per & 2)};
    const int K[2] = {k >> 1, partner(k, nc[2], per & 4)};
    T e[8], a[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int c = I[q & 1] + nc[0] * (J[(q >> 1) & 1] + nc[1] * K[q >> 2]);
        e[q] = ec[c];
        a[q] = ac[c];
    }
    return flux_corner_mean(e, a);
}

// Residual of the 4 cells of the quad at (i0, j, k): b - A x, faces in the
// order of stencil() (x-, x+, y-, y+, z-, z+).
template <class T>
__device__ __forceinline__ Quad<T> residual_quad(const T *__restrict__ x, const T *__restrict__ b,
                                                 const T *__restrict__ wx, const T *__restrict__ wy,
                                                 const T *__restrict__ wz, int nx, int ny, int nz,
                                                 int per, int i0, int j, int k)
{
    const int sy = nx, sz = nx * ny;
    const int c = i0 + sy * j + sz * k;
    const Quad<T> Z{{T(0), T(0), T(0), T(0)}};
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const int cw = i0 > 0 ? c - 1 : c + nx - 1;
    const int ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_s = j > 0 || (per & 2), has_n = j + 1 < ny || (per & 2);
    const int cs = j > 0 ? c - sy : c + sy * (ny - 1);
    const int cn = j + 1 < ny ? c + sy : c - sy * (ny - 1);
    const bool has_b = k > 0 || (per & 4), has_t = k + 1 < nz || (per & 4);
    const int cb = k > 0 ? c - sz : c + sz * (nz - 1);
    const int ct = k + 1 < nz ? c + sz : c - sz * (nz - 1);
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
// First red half-sweep of the coarse level from a zero correction, at coarse
// cell (I, J, K) with right-hand side bc: red cells get omega * (-bc / d), d
// the sum of the cell's face coefficients in the order every half-sweep uses
// (x low, x high, y low, y high, z low, z high; absent high faces skipped),
// black cells 0 -- the value the zero-start red half-sweep would write.
template <class T>
__device__ __forceinline__ T zero_start_red(const LevelView &L, int I, int J, int K, T bc, T omega)
{
    if (((I + J + K) & 1) != 0) return T(0);
    const int nx = L.nc[0], ny = L.nc[1], nz = L.nc[2], per = L.per;
    const int sy = nx, sz = nx * ny;
    const int c = I + nx * (J + ny * K);
    if (sizeof(T) == 8 && L.dinvc != nullptr) {
        // FP64 cycles: the coarse level's inverse diagonal (see relax_cell_inv)
        const T di = ((const T *)L.dinvc)[c];
        return di > T(0) ? omega * ((-bc) * di) : T(0);
    }
    const T *wx = (const T *)L.wc[0], *wy = (const T *)L.wc[1], *wz = (const T *)L.wc[2];
    T d = wx[c];
    if (I + 1 < nx) d += wx[c + 1];
    else if (per & 1) d += wx[c + 1 - nx];
    d += wy[c];
    if (J + 1 < ny) d += wy[c + sy];
    else if (per & 2) d += wy[c - sy * (ny - 1)];
    d += wz[c];
    if (K + 1 < nz) d += wz[c + sz];
    else if (per & 4) d += wz[c - sz * (nz - 1)];
    return d > T(0) ? omega * relax_div(-bc, d) : T(0);
}

template <class T>
__device__ __forceinline__ void restrict_pair(const LevelView &L, int crow, int J, int K, int P, T omega,
                                              bool go = true)
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
    T *bc = (T *)L.bc + ncx * crow + 2 * P;
    const T b0 = s0 * T(0.125), b1 = s1 * T(0.125);
    if (!go) return;  // (see half_quad)
    bc[0] = b0;
    bc[1] = b1;
    if (L.zr) {
        T *xc = (T *)L.xc + ncx * crow + 2 * P;
        xc[0] = zero_start_red<T>(L, 2 * P, J, K, b0, omega);
        xc[1] = zero_start_red<T>(L, 2 * P + 1, J, K, b1, omega);
    }
}

// Interpolation along x on one coarse row `er` for the 4 fine cells of the quad
// over coarse cells I0 = 2 qx and I0 + 1: own/partner pairs (I0, Im), (I0, I0+1),
// (I0+1, I0), (I0+1, Ip), Im / Ip the partners of fine cells 4 qx / 4 qx + 3.
template <class T>
__device__ __forceinline__ void lin_x(const T *__restrict__ er, int Im, int I0, int Ip, T out[4])
{
    const T a = er[Im], b = er[I0], c = er[I0 + 1], d = er[Ip];
    out[0] = lin(b, a);
    out[1] = lin(b, c);
    out[2] = lin(c, b);
    out[3] = lin(c, d);
}

// x += P e_c on the aligned quad (4 qx .. 4 qx + 3, j, k) of row `row`: same
// rounding order as prolong_at.  OUT: also add x to the outer iterate (see
// half_quad).
template <class T, bool OUT>
__device__ __forceinline__ void prolong_quad(const LevelView &L, int row, int j, int k, int qx,
                                             const OuterOut &po, bool go = true)
{
    const int nx = L.n[0], ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2], per = L.per;
    const T *__restrict__ ec = (const T *)L.xc;
    T *x = (T *)L.x;
    const int c = row * nx + 4 * qx;
    const int I0 = 2 * qx;
    const int Im = partner(4 * qx, ncx, per & 1), Ip = partner(4 * qx + 3, ncx, per & 1);
    const int J0 = j >> 1, J1 = partner(j, ncy, per & 2);
    const int K0 = k >> 1, K1 = partner(k, ncz, per & 4);
    T a00[4], a10[4], a01[4], a11[4];
    lin_x(ec + ncx * (J0 + ncy * K0), Im, I0, Ip, a00);
    lin_x(ec + ncx * (J1 + ncy * K0), Im, I0, Ip, a10);
    lin_x(ec + ncx * (J0 + ncy * K1), Im, I0, Ip, a01);
    lin_x(ec + ncx * (J1 + ncy * K1), Im, I0, Ip, a11);
    Quad<T> xq = ldq(x + c);
#pragma unroll
    for (int u = 0; u < 4; u++) {
        xq.v[u] += lin(lin(a00[u], a10[u]), lin(a01[u], a11[u]));
    }
    if (!go) return;  // (see half_quad)
    stq(x + c, xq);
    if constexpr (OUT) add_outer_quad<T>(po, c, xq.v, 0xF);
}

// Flux-conserving x += P e_c on the aligned quad (4 qx .. 4 qx + 3, j, k): the
// quad's 4 cells share the coarse x set {Im, I0, I0 + 1, Ip} on the 4 coarse
// rows (J0 or its partner, K0 or its partner).
template <class T, bool OUT>
__device__ __forceinline__ void prolong_quad_flux(const LevelView &L, int row, int j, int k, int qx,
                                                  const OuterOut &po)
{
    const int nx = L.n[0], ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2], per = L.per;
    const T *__restrict__ ec = (const T *)L.xc;
    const T *__restrict__ ac = (const T *)L.ac;
    T *x = (T *)L.x;
    const int c = row * nx + 4 * qx;
    const int I0 = 2 * qx;
    const int Ix[4] = {partner(4 * qx, ncx, per & 1), I0, I0 + 1, partner(4 * qx + 3, ncx, per & 1)};
    const int Jy[2] = {j >> 1, partner(j, ncy, per & 2)};
    const int Kz[2] = {k >> 1, partner(k, ncz, per & 4)};
    // coarse values: [row r = jy + 2 kz][x slot 0..3]
    T ev[4][4], av[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int base = ncx * (Jy[r & 1] + ncy * Kz[r >> 1]);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            ev[r][m] = ec[base + Ix[m]];
            av[r][m] = ac[base + Ix[m]];
        }
    }
    // own and partner x slot of each fine cell of the quad
    constexpr int own[4] = {1, 1, 2, 2}, par[4] = {0, 2, 1, 3};
    Quad<T> xq = ldq(x + c);
#pragma unroll
    for (int u = 0; u < 4; u++) {
        T e[8], a[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int r = ((q >> 1) & 1) + 2 * (q >> 2);
            const int m = (q & 1) ? par[u] : own[u];
            e[q] = ev[r][m];
            a[q] = av[r][m];
        }
        xq.v[u] += flux_corner_mean(e, a);
    }
    stq(x + c, xq);
    if constexpr (OUT) add_outer_quad<T>(po, c, xq.v, 0xF);
}

// x += P e_c on the 2 x 2 fine rows (2J + dy, 2K + dz) above coarse row (J, K),
// on the quad over the coarse cell pair (2P, 2P + 1).  The 4 fine rows share
// coarse rows: they use J and its two partners Jm, Jp (and K, Km, Kp), 9 coarse
// rows in all instead of 16.  Same rounding order as prolong_at.
template <class T>
__device__ __forceinline__ void prolong_block(const LevelView &L, int J, int K, int P, bool go = true)
{
    const int nx = L.n[0], ny = L.n[1], ncx = L.nc[0], ncy = L.nc[1], ncz = L.nc[2], per = L.per;
    const T *__restrict__ ec = (const T *)L.xc;
    T *x = (T *)L.x;
    const int I0 = 2 * P;
    const int Im = partner(4 * P, ncx, per & 1), Ip = partner(4 * P + 3, ncx, per & 1);
    const int Jr[3] = {partner(2 * J, ncy, per & 2), J, partner(2 * J + 1, ncy, per & 2)};
    const int Kr[3] = {partner(2 * K, ncz, per & 4), K, partner(2 * K + 1, ncz, per & 4)};
    // along x then y for each coarse plane Km, K, Kp: ey[kz][dy][u]
    T ey[3][2][4];
#pragma unroll
    for (int kz = 0; kz < 3; kz++) {
        T am[4], a0[4], ap[4];
        const T *plane = ec + ncx * ncy * Kr[kz];
        lin_x(plane + ncx * Jr[0], Im, I0, Ip, am);
        lin_x(plane + ncx * Jr[1], Im, I0, Ip, a0);
        lin_x(plane + ncx * Jr[2], Im, I0, Ip, ap);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            ey[kz][0][u] = lin(a0[u], am[u]);  // fine row 2J: partner J - 1 side
            ey[kz][1][u] = lin(a0[u], ap[u]);  // fine row 2J + 1: partner J + 1 side
        }
    }
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const int c = nx * ((2 * J + dy) + ny * (2 * K + dz)) + 4 * P;
            Quad<T> xq = ldq(x + c);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                xq.v[u] += lin(ey[1][dy][u], ey[dz ? 2 : 0][dy][u]);
            }
            if (go) stq(x + c, xq);
        }
}

}  // namespace gbmg
