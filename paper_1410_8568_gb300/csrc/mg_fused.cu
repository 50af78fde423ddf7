// mg_fused.cu -- one-pass red-black sweep (Sec. 2.3 item 5, red-black SOR):
// both colours of a full sweep in one launch, so the iterate, the right-hand
// side and the three face arrays stream through HBM once per sweep instead of
// once per colour.
//
// A sweep reads the iterate from one buffer and writes the new one to the
// other (ping-pong): every value the red half-sweep needs is then the old
// iterate, which no block overwrites.  A block owns a strip of R full rows of
// a chunk of planes and marches up the chunk in z.  At step k it relaxes the
// red cells of plane k (for its R rows and one halo row on each side) from the
// old iterate, and the black cells of plane k - 1 (its own rows) from the new
// red values: those of plane k - 1 in its rows and the halo rows (shared
// memory, a ring of 3 planes) and those of planes k - 2 and k in its own
// column (registers: a thread owns the same quad of every plane).  One block
// barrier per step.  The chunk's red half-sweep also covers the planes just
// below and above it (recomputed, as the halo rows are), so blocks never wait
// on one another.
//
// Every cell's new value comes from the same relax_cell call with the same
// operands as in the two half-sweep launches (mg_stencil.cuh), so the result
// is bitwise that of the red launch followed by the black launch.
#include "mg_kernels.h"
#include "mg_stencil.cuh"

namespace gbmg {

namespace {

// x after the half-sweep of `colour` on the aligned quad (4 qx .. 4 qx + 3, j,
// k): half_quad's arithmetic (same operands, same order), returned instead of
// stored.
template <class T>
__device__ __forceinline__ Quad<T> relax_quad_global(const T *__restrict__ x, const T *__restrict__ b,
                                                     const T *__restrict__ wx, const T *__restrict__ wy,
                                                     const T *__restrict__ wz, int nx, int ny, int nz, int per,
                                                     int j, int k, int qx, int colour, T omega, bool zero,
                                                     const T *__restrict__ dinv)
{
    const int sy = nx, sz = nx * ny;
    const int i0 = qx << 2;
    const int c = (j + ny * k) * nx + i0;
    const int par = (colour + j + k) & 1;
    const int c0 = c + par;
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const int cw = i0 > 0 ? c - 1 : c + nx - 1;
    const int ce = i0 + 4 < nx ? c + 4 : c + 4 - nx;
    const bool has_n = j + 1 < ny || (per & 2), has_t = k + 1 < nz || (per & 4);
    const bool has_s = j > 0 || (per & 2), has_b = k > 0 || (per & 4);
    const int ds = j > 0 ? -sy : sy * (ny - 1);
    const int dn = j + 1 < ny ? sy : -sy * (ny - 1);
    const int db = k > 0 ? -sz : sz * (nz - 1);
    const int dt = k + 1 < nz ? sz : -sz * (nz - 1);
    const Quad<T> fx = ldq(wx + c);
    const T fxe = has_e ? wx[ce] : T(0);
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
    return out;
}

// The black half-sweep of the quad at (j, k) whose values after the red
// half-sweep are xq, with its neighbours after the red half-sweep: the rows
// j - 1 and j + 1 of the plane (srow, nrow: full rows), its own row (orow, for
// the cells left and right of the quad) and its own column in planes k - 1
// and k + 1 (xbq, xtq).  Same operands, same order as half_quad's black launch.
template <class T>
__device__ __forceinline__ Quad<T> black_quad(const Quad<T> &xq, const T *orow, const T *srow, const T *nrow,
                                              const Quad<T> &xbq, const Quad<T> &xtq, const T *__restrict__ b,
                                              const T *__restrict__ wx, const T *__restrict__ wy,
                                              const T *__restrict__ wz, int nx, int ny, int nz, int per, int j,
                                              int k, int qx, T omega, const T *__restrict__ dinv)
{
    const int sy = nx, sz = nx * ny;
    const int i0 = qx << 2;
    const int c = (j + ny * k) * nx + i0;
    const int par = (1 + j + k) & 1;
    const int c0 = c + par;
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const int iw = i0 > 0 ? i0 - 1 : nx - 1;
    const int ie = i0 + 4 < nx ? i0 + 4 : i0 + 4 - nx;
    const int ce = c + (ie - i0);
    const bool has_n = j + 1 < ny || (per & 2), has_t = k + 1 < nz || (per & 4);
    const bool has_s = j > 0 || (per & 2), has_b = k > 0 || (per & 4);
    const int dn = j + 1 < ny ? sy : -sy * (ny - 1);
    const int dt = k + 1 < nz ? sz : -sz * (nz - 1);
    const Quad<T> fx = ldq(wx + c);
    const T fxe = has_e ? wx[ce] : T(0);
    const T b0 = b[c0], b1 = b[c0 + 2];
    const T fs0 = wy[c0], fs1 = wy[c0 + 2];
    const T fn0 = has_n ? wy[c0 + dn] : T(0), fn1 = has_n ? wy[c0 + 2 + dn] : T(0);
    const T fb0 = wz[c0], fb1 = wz[c0 + 2];
    const T ft0 = has_t ? wz[c0 + dt] : T(0), ft1 = has_t ? wz[c0 + 2 + dt] : T(0);
    const T xw = has_w ? orow[iw] : T(0), xe = has_e ? orow[ie] : T(0);
    const T xs0 = has_s ? srow[i0 + par] : T(0), xs1 = has_s ? srow[i0 + par + 2] : T(0);
    const T xn0 = has_n ? nrow[i0 + par] : T(0), xn1 = has_n ? nrow[i0 + par + 2] : T(0);
    const T xb0 = has_b ? (par ? xbq.v[1] : xbq.v[0]) : T(0), xb1 = has_b ? (par ? xbq.v[3] : xbq.v[2]) : T(0);
    const T xt0 = has_t ? (par ? xtq.v[1] : xtq.v[0]) : T(0), xt1 = has_t ? (par ? xtq.v[3] : xtq.v[2]) : T(0);
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
    return out;
}

// One block of a full sweep of grid view L: strip lb % fS of fR rows, chunk
// lb / fS of fKc planes.  B threads: thread t relaxes quad t % nq of slot row
// t / nq, slot 0 being the row below the strip and slot fR + 1 the row above.
template <class T, int B, bool OUT>
__device__ __forceinline__ void sweep_body(const LevelView &L, int lb, int dir, T omega, bool zero,
                                           const OuterOut &po, T *sm)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], per = L.per, nq = nx >> 2;
    const T *__restrict__ xin = (const T *)(dir ? L.x2 : L.x);
    T *__restrict__ xout = (T *)(dir ? L.x : L.x2);
    const T *__restrict__ b = (const T *)L.b;
    const T *__restrict__ wx = (const T *)L.w[0];
    const T *__restrict__ wy = (const T *)L.w[1];
    const T *__restrict__ wz = (const T *)L.w[2];
    const T *__restrict__ dinv = sizeof(T) == 8 ? (const T *)L.dinv : nullptr;
    const int R = L.fR, S = L.fS;
    const int chunk = fdiv(lb, L.dfS), strip = lb - chunk * S;
    const int j0 = strip * R, k0 = chunk * L.fKc;
    const int k1 = min(k0 + L.fKc, nz);
    const int t = (int)threadIdx.x;
    const int tr = fdiv(t, L.dfq), tq = t - tr * nq;
    const int slots = R + 2;
    const int j = j0 - 1 + tr;
    bool vrow = tr < slots;
    int jj = j;
    if (j < 0) {
        if (per & 2) jj = ny - 1;
        else vrow = false;
    } else if (j >= ny) {
        if (j == ny && (per & 2)) jj = 0;
        else vrow = false;
    }
    const bool owned = vrow && tr >= 1 && tr <= R && j < ny;
    const int rowlen = slots * nx;  // elements of one plane of the ring
    Quad<T> q0{{T(0), T(0), T(0), T(0)}}, q1 = q0, q2 = q0;  // planes k, k - 1, k - 2 of this quad
    int rk = (k0 + 2) % 3;  // ring slot of plane k (k = k0 - 1 first)
    for (int k = k0 - 1; k <= k1; k++) {
        int kk = k;
        bool vpl = true;
        if (k < 0) {
            if (per & 4) kk = nz - 1;
            else vpl = false;
        } else if (k >= nz) {
            if (per & 4) kk = 0;
            else vpl = false;
        }
        if (vrow && vpl) {
            q0 = relax_quad_global<T>(xin, b, wx, wy, wz, nx, ny, nz, per, jj, kk, tq, 0, omega, zero, dinv);
            stq(sm + rk * rowlen + tr * nx + (tq << 2), q0);
        }
        __syncthreads();
        const int kb = k - 1;
        if (owned && kb >= k0) {
            const int rp = rk == 0 ? 2 : rk - 1;  // ring slot of plane k - 1
            const T *plane = sm + rp * rowlen;
            const Quad<T> out = black_quad<T>(q1, plane + tr * nx, plane + (tr - 1) * nx, plane + (tr + 1) * nx,
                                              q2, q0, b, wx, wy, wz, nx, ny, nz, per, j, kb, tq, omega, dinv);
            const int c = (j + ny * kb) * nx + (tq << 2);
            stq(xout + c, out);
            if constexpr (OUT) add_outer_quad<T>(po, c, out.v, 0xF);
        }
        q2 = q1;
        q1 = q0;
        rk = rk == 2 ? 0 : rk + 1;
    }
}

template <class T, int B, bool MAYOUT>
__device__ __forceinline__ void sweep_entry(const LevelView &L, int lb, int dir, T omega, int flags, int cyc,
                                            const OuterView *__restrict__ ov, T *sm)
{
    // the whole block returns together (a grid's state is uniform), so the
    // barriers inside the body see every thread
    if (!in_cycle(L.st, cyc)) return;
    const bool zero = flags & kZeroGuess;
    if constexpr (MAYOUT) {
        if (last_cycle(L.st, cyc)) {
            sweep_body<T, B, true>(L, lb, dir, omega, zero, outer_out(ov[L.g]), sm);
            return;
        }
    }
    sweep_body<T, B, false>(L, lb, dir, omega, zero, OuterOut{}, sm);
}

template <class T, int B, bool MAYOUT>
__global__ void __launch_bounds__(B) k_sweep(const LevelView *__restrict__ lv, const int *__restrict__ start,
                                             int count, int dir, T omega, int flags, int cyc,
                                             const OuterView *__restrict__ ov,
                                             const __grid_constant__ LevelView one, int single)
{
    dep_entry();
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    T *sm = (T *)sweep_smem;
    if (single) {
        sweep_entry<T, B, MAYOUT>(one, blockIdx.x, dir, omega, flags, cyc, ov, sm);
        return;
    }
    const int e = find_entry(start, count);
    sweep_entry<T, B, MAYOUT>(lv[e], blockIdx.x - start[e], dir, omega, flags, cyc, ov, sm);
}

template <class T, int B, bool MAYOUT>
void launch_sweep_b(const Table &tb, int dir, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    // the ring: 3 planes of at most B / nq + ... rows; (fR + 2) nq <= B, so
    // 3 (fR + 2) nx <= 12 B elements
    const size_t smem = (size_t)12 * B * sizeof(T);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sweep<T, B, MAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int single = table_single(tb);
    launch_k(k_sweep<T, B, MAYOUT>, tb.blocks, B, smem, s, tb.lv, tb.start, tb.count, dir, (T)omega, flags,
             tb.cyc, ov, table_view(tb), single);
}

}  // namespace

bool sweep_fits(const int n[3], int per, int v, bool fp32)
{
    if (v < 1 || v >= kSweepVariants) return false;
    const SweepShape sh = sweep_shape(v);
    if (sh.tile_x) return fp32 && staged_fits(n, per);
    // rows of whole quads, at least one own row per strip, and an even number
    // of cells along every periodic axis (else the colours do not alternate
    // across the wrap)
    return (n[0] & 3) == 0 && n[1] >= 2 && n[2] >= 2 && 3 * (n[0] >> 2) <= sh.B &&
           !((per & 2) && (n[1] & 1)) && !((per & 4) && (n[2] & 1));
}

int sweep_layout(LevelView &v, int variant)
{
    const SweepShape sh = sweep_shape(variant);
    if (sh.tile_x) return staged_layout(v, sh.Kc);
    const int nq = v.n[0] >> 2, ny = v.n[1], nz = v.n[2];
    const int rmax = sh.B / nq - 2;
    const int strips = (ny + rmax - 1) / rmax;
    v.fR = (ny + strips - 1) / strips;
    v.fS = strips;
    const int chunks = (nz + sh.Kc - 1) / sh.Kc;
    v.fKc = (nz + chunks - 1) / chunks;
    v.dfS = make_fastdiv((unsigned)strips);
    v.dfq = make_fastdiv((unsigned)nq);
    return strips * ((nz + v.fKc - 1) / v.fKc);
}

int sweep_blocks(const int n[3], int variant)
{
    LevelView v;
    for (int d = 0; d < 3; d++) v.n[d] = n[d];
    return sweep_layout(v, variant);
}

template <class T>
void launch_sweep(const Table &tb, int dir, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    if (tb.blocks == 0) return;
    const SweepShape sh = sweep_shape(tb.variant);
    if (sh.tile_x) {
        // FP32 only: sweep_fits() offers the staged shapes to FP32 cycles alone
        if constexpr (sizeof(T) == 4) launch_sweep_staged(tb, dir, omega, flags, ov, s);
        return;
    }
    const bool mo = (flags & kOuter) != 0;
    if (sh.B == 1024) {
        if (mo) launch_sweep_b<T, 1024, true>(tb, dir, omega, flags, ov, s);
        else launch_sweep_b<T, 1024, false>(tb, dir, omega, flags, nullptr, s);
    } else {
        if (mo) launch_sweep_b<T, 512, true>(tb, dir, omega, flags, ov, s);
        else launch_sweep_b<T, 512, false>(tb, dir, omega, flags, nullptr, s);
    }
}

template void launch_sweep<float>(const Table &, int, double, int, const OuterView *, cudaStream_t);
template void launch_sweep<double>(const Table &, int, double, int, const OuterView *, cudaStream_t);

}  // namespace gbmg
