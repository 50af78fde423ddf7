// mg_staged.cu -- one-pass red-black sweep with staged operands (Sec. 2.3
// item 5, red-black SOR; FP32 cycles, finest level): both colours of a full
// sweep in one launch as in mg_fused.cu (a sweep reads one iterate buffer and
// writes the other), with every operand of a block's tile copied into shared
// memory by asynchronous 16-byte copies (cp.async) two planes ahead of the
// relaxation, so that the relaxation reads only shared memory and registers.
//
// A block owns a tile of kStX = 128 cells along x and up to kStR = 14 own rows
// along y, and marches up a chunk of planes in z.  Its shared memory holds two
// rings of plane slots: the tile's rows of the iterate (8 cells beyond the tile
// on each side in x, two rows beyond it on each side in y; 6 slots) and of the
// x faces, b, y faces and z faces (with the halos that the relaxation of the
// tile and of its halo cells reads; 4 slots).  Step k:
//   red:   the red cells of plane k, from the old iterate: every quad of the
//          own rows and of one halo row on each side (a warp per row, a thread
//          per quad), and the quads just west and east of the tile in the own
//          rows (one more warp); the new values go into the iterate slot in
//          place (red cells read only black cells, whose old values stay);
//   a block barrier, after which the copies of plane k + 4 are issued into the
//          slots that no step reads any more;
//   black: the black cells of plane k - 1 of the own rows and columns: their
//          in-plane neighbours (new red values) from the iterate slot of plane
//          k - 1, everything else from the thread's registers (b and the faces
//          kept from its red relaxation of plane k - 1, whose quad holds the
//          black cells too; the z faces above and the z neighbours from its red
//          relaxations of planes k - 2 and k); both colours go to the other
//          iterate buffer.
// The red cells of the halo rows, halo quads and the planes just below and
// above the chunk are computed by every block that needs them, so blocks never
// wait on one another; a thread's copies of a plane are waited for
// (cp.async.wait_group) before the barrier that precedes their first use, so
// the block's only waits are its barriers and its own copies.
//
// Every cell's new value comes from relax_cell with the same operands as in
// the red and black half-sweep launches, so the result is bitwise theirs.
#include "mg_bulk.cuh"  // smem_u32
#include "mg_kernels.h"
#include "mg_stencil.cuh"

namespace gbmg {

namespace {

constexpr int kStX = 128;  // cells per tile along x
constexpr int kStR = 14;   // own rows per tile (at most)
constexpr int kStQ = kStX / 4;
constexpr int kStRowWarps = kStR + 2;         // a warp per row: own rows and the two halo rows
constexpr int kStNT = (kStRowWarps + 1) * 32;  // relaxing threads (row warps + the halo-quad warp)
constexpr int kStThreads = kStNT;
// two rings of plane slots: the iterate (6 planes) and the faces and b (4 planes)
constexpr int kStXSlots = 6, kStFSlots = 4;
// row widths (floats) of the slot arrays; first cell x0 - 8 (iterate) or x0 - 4
constexpr int kStWX = kStX + 16;  // iterate: x0 - 8 .. x0 + X + 8
constexpr int kStWF = kStX + 12;  // x faces: x0 - 4 .. x0 + X + 8
constexpr int kStWC = kStX + 8;   // b, y faces, z faces: x0 - 4 .. x0 + X + 4
constexpr int kStXSlot = (kStR + 4) * kStWX;          // iterate, rows y0 - 2 .. y0 + R + 1
constexpr int kStOFX = 0;                             // x faces, rows y0 - 1 .. y0 + R
constexpr int kStOB = kStOFX + (kStR + 2) * kStWF;    // b, rows y0 - 1 .. y0 + R
constexpr int kStOFY = kStOB + (kStR + 2) * kStWC;    // y faces, rows y0 - 1 .. y0 + R + 1
constexpr int kStOFZ = kStOFY + (kStR + 3) * kStWC;   // z faces, rows y0 - 1 .. y0 + R
constexpr int kStFSlot = kStOFZ + (kStR + 2) * kStWC;
constexpr int kStFBase = kStXSlots * kStXSlot;        // the face ring follows the iterate ring
constexpr size_t kStSmem = (size_t)(kStFBase + kStFSlots * kStFSlot) * sizeof(float);
constexpr int kStXChunks = (kStR + 4) * (kStWX / 4);
constexpr int kStChunks = kStXChunks + (kStR + 2) * (kStWF / 4) + 2 * (kStR + 2) * (kStWC / 4) + (kStR + 3) * (kStWC / 4);
constexpr int kStRounds = (kStChunks + kStNT - 1) / kStNT;
static_assert(kStQ == 32, "a row of the tile is one warp of quads");
static_assert(kStXSlot % 4 == 0 && kStOB % 4 == 0 && kStOFY % 4 == 0 && kStOFZ % 4 == 0 && kStFSlot % 4 == 0,
              "16-byte aligned slot arrays");
static_assert(kStSmem <= 232448, "shared memory of one block");
static_assert(sweep_shape(7).B == kStThreads && sweep_shape(7).tile_x == kStX, "the staged launch shapes");

// The half-sweep value of an aligned quad of the colour whose cells sit at
// offsets par and par + 2: relax_quad_global's selection and relax_cell
// calls, on operands already loaded (neighbour quads, zero where absent).
__device__ __forceinline__ Quad<float> relax_quad_vals(const Quad<float> &xq, float xw, float xe,
                                                       const Quad<float> &xs, const Quad<float> &xn,
                                                       const Quad<float> &xb, const Quad<float> &xt,
                                                       const Quad<float> &fx, float fxe, const Quad<float> &bq,
                                                       const Quad<float> &fs, const Quad<float> &fn,
                                                       const Quad<float> &fb, const Quad<float> &ft, int par,
                                                       float omega)
{
    const float xc0 = par ? xq.v[1] : xq.v[0], xc1 = par ? xq.v[3] : xq.v[2];
    const float xl0 = par ? xq.v[0] : xw, xr0 = par ? xq.v[2] : xq.v[1];
    const float xl1 = par ? xq.v[2] : xq.v[1], xr1 = par ? xe : xq.v[3];
    const float fl0 = par ? fx.v[1] : fx.v[0], fr0 = par ? fx.v[2] : fx.v[1];
    const float fl1 = par ? fx.v[3] : fx.v[2], fr1 = par ? fxe : fx.v[3];
    const float v0 = relax_cell(xc0, xl0, xr0, fl0, fr0, par ? fs.v[1] : fs.v[0], par ? fn.v[1] : fn.v[0],
                                par ? fb.v[1] : fb.v[0], par ? ft.v[1] : ft.v[0], par ? xs.v[1] : xs.v[0],
                                par ? xn.v[1] : xn.v[0], par ? xb.v[1] : xb.v[0], par ? xt.v[1] : xt.v[0],
                                par ? bq.v[1] : bq.v[0], omega);
    const float v1 = relax_cell(xc1, xl1, xr1, fl1, fr1, par ? fs.v[3] : fs.v[2], par ? fn.v[3] : fn.v[2],
                                par ? fb.v[3] : fb.v[2], par ? ft.v[3] : ft.v[2], par ? xs.v[3] : xs.v[2],
                                par ? xn.v[3] : xn.v[2], par ? xb.v[3] : xb.v[2], par ? xt.v[3] : xt.v[2],
                                par ? bq.v[3] : bq.v[2], omega);
    Quad<float> out = xq;
    out.v[0] = par ? xq.v[0] : v0;
    out.v[1] = par ? v0 : xq.v[1];
    out.v[2] = par ? xq.v[2] : v1;
    out.v[3] = par ? v1 : xq.v[3];
    return out;
}

__device__ __forceinline__ Quad<float> ldq_if(const float *p, bool on)
{
    Quad<float> q = ldq(p);
    if (!on) q = Quad<float>{{0.f, 0.f, 0.f, 0.f}};
    return q;
}

// Geometry of one block: tile x0, own rows y0 .. y0 + nown - 1, chunk planes
// k0 .. k1 - 1.
struct StTile {
    int x0, y0, nown, k0, k1;
};

__device__ __forceinline__ StTile st_tile(const LevelView &L, int lb)
{
    // fS tiles per plane range: fS = strips x x-tiles, dfq divides by the x-tiles
    const int chunk = fdiv(lb, L.dfS), tile = lb - chunk * L.fS;
    const int xtiles = L.n[0] / kStX;
    const int strip = fdiv(tile, L.dfq), xt = tile - strip * xtiles;
    StTile T;
    T.x0 = xt * kStX;
    T.y0 = strip * L.fR;
    T.nown = min(L.fR, L.n[1] - T.y0);
    T.k0 = chunk * L.fKc;
    T.k1 = min(T.k0 + L.fKc, L.n[2]);
    return T;
}

// Wrapped index of i along an axis of n cells, or -1 outside a non-periodic axis.
__device__ __forceinline__ int st_wrap(int i, int n, bool periodic)
{
    if (i >= 0 && i < n) return i;
    if (!periodic) return -1;
    i %= n;
    return i < 0 ? i + n : i;
}

template <bool OUT>
__device__ __forceinline__ void staged_body(const LevelView &L, int lb, int dir, float omega, bool zero,
                                            const OuterOut &po, unsigned char *smem)
{
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], per = L.per;
    const float *__restrict__ xin = (const float *)(dir ? L.x2 : L.x);
    float *__restrict__ xout = (float *)(dir ? L.x : L.x2);
    float *slots = (float *)smem;
    const StTile T = st_tile(L, lb);
    const int np = T.k1 - T.k0 + 4;  // planes staged: k0 - 2 .. k1 + 1
    const int t = (int)threadIdx.x, warp = t >> 5, lane = t & 31;
    const size_t plane = (size_t)nx * ny;
    // this thread's 16-byte chunks of every staged plane: source (plane 0) and
    // slot offset; null source = not copied
    const float *csrc[kStRounds];
    int cdst[kStRounds];
    bool cx[kStRounds];  // an iterate chunk (else faces or b)
#pragma unroll
    for (int m = 0; m < kStRounds; m++) {
        int f = t + m * kStNT;
        csrc[m] = nullptr;
        cdst[m] = 0;
        cx[m] = f < kStXChunks;
        if (f >= kStChunks) continue;
        int a, rows, W, hw, off;
        const float *base;
        const int c0 = kStXChunks, c1 = c0 + (kStR + 2) * (kStWF / 4), c2 = c1 + (kStR + 2) * (kStWC / 4),
                  c3 = c2 + (kStR + 3) * (kStWC / 4);
        if (f < c0) { a = 0; W = kStWX; hw = 8; off = 0; base = xin; }
        else if (f < c1) { a = 1; f -= c0; W = kStWF; hw = 4; off = kStOFX; base = (const float *)L.w[0]; }
        else if (f < c2) { a = 2; f -= c1; W = kStWC; hw = 4; off = kStOB; base = (const float *)L.b; }
        else if (f < c3) { a = 3; f -= c2; W = kStWC; hw = 4; off = kStOFY; base = (const float *)L.w[1]; }
        else { a = 4; f -= c3; W = kStWC; hw = 4; off = kStOFZ; base = (const float *)L.w[2]; }
        if (a == 0 && zero) continue;
        const int cpr = W / 4, s = f / cpr, cc = f - s * cpr;
        rows = a == 0 ? T.nown + 4 : a == 3 ? T.nown + 3 : T.nown + 2;
        if (s >= rows) continue;
        const int jj = st_wrap(T.y0 + (a == 0 ? -2 : -1) + s, ny, per & 2);
        const int xg = st_wrap(T.x0 - hw + 4 * cc, nx, per & 1);
        if (jj < 0 || xg < 0) continue;
        csrc[m] = base + (size_t)jj * nx + xg;
        cdst[m] = off + s * W + 4 * cc;
    }
    // stage plane i: iterate into slot i % 6 of its ring, the rest into slot i % 4
    auto stage = [&](int i) {
        const int kk = st_wrap(T.k0 - 2 + i, nz, per & 4);
        if (kk >= 0) {
            const unsigned sbx = smem_u32(slots + (size_t)(i % kStXSlots) * kStXSlot);
            const unsigned sbf = smem_u32(slots + kStFBase + (size_t)(i % kStFSlots) * kStFSlot);
#pragma unroll
            for (int m = 0; m < kStRounds; m++)
                if (csrc[m])
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((cx[m] ? sbx : sbf) +
                                                                                   4u * (unsigned)cdst[m]),
                                 "l"(csrc[m] + (size_t)kk * plane)
                                 : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // planes 0 .. 2 before the first step; plane i + 4 after the barrier of
    // step i (its slots were read for the last time before it), waited for
    // before the barrier of step i + 2
    stage(0);
    stage(1);
    stage(2);
    stage(3);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    stage(4);

    // relaxing warps: row warps 0 .. R + 1 (slot row tr = warp: row y0 - 1 + tr),
    // and the halo-quad warp (lane l < 2 nown: own row 1 + l / 2, west or east quad)
    const bool halo = warp == kStRowWarps;
    int tr, px, pc;
    int i0;       // first cell of the quad (global, wrapped)
    bool qv;      // the quad exists
    if (!halo) {
        tr = warp;
        i0 = T.x0 + 4 * lane;
        px = 8 + 4 * lane;
        pc = 4 + 4 * lane;
        qv = tr <= T.nown + 1;
    } else {
        tr = 1 + (lane >> 1);
        const bool east = lane & 1;
        const int ig = east ? T.x0 + kStX : T.x0 - 4;
        i0 = st_wrap(ig, nx, per & 1);
        px = east ? kStX + 8 : 4;
        pc = east ? kStX + 4 : 0;
        qv = lane < 2 * T.nown && i0 >= 0;
    }
    const int j = st_wrap(T.y0 - 1 + tr, ny, per & 2);
    qv = qv && j >= 0;
    const bool own = !halo && tr >= 1 && tr <= T.nown;
    const bool has_w = i0 > 0 || (per & 1), has_e = i0 + 4 < nx || (per & 1);
    const bool has_s = j > 0 || (per & 2), has_n = j + 1 < ny || (per & 2);

    // step r: red of staged plane r (k = k0 - 2 + r), black of plane r - 1.
    // The black relaxation of plane k - 1 takes its b and face operands from the
    // thread's registers (kept from its red relaxation of plane k - 1: the black
    // cells of a plane sit in the red cells' quads), its z faces above from the
    // red relaxation of plane k, and its z neighbours from the red values of
    // planes k - 2 and k (the same cells of the quad); only its in-plane
    // neighbours come from shared memory.
    const Quad<float> z4{{0.f, 0.f, 0.f, 0.f}};
    Quad<float> rq1 = z4;             // red quad of plane k - 1 (new red cells, old black cells)
    float rv1a = 0.f, rv1b = 0.f;     // red values of plane k - 1
    float rv2a = 0.f, rv2b = 0.f;     // red values of plane k - 2
    Quad<float> cfx = z4;             // plane k - 1: x faces of the quad,
    float cfxe = 0.f;                 // the face east of it,
    float cb0 = 0.f, cb1 = 0.f, cs0 = 0.f, cs1 = 0.f, cn0 = 0.f, cn1 = 0.f, cz0 = 0.f, cz1 = 0.f;  // b, y, z faces at its black cells
    for (int r = 1; r <= np - 2; r++) {
        const int k = T.k0 - 2 + r;
        const float *Xk = slots + (size_t)(r % kStXSlots) * kStXSlot;
        const float *Xm = slots + (size_t)((r - 1) % kStXSlots) * kStXSlot;
        const float *Xp = slots + (size_t)((r + 1) % kStXSlots) * kStXSlot;
        const float *Sk = slots + kStFBase + (size_t)(r % kStFSlots) * kStFSlot;
        const float *Sp = slots + kStFBase + (size_t)((r + 1) % kStFSlots) * kStFSlot;
        const int kk = st_wrap(k, nz, per & 4);
        Quad<float> rq0 = z4, nfx = z4;
        float nfxe = 0.f, rv0a = 0.f, rv0b = 0.f;
        float nb0 = 0.f, nb1 = 0.f, ns0 = 0.f, ns1 = 0.f, nn0 = 0.f, nn1 = 0.f, nz0 = 0.f, nz1 = 0.f;
        float tz0 = 0.f, tz1 = 0.f;  // z faces of plane k at its red cells: the black cells of k - 1 below them
        if (qv && kk >= 0) {
            const bool has_b = kk > 0 || (per & 4), has_t = kk + 1 < nz || (per & 4);
            const int par = (j + kk) & 1;
            float *xr = (float *)Xk + (tr + 1) * kStWX + px;
            const Quad<float> xq = zero ? z4 : ldq(xr);
            const float xw = (!zero && has_w) ? xr[-1] : 0.f, xe = (!zero && has_e) ? xr[4] : 0.f;
            const Quad<float> xs = ldq_if(xr - kStWX, !zero && has_s), xn = ldq_if(xr + kStWX, !zero && has_n);
            // old x of plane k - 1: its black cells are unchanged in the red quad of k - 1
            Quad<float> xb = z4;
            if (!zero && has_b) xb = r == 1 ? ldq(Xm + (tr + 1) * kStWX + px) : rq1;
            const Quad<float> xt = ldq_if(Xp + (tr + 1) * kStWX + px, !zero && has_t);
            const float *fr = Sk + kStOFX + tr * kStWF + (px - 4);
            nfx = ldq(fr);
            nfxe = has_e ? fr[4] : 0.f;
            const Quad<float> bq = ldq(Sk + kStOB + tr * kStWC + pc);
            const Quad<float> fs = ldq(Sk + kStOFY + tr * kStWC + pc);
            const Quad<float> fn = ldq_if(Sk + kStOFY + (tr + 1) * kStWC + pc, has_n);
            const Quad<float> fb = ldq(Sk + kStOFZ + tr * kStWC + pc);
            const Quad<float> ft = ldq_if(Sp + kStOFZ + tr * kStWC + pc, has_t);
            rq0 = relax_quad_vals(xq, xw, xe, xs, xn, xb, xt, nfx, nfxe, bq, fs, fn, fb, ft, par, omega);
            rv0a = par ? rq0.v[1] : rq0.v[0];
            rv0b = par ? rq0.v[3] : rq0.v[2];
            // the black cells of this quad (offsets 1 - par), for the next step
            nb0 = par ? bq.v[0] : bq.v[1];
            nb1 = par ? bq.v[2] : bq.v[3];
            ns0 = par ? fs.v[0] : fs.v[1];
            ns1 = par ? fs.v[2] : fs.v[3];
            nn0 = par ? fn.v[0] : fn.v[1];
            nn1 = par ? fn.v[2] : fn.v[3];
            nz0 = par ? fb.v[0] : fb.v[1];
            nz1 = par ? fb.v[2] : fb.v[3];
            tz0 = par ? fb.v[1] : fb.v[0];
            tz1 = par ? fb.v[3] : fb.v[2];
            if (zero) {
                stq(xr, rq0);  // the black cells' zero values too
            } else {
                xr[par] = rv0a;
                xr[par + 2] = rv0b;
            }
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // plane r + 2 (this thread's chunks)
        __syncthreads();
        if (r + 4 < np) stage(r + 4);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        const int kb = k - 1;
        if (own && r >= 3) {  // black of planes k0 .. k1 - 1: cells at offsets pb, pb + 2
            const bool has_b = kb > 0 || (per & 4), has_t = kb + 1 < nz || (per & 4);
            const int pb = (1 + j + kb) & 1;
            const float *xr = Xm + (tr + 1) * kStWX + px;
            const float xw = has_w ? xr[-1] : 0.f, xe = has_e ? xr[4] : 0.f;
            const Quad<float> xs = ldq_if(xr - kStWX, has_s), xn = ldq_if(xr + kStWX, has_n);
            const Quad<float> &xq = rq1;
            const float xc0 = pb ? xq.v[1] : xq.v[0], xc1 = pb ? xq.v[3] : xq.v[2];
            const float xl0 = pb ? xq.v[0] : xw, xr0 = pb ? xq.v[2] : xq.v[1];
            const float xl1 = pb ? xq.v[2] : xq.v[1], xr1 = pb ? xe : xq.v[3];
            const float fl0 = pb ? cfx.v[1] : cfx.v[0], fr0 = pb ? cfx.v[2] : cfx.v[1];
            const float fl1 = pb ? cfx.v[3] : cfx.v[2], fr1 = pb ? cfxe : cfx.v[3];
            const float v0 = relax_cell(xc0, xl0, xr0, fl0, fr0, cs0, cn0, cz0, has_t ? tz0 : 0.f,
                                        pb ? xs.v[1] : xs.v[0], pb ? xn.v[1] : xn.v[0], has_b ? rv2a : 0.f,
                                        has_t ? rv0a : 0.f, cb0, omega);
            const float v1 = relax_cell(xc1, xl1, xr1, fl1, fr1, cs1, cn1, cz1, has_t ? tz1 : 0.f,
                                        pb ? xs.v[3] : xs.v[2], pb ? xn.v[3] : xn.v[2], has_b ? rv2b : 0.f,
                                        has_t ? rv0b : 0.f, cb1, omega);
            Quad<float> out = xq;
            out.v[0] = pb ? xq.v[0] : v0;
            out.v[1] = pb ? v0 : xq.v[1];
            out.v[2] = pb ? xq.v[2] : v1;
            out.v[3] = pb ? v1 : xq.v[3];
            const int c = (j + ny * kb) * nx + i0;
            stq(xout + c, out);
            if constexpr (OUT) add_outer_quad<float>(po, c, out.v, 0xF);
        }
        cfx = nfx;
        cfxe = nfxe;
        cb0 = nb0; cb1 = nb1; cs0 = ns0; cs1 = ns1; cn0 = nn0; cn1 = nn1; cz0 = nz0; cz1 = nz1;
        rv2a = rv1a; rv2b = rv1b;
        rv1a = rv0a; rv1b = rv0b;
        rq1 = rq0;
    }
}

template <bool MAYOUT>
__device__ __forceinline__ void staged_entry(const LevelView &L, int lb, int dir, float omega, int flags, int cyc,
                                             const OuterView *__restrict__ ov, unsigned char *smem)
{
    // the whole block returns together (a grid's state is uniform)
    if (!in_cycle(L.st, cyc)) return;
    const bool zero = flags & kZeroGuess;
    if constexpr (MAYOUT) {
        if (last_cycle(L.st, cyc)) {
            staged_body<true>(L, lb, dir, omega, zero, outer_out(ov[L.g]), smem);
            return;
        }
    }
    staged_body<false>(L, lb, dir, omega, zero, OuterOut{}, smem);
}

template <bool MAYOUT>
__global__ void __launch_bounds__(kStThreads, 1)
    k_sweep_staged(const LevelView *__restrict__ lv, const int *__restrict__ start, int count, int dir, float omega,
                   int flags, int cyc, const OuterView *__restrict__ ov, const __grid_constant__ LevelView one,
                   int single)
{
    // the next grid is allowed only as the blocks finish (dep_release, or the
    // block's exit): its blocks would otherwise sit on this kernel's SMs, in
    // the threads and registers a staged block leaves free, for the whole
    // march, taking issue slots from a kernel that is bound by them
    dep_wait();
    extern __shared__ __align__(128) unsigned char staged_smem[];
    if (single) {
        staged_entry<MAYOUT>(one, blockIdx.x, dir, omega, flags, cyc, ov, staged_smem);
    } else {
        const int e = find_entry(start, count);
        staged_entry<MAYOUT>(lv[e], blockIdx.x - start[e], dir, omega, flags, cyc, ov, staged_smem);
    }
    dep_release();
}

template <bool MAYOUT>
void launch_staged_b(const Table &tb, int dir, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sweep_staged<MAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStSmem);
        attr = true;
    }
    launch_k(k_sweep_staged<MAYOUT>, tb.blocks, kStThreads, kStSmem, s, tb.lv, tb.start, tb.count, dir,
             (float)omega, flags, tb.cyc, ov, table_view(tb), table_single(tb));
}

}  // namespace

bool staged_fits(const int n[3], int per)
{
    // whole tiles along x, and an even number of cells along every periodic
    // axis (else the colours do not alternate across the wrap)
    return n[0] % kStX == 0 && n[1] >= 2 && n[2] >= 2 && !((per & 2) && (n[1] & 1)) && !((per & 4) && (n[2] & 1));
}

int staged_layout(LevelView &v, int kc)
{
    const int ny = v.n[1], nz = v.n[2];
    const int strips = (ny + kStR - 1) / kStR;
    v.fR = (ny + strips - 1) / strips;
    const int xtiles = v.n[0] / kStX;
    v.fS = strips * xtiles;
    const int chunks = (nz + kc - 1) / kc;
    v.fKc = (nz + chunks - 1) / chunks;
    v.dfS = make_fastdiv((unsigned)v.fS);
    v.dfq = make_fastdiv((unsigned)xtiles);
    return v.fS * ((nz + v.fKc - 1) / v.fKc);
}

void launch_sweep_staged(const Table &tb, int dir, double omega, int flags, const OuterView *ov, cudaStream_t s)
{
    if (tb.blocks == 0) return;
    if (flags & kOuter) launch_staged_b<true>(tb, dir, omega, flags, ov, s);
    else launch_staged_b<false>(tb, dir, omega, flags, nullptr, s);
}

}  // namespace gbmg
