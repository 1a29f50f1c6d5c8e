// Paired-cell FP32 3D stage kernel for the RKL2 conduction super-step: the
// tile body, the kernel template and its launch helpers, shared by the
// translation units that instantiate it (rkl_x2.cu: the classical flux and
// the ensemble kernel; rkl_x2_sat.cu: the saturated flux), so that the
// instantiations compile in parallel.
//
// Same z-march and plane-bundle pipeline as the tiled kernel, but each
// thread owns two neighbouring cells in x (columns 2l, 2l + 1 of a 64 x TY
// tile, one warp per row, five CTAs per SM) and evaluates their faces,
// divergence and recurrence with the packed
// FP32 pair instructions of sm_100+ (add/sub/mul/fma .f32x2), so one
// instruction serves both cells.  Shared-memory reads are 64-bit pairs.
// The x-face below a pair comes from the lane to the left by a warp shuffle
// (lane 0 from the tile's boundary faces), the y-face below from the row
// below through shared memory, the z-face below from the previous plane.
//
// The per-tile body (tile_x2) is also the work item of the persistent
// ensemble kernel (rkl_ensemble.cu).
//
// LIM: MC-limited transverse gradients at every face (Appendix C, the
// limiter floor at +inf).  The per-cell quantities that the unlimited form
// carries as centred differences T+ - T- become the cells' limited slopes
// MC(T+ - T0, T0 - T-), and a face takes MC of its two cells' slopes / dx
// instead of their sum / (4 dx): the same four one-sided differences per
// transverse direction.  A cell's slope is limited once per plane where the
// thread owns the cell (and again where a neighbouring face needs a cell of
// the next row or column); the kernel carries halves of the slopes
// (mc_half), which changes no rounding.
#pragma once

#include <algorithm>

#include "rkl_launch.h"
#include "rkl_pair.cuh"
#include "rkl_x2.cuh"

namespace rkl {
namespace x2 {

// --------------------------------------------------------------------------
// shared memory and copies


// Half the MC limit: MC(a, b) / 2 = sign(a) min(|a + b| / 4, |a|, |b|) if
// a b > 0, else 0.  Both factors 2 of MC are powers of two, so they move
// into the callers' constants without changing a rounding.
__device__ __forceinline__ float mc_half(float a, float b)
{
    const float m = fminf(0.25f * fabsf(a + b), fminf(fabsf(a), fabsf(b)));
    return a * b > 0.f ? copysignf(m, a) : 0.f;
}

// Per-cell transverse slope along one axis from the cell (T0) and its two
// neighbours: the centred difference T+ - T- (unscaled), or with LIM half
// the limited slope, MC(T+ - T0, T0 - T-) / 2.
template <bool LIM>
__device__ __forceinline__ float2 cslope(float2 Tp, float2 T0, float2 Tm)
{
    if (!LIM) return sub2(Tp, Tm);
    const float2 up = sub2(Tp, T0), dn = sub2(T0, Tm);
    return make_float2(mc_half(up.x, dn.x), mc_half(up.y, dn.y));
}
template <bool LIM>
__device__ __forceinline__ float cslope1(float Tp, float T0, float Tm)
{
    return LIM ? mc_half(Tp - T0, T0 - Tm) : Tp - Tm;
}
// Transverse gradient at a face from its two cells' slopes: their sum
// times 1 / (4 dx) (i4), or with LIM MC of the two limited slopes / dx =
// 4 mc_half of the halves / dx (i1 = 4 / dx).
template <bool LIM>
__device__ __forceinline__ float2 fgrad(float2 sL, float2 sR, float2 i4, float2 i1)
{
    if (!LIM) return mul2(add2(sL, sR), i4);
    return mul2(make_float2(mc_half(sL.x, sR.x), mc_half(sL.y, sR.y)), i1);
}

// Copy tasks fixed per thread for the whole tile, grouped by ring so that a
// thread's slot s always feeds the same ring (its slot offset is known at
// compile time): slot 0 a 16-byte chunk of T (TY + 2 rows x 18 chunks, halo
// ring included), slots 1-3 chunks of bx, by, bz, slots 4-5 chunks of Y0,
// Y_{j-2}, M(Y0) (3 x TY rows x 16).  Rows must start on a
// 16-byte boundary (nx % 4 == 0); chunks past the grid edge wrap
// (periodic), hold the ghost value (Dirichlet T), repeat the nearest
// interior b (Dirichlet, past the x edge) or are skipped (Y).  The smem
// address is 16-byte aligned, so its low bits carry the task's flags.
enum : unsigned { TK_VALID = 1u, TK_GHOST = 2u, TK_BCAST = 4u, TK_FLAGS = 15u, TK_T = 16u, TK_Y = 32u };
struct Task {
    const float* src;     // chunk address in plane 0
    unsigned dst;         // smem byte address in slot 0 | flags
};
constexpr int kTT = ROWS * CPR;                  // 180 T chunks
constexpr int kTBc = 3 * ROWS * CPR;             // 540 b chunks
constexpr int kY = 3 * TY * (TX / 4);            // 384 Y chunks
constexpr int kSlotB = 1, kSlotY = 4, kSlots = 6;
static_assert(kTT <= NTHREADS && kTBc <= 3 * NTHREADS && kY <= 2 * NTHREADS, "task slots");

template <int MODE, class SM>
__device__ __forceinline__ Task make_task(const SM& sm, const KGrid<float>& g, const FastArgs& a, int s, int tid,
                                          int i0, int j0)
{
    constexpr int TX = SM::TX, TY = SM::TY, CPR = SM::CPR, ROWS = SM::ROWS;
    constexpr int kTT = ROWS * CPR, kTBc = 3 * ROWS * CPR, kY = 3 * TY * (TX / 4);
    static_assert(kTT <= NTHREADS && kTBc <= 3 * NTHREADS && kY <= 2 * NTHREADS, "task slots");
    Task k{nullptr, 0u};
    const int nx = g.n[0], ny = g.n[1];
    if (s < kSlotY) {
        const int t = s == 0 ? tid : tid + (s - kSlotB) * NTHREADS;
        if (t >= (s == 0 ? kTT : kTBc)) return k;
        const int arr = s == 0 ? 0 : 1 + t / (ROWS * CPR), r = t % (ROWS * CPR);
        const int row = r / CPR - 1, c = (r % CPR) * 4 - 4;
        int gy = j0 + row, gx = i0 + c;
        bool ghost = false;
        if (gy < 0 || gy >= ny) {
            if (g.bc == 1) { ghost = true; gy = gy < 0 ? 0 : ny - 1; } else gy = pmod(gy, ny);
        }
        bool xghost = false;
        if (gx < 0 || gx >= nx) {
            // Dirichlet: a chunk past the x edge is ghosts only; b there
            // repeats the nearest interior cell (broadcast of one element)
            if (g.bc == 1) { ghost = xghost = true; gx = gx < 0 ? 0 : nx - 1; } else gx = pmod(gx, nx);
        }
        const int64_t rowoff = (int64_t)gy * nx + gx;
        if (arr == 0) {
            k.src = a.Tin + rowoff;
            k.dst = smem_u32(&sm.T[0][SM::off(row, c)]) | TK_VALID | (ghost ? TK_GHOST : 0u);
        } else {
            k.src = a.b + (int64_t)(arr - 1) * g.ncell + rowoff;
            k.dst = smem_u32(&sm.B[0][arr - 1][SM::off(row, c)]) | TK_VALID | (xghost ? TK_BCAST : 0u);
        }
        return k;
    }
    const int t = tid + (s - kSlotY) * NTHREADS;
    if (MODE != 2 || t >= kY) return k;
    const int arr = t / (TY * (TX / 4)), r = t % (TY * (TX / 4));
    const int row = r / (TX / 4), c = (r % (TX / 4)) * 4;
    if (j0 + row >= ny || i0 + c >= nx) return k;
    const float* base = arr == 0 ? a.Y0 : (arr == 1 ? a.Yjm2 : a.MY0in);
    k.src = base + (int64_t)(j0 + row) * nx + i0 + c;
    k.dst = smem_u32(&sm.Y[0][arr][row * TX + c]) | TK_VALID;
    return k;
}

struct PlaneOff {
    int64_t t, b;
    bool zghost;
};

__device__ __forceinline__ PlaneOff plane_offsets(const KGrid<float>& g, int kk)
{
    const int nz = g.n[2];
    PlaneOff o{0, 0, false};
    int kz = kk;
    if (kk < 0 || kk >= nz) {
        if (g.bc == 1) { o.zghost = true; kz = kk < 0 ? 0 : nz - 1; }
        else kz = pmod(kk, nz);
    }
    o.t = o.b = (int64_t)kz * g.plane;
    return o;
}

// Bulk-copy tasks (periodic grids with nx >= 72): thread t < 4 (TY + 2) +
// 3 TY owns one smem row of a bundle -- rows -1 .. TY of T and of bx, by,
// bz (72 columns from i0 - 4, wrapped into at most two pieces) and rows
// 0 .. TY - 1 of Y0, Y_{j-2}, M(Y0) -- copied by the TMA engine straight
// into the ring slot.
constexpr int kRowTB = 4 * ROWS;
struct RowTask {
    const float* s1;      // first piece, plane 0
    const float* s2;      // second piece (wrapped part of a halo row)
    unsigned d1, d2;      // smem byte addresses in slot 0
    unsigned n1, n2;      // bytes (0: no piece)
    unsigned flags;       // TK_T, TK_Y or 0 (b)
};

template <int MODE, class SM>
__device__ __forceinline__ RowTask make_rowtask(const SM& sm, const KGrid<float>& g, const FastArgs& a, int t, int i0,
                                                int j0)
{
    RowTask k{nullptr, nullptr, 0u, 0u, 0u, 0u, 0u};
    const int nx = g.n[0], ny = g.n[1];
    if (t < kRowTB) {
        const int arr = t / ROWS, row = t % ROWS - 1;
        const float* base = (arr == 0 ? a.Tin : a.b + (int64_t)(arr - 1) * g.ncell) + (int64_t)pmod(j0 + row, ny) * nx;
        const unsigned dst = arr == 0 ? smem_u32(&sm.T[0][(row + 1) * SXS]) : smem_u32(&sm.B[0][arr - 1][(row + 1) * SXS]);
        const int x0 = i0 - 4;
        if (x0 < 0) {                       // columns nx-4 .. nx-1, then 0 .. 67
            k.s1 = base + (nx - 4);
            k.n1 = 16u;
            k.s2 = base;
            k.d2 = dst + 16u;
            k.n2 = (unsigned)(SXS - 4) * 4u;
        } else if (x0 + SXS > nx) {         // columns x0 .. nx-1, then 0 ..
            k.s1 = base + x0;
            k.n1 = (unsigned)(nx - x0) * 4u;
            k.s2 = base;
            k.d2 = dst + k.n1;
            k.n2 = (unsigned)(x0 + SXS - nx) * 4u;
        } else {
            k.s1 = base + x0;
            k.n1 = (unsigned)SXS * 4u;
        }
        k.d1 = dst;
        k.flags = arr == 0 ? TK_T : 0u;
        return k;
    }
    const int u = t - kRowTB;
    if (MODE != 2 || u >= 3 * TY) return k;
    const int arr = u / TY, row = u % TY;
    if (j0 + row >= ny) return k;
    const float* base = arr == 0 ? a.Y0 : (arr == 1 ? a.Yjm2 : a.MY0in);
    k.s1 = base + (int64_t)(j0 + row) * nx + i0;
    k.d1 = smem_u32(&sm.Y[0][arr][row * TX]);
    k.n1 = (unsigned)min(TX, nx - i0) * 4u;
    k.flags = TK_Y;
    return k;
}

// One task of slot s in the general (Dirichlet) case; off is the slot
// offset of the task's ring.
__device__ __forceinline__ void issue(const Task& k, int s, const PlaneOff& po, unsigned off, bool withY,
                                      float bcv)
{
    const unsigned f = k.dst & TK_FLAGS;
    if (!(f & TK_VALID)) return;
    const unsigned d = (k.dst & ~TK_FLAGS) + off;
    if (s >= kSlotY) {
        if (withY) cp16(d, k.src + po.t);
    } else if (s == 0) {
        if (po.zghost || (f & TK_GHOST)) st4(d, bcv);
        else cp16(d, k.src + po.t);
    } else {
        if (f & TK_BCAST) st4(d, __ldcg(k.src + po.b));
        else cp16(d, k.src + po.b);
    }
}

// --------------------------------------------------------------------------
// per-plane quantities of a thread's cell pair

// Quantities carried from one plane to the next (needed by the z-face and
// the z-differences): T of the pair, of column 2l+2 and one row up, the
// pair's x/y slopes (cslope) and b.
struct QZ {
    float2 To;        // T at columns (2l, 2l+1)
    float Tr;         // T at column 2l+2
    float2 TU;        // T one row up
    float2 gxo, gyo;  // x / y slopes at the pair
    float2 bo[3];     // b at the pair
};

// Quantities of the current plane needed only by its x- and y-faces
// (read at the start of the plane's step, not carried).
struct QXY {
    float2 gyR;       // y slopes at (2l+1, 2l+2)
    float2 gxU;       // x slopes one row up
    float bR[3];      // b at column 2l+2
    float2 bU[3];     // b one row up
};

template <bool LIM, class SM>
__device__ __forceinline__ QZ read_qz(const SM& sm, int ts, int bs, int c, int r)
{
    const float* T = sm.T[ts];
    QZ q;
    const float2 Tc = lds2(&T[SM::off(r, c)]);
    const float2 Tl = lds2(&T[SM::off(r, c - 2)]);
    const float2 Trr = lds2(&T[SM::off(r, c + 2)]);
    const float2 Tu = lds2(&T[SM::off(r + 1, c)]);
    const float2 Td = lds2(&T[SM::off(r - 1, c)]);
    q.To = Tc;
    q.Tr = Trr.x;
    q.TU = Tu;
    q.gxo = cslope<LIM>(make_float2(Tc.y, Trr.x), Tc, make_float2(Tl.y, Tc.x));
    q.gyo = cslope<LIM>(Tu, Tc, Td);
#pragma unroll
    for (int e = 0; e < 3; ++e) q.bo[e] = lds2(&sm.B[bs][e][SM::off(r, c)]);
    return q;
}

template <bool LIM, class SM>
__device__ __forceinline__ QXY read_qxy(const SM& sm, int ts, int bs, int c, int r, const QZ& z)
{
    const float* T = sm.T[ts];
    QXY q;
    const float2 Td = lds2(&T[SM::off(r - 1, c)]);
    const float2 Tur = lds2(&T[SM::off(r + 1, c + 2)]);
    const float2 Tdr = lds2(&T[SM::off(r - 1, c + 2)]);
    const float2 Tul = lds2(&T[SM::off(r + 1, c - 2)]);
    if (LIM)    // column 2l+1's limited slope is the pair's own
        q.gyR = make_float2(z.gyo.y, cslope1<LIM>(Tur.x, z.Tr, Tdr.x));
    else
        q.gyR = cslope<LIM>(make_float2(z.TU.y, Tur.x), make_float2(z.To.y, z.Tr), make_float2(Td.y, Tdr.x));
    q.gxU = cslope<LIM>(make_float2(z.TU.y, Tur.x), z.TU, make_float2(Tul.y, z.TU.x));
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const float* B = sm.B[bs][e];
        q.bR[e] = B[SM::off(r, c + 2)];
        q.bU[e] = lds2(&B[SM::off(r + 1, c)]);
    }
    return q;
}

// Boundary faces of the tile, straight from smem: the y-face pair between
// row -1 and row 0 at columns (c, c+1), and the x-face between columns -1
// and 0 at row r.
template <bool SP, bool SAT, bool LIM, class SM>
__device__ __forceinline__ float2 low_yface2(const SM& sm, const KGrid<float>& g, const KPhys<float>& p,
                                             const FaceK& fk, int tm, int tc, int tp, int bs, int c)
{
    const float* T = sm.T[tc];
    const float2 TL = lds2(&T[SM::off(-1, c)]), TR = lds2(&T[SM::off(0, c)]);
    const float2 Ll = lds2(&T[SM::off(-1, c - 2)]), Lr = lds2(&T[SM::off(-1, c + 2)]);
    const float2 Rl = lds2(&T[SM::off(0, c - 2)]), Rr = lds2(&T[SM::off(0, c + 2)]);
    const float2 gxL = cslope<LIM>(make_float2(TL.y, Lr.x), TL, make_float2(Ll.y, TL.x));
    const float2 gxR = cslope<LIM>(make_float2(TR.y, Rr.x), TR, make_float2(Rl.y, TR.x));
    const float2 gzL = cslope<LIM>(lds2(&sm.T[tp][SM::off(-1, c)]), TL, lds2(&sm.T[tm][SM::off(-1, c)]));
    const float2 gzR = cslope<LIM>(lds2(&sm.T[tp][SM::off(0, c)]), TR, lds2(&sm.T[tm][SM::off(0, c)]));
    float2 b[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) b[e] = add2(lds2(&sm.B[bs][e][SM::off(-1, c)]), lds2(&sm.B[bs][e][SM::off(0, c)]));
    return face2s<SP, SAT>(TL, TR, mul2(sub2(TR, TL), bc2(g.inv_dx[1])),
                           fgrad<LIM>(gxL, gxR, bc2(g.inv_4dx[0]), bc2(4.f * g.inv_dx[0])),
                           fgrad<LIM>(gzL, gzR, bc2(g.inv_4dx[2]), bc2(4.f * g.inv_dx[2])), b[1], b[0], b[2], fk, p);
}

template <bool SP, bool SAT, bool LIM, class SM>
__device__ __forceinline__ float low_xface(const SM& sm, const KGrid<float>& g, const KPhys<float>& p,
                                           const FaceK& fk, int tm, int tc, int tp, int bs, int r)
{
    const float* T = sm.T[tc];
    const float TL = T[SM::off(r, -1)], TR = T[SM::off(r, 0)];
    const float gyL = cslope1<LIM>(T[SM::off(r + 1, -1)], TL, T[SM::off(r - 1, -1)]);
    const float gyR = cslope1<LIM>(T[SM::off(r + 1, 0)], TR, T[SM::off(r - 1, 0)]);
    const float gzL = cslope1<LIM>(sm.T[tp][SM::off(r, -1)], TL, sm.T[tm][SM::off(r, -1)]);
    const float gzR = cslope1<LIM>(sm.T[tp][SM::off(r, 0)], TR, sm.T[tm][SM::off(r, 0)]);
    const float gy = LIM ? mc_half(gyL, gyR) * (4.f * g.inv_dx[1]) : (gyL + gyR) * g.inv_4dx[1];
    const float gz = LIM ? mc_half(gzL, gzR) * (4.f * g.inv_dx[2]) : (gzL + gzR) * g.inv_4dx[2];
    float b[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) b[e] = sm.B[bs][e][SM::off(r, -1)] + sm.B[bs][e][SM::off(r, 0)];
    // the packed form on a duplicated scalar costs what the scalar form does
    return face2s<SP, SAT>(bc2(TL), bc2(TR), bc2((TR - TL) * g.inv_dx[0]), bc2(gy), bc2(gz), bc2(b[0]), bc2(b[1]),
                           bc2(b[2]), fk, p)
        .x;
}

}  // namespace x2

// --------------------------------------------------------------------------
// one tile: columns [i0, i0 + 64), rows [j0, j0 + 8), planes [z0, z0 + nzc)

// TMA tensor copy of one box into shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

namespace x2 {
// Tensor-map bundles (TB): the TMA engine fills the halo ring of a tile that
// touches the grid's edge with zeros where a box leaves the grid; the
// periodic images of those cells come from per-thread 16-byte chunks, at
// most one per thread.  For each of T, bx, by, bz: the chunk holding column
// -1 (x-left edge, i0 == 0) or column nx - i0 (x-right edge) in rows -1 ..
// TY, and the whole row -1 (y-low edge) or row ny - j0 (y-high edge) except
// the chunks already listed.  Needs nx > TX and ny > TY (a tile has at most
// one x edge and one y edge): at most 4 (6 + 17) = 92 chunks, taken by the
// threads of warps 1 .. 3.
struct FixTask {
    const float* src;     // chunk in plane 0 (wrapped coordinates), nullptr: none
    unsigned dst;         // smem byte address in ring slot 0
    unsigned bring;       // 1: the chunk belongs to the b ring, 0: to the T ring
};

template <class SM>
__device__ __forceinline__ FixTask make_fix(const SM& sm, const KGrid<float>& g, const FastArgs& a, int tid, int i0,
                                            int j0)
{
    FixTask f{nullptr, 0u, 0u};
    const int nx = g.n[0], ny = g.n[1];
    const int xl = i0 == 0, xr = nx - i0 <= TX, yl = j0 == 0, yh = ny - j0 <= TY;
    const int kr = (nx - i0 + 4) / 4;                   // chunk of column nx - i0 (smem column nx - i0 + 4)
    const int ny_ch = CPR - xl - xr;                    // y-strip chunks not in an x strip
    const int nxs = (xl + xr) * ROWS, n = nxs + (yl + yh) * ny_ch;
    // chunks go to warps 1 .. 3 (warp 0 issues the plane's tensor copies)
    const int t = tid - 32;
    if (t < 0 || t >= 4 * n) return f;
    const int arr = t / n, i = t % n;
    int row, k;
    if (i < nxs) {
        row = i % ROWS - 1;
        k = (i / ROWS == 0 && xl) ? 0 : kr;
    } else {
        const int jj = i - nxs;
        row = (jj / ny_ch == 0 && yl) ? -1 : ny - j0;
        k = jj % ny_ch + xl;
        if (xr && k >= kr) ++k;
    }
    const int gx = pmod(i0 + 4 * k - 4, nx), gy = pmod(j0 + row, ny);
    const float* base = arr == 0 ? a.Tin : a.b + (int64_t)(arr - 1) * g.ncell;
    f.src = base + (int64_t)gy * nx + gx;
    f.dst = arr == 0 ? smem_u32(&sm.T[0][(row + 1) * SXS + 4 * k]) : smem_u32(&sm.B[0][arr - 1][(row + 1) * SXS + 4 * k]);
    f.bring = arr == 0 ? 0u : 1u;
    return f;
}
}  // namespace x2

// YT: the Y0 / Y_{j-2} / M(Y0) bundle of each plane is one tensor copy per
// array issued by a single thread (ym: tensor maps in kernel-parameter space)
// instead of per-thread 16-byte copies; plane q completes on ybar[q & 3].
// TB: every bundle of each plane (T and b with their halo ring, and the Y
// arrays) is a tensor copy; lanes 0-6 of warp 0 issue one box each after
// lane 0 announced the plane's bytes on its barrier, every thread waits for
// the barrier, and the wrapped halo chunks (make_fix) are stored over the
// zero fill before the plane's first reader passes the CTA barrier.
// Periodic grids with nx > TX and ny > TY only.
// TXW: tile width, 64 (one warp per row) or 32 (two rows of 16 lanes per
// warp, 8 rows per tile; per-thread copies only).
template <bool SP, bool SAT, int MODE, int PD, bool BULK = false, bool YT = false, bool LIM = false,
          bool TB = false, int TXW = x2::TX>
__device__ __forceinline__ void tile_x2(x2::SmemT<PD, TXW, TB ? x2::PSTR : x2::plane_of(TXW)>& sm,
                                        const KGrid<float>& g, const KPhys<float>& p, const x2::FastArgs& a,
                                        KCoef<float> cf, unsigned* status, int i0, int j0, int z0, int nzc,
                                        const x2::YMaps* ym = nullptr, const x2::TMaps* tm = nullptr)
{
    using namespace x2;
    static_assert(TXW == x2::TX || !(BULK || YT || TB), "32-column tiles use per-thread copies");
    using SM = SmemT<PD, TXW, TB ? PSTR : plane_of(TXW)>;
    // the tile's geometry (shadows the 64-column defaults of namespace x2)
    constexpr int TX = SM::TX, TY = SM::TY, LPR = SM::LPR;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lx = tid % LPR;                   // pair index in the row
    const int r = tid / LPR;                    // row of the tile
    const int c = 2 * lx;
    const int nx = g.n[0], ny = g.n[1];

    if (MODE != 0 && a.coef_tab) {
        const float* t = a.coef_tab + 4 * a.j;
        cf.mu = t[0]; cf.nu = t[1]; cf.mt = t[2]; cf.gt = t[3];
    }

    static_assert(!(TB && (BULK || YT)), "tensor-map bundles replace the other copy paths");
    constexpr bool kYT = YT && MODE == 2 && !BULK;
    constexpr int kTk = (BULK || TB) ? 1 : (kYT ? kSlotY : kSlots);
    Task tk[kTk];
    RowTask rt{};
    FixTask fx{nullptr, 0u, 0u};
    float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (TB) {
        fx = make_fix(sm, g, a, tid, i0, j0);
        if (fx.src && (((uintptr_t)fx.src & 15u) != 0u || (fx.dst & 15u) != 0u)) {   // 16-byte chunks only
            atomicOr(status, ST_TIMEOUT);
            fx.src = nullptr;
        }
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < PD + 2; ++i) mbar_init(smem_u32(&sm.bar[i]), 1u);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        }
        __syncthreads();
    } else if constexpr (BULK) {
        rt = make_rowtask<MODE>(sm, g, a, tid, i0, j0);
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < PD + 2; ++i) mbar_init(smem_u32(&sm.bar[i]), 1u);
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int s = 0; s < kTk; ++s) tk[s] = make_task<MODE>(sm, g, a, s, tid, i0, j0);
        if constexpr (kYT) {
            if (tid == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&sm.ybar[i]), 1u);
                asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            }
            __syncthreads();
        }
    }
    // bundle q completes phase (q + 1) / (PD + 2) of barrier (q + 1) % (PD + 2)
    auto bar_of = [&](int q) { return smem_u32(&sm.bar[(q + 1) % (PD + 2)]); };
    auto wait_bundle = [&](int q) {
        if (!mbar_wait(bar_of(q), (unsigned)(((q + 1) / (PD + 2)) & 1))) atomicOr(status, ST_TIMEOUT);
    };
    const unsigned ybytes =
        MODE == 2 ? 3u * (unsigned)min(TY, ny - j0) * (unsigned)min(TX, nx - i0) * 4u : 0u;

    constexpr int PS = SM::PSTRIDE;
    // slot of plane q >= -1 in a ring of n (a mask when n is a power of two)
    auto slot = [](int q, int n) { return (n & (n - 1)) == 0 ? (q + 1) & (n - 1) : (q + 1) % n; };
    auto tslot = [&](int q) { return slot(q, SM::NT); };
    auto bslot = [&](int q) { return slot(q, SM::NB); };
    auto yslot = [&](int q) { return slot(q, SM::NY); };
    // Periodic grids have no ghost or broadcast tasks: every task is one
    // 16-byte copy, issued without branches (the slot offset selected by
    // the task's array, invalid and skipped-Y tasks predicated off).
    const bool plain = g.bc == 0;
    auto load = [&](int q, bool withY) {
        const PlaneOff po = plane_offsets(g, z0 + q);
        const unsigned ts = (unsigned)(tslot(q) * PS * 4);
        const unsigned bs = (unsigned)(bslot(q) * 3 * PS * 4);
        const unsigned ys = (unsigned)(yslot(q) * 3 * TY * TX * 4);
        if constexpr (TB) {
            if (r == 0) {
                // only the stages j >= 2 read the Y bundles (and only they
                // are given the Y tensor maps)
                const bool ytm = MODE == 2 && withY;
                const unsigned bar = bar_of(q);
                if (lane == 0) mbar_expect_tx(bar, 4u * PLANE * 4u + (ytm ? 3u * TY * TX * 4u : 0u));
                __syncwarp();
                if (lane < (ytm ? 7 : 4)) {
                    int kz = z0 + q;                    // periodic: wrap the plane index
                    kz += kz < 0 ? g.n[2] : 0;
                    kz -= kz >= g.n[2] ? g.n[2] : 0;
                    unsigned dst;
                    if (lane == 0) dst = smem_u32(&sm.T[0][0]) + ts;
                    else if (lane < 4) dst = smem_u32(&sm.B[0][lane - 1][0]) + bs;
                    else dst = smem_u32(&sm.Y[0][lane - 4][0]) + ys;
                    // a tensor copy needs a 128-byte aligned destination: a
                    // layout that breaks this reports a timeout instead of
                    // faulting (the plane's barrier then never completes)
                    if ((dst & 127u) == 0u)
                        tma_load_3d(dst, &tm->m[lane], lane < 4 ? i0 - 4 : i0, lane < 4 ? j0 - 1 : j0, kz, bar);
                    else
                        atomicOr(status, ST_TIMEOUT);
                }
            }
        } else if constexpr (BULK) {
            const unsigned bar = bar_of(q);
            if (tid == 0) mbar_expect_tx(bar, (unsigned)(kRowTB * SXS * 4) + (withY ? ybytes : 0u));
            const unsigned off = (rt.flags & TK_T) ? ts : ((rt.flags & TK_Y) ? ys : bs);
            if (rt.n1 && (withY || !(rt.flags & TK_Y))) {
                bulk_g2s(rt.d1 + off, rt.s1 + po.t, rt.n1, bar);
                if (rt.n2) bulk_g2s(rt.d2 + off, rt.s2 + po.t, rt.n2, bar);
            }
        } else if (plain) {
            // periodic: only the valid flag is set, so dst + off - 1 is the address
#pragma unroll
            for (int s = 0; s < kTk; ++s) {
                const unsigned off = (s == 0 ? ts : (s < kSlotY ? bs : ys)) - TK_VALID;
                const bool on = (tk[s].dst & TK_VALID) && (s < kSlotY || withY);
                if (on) cp16(tk[s].dst + off, tk[s].src + po.t);
            }
        } else {
#pragma unroll
            for (int s = 0; s < kTk; ++s) issue(tk[s], s, po, s == 0 ? ts : (s < kSlotY ? bs : ys), withY, g.bcv);
        }
        if constexpr (kYT) {
            // planes with Y lie inside the grid (0 <= z0 + q < nz): no wrap
            if (withY && tid == 0) {
                const unsigned bar = smem_u32(&sm.ybar[q & 3]);
                mbar_expect_tx(bar, 3u * TY * TX * 4u);
                const unsigned dst = smem_u32(&sm.Y[0][0][0]) + ys;
#pragma unroll
                for (int arr = 0; arr < 3; ++arr)
                    tma_load_3d(dst + (unsigned)(arr * TY * TX * 4), &ym->m[arr], i0, j0, z0 + q, bar);
            }
        }
    };

    // TB: the wrapped halo chunk of plane q (read in one 16-byte load, stored
    // over the zero fill once the plane's boxes have landed)
    auto fix_src = [&](int q) {
        int kz = z0 + q;
        kz += kz < 0 ? g.n[2] : 0;
        kz -= kz >= g.n[2] ? g.n[2] : 0;
        return reinterpret_cast<const float4*>(fx.src + (int64_t)kz * g.plane);
    };
    auto fix_store = [&](int q, float4 v) {
        const unsigned d = fx.dst + (fx.bring ? (unsigned)(bslot(q) * 3 * PS * 4) : (unsigned)(tslot(q) * PS * 4));
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(d), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                     : "memory");
        // the next box into this slot is written by the async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    };

    // planes -1 .. PD in flight; -1 and 0 must land before the first reads
    load(-1, false);
    cp_commit();
#pragma unroll
    for (int k = 0; k <= PD; ++k) {
        if (k <= nzc) load(k, k < nzc);
        cp_commit();
    }
    if constexpr (TB) {
        if (fx.src) {
            const float4 f0 = __ldg(fix_src(-1)), f1 = __ldg(fix_src(0));
            wait_bundle(-1);
            wait_bundle(0);
            fix_store(-1, f0);
            fix_store(0, f1);
            if (1 <= nzc) fv = __ldg(fix_src(1));
        } else {
            wait_bundle(-1);
            wait_bundle(0);
        }
    } else if constexpr (BULK) {
        wait_bundle(-1);
        wait_bundle(0);
    } else {
        cp_wait<PD>();
    }
    __syncthreads();

    const float2 idx2 = bc2(g.inv_dx[0]), idy2 = bc2(g.inv_dx[1]), idz2 = bc2(g.inv_dx[2]);
    const float2 i4x = bc2(g.inv_4dx[0]), i4y = bc2(g.inv_4dx[1]), i4z = bc2(g.inv_4dx[2]);
    // with LIM, limited face gradients take 4 / dx (fgrad)
    const float2 ilx = bc2(4.f * g.inv_dx[0]), ily = bc2(4.f * g.inv_dx[1]), ilz = bc2(4.f * g.inv_dx[2]);
    // fluxes in face2s units; cm = -fscale / dx turns their differences into M
    const FaceK fk = face_consts<SP, SAT>(p);
    const float2 cmx = bc2(-fk.fscale * g.inv_dx[0]), cmy = bc2(-fk.fscale * g.inv_dx[1]);
    const float2 cmz = bc2(-fk.fscale * g.inv_dx[2]);

    QZ A = read_qz<LIM>(sm, tslot(-1), bslot(-1), c, r);
    QZ B = read_qz<LIM>(sm, tslot(0), bslot(0), c, r);
    float2 Fz_lo = face2s<SP, SAT>(A.To, B.To, mul2(sub2(B.To, A.To), idz2), fgrad<LIM>(A.gxo, B.gxo, i4x, ilx),
                                   fgrad<LIM>(A.gyo, B.gyo, i4y, ily), add2(A.bo[2], B.bo[2]),
                                   add2(A.bo[0], B.bo[0]), add2(A.bo[1], B.bo[1]), fk, p);
    float2 TmO = A.To, TmU = A.TU;
    float TmR = A.Tr;

    const bool in0 = (j0 + r < ny) && (i0 + c < nx);   // nx % 4 == 0: both cells or none
    int64_t cbase = ((int64_t)z0 * ny + (j0 + r)) * nx + (i0 + c);

    // Plane q's divergence needs the y-face below each row (written by the
    // warp below) and, for lane 0, the tile's left boundary face; both are
    // read after the next plane's barrier, so each plane costs one barrier.
    // Pending between the two: the known part of the divergence, T and the
    // Y0 / Y_{j-2} / M(Y0) values of the pair, and its output offset.
    float2 pend = bc2(0.f), pTo = bc2(0.f), py0 = bc2(0.f), pyjm2 = bc2(0.f), pmy0 = bc2(0.f);
    int64_t pcb = 0;
    // Status of the values written, reported once at the end of the tile:
    // the sum of (y - y) stays 0 unless some y was NaN or +-Inf, the running
    // minimum flags y <= 0 (Spitzer conductivity needs T > 0).
    float2 nfacc = bc2(0.f);
    float mnacc = INFINITY;
    auto finish = [&](int qp) {
        const int par = qp & 1;
        float2 M = fma2(lds2(&sm.Fy[par][r][c]), bc2(-cmy.x), pend);
        if (lx == 0) M.x = fmaf(sm.FxLo[par][r], -cmx.x, M.x);
        if (in0) {
            float2* out = reinterpret_cast<float2*>(a.out + pcb);
            if (MODE == 0) {
                *out = M;
            } else if (MODE == 1) {
                if (a.MY0out) *reinterpret_cast<float2*>(a.MY0out + pcb) = M;
                const float2 y = fma2(bc2(cf.mt), M, pTo);
                nfacc = add2(nfacc, sub2(y, y));
                if (SP) mnacc = fminf(mnacc, fminf(y.x, y.y));
                *out = y;
            } else {
                const float2 inc = fma2(bc2(cf.mu), sub2(pTo, py0),
                                        fma2(bc2(cf.nu), sub2(pyjm2, py0), fma2(bc2(cf.mt), M, mul2(bc2(cf.gt), pmy0))));
                const float2 y = add2(py0, inc);
                nfacc = add2(nfacc, sub2(y, y));
                if (SP) mnacc = fminf(mnacc, fminf(y.x, y.y));
                *out = y;
            }
        }
    };

    // one plane: cur holds plane q, nxt receives plane q + 1
    auto step = [&](int q, QZ& cur, QZ& nxt) {
        if constexpr (TB) {
            wait_bundle(q + 1);                     // bundle q + 1 has landed
            if (fx.src) fix_store(q + 1, fv);
        } else if constexpr (BULK) {
            wait_bundle(q + 1);
        } else {
            cp_wait<PD - 1>();
        }
        if constexpr (kYT) {
            // plane q's Y bundle (read after the barrier); a polling wait,
            // bounded, that records a timeout and lets the tile finish
            if (tid == 0) {
                const unsigned bar = smem_u32(&sm.ybar[q & 3]);
                bool ok = false;
                for (int it = 0; it < (1 << 24) && !ok; ++it) ok = mbar_try_wait(bar, (unsigned)((q >> 2) & 1));
                if (!ok) atomicOr(status, ST_TIMEOUT);
            }
        }
        __syncthreads();
        // the slots of bundle q + PD + 1 held planes no thread reads any more
        if (q + PD + 1 <= nzc) load(q + PD + 1, q + PD + 1 < nzc);
        cp_commit();
        if constexpr (TB) {
            if (fx.src && q + 2 <= nzc) fv = __ldg(fix_src(q + 2));
        }
        if (q > 0) finish(q - 1);

        const float2 TmRp = make_float2(TmO.y, TmR);
        const QXY cx = read_qxy<LIM>(sm, tslot(q), bslot(q), c, r, cur);
        nxt = read_qz<LIM>(sm, tslot(q + 1), bslot(q + 1), c, r);
        const float2 TR = make_float2(cur.To.y, cur.Tr);
        const float2 gzo = cslope<LIM>(nxt.To, cur.To, TmO);
        const float2 TRn = make_float2(nxt.To.y, nxt.Tr);
        const float2 gzR = LIM ? make_float2(gzo.y, cslope1<LIM>(TRn.y, TR.y, TmRp.y)) : cslope<LIM>(TRn, TR, TmRp);
        const float2 gzU = cslope<LIM>(nxt.TU, cur.TU, TmU);

        // +x faces of the pair
        const float2 Fx = face2s<SP, SAT>(
            cur.To, TR, mul2(sub2(TR, cur.To), idx2), fgrad<LIM>(cur.gyo, cx.gyR, i4y, ily),
            fgrad<LIM>(gzo, gzR, i4z, ilz),
            add2(cur.bo[0], make_float2(cur.bo[0].y, cx.bR[0])), add2(cur.bo[1], make_float2(cur.bo[1].y, cx.bR[1])),
            add2(cur.bo[2], make_float2(cur.bo[2].y, cx.bR[2])), fk, p);
        // +y faces
        const float2 Fy = face2s<SP, SAT>(cur.To, cur.TU, mul2(sub2(cur.TU, cur.To), idy2),
                                          fgrad<LIM>(cur.gxo, cx.gxU, i4x, ilx), fgrad<LIM>(gzo, gzU, i4z, ilz),
                                          add2(cur.bo[1], cx.bU[1]), add2(cur.bo[0], cx.bU[0]),
                                          add2(cur.bo[2], cx.bU[2]), fk, p);
        // +z faces
        const float2 Fz = face2s<SP, SAT>(cur.To, nxt.To, mul2(sub2(nxt.To, cur.To), idz2),
                                          fgrad<LIM>(cur.gxo, nxt.gxo, i4x, ilx),
                                          fgrad<LIM>(cur.gyo, nxt.gyo, i4y, ily),
                                          add2(cur.bo[2], nxt.bo[2]), add2(cur.bo[0], nxt.bo[0]),
                                          add2(cur.bo[1], nxt.bo[1]), fk, p);

        // the tile's bottom y-faces and left x-faces: one extra face each,
        // taken by warps on different schedulers from plane to plane
        const int par = q & 1;
        const int wy = q & (TY - 1), wx = (q + TY / 2) & (TY - 1);
        if (r == wy) {
            *reinterpret_cast<float2*>(&sm.Fy[par][0][c]) =
                low_yface2<SP, SAT, LIM>(sm, g, p, fk, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), c);
        } else if (r == wx && lx < TY) {
            sm.FxLo[par][lx] =
                low_xface<SP, SAT, LIM>(sm, g, p, fk, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), lx);
        }
        if (MODE == 2) {
            const int ys = yslot(q);
            py0 = lds2(&sm.Y[ys][0][r * TX + c]);
            pyjm2 = lds2(&sm.Y[ys][1][r * TX + c]);
            pmy0 = lds2(&sm.Y[ys][2][r * TX + c]);
        }
        *reinterpret_cast<float2*>(&sm.Fy[par][r + 1][c]) = Fy;
        const float fxl = __shfl_up_sync(0xffffffffu, Fx.y, 1, LPR);
        // divergence without the y-face below (and, on a row's first lane, the left face)
        const float2 Fx_lo = make_float2(lx == 0 ? 0.f : fxl, Fx.x);
        pend = fma2(sub2(Fx, Fx_lo), cmx, fma2(Fy, cmy, mul2(sub2(Fz, Fz_lo), cmz)));
        pTo = cur.To;
        pcb = cbase;
        cbase += g.plane;
        Fz_lo = Fz;
        TmO = cur.To;
        TmR = cur.Tr;
        TmU = cur.TU;
    };

    int q = 0;
    for (; q + 1 < nzc; q += 2) {
        step(q, B, A);
        step(q + 1, A, B);
    }
    if (q < nzc) step(q, B, A);
    if constexpr (!BULK && !TB) cp_wait<0>();
    __syncthreads();
    finish(nzc - 1);
    if constexpr (BULK || TB) {
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < PD + 2; ++i) mbar_inval(smem_u32(&sm.bar[i]));
        }
    }
    if constexpr (kYT) {
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) mbar_inval(smem_u32(&sm.ybar[i]));
        }
    }
    if (MODE != 0) {
        const bool bad_nf = nfacc.x != 0.f || nfacc.y != 0.f;
        const bool bad_np = SP && !(mnacc > 0.f);
        if (bad_nf || bad_np) atomicOr(status, (bad_nf ? ST_NONFINITE : 0u) | (bad_np ? ST_NONPOSITIVE : 0u));
    }
    __syncthreads();
}

namespace {

// OCC selects the build: 2 the default (x2::kCtasPerSm CTAs per SM, two
// planes in flight), 3 six CTAs per SM at up to 80 registers with one plane
// in flight, 4 the MC-limited faces (LIM; two planes in flight, five CTAs
// per SM: 0.173 ms per 256^3 stage against 0.178 ms at four CTAs with 128
// registers).
// BULK: bundles copied by the TMA engine (periodic grids with nx >= 72).
// 6: the default build with 32-column tiles (two rows per warp).
constexpr int ctas_per_sm(int occ) { return (occ == 2 || occ == 6) ? x2::kCtasPerSm : (occ == 4 ? 5 : 6); }
constexpr int occ_pd(int occ) { return occ == 3 ? 1 : x2::kPD; }
constexpr int occ_txw(int occ) { return occ == 6 ? 32 : x2::TX; }

// TB: all bundles copied from tensor maps (maps: x2::TMaps, else x2::YMaps)
template <bool TB>
using MapsT = typename std::conditional<TB, x2::TMaps, x2::YMaps>::type;

template <bool SP, bool SAT, int MODE, int OCC, bool BULK, bool YT = false, bool TB = false>
__global__ void __launch_bounds__(x2::NTHREADS, ctas_per_sm(OCC))
stage_x2_kernel(KGrid<float> g, KPhys<float> p, x2::FastArgs a, KCoef<float> cf, unsigned* status, int nzchunk,
                const __grid_constant__ MapsT<TB> maps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];     // tensor copies land 128-byte aligned
    constexpr int PD = occ_pd(OCC);
    constexpr bool LIM = OCC == 4;
    constexpr int TXW = occ_txw(OCC);
    using SMT = x2::SmemT<PD, TXW, TB ? x2::PSTR : x2::plane_of(TXW)>;
    SMT& sm = *reinterpret_cast<SMT*>(smem_raw);
    const x2::YMaps* ym = nullptr;
    const x2::TMaps* tm = nullptr;
    if constexpr (TB) tm = &maps;
    else ym = &maps;
    if (nzchunk > 0) {
        // one tile column, one chunk of nzchunk planes per CTA
        const int z0 = blockIdx.z * nzchunk;
        tile_x2<SP, SAT, MODE, PD, BULK, YT, LIM, TB, TXW>(sm, g, p, a, cf, status, blockIdx.x * SMT::TX,
                                                           blockIdx.y * SMT::TY, z0, min(nzchunk, g.n[2] - z0), ym,
                                                           tm);
        return;
    }
    // Balanced schedule: the column-planes (tile column, plane) in column-major
    // order are split into gridDim.x equal runs; each CTA marches its run,
    // switching columns where the run crosses one, so every CTA carries the
    // same number of planes and no partial last wave is left.
    const int ntx = (g.n[0] + SMT::TX - 1) / SMT::TX;
    const int nz = g.n[2];
    const int64_t U = (int64_t)ntx * ((g.n[1] + SMT::TY - 1) / SMT::TY) * nz;
    int64_t u = U * blockIdx.x / gridDim.x;
    const int64_t u1 = U * (blockIdx.x + 1) / gridDim.x;
    while (u < u1) {
        const int64_t col = u / nz;
        const int z0 = (int)(u - col * nz);
        const int nzc = (int)min((int64_t)(nz - z0), u1 - u);
        tile_x2<SP, SAT, MODE, PD, BULK, YT, LIM, TB, TXW>(sm, g, p, a, cf, status, (int)(col % ntx) * SMT::TX,
                                                           (int)(col / ntx) * SMT::TY, z0, nzc, ym, tm);
        u += nzc;
    }
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

template <bool SP, bool SAT, int MODE, int OCC, bool BULK, bool YT = false, bool TB = false>
cudaError_t launch3(const KGrid<float>& g, const KPhys<float>& p, const x2::FastArgs& a, const KCoef<float>& cf,
                    unsigned* status, int nzchunk, cudaStream_t st, const MapsT<TB>& ym)
{
    constexpr int kCtasPerSm = ctas_per_sm(OCC);
    using SMT = x2::SmemT<occ_pd(OCC), occ_txw(OCC), TB ? x2::PSTR : x2::plane_of(occ_txw(OCC))>;
    const int smem = (int)sizeof(SMT);
    static bool attr_set = false;       // the attribute is per function, set once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(stage_x2_kernel<SP, SAT, MODE, OCC, BULK, YT, TB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntx = (g.n[0] + SMT::TX - 1) / SMT::TX, nty = (g.n[1] + SMT::TY - 1) / SMT::TY;
    dim3 grid(ntx, nty, nzchunk > 0 ? (g.n[2] + nzchunk - 1) / nzchunk : 1);
    if (nzchunk <= 0) {
        // balanced: one wave of resident CTAs, each run at least 8 planes long
        const int64_t U = (int64_t)ntx * nty * g.n[2];
        grid = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)kCtasPerSm * sm_count(), U / 8)), 1, 1);
        nzchunk = 0;
    }
    stage_x2_kernel<SP, SAT, MODE, OCC, BULK, YT, TB><<<grid, x2::NTHREADS, smem, st>>>(g, p, a, cf, status,
                                                                                   nzchunk, ym);
    return cudaGetLastError();
}

// ym: tensor maps of the Y arrays for the stages j >= 2 of the default
// build (OCC 2, no bulk copies), or nullptr for per-thread Y copies; tm:
// tensor maps of every bundle (OCC 2, periodic, nx > TX, ny > TY), or
// nullptr.
template <bool SP, bool SAT, int OCC, bool BULK>
cudaError_t launch_mode(int mode, const KGrid<float>& g, const KPhys<float>& p, const x2::FastArgs& a,
                        const KCoef<float>& cf, unsigned* status, int nzchunk, cudaStream_t st,
                        const x2::YMaps* ym = nullptr, const x2::TMaps* tm = nullptr)
{
    if constexpr (OCC == 2 && !BULK) {
        if (tm) {
            if (mode == 0) return launch3<SP, SAT, 0, OCC, BULK, false, true>(g, p, a, cf, status, nzchunk, st, *tm);
            if (mode == 1) return launch3<SP, SAT, 1, OCC, BULK, false, true>(g, p, a, cf, status, nzchunk, st, *tm);
            return launch3<SP, SAT, 2, OCC, BULK, false, true>(g, p, a, cf, status, nzchunk, st, *tm);
        }
    }
    static const x2::YMaps none{};
    if (mode == 0) return launch3<SP, SAT, 0, OCC, BULK>(g, p, a, cf, status, nzchunk, st, none);
    if (mode == 1) return launch3<SP, SAT, 1, OCC, BULK>(g, p, a, cf, status, nzchunk, st, none);
    if constexpr (OCC == 2 && !BULK) {
        if (ym) return launch3<SP, SAT, 2, OCC, BULK, true>(g, p, a, cf, status, nzchunk, st, *ym);
    }
    return launch3<SP, SAT, 2, OCC, BULK>(g, p, a, cf, status, nzchunk, st, none);
}

}  // namespace

// The MC-limited launches (rkl_x2_lim.cu).
cudaError_t launch_x2_lim(bool spitzer, bool saturate, int mode, const KGrid<float>& g, const KPhys<float>& p,
                          const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                          cudaStream_t st);

// The saturated-flux launches (rkl_x2_sat.cu).
cudaError_t launch_x2_sat(bool spitzer, int occ, bool bulk, int mode, const KGrid<float>& g, const KPhys<float>& p,
                          const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                          cudaStream_t st, const x2::YMaps* ym, const x2::TMaps* tm);

}  // namespace rkl
