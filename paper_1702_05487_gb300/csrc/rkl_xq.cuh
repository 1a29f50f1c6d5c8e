// Row-pair FP32 3D stage kernel for the RKL2 conduction super-step:
// shared-memory layout, tile body, kernel template and launch helpers,
// shared by the translation units that instantiate it (rkl_xq.cu: the
// classical flux and the ensemble kernel; rkl_xq_sat.cu: the saturated flux;
// rkl_xq_lim.cu: the MC-limited transverse gradients), so that the
// instantiations compile in parallel.
//
// The kernel runs the paired-cell kernel's arithmetic with each thread owning two cell pairs,
// (2l, 2l + 1) in rows 2w and 2w + 1 of a 64 x 8 tile (lane l, warp w).
// With 32-column tiles (for grids whose width is an odd multiple of 32) a
// warp holds two row pairs side by side in its lane halves: lanes 0-15 rows
// 4w, 4w + 1 and lanes 16-31 rows 4w + 2, 4w + 3 of a 32 x 16 tile.
//
// What a thread shares between its two rows instead of reading or
// exchanging it: the y-face between them (its own, in registers; only row
// 2w's lower face comes from the warp below through shared memory), row
// 2w + 1's T, slopes and b as row 2w's "one row up" quantities, and the
// per-plane bookkeeping (ring slots, copy issue, plane offsets, loop) over
// four cells instead of two.  The copy tasks are positions of a plane (a
// 16-byte chunk of a tile row with its halo), each issuing the same chunk of
// T, bx, by and bz (and of Y0, Y_{j-2}, M(Y0)), so a thread holds three
// 32-bit offset pairs instead of six pointer tasks.  Three CTAs of 70 KB per
// SM.  Every shared-memory row that a row of lanes reads starts on a
// 128-byte boundary (the T and b planes keep their rows' halo chunks apart
// from the interior rows), so that a 256-byte row is two wavefronts.  The
// saturated builds for kappa_perp = 0 leave out the perpendicular terms at
// compile time (the same bits for finite values); the limited builds (the
// MC limiter at every face) carry half the limited slopes, as the
// paired-cell kernel's limited build does.
//
// Every face flux, slope, divergence term and recurrence update is the
// same operation on the same operands, in the same order, as in the
// paired-cell kernel (rkl_x2_tile.cuh), so the two kernels write the same
// bits.  Periodic grids with nx % 4 == 0 and fewer than 2^31 cells.
#pragma once

#include <algorithm>

#include "rkl_x2_tile.cuh"

namespace rkl {
namespace xq {

using x2::add2;
using x2::bc2;
using x2::cp16;
using x2::cp_commit;
using x2::cp_wait;
using x2::fma2;
using x2::lds2;
using x2::mul2;
using x2::smem_u32;
using x2::sub2;

constexpr int NTHREADS = 128;
constexpr int NWARPS = NTHREADS / 32;
constexpr int PD = 2;                   // planes in flight
constexpr int kCtasPerSm = 3;

// Geometry and rings of one tile TXW columns wide (64 or 32): TXW / 2 lanes
// per row pair, 32 / (TXW / 2) row pairs per warp.  Rings: T planes q-1,
// q, q+1 and those in flight; b planes q, q+1 and those in flight; Y planes
// q and those in flight (a plane's Y bundle is issued one plane after its T
// and b, as it is read one plane later).
template <int TXW>
struct SmemQ {
    static constexpr int TX = TXW, LPR = TXW / 2, SEGS = 32 / LPR;
    static constexpr int TY = 2 * SEGS * NWARPS;        // 8 rows (64 columns) or 16 (32 columns)
    static constexpr int NRP = TY / 2;                  // row pairs
    // A plane: the interior rows (-1 .. TY, TX floats each, 128-byte
    // aligned so that a row of lanes reads a row in two shared-memory
    // wavefronts), then the rows' halo chunks (the 4 columns left and the 4
    // right of each row), padded to a 128-byte multiple.
    static constexpr int CPR = (TX + 8) / 4;            // 16-byte chunks of a row with its halo
    static constexpr int ROWS = TY + 2;
    static constexpr int HALO = ROWS * TX;              // first halo chunk of a plane
    static constexpr int PLANE = (ROWS * (TX + 8) + 31) / 32 * 32;
    static constexpr int kPos = ROWS * CPR;             // T / b chunk positions of a plane (180)
    static constexpr int kYPos = TY * (TX / 4);         // Y chunk positions (128: one per thread)
    static_assert(kPos <= 2 * NTHREADS && kYPos == NTHREADS, "copy positions");
    static constexpr int NT = 3 + PD, NB = 2 + PD, NY = 1 + PD;
    alignas(128) float T[NT][PLANE];
    alignas(128) float B[NB][3][PLANE];
    // rows of TX floats read as 64-bit pairs by a whole row of lanes: on
    // 128-byte boundaries a row is two shared-memory wavefronts, not three
    alignas(128) float Y[NY][3][TY * TX];
    alignas(128) float Fy[2][NRP + 1][TX];   // row k: lower y-face of row 2k (k = 0: the tile's boundary)
    float FxLo[2][TY];              // x-faces on the tile's left boundary
    // offset of interior cell (row r, column c), 0 <= c < TX, in a plane
    __device__ static int offI(int r, int c) { return (r + 1) * TX + c; }
    // offset of any cell of a row with its halo, -4 <= c < TX + 4
    __device__ static int off(int r, int c)
    {
        return (c >= 0 && c < TX) ? offI(r, c) : HALO + (r + 1) * 8 + (c < 0 ? c + 4 : c - TX + 4);
    }
};
using Smem = SmemQ<64>;

// A thread's two rows of one plane: T, the x / y slopes (centred
// differences) and b at the pair of each row, T at column c + 2, and T one
// row above the upper row.
struct QZ2 {
    float2 T0, T1;
    float r0, r1;
    float2 TU;
    float2 gx0, gx1, gy0, gy1;
    float2 b0[3], b1[3];
};

template <bool LIM, class SM>
__device__ __forceinline__ QZ2 read_qz2(const SM& sm, int ts, int bs, int c, int ra)
{
    const int rb = ra + 1;
    const float* T = sm.T[ts];
    QZ2 q;
    const float2 Td = lds2(&T[SM::offI(ra - 1, c)]);
    const float2 Tc0 = lds2(&T[SM::offI(ra, c)]);
    const float2 Tc1 = lds2(&T[SM::offI(rb, c)]);
    const float2 Tu = lds2(&T[SM::offI(rb + 1, c)]);
    const float l0 = T[SM::off(ra, c - 1)], l1 = T[SM::off(rb, c - 1)];
    q.r0 = T[SM::off(ra, c + 2)];
    q.r1 = T[SM::off(rb, c + 2)];
    q.T0 = Tc0;
    q.T1 = Tc1;
    q.TU = Tu;
    q.gx0 = x2::cslope<LIM>(make_float2(Tc0.y, q.r0), Tc0, make_float2(l0, Tc0.x));
    q.gx1 = x2::cslope<LIM>(make_float2(Tc1.y, q.r1), Tc1, make_float2(l1, Tc1.x));
    q.gy0 = x2::cslope<LIM>(Tc1, Tc0, Td);
    q.gy1 = x2::cslope<LIM>(Tu, Tc1, Tc0);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        q.b0[e] = lds2(&sm.B[bs][e][SM::offI(ra, c)]);
        q.b1[e] = lds2(&sm.B[bs][e][SM::offI(rb, c)]);
    }
    return q;
}

// Copy positions of a thread: T / b positions tid and tid + 128 (rows -1 ..
// TY of the tile with a 4-column halo on each side, wrapped periodically),
// Y position tid.  src: element offset in plane 0; dst: byte offset in a
// ring slot; ~0u: no position.
struct Pos {
    unsigned src, dst;
};

template <class SM>
__device__ __forceinline__ Pos tb_pos(const KGrid<float>& g, int t, int i0, int j0)
{
    if (t >= SM::kPos) return Pos{0u, ~0u};
    const int row = t / SM::CPR - 1, cc = (t % SM::CPR) * 4 - 4;
    const int gy = x2::pmod(j0 + row, g.n[1]), gx = x2::pmod(i0 + cc, g.n[0]);
    return Pos{(unsigned)gy * (unsigned)g.n[0] + (unsigned)gx, (unsigned)(SM::off(row, cc) * 4)};
}

template <class SM>
__device__ __forceinline__ Pos y_pos(const KGrid<float>& g, int t, int i0, int j0)
{
    constexpr int TX = SM::TX;
    const int row = t / (TX / 4), cc = (t % (TX / 4)) * 4;
    if (j0 + row >= g.n[1] || i0 + cc >= g.n[0]) return Pos{0u, ~0u};
    return Pos{(unsigned)(j0 + row) * (unsigned)g.n[0] + (unsigned)(i0 + cc), (unsigned)((row * TX + cc) * 4)};
}

template <bool SP, bool SAT, int MODE, int TXW, bool KP0 = false, bool LIM = false>
__device__ __forceinline__ void tile_q(SmemQ<TXW>& sm, const KGrid<float>& g, const KPhys<float>& p,
                                       const x2::FastArgs& a, KCoef<float> cf, unsigned* status, int i0, int j0,
                                       int z0, int nzc)
{
    using Smem = SmemQ<TXW>;
    constexpr int TX = Smem::TX, TY = Smem::TY, LPR = Smem::LPR, SEGS = Smem::SEGS;
    constexpr int PLANE = Smem::PLANE;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lx = lane % LPR;                  // pair index in the row
    const int w = tid >> 5;
    const int rp = w * SEGS + lane / LPR;       // row pair: rows 2 rp, 2 rp + 1
    const int ra = 2 * rp, rb = ra + 1;
    const int c = 2 * lx;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];

    if (MODE != 0 && a.coef_tab) {
        const float* t = a.coef_tab + 4 * a.j;
        cf.mu = t[0]; cf.nu = t[1]; cf.mt = t[2]; cf.gt = t[3];
    }

    const Pos p0 = tb_pos<Smem>(g, tid, i0, j0), p1 = tb_pos<Smem>(g, tid + NTHREADS, i0, j0);
    const Pos py = MODE == 2 ? y_pos<Smem>(g, tid, i0, j0) : Pos{0u, ~0u};
    const float* bxp = a.b;
    const float* byp = a.b + g.ncell;
    const float* bzp = a.b + 2 * g.ncell;
    const unsigned plane = (unsigned)g.plane;
    const unsigned tbase = smem_u32(&sm.T[0][0]), bbase = smem_u32(&sm.B[0][0][0]), ybase = smem_u32(&sm.Y[0][0][0]);

    auto tslot = [](int q) { return (q + 1) % Smem::NT; };
    auto bslot = [](int q) { return (q + 1) & (Smem::NB - 1); };
    auto yslot = [](int q) { return q % Smem::NY; };
    static_assert((Smem::NB & (Smem::NB - 1)) == 0, "b ring size a power of two");

    // T and b of plane k, and (stages j >= 2) the Y bundle of plane k - 1
    auto load = [&](int k) {
        int kz = z0 + k;                        // periodic: wrap the plane index
        kz += kz < 0 ? nz : 0;
        kz -= kz >= nz ? nz : 0;
        const unsigned pt = (unsigned)kz * plane;
        const unsigned ts = tbase + (unsigned)(tslot(k) * PLANE * 4);
        const unsigned bs = bbase + (unsigned)(bslot(k) * 3 * PLANE * 4);
        {
            const unsigned x = p0.src + pt;
            cp16(ts + p0.dst, a.Tin + x);
            cp16(bs + p0.dst, bxp + x);
            cp16(bs + PLANE * 4 + p0.dst, byp + x);
            cp16(bs + 2 * PLANE * 4 + p0.dst, bzp + x);
        }
        if (p1.dst != ~0u) {
            const unsigned x = p1.src + pt;
            cp16(ts + p1.dst, a.Tin + x);
            cp16(bs + p1.dst, bxp + x);
            cp16(bs + PLANE * 4 + p1.dst, byp + x);
            cp16(bs + 2 * PLANE * 4 + p1.dst, bzp + x);
        }
        if (MODE == 2 && k >= 1 && py.dst != ~0u) {
            // plane k - 1 lies inside the chunk, so inside the grid
            const unsigned x = py.src + (unsigned)(z0 + k - 1) * plane;
            const unsigned ys = ybase + (unsigned)(yslot(k - 1) * 3 * TY * TX * 4);
            cp16(ys + py.dst, a.Y0 + x);
            cp16(ys + TY * TX * 4 + py.dst, a.Yjm2 + x);
            cp16(ys + 2 * TY * TX * 4 + py.dst, a.MY0in + x);
        }
    };

    // groups: plane -1, then planes 0 .. PD; plane k's group also carries
    // the Y bundle of plane k - 1
    load(-1);
    cp_commit();
#pragma unroll
    for (int k = 0; k <= PD; ++k) {
        if (k <= nzc) load(k);
        cp_commit();
    }
    cp_wait<PD>();
    __syncthreads();

    const float2 idx2 = bc2(g.inv_dx[0]), idy2 = bc2(g.inv_dx[1]), idz2 = bc2(g.inv_dx[2]);
    const float2 i4x = bc2(g.inv_4dx[0]), i4y = bc2(g.inv_4dx[1]), i4z = bc2(g.inv_4dx[2]);
    // with LIM, limited face gradients take 4 / dx (x2::fgrad)
    const float2 ilx = bc2(4.f * g.inv_dx[0]), ily = bc2(4.f * g.inv_dx[1]), ilz = bc2(4.f * g.inv_dx[2]);
    const x2::FaceK fk = x2::face_consts<SP, SAT>(p);
    const float2 cmx = bc2(-fk.fscale * g.inv_dx[0]), cmy = bc2(-fk.fscale * g.inv_dx[1]);
    const float2 cmz = bc2(-fk.fscale * g.inv_dx[2]);

    QZ2 A = read_qz2<LIM>(sm, tslot(-1), bslot(-1), c, ra);
    QZ2 B = read_qz2<LIM>(sm, tslot(0), bslot(0), c, ra);
    float2 Fzl0 = x2::face2s<SP, SAT, KP0>(A.T0, B.T0, mul2(sub2(B.T0, A.T0), idz2), x2::fgrad<LIM>(A.gx0, B.gx0, i4x, ilx),
                                      x2::fgrad<LIM>(A.gy0, B.gy0, i4y, ily), add2(A.b0[2], B.b0[2]),
                                      add2(A.b0[0], B.b0[0]), add2(A.b0[1], B.b0[1]), fk, p);
    float2 Fzl1 = x2::face2s<SP, SAT, KP0>(A.T1, B.T1, mul2(sub2(B.T1, A.T1), idz2), x2::fgrad<LIM>(A.gx1, B.gx1, i4x, ilx),
                                      x2::fgrad<LIM>(A.gy1, B.gy1, i4y, ily), add2(A.b1[2], B.b1[2]),
                                      add2(A.b1[0], B.b1[0]), add2(A.b1[1], B.b1[1]), fk, p);
    // plane q - 1 of the z-march: T of both pairs, at column c + 2, one row up
    float2 Tm0 = A.T0, Tm1 = A.T1, TmU = A.TU;
    float Tmr0 = A.r0, Tmr1 = A.r1;

    const bool inx = i0 + c < nx;               // nx % 4 == 0: both cells or none
    const bool in0 = inx && j0 + ra < ny, in1 = inx && j0 + rb < ny;
    int64_t cbase = ((int64_t)z0 * ny + (j0 + ra)) * nx + (i0 + c);

    // Pending between a plane and the next barrier: the divergence without
    // row 2w's lower y-face and without the left boundary face (lane 0),
    // the Y0 / Y_{j-2} / M(Y0) values of both pairs, the output offset.
    float2 pend0 = bc2(0.f), pend1 = bc2(0.f);
    float2 y00 = bc2(0.f), y01 = bc2(0.f), yj0 = bc2(0.f), yj1 = bc2(0.f), my0 = bc2(0.f), my1 = bc2(0.f);
    int64_t pcb = 0;
    float2 nfacc = bc2(0.f);
    float mnacc = INFINITY;

    auto emit = [&](int64_t o, float2 M, float2 To, float2 py0, float2 pyjm2, float2 pmy0) {
        float2* out = reinterpret_cast<float2*>(a.out + o);
        if (MODE == 0) {
            *out = M;
        } else if (MODE == 1) {
            if (a.MY0out) *reinterpret_cast<float2*>(a.MY0out + o) = M;
            const float2 y = fma2(bc2(cf.mt), M, To);
            nfacc = add2(nfacc, sub2(y, y));
            if (SP) mnacc = fminf(mnacc, fminf(y.x, y.y));
            *out = y;
        } else {
            const float2 inc = fma2(bc2(cf.mu), sub2(To, py0),
                                    fma2(bc2(cf.nu), sub2(pyjm2, py0), fma2(bc2(cf.mt), M, mul2(bc2(cf.gt), pmy0))));
            const float2 y = add2(py0, inc);
            nfacc = add2(nfacc, sub2(y, y));
            if (SP) mnacc = fminf(mnacc, fminf(y.x, y.y));
            *out = y;
        }
    };
    // Tm0 / Tm1 hold T of plane qp when finish(qp) runs
    auto finish = [&](int qp) {
        const int par = qp & 1;
        float2 M0 = fma2(lds2(&sm.Fy[par][rp][c]), bc2(-cmy.x), pend0);
        float2 M1 = pend1;
        if (lx == 0) {
            M0.x = fmaf(sm.FxLo[par][ra], -cmx.x, M0.x);
            M1.x = fmaf(sm.FxLo[par][rb], -cmx.x, M1.x);
        }
        if (in0) emit(pcb, M0, Tm0, y00, yj0, my0);
        if (in1) emit(pcb + nx, M1, Tm1, y01, yj1, my1);
    };

    // one plane: cur holds plane q, nxt receives plane q + 1
    auto step = [&](int q, QZ2& cur, QZ2& nxt) {
        cp_wait<PD - 1>();
        __syncthreads();
        // the slots of plane q + PD + 1 held planes no thread reads any more
        if (q + PD + 1 <= nzc) load(q + PD + 1);
        cp_commit();
        if (q > 0) finish(q - 1);

        const int ts = tslot(q), bs = bslot(q);
        // plane q beyond the pairs' own quantities
        const float* T = sm.T[ts];
        const float Tdr = T[Smem::off(ra - 1, c + 2)];      // row 2w - 1, column c + 2
        const float Tur = T[Smem::off(rb + 1, c + 2)];      // row 2w + 2, column c + 2
        const float Tul = T[Smem::off(rb + 1, c - 1)];      // row 2w + 2, column c - 1
        float bR0[3], bR1[3];
        float2 bU1[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float* Bp = sm.B[bs][e];
            bR0[e] = Bp[Smem::off(ra, c + 2)];
            bR1[e] = Bp[Smem::off(rb, c + 2)];
            bU1[e] = lds2(&Bp[Smem::offI(rb + 1, c)]);
        }
        nxt = read_qz2<LIM>(sm, tslot(q + 1), bslot(q + 1), c, ra);

        // z slopes over planes q - 1 .. q + 1 (centred differences, or with
        // LIM half the limited slopes)
        const float2 gz0 = x2::cslope<LIM>(nxt.T0, cur.T0, Tm0), gz1 = x2::cslope<LIM>(nxt.T1, cur.T1, Tm1);
        const float2 gzR0 = make_float2(gz0.y, x2::cslope1<LIM>(nxt.r0, cur.r0, Tmr0));
        const float2 gzR1 = make_float2(gz1.y, x2::cslope1<LIM>(nxt.r1, cur.r1, Tmr1));
        const float2 gzU1 = x2::cslope<LIM>(nxt.TU, cur.TU, TmU);
        // y slopes at columns (c + 1, c + 2) (column c + 1's is the pair's
        // own), x slopes one row up
        const float2 gyR0 = make_float2(cur.gy0.y, x2::cslope1<LIM>(cur.r1, cur.r0, Tdr));
        const float2 gyR1 = make_float2(cur.gy1.y, x2::cslope1<LIM>(Tur, cur.r1, cur.r0));
        const float2 gxU1 = x2::cslope<LIM>(make_float2(cur.TU.y, Tur), cur.TU, make_float2(Tul, cur.TU.x));

        // +x faces of both pairs
        const float2 TR0 = make_float2(cur.T0.y, cur.r0), TR1 = make_float2(cur.T1.y, cur.r1);
        const float2 Fx0 = x2::face2s<SP, SAT, KP0>(
            cur.T0, TR0, mul2(sub2(TR0, cur.T0), idx2), x2::fgrad<LIM>(cur.gy0, gyR0, i4y, ily), x2::fgrad<LIM>(gz0, gzR0, i4z, ilz),
            add2(cur.b0[0], make_float2(cur.b0[0].y, bR0[0])), add2(cur.b0[1], make_float2(cur.b0[1].y, bR0[1])),
            add2(cur.b0[2], make_float2(cur.b0[2].y, bR0[2])), fk, p);
        const float2 Fx1 = x2::face2s<SP, SAT, KP0>(
            cur.T1, TR1, mul2(sub2(TR1, cur.T1), idx2), x2::fgrad<LIM>(cur.gy1, gyR1, i4y, ily), x2::fgrad<LIM>(gz1, gzR1, i4z, ilz),
            add2(cur.b1[0], make_float2(cur.b1[0].y, bR1[0])), add2(cur.b1[1], make_float2(cur.b1[1].y, bR1[1])),
            add2(cur.b1[2], make_float2(cur.b1[2].y, bR1[2])), fk, p);
        // +y faces: between the two rows, and above the upper row
        const float2 Fy0 = x2::face2s<SP, SAT, KP0>(cur.T0, cur.T1, mul2(sub2(cur.T1, cur.T0), idy2),
                                               x2::fgrad<LIM>(cur.gx0, cur.gx1, i4x, ilx), x2::fgrad<LIM>(gz0, gz1, i4z, ilz),
                                               add2(cur.b0[1], cur.b1[1]), add2(cur.b0[0], cur.b1[0]),
                                               add2(cur.b0[2], cur.b1[2]), fk, p);
        const float2 Fy1 = x2::face2s<SP, SAT, KP0>(cur.T1, cur.TU, mul2(sub2(cur.TU, cur.T1), idy2),
                                               x2::fgrad<LIM>(cur.gx1, gxU1, i4x, ilx), x2::fgrad<LIM>(gz1, gzU1, i4z, ilz),
                                               add2(cur.b1[1], bU1[1]), add2(cur.b1[0], bU1[0]),
                                               add2(cur.b1[2], bU1[2]), fk, p);
        // +z faces
        const float2 Fz0 = x2::face2s<SP, SAT, KP0>(cur.T0, nxt.T0, mul2(sub2(nxt.T0, cur.T0), idz2),
                                               x2::fgrad<LIM>(cur.gx0, nxt.gx0, i4x, ilx), x2::fgrad<LIM>(cur.gy0, nxt.gy0, i4y, ily),
                                               add2(cur.b0[2], nxt.b0[2]), add2(cur.b0[0], nxt.b0[0]),
                                               add2(cur.b0[1], nxt.b0[1]), fk, p);
        const float2 Fz1 = x2::face2s<SP, SAT, KP0>(cur.T1, nxt.T1, mul2(sub2(nxt.T1, cur.T1), idz2),
                                               x2::fgrad<LIM>(cur.gx1, nxt.gx1, i4x, ilx), x2::fgrad<LIM>(cur.gy1, nxt.gy1, i4y, ily),
                                               add2(cur.b1[2], nxt.b1[2]), add2(cur.b1[0], nxt.b1[0]),
                                               add2(cur.b1[1], nxt.b1[1]), fk, p);

        // the tile's bottom y-faces and left x-faces, by warps that rotate
        // over the schedulers from plane to plane (32-column tiles: one
        // warp, its lower half the y-faces, its upper half the x-faces)
        const int par = q & 1;
        const bool ydo = SEGS == 1 ? w == (q & 3) : (w == (q & 3) && rp == SEGS * w);
        const bool xdo = SEGS == 1 ? (w == ((q + 2) & 3) && lx < TY) : (w == (q & 3) && rp != SEGS * w);
        if (ydo) {
            *reinterpret_cast<float2*>(&sm.Fy[par][0][c]) =
                x2::low_yface2<SP, SAT, LIM>(sm, g, p, fk, tslot(q - 1), ts, tslot(q + 1), bs, c);
        } else if (xdo) {
            sm.FxLo[par][lx] = x2::low_xface<SP, SAT, LIM>(sm, g, p, fk, tslot(q - 1), ts, tslot(q + 1), bs, lx);
        }
        if (MODE == 2) {
            const float* Yp = sm.Y[yslot(q)][0];
            y00 = lds2(&Yp[ra * TX + c]);
            y01 = lds2(&Yp[rb * TX + c]);
            yj0 = lds2(&Yp[TY * TX + ra * TX + c]);
            yj1 = lds2(&Yp[TY * TX + rb * TX + c]);
            my0 = lds2(&Yp[2 * TY * TX + ra * TX + c]);
            my1 = lds2(&Yp[2 * TY * TX + rb * TX + c]);
        }
        *reinterpret_cast<float2*>(&sm.Fy[par][rp + 1][c]) = Fy1;
        const float fl0 = __shfl_up_sync(0xffffffffu, Fx0.y, 1, LPR);
        const float fl1 = __shfl_up_sync(0xffffffffu, Fx1.y, 1, LPR);
        const float2 Fxl0 = make_float2(lx == 0 ? 0.f : fl0, Fx0.x);
        const float2 Fxl1 = make_float2(lx == 0 ? 0.f : fl1, Fx1.x);
        pend0 = fma2(sub2(Fx0, Fxl0), cmx, fma2(Fy0, cmy, mul2(sub2(Fz0, Fzl0), cmz)));
        pend1 = fma2(sub2(Fx1, Fxl1), cmx, fma2(Fy1, cmy, mul2(sub2(Fz1, Fzl1), cmz)));
        pend1 = fma2(Fy0, bc2(-cmy.x), pend1);      // row 2w + 1's lower face is Fy0
        pcb = cbase;
        cbase += g.plane;
        Fzl0 = Fz0;
        Fzl1 = Fz1;
        Tm0 = cur.T0;
        Tm1 = cur.T1;
        Tmr0 = cur.r0;
        Tmr1 = cur.r1;
        TmU = cur.TU;
    };

    int q = 0;
    for (; q + 1 < nzc; q += 2) {
        step(q, B, A);
        step(q + 1, A, B);
    }
    if (q < nzc) step(q, B, A);
    cp_wait<0>();
    __syncthreads();
    finish(nzc - 1);
    if (MODE != 0) {
        const bool bad_nf = nfacc.x != 0.f || nfacc.y != 0.f;
        const bool bad_np = SP && !(mnacc > 0.f);
        if (bad_nf || bad_np) atomicOr(status, (bad_nf ? ST_NONFINITE : 0u) | (bad_np ? ST_NONPOSITIVE : 0u));
    }
    __syncthreads();
}

template <bool SP, bool SAT, int MODE, int TXW, bool KP0, bool LIM>
__global__ void __launch_bounds__(NTHREADS, kCtasPerSm)
stage_q_kernel(KGrid<float> g, KPhys<float> p, x2::FastArgs a, KCoef<float> cf, unsigned* status, int nzchunk)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemQ<TXW>& sm = *reinterpret_cast<SmemQ<TXW>*>(smem_raw);
    const int z0 = blockIdx.z * nzchunk;
    tile_q<SP, SAT, MODE, TXW, KP0, LIM>(sm, g, p, a, cf, status, blockIdx.x * SmemQ<TXW>::TX, blockIdx.y * SmemQ<TXW>::TY,
                               z0, min(nzchunk, g.n[2] - z0));
}

template <bool SP, bool SAT, int MODE, int TXW, bool KP0, bool LIM>
cudaError_t launch_q(const KGrid<float>& g, const KPhys<float>& p, const x2::FastArgs& a, const KCoef<float>& cf,
                     unsigned* status, int nzchunk, cudaStream_t st)
{
    using SM = SmemQ<TXW>;
    const int smem = (int)sizeof(SM);
    static bool attr_set = false;       // the attribute is per function, set once
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(stage_q_kernel<SP, SAT, MODE, TXW, KP0, LIM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((g.n[0] + SM::TX - 1) / SM::TX, (g.n[1] + SM::TY - 1) / SM::TY, (g.n[2] + nzchunk - 1) / nzchunk);
    stage_q_kernel<SP, SAT, MODE, TXW, KP0, LIM><<<grid, NTHREADS, smem, st>>>(g, p, a, cf, status, nzchunk);
    return cudaGetLastError();
}

template <bool SP, bool SAT, int TXW, bool KP0, bool LIM = false>
cudaError_t launch_q_mode(int mode, const KGrid<float>& g, const KPhys<float>& p, const x2::FastArgs& a,
                          const KCoef<float>& cf, unsigned* status, int nzchunk, cudaStream_t st)
{
    if (mode == 0) return launch_q<SP, SAT, 0, TXW, KP0, LIM>(g, p, a, cf, status, nzchunk, st);
    if (mode == 1) return launch_q<SP, SAT, 1, TXW, KP0, LIM>(g, p, a, cf, status, nzchunk, st);
    return launch_q<SP, SAT, 2, TXW, KP0, LIM>(g, p, a, cf, status, nzchunk, st);
}

// Launches of the builds compiled in rkl_xq_sat.cu (saturated flux; kp0:
// the kappa_perp = 0 form) and rkl_xq_lim.cu (MC limiter at every face,
// 64-column tiles).
cudaError_t launch_q_sat(bool sp, bool kp0, int txw, int mode, const KGrid<float>& g, const KPhys<float>& p,
                         const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                         cudaStream_t st);
cudaError_t launch_q_lim(bool sp, bool sat, int mode, const KGrid<float>& g, const KPhys<float>& p,
                         const x2::FastArgs& a, const KCoef<float>& cf, unsigned* status, int nzchunk,
                         cudaStream_t st);

}  // namespace xq
}  // namespace rkl
