// Two-stage paired-cell FP32 3D kernel: stages j and j + 1 of the RKL2
// recurrence (Eq. rkl2scheme) in one pass over the grid (temporal blocking).
//
// A CTA owns a 60 x 7 block of columns and marches it through a chunk of z
// planes.  Nine "A" warps evaluate stage j on the 64 x 9 region around the
// owned block (rows -1 .. 7, columns -2 .. 61 relative to it) from Y_{j-1},
// Y_{j-2}, Y_0, M(Y_0) and b streamed through shared memory, and keep each
// finished plane of Y_j in a shared-memory ring.  Seven "B" warps follow
// four planes behind and evaluate stage j + 1 on the owned rows from that
// ring.  Both stages write their owned cells (Y_j is the next pass's
// Y_{j-2}); per two stages the grid arrays cross HBM once, 36 bytes per cell
// instead of 2 x 32.  The price is the halo ring of stage j (64 x 9
// computed for 60 x 7 kept), the idle lanes of stage j + 1 (64 x 7 for
// 60 x 7) and the planes of the chunk's two z-halos.  16 warps keep the
// register budget at 128 per thread.
//
// Per pair of faces the arithmetic is the one of the single-stage kernel
// (packed f32x2, face2).  Periodic grids only, nx % 4 == 0.
#include <algorithm>

#include "rkl_launch.h"
#include "rkl_pair.cuh"

namespace rkl {
namespace x2t {

using namespace x2;

constexpr int TXC = 64;                  // computed columns per row (32 lanes x 2)
constexpr int OX = 60;                   // owned columns, tile stride in x
constexpr int OY = 7;                    // owned rows, tile stride in y (= B rows)
constexpr int RA = OY + 2;               // A rows -1 .. OY
constexpr int RT = OY + 4;               // loaded Y_{j-1} / b rows -2 .. OY + 1
constexpr int SX = 72;                   // Y_{j-1}, b, Y_j rows: columns -4 .. 67 of the owned block
constexpr int SY = 68;                   // Y0 / Y_{j-2} / M(Y0) rows: columns -4 .. 63
constexpr int WA = RA, WB = OY, NW = WA + WB, NTH = 32 * NW;    // 512 threads
// ring slots: Y_{j-1}, b and the Y arrays span planes t-5 .. t+2 of iteration
// t (B warps read plane t-4, A warps t-2 .. t, planes t+1, t+2 in flight);
// the Y_j ring holds B's planes t-5 .. t-3 and the one A finishes
constexpr int NT = 8, NB = 8, NYR = 8, NJ = 4;     // powers of two: slots are masks
constexpr int PLT = RT * SX;
constexpr int PLY = RA * SY;
constexpr int PLJ = RA * SX;

struct Smem {
    float T[NT][PLT];
    float B[NB][3][PLT];
    float Y[NYR][3][PLY];
    float J[NJ][PLJ];
    float Fy[2][2][RA + 1][TXC];         // [stage][parity][face row][column]
    float Fx[2][RA];                     // A's left-boundary x-faces [parity][row + 1]
};

struct Args {
    const float* Tin;       // Y_{j-1}
    const float* b;         // [3][ncell]
    const float* Y0;
    const float* Yjm2;
    const float* MY0;
    float* outA;            // Y_j
    float* outB;            // Y_{j+1}
    const float* coef_tab;  // stage coefficients at coef_tab[4 j]
    int j;
};

// copy tasks: Y_{j-1} and b (4 arrays x RT rows x 18 chunks), Y0, Y_{j-2},
// M(Y0) (3 arrays x RA rows x 17 chunks); every chunk wraps (periodic)
constexpr int kTB = 4 * RT * (SX / 4);
constexpr int kYT = 3 * RA * (SY / 4);
constexpr int kSlots = (kTB + kYT + NTH - 1) / NTH;    // 3 (1251 tasks)
enum : unsigned { RING_T = 0, RING_B = 1, RING_Y = 2, RING_NONE = 3 };
struct Task {
    const float* src;       // chunk address in plane 0
    unsigned dst;           // smem byte address in slot 0
    unsigned ring;
};

__device__ __forceinline__ int pmodi(int v, int n) { return pmod(v, n); }

__device__ __forceinline__ Task make_task(const Smem& sm, const KGrid<float>& g, const Args& a, int t, int i0,
                                          int j0)
{
    Task k{nullptr, 0u, RING_NONE};
    const int nx = g.n[0], ny = g.n[1];
    if (t < kTB) {
        const int arr = t / (RT * (SX / 4)), rr = t % (RT * (SX / 4));
        const int row = rr / (SX / 4) - 2, ch = rr % (SX / 4);
        const int64_t o = (int64_t)pmodi(j0 + row, ny) * nx + pmodi(i0 - 4 + 4 * ch, nx);
        if (arr == 0) {
            k.src = a.Tin + o;
            k.dst = smem_u32(&sm.T[0][(row + 2) * SX + 4 * ch]);
            k.ring = RING_T;
        } else {
            k.src = a.b + (int64_t)(arr - 1) * g.ncell + o;
            k.dst = smem_u32(&sm.B[0][arr - 1][(row + 2) * SX + 4 * ch]);
            k.ring = RING_B;
        }
        return k;
    }
    t -= kTB;
    if (t >= kYT) return k;
    const int arr = t / (RA * (SY / 4)), rr = t % (RA * (SY / 4));
    const int row = rr / (SY / 4) - 1, ch = rr % (SY / 4);
    const int64_t o = (int64_t)pmodi(j0 + row, ny) * nx + pmodi(i0 - 4 + 4 * ch, nx);
    k.src = (arr == 0 ? a.Y0 : (arr == 1 ? a.Yjm2 : a.MY0)) + o;
    k.dst = smem_u32(&sm.Y[0][arr][(row + 1) * SY + 4 * ch]);
    k.ring = RING_Y;
    return k;
}

// Quantities of a cell pair carried from plane to plane (as in the
// single-stage kernel): T of the pair, of column c+2 and one row up, the
// pair's centred x/y differences and b.
struct QZ {
    float2 To;
    float Tr;
    float2 TU;
    float2 gxo, gyo;
    float2 bo[3];
};
struct QXY {
    float2 gyR, gxU;
    float bR[3];
    float2 bU[3];
};

// A plane view: element (r, c) at p[r * SX + c] (p points at row 0, column 0
// of the computed region).
__device__ __forceinline__ float2 at2(const float* p, int r, int c) { return lds2(p + r * SX + c); }
__device__ __forceinline__ float at1(const float* p, int r, int c) { return p[r * SX + c]; }

__device__ __forceinline__ QZ read_qz(const float* T, const float* const B[3], int c, int r)
{
    QZ q;
    const float2 Tc = at2(T, r, c), Tl = at2(T, r, c - 2), Trr = at2(T, r, c + 2);
    const float2 Tu = at2(T, r + 1, c), Td = at2(T, r - 1, c);
    q.To = Tc;
    q.Tr = Trr.x;
    q.TU = Tu;
    q.gxo = sub2(make_float2(Tc.y, Trr.x), make_float2(Tl.y, Tc.x));
    q.gyo = sub2(Tu, Td);
#pragma unroll
    for (int e = 0; e < 3; ++e) q.bo[e] = at2(B[e], r, c);
    return q;
}

__device__ __forceinline__ QXY read_qxy(const float* T, const float* const B[3], int c, int r, const QZ& z)
{
    QXY q;
    const float2 Td = at2(T, r - 1, c), Tur = at2(T, r + 1, c + 2), Tdr = at2(T, r - 1, c + 2);
    const float2 Tul = at2(T, r + 1, c - 2);
    q.gyR = sub2(make_float2(z.TU.y, Tur.x), make_float2(Td.y, Tdr.x));
    q.gxU = sub2(make_float2(z.TU.y, Tur.x), make_float2(Tul.y, z.TU.x));
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        q.bR[e] = at1(B[e], r, c + 2);
        q.bU[e] = at2(B[e], r + 1, c);
    }
    return q;
}

// y-face pair between rows rl-1 and rl at columns (c, c+1)
template <bool SP, bool SAT>
__device__ __forceinline__ float2 low_yface2(const float* Tm, const float* Tc, const float* Tp, const float* const B[3],
                                             const KGrid<float>& g, const KPhys<float>& p, int rl, int c)
{
    const float2 TL = at2(Tc, rl - 1, c), TR = at2(Tc, rl, c);
    const float2 Ll = at2(Tc, rl - 1, c - 2), Lr = at2(Tc, rl - 1, c + 2);
    const float2 Rl = at2(Tc, rl, c - 2), Rr = at2(Tc, rl, c + 2);
    const float2 gxL = sub2(make_float2(TL.y, Lr.x), make_float2(Ll.y, TL.x));
    const float2 gxR = sub2(make_float2(TR.y, Rr.x), make_float2(Rl.y, TR.x));
    const float2 gzL = sub2(at2(Tp, rl - 1, c), at2(Tm, rl - 1, c));
    const float2 gzR = sub2(at2(Tp, rl, c), at2(Tm, rl, c));
    float2 b[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) b[e] = mul2(bc2(0.5f), add2(at2(B[e], rl - 1, c), at2(B[e], rl, c)));
    return face2<SP, SAT>(TL, TR, mul2(sub2(TR, TL), bc2(g.inv_dx[1])), mul2(add2(gxL, gxR), bc2(g.inv_4dx[0])),
                          mul2(add2(gzL, gzR), bc2(g.inv_4dx[2])), b[1], b[0], b[2], p);
}

// x-face between columns -1 and 0 at row r
template <bool SP, bool SAT>
__device__ __forceinline__ float low_xface(const float* Tm, const float* Tc, const float* Tp, const float* const B[3],
                                           const KGrid<float>& g, const KPhys<float>& p, int r)
{
    const float TL = at1(Tc, r, -1), TR = at1(Tc, r, 0);
    const float gyL = at1(Tc, r + 1, -1) - at1(Tc, r - 1, -1);
    const float gyR = at1(Tc, r + 1, 0) - at1(Tc, r - 1, 0);
    const float gzL = at1(Tp, r, -1) - at1(Tm, r, -1);
    const float gzR = at1(Tp, r, 0) - at1(Tm, r, 0);
    float b[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) b[e] = 0.5f * (at1(B[e], r, -1) + at1(B[e], r, 0));
    return face_flux<float, SP, SAT>(TL, TR, (TR - TL) * g.inv_dx[0], (gyL + gyR) * g.inv_4dx[1],
                                     (gzL + gzR) * g.inv_4dx[2], b[0], b[1], b[2], p);
}

// Per-warp state of one stage's z-march (the two carried planes live in
// the caller, which swaps their roles from one iteration to the next).
struct March {
    float2 Fz_lo, TmO, TmU;
    float TmR;
    float2 pend, pTo, py0, pyjm2, pmy0;
    float2 nfacc;
    float mnacc;
};

}  // namespace x2t

namespace {

using namespace x2t;

// One tile: owned columns [i0, i0 + 60), rows [j0, j0 + 7), planes [z0, z0 + nzc).
template <bool SP, bool SAT>
__device__ __forceinline__ void tile_x2t(Smem& sm, const KGrid<float>& g, const KPhys<float>& p, const Args& a,
                                         unsigned* status, int i0, int j0, int z0, int nzc)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const bool roleA = warp < WA;
    const int r = roleA ? warp - 1 : warp - WA;      // A rows -1 .. OY, B rows 0 .. OY - 1
    const int c = 2 * lane;                           // pair (c, c+1), columns i0 - 2 + c
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int st = roleA ? 0 : 1;                     // Fy stage index

    KCoef<float> cf;
    {
        const float* t = a.coef_tab + 4 * (a.j + (roleA ? 0 : 1));
        cf.mu = t[0]; cf.nu = t[1]; cf.mt = t[2]; cf.gt = t[3];
    }
    float* const out = roleA ? a.outA : a.outB;
    // owned pair: rows 0 .. OY - 1, lanes 1 .. 30, inside the grid (nx % 4 == 0:
    // both cells of a pair or neither)
    const bool own_xy = r >= 0 && r < OY && lane >= 1 && lane <= 30 && j0 + r < ny && i0 - 2 + c < nx;

    Task tk[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) tk[s] = make_task(sm, g, a, tid + s * NTH, i0, j0);

    auto ring = [](int q, int n) { return q & (n - 1); };          // n a power of two
    auto load = [&](int q, bool withY) {
        const int64_t zo = (int64_t)pmod(z0 + q, nz) * g.plane;
        const unsigned ts = (unsigned)(ring(q, NT) * PLT * 4);
        const unsigned bs = (unsigned)(ring(q, NB) * 3 * PLT * 4);
        const unsigned ys = (unsigned)(ring(q, NYR) * 3 * PLY * 4);
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const unsigned rg = tk[s].ring;
            const unsigned off = rg == RING_T ? ts : (rg == RING_B ? bs : ys);
            if (rg < RING_Y || (rg == RING_Y && withY)) cp16(tk[s].dst + off, tk[s].src + zo);
        }
    };
    // plane views (row 0, column 0 of the computed region)
    auto Tv = [&](int q) -> const float* { return &sm.T[ring(q, NT)][2 * SX + 2]; };
    auto Jv = [&](int q) -> const float* { return &sm.J[ring(q, NJ)][1 * SX + 2]; };
    auto Bv = [&](int q, const float* (&B)[3]) {
#pragma unroll
        for (int e = 0; e < 3; ++e) B[e] = &sm.B[ring(q, NB)][e][2 * SX + 2];
    };
    auto Yv = [&](int q, int arr) -> const float* { return &sm.Y[ring(q, NYR)][arr][1 * SY + 2]; };

    const float2 idx2 = bc2(g.inv_dx[0]), idy2 = bc2(g.inv_dx[1]), idz2 = bc2(g.inv_dx[2]);
    const float2 i4x = bc2(g.inv_4dx[0]), i4y = bc2(g.inv_4dx[1]), i4z = bc2(g.inv_4dx[2]);
    const float2 half = bc2(0.5f);

    March m;
    m.nfacc = bc2(0.f);
    m.mnacc = INFINITY;
    m.pend = m.pTo = m.py0 = m.pyjm2 = m.pmy0 = bc2(0.f);

    // the +z face between two carried planes
    auto zface = [&](const QZ& lo, const QZ& hi) {
        return face2<SP, SAT>(lo.To, hi.To, mul2(sub2(hi.To, lo.To), idz2), mul2(add2(lo.gxo, hi.gxo), i4x),
                              mul2(add2(lo.gyo, hi.gyo), i4y), mul2(half, add2(lo.bo[2], hi.bo[2])),
                              mul2(half, add2(lo.bo[0], hi.bo[0])), mul2(half, add2(lo.bo[1], hi.bo[1])), p);
    };
    // carried planes qlo (into lo) and qlo + 1 (into hi) and the z-face between them
    auto start = [&](const float* Tlo, const float* Thi, int qlo, QZ& lo, QZ& hi) {
        const float* Blo[3];
        const float* Bhi[3];
        Bv(qlo, Blo);
        Bv(qlo + 1, Bhi);
        lo = read_qz(Tlo, Blo, c, r);
        hi = read_qz(Thi, Bhi, c, r);
        m.Fz_lo = zface(lo, hi);
        m.TmO = lo.To;
        m.TmU = lo.TU;
        m.TmR = lo.Tr;
    };

    // faces of plane q with cur holding plane q; nxt receives plane q + 1.
    // Tm/Tc/Tn: views of planes q-1, q, q+1; the y-faces below row rl (the
    // stage's lowest row) and, for stage A, the x-faces left of column 0
    // come from one warp each.
    auto faces = [&](int q, QZ& cur, QZ& nxt, const float* Tm, const float* Tc, const float* Tn, int rl) {
        const float* Bc[3];
        const float* Bn[3];
        Bv(q, Bc);
        Bv(q + 1, Bn);
        const float2 TmRp = make_float2(m.TmO.y, m.TmR);
        const QXY cx = read_qxy(Tc, Bc, c, r, cur);
        nxt = read_qz(Tn, Bn, c, r);
        const float2 gzo = sub2(nxt.To, m.TmO);
        const float2 gzR = sub2(make_float2(nxt.To.y, nxt.Tr), TmRp);
        const float2 gzU = sub2(nxt.TU, m.TmU);
        const float2 TR = make_float2(cur.To.y, cur.Tr);
        const float2 Fx = face2<SP, SAT>(
            cur.To, TR, mul2(sub2(TR, cur.To), idx2), mul2(add2(cur.gyo, cx.gyR), i4y), mul2(add2(gzo, gzR), i4z),
            mul2(half, add2(cur.bo[0], make_float2(cur.bo[0].y, cx.bR[0]))),
            mul2(half, add2(cur.bo[1], make_float2(cur.bo[1].y, cx.bR[1]))),
            mul2(half, add2(cur.bo[2], make_float2(cur.bo[2].y, cx.bR[2]))), p);
        const float2 Fy = face2<SP, SAT>(cur.To, cur.TU, mul2(sub2(cur.TU, cur.To), idy2),
                                         mul2(add2(cur.gxo, cx.gxU), i4x), mul2(add2(gzo, gzU), i4z),
                                         mul2(half, add2(cur.bo[1], cx.bU[1])), mul2(half, add2(cur.bo[0], cx.bU[0])),
                                         mul2(half, add2(cur.bo[2], cx.bU[2])), p);
        const float2 Fz = zface(cur, nxt);
        const int par = (q + 2) & 1;
        const int wbase = roleA ? 0 : WA, nwr = roleA ? WA : WB;
        const int w = warp - wbase;
        if (w == (q + 2) % nwr) {
            *reinterpret_cast<float2*>(&sm.Fy[st][par][0][c]) = low_yface2<SP, SAT>(Tm, Tc, Tn, Bc, g, p, rl, c);
        } else if (roleA && w == (q + 2 + WA / 2) % nwr && lane < RA) {
            sm.Fx[par][lane] = low_xface<SP, SAT>(Tm, Tc, Tn, Bc, g, p, lane - 1);
        }
        *reinterpret_cast<float2*>(&sm.Fy[st][par][r - rl + 1][c]) = Fy;
        const float fxl = __shfl_up_sync(0xffffffffu, Fx.y, 1);
        const float2 Fx_lo = make_float2(lane == 0 ? 0.f : fxl, Fx.x);
        m.pend = fma2(sub2(Fx, Fx_lo), idx2, fma2(Fy, idy2, mul2(sub2(Fz, m.Fz_lo), idz2)));
        m.pTo = cur.To;
        m.Fz_lo = Fz;
        m.TmO = cur.To;
        m.TmR = cur.Tr;
        m.TmU = cur.TU;
    };

    // divergence and recurrence of the pending plane q
    auto finish = [&](int q, int rl) -> float2 {
        const int par = (q + 2) & 1;
        float2 div = sub2(m.pend, mul2(lds2(&sm.Fy[st][par][r - rl][c]), idy2));
        if (roleA && lane == 0) div.x -= sm.Fx[par][r + 1] * g.inv_dx[0];
        const float2 M = mul2(bc2(-1.f), div);
        const float2 inc = fma2(bc2(cf.mu), sub2(m.pTo, m.py0),
                                fma2(bc2(cf.nu), sub2(m.pyjm2, m.py0), fma2(bc2(cf.mt), M, mul2(bc2(cf.gt), m.pmy0))));
        const float2 y = add2(m.py0, inc);
        if (own_xy && q >= 0 && q < nzc) {
            *reinterpret_cast<float2*>(out + (((int64_t)(z0 + q) * ny + (j0 + r)) * nx + (i0 - 2 + c))) = y;
            m.nfacc = add2(m.nfacc, sub2(y, y));
            if (SP) m.mnacc = fminf(m.mnacc, fminf(y.x, y.y));
        }
        return y;
    };

    // The loop body, for one iteration t with (cur, nxt) roles of the carried planes.
    auto iter = [&](int t, QZ& cur, QZ& nxt) {
        cp_wait<1>();                       // bundle t has landed
        __syncthreads();
        if (t + 2 <= nzc + 1) load(t + 2, t + 2 <= nzc);
        cp_commit();
        if (roleA) {
            if (t >= 1 && t <= nzc + 2) {
                const float2 y = finish(t - 2, -1);
                *reinterpret_cast<float2*>(&sm.J[ring(t - 2, NJ)][(r + 1) * SX + c + 2]) = y;
            }
            if (t <= nzc + 1) {
                const int q = t - 1;
                m.py0 = lds2(Yv(q, 0) + r * SY + c);
                m.pyjm2 = lds2(Yv(q, 1) + r * SY + c);
                m.pmy0 = lds2(Yv(q, 2) + r * SY + c);
                faces(q, cur, nxt, Tv(q - 1), Tv(q), Tv(q + 1), -1);
            }
        } else {
            if (t >= 5) finish(t - 5, 0);
            if (t == 3) {
                start(Jv(-1), Jv(0), -1, cur, nxt);
            } else if (t >= 4) {
                const int q = t - 4;
                // Y_{j-1} at the cell (the stage's Y_{j-2}) from the Y_{j-1} ring
                m.py0 = lds2(Yv(q, 0) + r * SY + c);
                m.pyjm2 = lds2(Tv(q) + r * SX + c);
                m.pmy0 = lds2(Yv(q, 2) + r * SY + c);
                faces(q, cur, nxt, Jv(q - 1), Jv(q), Jv(q + 1), 0);
            }
        }
    };

    // planes -2 .. 1 in flight; -2 and -1 must land before stage A starts
#pragma unroll
    for (int k = -2; k <= 1; ++k) {
        if (k <= nzc + 1) load(k, k >= -1 && k <= nzc);
        cp_commit();
    }
    cp_wait<2>();
    __syncthreads();
    QZ qa, qb;
    if (roleA) start(Tv(-2), Tv(-1), -2, qa, qb);
    const int tend = nzc + 3;
    for (int t = 0; t <= tend; t += 2) {
        iter(t, qb, qa);
        if (t + 1 <= tend) iter(t + 1, qa, qb);
    }
    cp_wait<0>();
    __syncthreads();
    if (!roleA) finish(nzc - 1, 0);
    const bool bad_nf = m.nfacc.x != 0.f || m.nfacc.y != 0.f;
    const bool bad_np = SP && !(m.mnacc > 0.f);
    if (bad_nf || bad_np) atomicOr(status, (bad_nf ? ST_NONFINITE : 0u) | (bad_np ? ST_NONPOSITIVE : 0u));
    __syncthreads();
}

template <bool SP, bool SAT>
__global__ void __launch_bounds__(x2t::NTH, 1)
stage_pair_kernel(KGrid<float> g, KPhys<float> p, x2t::Args a, unsigned* status, int nzchunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    x2t::Smem& sm = *reinterpret_cast<x2t::Smem*>(smem_raw);
    // columns the A warps never write (the Y_j ring's outer columns) stay 0
    for (int i = threadIdx.x; i < x2t::NJ * x2t::PLJ; i += blockDim.x) (&sm.J[0][0])[i] = 0.f;
    __syncthreads();
    const int z0 = blockIdx.z * nzchunk;
    tile_x2t<SP, SAT>(sm, g, p, a, status, blockIdx.x * x2t::OX, blockIdx.y * x2t::OY, z0,
                      min(nzchunk, g.n[2] - z0));
}

template <bool SP, bool SAT>
cudaError_t launch_pair_t(const KGrid<float>& g, const KPhys<float>& p, const x2t::Args& a, unsigned* status,
                          int nzchunk, cudaStream_t st)
{
    const int smem = (int)sizeof(x2t::Smem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(stage_pair_kernel<SP, SAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((g.n[0] + x2t::OX - 1) / x2t::OX, (g.n[1] + x2t::OY - 1) / x2t::OY, (g.n[2] + nzchunk - 1) / nzchunk);
    stage_pair_kernel<SP, SAT><<<grid, x2t::NTH, smem, st>>>(g, p, a, status, nzchunk);
    return cudaGetLastError();
}

}  // namespace

bool pair_stage_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return c.dtype == 0 && c.ndim == 3 && !c.limiter && g.bc == 0 && (g.n[0] % 4) == 0;
}

cudaError_t launch_stage_pair(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p, const StageIO& io,
                              void* Yj1, unsigned* status, int nzchunk, cudaStream_t st)
{
    x2t::Args a;
    a.Tin = static_cast<const float*>(io.Yjm1);
    a.b = static_cast<const float*>(io.b);
    a.Y0 = static_cast<const float*>(io.Y0);
    a.Yjm2 = static_cast<const float*>(io.Yjm2);
    a.MY0 = static_cast<const float*>(io.MY0);
    a.outA = static_cast<float*>(io.Yj);
    a.outB = static_cast<float*>(Yj1);
    a.coef_tab = static_cast<const float*>(io.coef_tab);
    a.j = io.j;
    if (nzchunk < 1) nzchunk = 32;
    if (c.spitzer) {
        if (c.saturate) return launch_pair_t<true, true>(g, p, a, status, nzchunk, st);
        return launch_pair_t<true, false>(g, p, a, status, nzchunk, st);
    }
    if (c.saturate) return launch_pair_t<false, true>(g, p, a, status, nzchunk, st);
    return launch_pair_t<false, false>(g, p, a, status, nzchunk, st);
}

}  // namespace rkl
