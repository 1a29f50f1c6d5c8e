// Tiled FP32 3D stage kernel for the RKL2 conduction super-step.
//
// Each CTA owns a TX x TY column of cells in xy and marches through a chunk
// of NZC planes in z.  A three-deep cp.async pipeline stages plane bundles
// into shared memory: T = Y_{j-1} and the three b planes with a one-cell
// halo ring (periodic wrap or Dirichlet ghost applied at load time), and the
// pointwise registers Y_0, Y_{j-2}, M(Y_0).  Every face flux is evaluated
// exactly once: each thread computes the +x, +y and +z faces of its cell
// from per-cell quantities carried in registers along z (T, the centred
// transverse differences and b of its own, +x and +y neighbours); two warps
// add the faces on the tile's low x and y boundary.  The +x/+y fluxes are
// exchanged through shared memory for the divergence, the -z flux is the
// previous plane's +z flux, and the RKL2 recurrence is applied in registers
// before the single coalesced store of Y_j.
#include "rkl_launch.h"

namespace rkl {
namespace {

constexpr int TX = 32;                 // tile width (x), one warp per row
constexpr int TY = 8;                  // tile height (y), one row per warp
constexpr int NTHREADS = TX * TY;
constexpr int SXS = 40;                // smem row stride: halo at 3, interior 4..35, halo at 36
constexpr int ROWS = TY + 2;
constexpr int PLANE = ROWS * SXS;
constexpr int NZC = 32;                // planes per CTA

__device__ __forceinline__ int off(int iy, int ix) { return (iy + 1) * SXS + ix + 4; }

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ int pmod(int v, int n)
{
    int r = v % n;
    return r < 0 ? r + n : r;
}

struct FastArgs {
    const float* Tin;      // field whose M is taken (Y_{j-1}, or Y_0 at stage 1)
    const float* b;        // [3][ncell]
    const float* Y0;
    const float* Yjm2;
    const float* MY0in;
    float* MY0out;         // stage 1 only
    float* out;            // Y_j, or M(T) in mode 0
    const float* coef_tab; // if non-null: stage coefficients at coef_tab[4 j]
    int j;
};

struct Smem {
    float T[4][PLANE];
    float B[3][3][PLANE];
    float Y[3][3][NTHREADS];
    float Fx[2][TY][TX + 1];
    float Fy[2][TY + 1][TX];
};

// Plane bookkeeping of one bundle: element offsets of the T plane and of
// the b plane (they differ only for Dirichlet ghost planes, where T is the
// ghost value and b copies the nearest interior plane).
struct PlaneOff {
    int64_t t, b;
    bool zghost;
};

__device__ __forceinline__ PlaneOff plane_offsets(const KGrid<float>& g, int kk)
{
    const int nz = g.n[2];
    PlaneOff o{0, 0, false};
    int kz = kk, kzb = kk;
    if (kk < 0 || kk >= nz) {
        if (g.bc == 1) {
            o.zghost = true;
            kz = kzb = kk < 0 ? 0 : nz - 1;
        } else {
            kz = kzb = pmod(kk, nz);
        }
    }
    o.t = (int64_t)kz * g.plane;
    o.b = (int64_t)kzb * g.plane;
    return o;
}

// Copy tasks of the full-tile path, fixed per thread for the whole z-march.
// A bundle is 4 arrays (T, bx, by, bz) x (10 rows x 8 chunks of 16 B + 20
// halo cells of 4 B) = 400 tasks, plus 3 x 64 chunks of Y0, Y_{j-2}, M(Y0).
// Thread t owns T/b tasks t and t + 256 and Y task t (t < 192).
enum : unsigned { TK_VALID = 1u, TK_CHUNK = 2u, TK_T = 4u, TK_GHOST = 8u, TK_BCAST = 16u };
struct Task {
    const float* src;   // element address in plane 0 (the bundle's plane offset is added)
    unsigned dst;       // shared-memory byte address in slot 0
    unsigned flags;
};

__device__ __forceinline__ Task make_tb_task(const Smem& sm, const KGrid<float>& g, const FastArgs& a, int t,
                                             int i0, int j0)
{
    Task k{nullptr, 0u, 0u};
    if (t >= 400) return k;
    const int nx = g.n[0], ny = g.n[1];
    const bool dir = g.bc == 1;
    int arr = t / 100, r = t % 100;
    int iy, ix;
    bool chunk = r < 80;
    if (chunk) { iy = r / 8 - 1; ix = (r % 8) * 4; }
    else { r -= 80; iy = r / 2 - 1; ix = (r & 1) ? TX : -1; }
    int gy = j0 + iy, gx = i0 + ix;
    bool ghost = false;
    if (gy < 0 || gy >= ny) {
        if (dir) { ghost = true; gy = gy < 0 ? 0 : ny - 1; } else gy = pmod(gy, ny);
    }
    bool xghost = false;
    if (gx < 0 || gx >= nx) {
        if (dir) { ghost = xghost = true; gx = gx < 0 ? 0 : nx - 1; } else gx = pmod(gx, nx);
    }
    const int64_t row = (int64_t)gy * nx + gx;
    k.flags = TK_VALID | (chunk ? TK_CHUNK : 0u);
    if (arr == 0) {
        k.flags |= TK_T | (ghost ? TK_GHOST : 0u);
        k.src = a.Tin + row;
        k.dst = smem_u32(&sm.T[0][off(iy, ix)]);
    } else {
        // Dirichlet: b past the x edge repeats the nearest interior cell
        k.flags |= xghost ? TK_BCAST : 0u;
        k.src = a.b + (int64_t)(arr - 1) * g.ncell + row;
        k.dst = smem_u32(&sm.B[0][arr - 1][off(iy, ix)]);
    }
    return k;
}

template <int MODE>
__device__ __forceinline__ Task make_y_task(const Smem& sm, const KGrid<float>& g, const FastArgs& a, int t,
                                            int i0, int j0)
{
    Task k{nullptr, 0u, 0u};
    if (MODE != 2 || t >= 192) return k;
    int arr = t / 64, r = t % 64;
    int iy = r / 8, ix = (r % 8) * 4;
    // a 16-byte chunk lies wholly inside or wholly outside the grid (nx % 4 == 0)
    if (j0 + iy >= g.n[1] || i0 + ix >= g.n[0]) return k;
    const float* base = arr == 0 ? a.Y0 : (arr == 1 ? a.Yjm2 : a.MY0in);
    k.src = base + (int64_t)(j0 + iy) * g.n[0] + i0 + ix;
    k.dst = smem_u32(&sm.Y[0][arr][iy * TX + ix]);
    k.flags = TK_VALID | TK_CHUNK;
    return k;
}

__device__ __forceinline__ void st_shared(unsigned d, float v) { asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(d), "f"(v)); }
__device__ __forceinline__ void st_shared4(unsigned d, float v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};\n" ::"r"(d), "f"(v));
}
__device__ __forceinline__ void cp16a(unsigned d, const void* s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(s));
}
__device__ __forceinline__ void cp4a(unsigned d, const void* s)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(s));
}

__device__ __forceinline__ void issue_tb(const Task& k, const PlaneOff& po, unsigned tslot_bytes,
                                         unsigned bslot_bytes, float bcv)
{
    if (!(k.flags & TK_VALID)) return;
    const bool isT = k.flags & TK_T;
    const unsigned d = k.dst + (isT ? tslot_bytes : bslot_bytes);
    if (isT && (po.zghost || (k.flags & TK_GHOST))) {
        if (k.flags & TK_CHUNK) st_shared4(d, bcv); else st_shared(d, bcv);
        return;
    }
    const float* s = k.src + (isT ? po.t : po.b);
    if (k.flags & TK_BCAST) {
        const float v = __ldcg(s);
        if (k.flags & TK_CHUNK) st_shared4(d, v); else st_shared(d, v);
        return;
    }
    if (k.flags & TK_CHUNK) cp16a(d, s); else cp4a(d, s);
}

__device__ __forceinline__ void issue_y(const Task& k, int64_t poff, unsigned yslot_bytes)
{
    if (k.flags & TK_VALID) cp16a(k.dst + yslot_bytes, k.src + poff);
}

// Rows not 16-byte aligned (nx % 4 != 0):
// stage the bundle of plane kk element by element with wrap / ghost per element.
template <int MODE>
__device__ __forceinline__ void load_bundle_ragged(Smem& sm, const KGrid<float>& g, const FastArgs& a, int kk,
                                                   int tslot, int bslot, int yslot, bool withY, int i0, int j0)
{
    const int nx = g.n[0], ny = g.n[1];
    const int tid = threadIdx.x;
    const bool dir = g.bc == 1;
    const PlaneOff po = plane_offsets(g, kk);
    float* dT = sm.T[tslot];
    for (int t = tid; t < 4 * ROWS * (TX + 2); t += NTHREADS) {
        int arr = t / (ROWS * (TX + 2)), r = t % (ROWS * (TX + 2));
        int iy = r / (TX + 2) - 1, ix = r % (TX + 2) - 1;
        float* dst = arr == 0 ? dT : sm.B[bslot][arr - 1];
        const float* base = arr == 0 ? a.Tin : a.b + (int64_t)(arr - 1) * g.ncell;
        int gy = j0 + iy, gx = i0 + ix;
        bool ghost = po.zghost;
        if (gy < 0 || gy >= ny) {
            if (dir) { ghost = true; gy = gy < 0 ? 0 : ny - 1; } else gy = pmod(gy, ny);
        }
        if (gx < 0 || gx >= nx) {
            if (dir) { ghost = true; gx = gx < 0 ? 0 : nx - 1; } else gx = pmod(gx, nx);
        }
        float* d = dst + off(iy, ix);
        if (arr == 0) {
            if (ghost) { *d = g.bcv; continue; }
            cp4(d, base + po.t + (int64_t)gy * nx + gx);
        } else {
            cp4(d, base + po.b + (int64_t)gy * nx + gx);
        }
    }
    if (withY && MODE == 2) {
        for (int t = tid; t < 3 * NTHREADS; t += NTHREADS) {
            int arr = t / NTHREADS, r = t % NTHREADS;
            int iy = r / TX, ix = r % TX;
            int gy = j0 + iy, gx = i0 + ix;
            float* d = &sm.Y[yslot][arr][r];
            if (gy >= ny || gx >= nx) { *d = 0.f; continue; }
            const float* base = arr == 0 ? a.Y0 : (arr == 1 ? a.Yjm2 : a.MY0in);
            cp4(d, base + po.t + (int64_t)gy * nx + gx);
        }
    }
}

// Per-cell quantities of one plane for this thread's cell (own), its +x
// neighbour (R) and +y neighbour (U).  gx/gy are unscaled centred
// differences T(+1) - T(-1).
struct PlaneQ {
    float To, TR, TU;
    float gxo, gyo, gyR, gxU;
    float bo[3], bR[3], bU[3];
};

__device__ __forceinline__ PlaneQ read_plane(const Smem& sm, int tslot, int bslot, int ix, int iy)
{
    const float* T = sm.T[tslot];
    PlaneQ q;
    q.To = T[off(iy, ix)];
    q.TR = T[off(iy, ix + 1)];
    q.TU = T[off(iy + 1, ix)];
    float TRU = T[off(iy + 1, ix + 1)];
    q.gxo = q.TR - T[off(iy, ix - 1)];
    q.gyo = q.TU - T[off(iy - 1, ix)];
    q.gyR = TRU - T[off(iy - 1, ix + 1)];
    q.gxU = TRU - T[off(iy + 1, ix - 1)];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const float* B = sm.B[bslot][e];
        q.bo[e] = B[off(iy, ix)];
        q.bR[e] = B[off(iy, ix + 1)];
        q.bU[e] = B[off(iy + 1, ix)];
    }
    return q;
}

// x-face between local cells (ix, iy) and (ix + 1, iy) straight from smem
// (used for the tile's low-x boundary faces).
template <bool SP, bool SAT>
__device__ __forceinline__ float face_x_smem(const Smem& sm, const KGrid<float>& g, const KPhys<float>& p,
                                             int tm, int tc, int tp, int bc, int ix, int iy)
{
    const float* T = sm.T[tc];
    float TL = T[off(iy, ix)], TR = T[off(iy, ix + 1)];
    float gyL = T[off(iy + 1, ix)] - T[off(iy - 1, ix)];
    float gyR = T[off(iy + 1, ix + 1)] - T[off(iy - 1, ix + 1)];
    float gzL = sm.T[tp][off(iy, ix)] - sm.T[tm][off(iy, ix)];
    float gzR = sm.T[tp][off(iy, ix + 1)] - sm.T[tm][off(iy, ix + 1)];
    const float* Bx = sm.B[bc][0];
    const float* By = sm.B[bc][1];
    const float* Bz = sm.B[bc][2];
    return face_flux<float, SP, SAT>(TL, TR, (TR - TL) * g.inv_dx[0], (gyL + gyR) * g.inv_4dx[1],
                                     (gzL + gzR) * g.inv_4dx[2], 0.5f * (Bx[off(iy, ix)] + Bx[off(iy, ix + 1)]),
                                     0.5f * (By[off(iy, ix)] + By[off(iy, ix + 1)]),
                                     0.5f * (Bz[off(iy, ix)] + Bz[off(iy, ix + 1)]), p);
}

// y-face between local cells (ix, iy) and (ix, iy + 1) straight from smem.
template <bool SP, bool SAT>
__device__ __forceinline__ float face_y_smem(const Smem& sm, const KGrid<float>& g, const KPhys<float>& p,
                                             int tm, int tc, int tp, int bc, int ix, int iy)
{
    const float* T = sm.T[tc];
    float TL = T[off(iy, ix)], TR = T[off(iy + 1, ix)];
    float gxL = T[off(iy, ix + 1)] - T[off(iy, ix - 1)];
    float gxR = T[off(iy + 1, ix + 1)] - T[off(iy + 1, ix - 1)];
    float gzL = sm.T[tp][off(iy, ix)] - sm.T[tm][off(iy, ix)];
    float gzR = sm.T[tp][off(iy + 1, ix)] - sm.T[tm][off(iy + 1, ix)];
    const float* Bx = sm.B[bc][0];
    const float* By = sm.B[bc][1];
    const float* Bz = sm.B[bc][2];
    return face_flux<float, SP, SAT>(TL, TR, (TR - TL) * g.inv_dx[1], (gxL + gxR) * g.inv_4dx[0],
                                     (gzL + gzR) * g.inv_4dx[2], 0.5f * (By[off(iy, ix)] + By[off(iy + 1, ix)]),
                                     0.5f * (Bx[off(iy, ix)] + Bx[off(iy + 1, ix)]),
                                     0.5f * (Bz[off(iy, ix)] + Bz[off(iy + 1, ix)]), p);
}

// Transverse gradient of a face from the four one-sided differences at its
// two cells (L, R) along axis e: their average, or where the limiter is on
// (Appendix C) the MC limit of the MC limits taken at L and at R.
__device__ __forceinline__ float tgrad(float TL, float TR, float Lp, float Lm, float Rp, float Rm, float inv_dx,
                                       float inv_4dx, bool limit)
{
    if (limit) return mc_limit(mc_limit(Lp - TL, TL - Lm), mc_limit(Rp - TR, TR - Rm)) * inv_dx;
    return (Lp + Rp - Lm - Rm) * inv_4dx;
}

// Face flux along DIR (0 x, 1 y, 2 z) between local cell (ix, iy) of plane
// tc and its +DIR neighbour, every value straight from the smem ring, with
// MC-limited transverse gradients at faces whose lower temperature is below
// the floor.  tm / tp: T slots of the planes below / above tc; bc / bp: b
// slots of plane tc and of the plane above (z-faces take b there).
template <bool SP, bool SAT, int DIR>
__device__ __forceinline__ float face_lim(const Smem& sm, const KGrid<float>& g, const KPhys<float>& p, int tm,
                                          int tc, int tp, int bc, int bp, int ix, int iy)
{
    const float* T = sm.T[tc];
    const int jx = DIR == 0 ? ix + 1 : ix, jy = DIR == 1 ? iy + 1 : iy;
    const float* TRp = DIR == 2 ? sm.T[tp] : T;          // plane of the R cell
    const float TL = T[off(iy, ix)], TR = TRp[off(jy, jx)];
    const bool limit = p.limiter && fminf(TL, TR) < p.lfloor;
    const float gn = (TR - TL) * g.inv_dx[DIR];
    float g1, g2;
    if (DIR == 0) {
        g1 = tgrad(TL, TR, T[off(iy + 1, ix)], T[off(iy - 1, ix)], T[off(iy + 1, jx)], T[off(iy - 1, jx)],
                   g.inv_dx[1], g.inv_4dx[1], limit);
        g2 = tgrad(TL, TR, sm.T[tp][off(iy, ix)], sm.T[tm][off(iy, ix)], sm.T[tp][off(iy, jx)],
                   sm.T[tm][off(iy, jx)], g.inv_dx[2], g.inv_4dx[2], limit);
    } else if (DIR == 1) {
        g1 = tgrad(TL, TR, T[off(iy, ix + 1)], T[off(iy, ix - 1)], T[off(jy, ix + 1)], T[off(jy, ix - 1)],
                   g.inv_dx[0], g.inv_4dx[0], limit);
        g2 = tgrad(TL, TR, sm.T[tp][off(iy, ix)], sm.T[tm][off(iy, ix)], sm.T[tp][off(jy, ix)],
                   sm.T[tm][off(jy, ix)], g.inv_dx[2], g.inv_4dx[2], limit);
    } else {
        g1 = tgrad(TL, TR, T[off(iy, ix + 1)], T[off(iy, ix - 1)], TRp[off(iy, ix + 1)], TRp[off(iy, ix - 1)],
                   g.inv_dx[0], g.inv_4dx[0], limit);
        g2 = tgrad(TL, TR, T[off(iy + 1, ix)], T[off(iy - 1, ix)], TRp[off(iy + 1, ix)], TRp[off(iy - 1, ix)],
                   g.inv_dx[1], g.inv_4dx[1], limit);
    }
    const int br = DIR == 2 ? bp : bc;
    float bf[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) bf[e] = 0.5f * (sm.B[bc][e][off(iy, ix)] + sm.B[br][e][off(jy, jx)]);
    // normal component first, then the transverse ones in axis order
    const int t1 = DIR == 0 ? 1 : 0, t2 = DIR == 2 ? 1 : 2;
    return face_flux<float, SP, SAT>(TL, TR, gn, g1, g2, bf[DIR], bf[t1], bf[t2], p);
}

// MODE 0: out = M(Tin); 1: stage 1 (MY0out = M, out = Y0 + mt M); 2: stage j.
// LIM: slope-limited transverse gradients, every face from shared memory.
template <bool SP, bool SAT, int MODE, bool LIM>
__global__ void __launch_bounds__(NTHREADS, 3)
stage_fast_kernel(KGrid<float> g, KPhys<float> p, FastArgs a, KCoef<float> cf, unsigned* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);

    const int tid = threadIdx.x;
    const int ix = tid & (TX - 1);
    const int iy = tid >> 5;
    const int i0 = blockIdx.x * TX;
    const int j0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * NZC;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int nzc = min(NZC, nz - z0);
    // 16-byte chunks need rows that start on a 16-byte boundary; partially
    // filled tiles are fine (chunks past the edge wrap or hold ghosts whole)
    const bool fastx = (nx & 3) == 0;

    if (MODE != 0 && a.coef_tab) {
        const float* t = a.coef_tab + 4 * a.j;
        cf.mu = t[0]; cf.nu = t[1]; cf.mt = t[2]; cf.gt = t[3];
    }

    // bundles are indexed by local plane q = kk - z0 in [-1, nzc]
    auto tslot = [](int q) { return (q + 1) & 3; };
    auto bslot = [](int q) { return (q + 1) % 3; };
    auto yslot = [](int q) { return (q + 3) % 3; };

    Task tk0{nullptr, 0u, 0u}, tk1{nullptr, 0u, 0u}, tky{nullptr, 0u, 0u};
    if (fastx) {
        tk0 = make_tb_task(sm, g, a, tid, i0, j0);
        tk1 = make_tb_task(sm, g, a, tid + NTHREADS, i0, j0);
        tky = make_y_task<MODE>(sm, g, a, tid, i0, j0);
    }
    auto load = [&](int q, bool withY) {
        if (fastx) {
            const PlaneOff po = plane_offsets(g, z0 + q);
            const unsigned ts = (unsigned)(tslot(q) * PLANE * 4);
            const unsigned bs = (unsigned)(bslot(q) * 3 * PLANE * 4);
            issue_tb(tk0, po, ts, bs, g.bcv);
            issue_tb(tk1, po, ts, bs, g.bcv);
            if (withY) issue_y(tky, po.t, (unsigned)(yslot(q) * 3 * NTHREADS * 4));
        } else {
            load_bundle_ragged<MODE>(sm, g, a, z0 + q, tslot(q), bslot(q), yslot(q), withY, i0, j0);
        }
    };

    load(-1, false);
    cp_commit();
    load(0, true);
    cp_commit();
    load(1, nzc > 1);
    cp_commit();
    cp_wait<0>();
    __syncthreads();

    PlaneQ prv = read_plane(sm, tslot(-1), bslot(-1), ix, iy);
    PlaneQ cur = read_plane(sm, tslot(0), bslot(0), ix, iy);
    // z-face between planes z0 - 1 and z0
    float Fz_lo;
    if (LIM) {
        Fz_lo = face_lim<SP, SAT, 2>(sm, g, p, 0, tslot(-1), tslot(0), bslot(-1), bslot(0), ix, iy);
    } else {
        Fz_lo = face_flux<float, SP, SAT>(
            prv.To, cur.To, (cur.To - prv.To) * g.inv_dx[2], (prv.gxo + cur.gxo) * g.inv_4dx[0],
            (prv.gyo + cur.gyo) * g.inv_4dx[1], 0.5f * (prv.bo[2] + cur.bo[2]), 0.5f * (prv.bo[0] + cur.bo[0]),
            0.5f * (prv.bo[1] + cur.bo[1]), p);
    }
    float TmO = prv.To, TmR = prv.TR, TmU = prv.TU;

    const bool inside = (i0 + ix < nx) && (j0 + iy < ny);
    for (int q = 0; q < nzc; ++q) {
        // prefetch bundle q + 2 (T and b are needed up to q = nzc)
        if (q + 2 <= nzc) load(q + 2, q + 2 < nzc);
        cp_commit();
        cp_wait<1>();
        __syncthreads();

        PlaneQ nxt = read_plane(sm, tslot(q + 1), bslot(q + 1), ix, iy);
        const float gzo = nxt.To - TmO, gzR = nxt.TR - TmR, gzU = nxt.TU - TmU;

        float Fx, Fy, Fz;
        if (LIM) {
            const int tm = tslot(q - 1), tc = tslot(q), tp = tslot(q + 1), bc = bslot(q), bp = bslot(q + 1);
            Fx = face_lim<SP, SAT, 0>(sm, g, p, tm, tc, tp, bc, bp, ix, iy);
            Fy = face_lim<SP, SAT, 1>(sm, g, p, tm, tc, tp, bc, bp, ix, iy);
            Fz = face_lim<SP, SAT, 2>(sm, g, p, tm, tc, tp, bc, bp, ix, iy);
        } else {
            // +x face
            Fx = face_flux<float, SP, SAT>(
                cur.To, cur.TR, (cur.TR - cur.To) * g.inv_dx[0], (cur.gyo + cur.gyR) * g.inv_4dx[1],
                (gzo + gzR) * g.inv_4dx[2], 0.5f * (cur.bo[0] + cur.bR[0]), 0.5f * (cur.bo[1] + cur.bR[1]),
                0.5f * (cur.bo[2] + cur.bR[2]), p);
            // +y face
            Fy = face_flux<float, SP, SAT>(
                cur.To, cur.TU, (cur.TU - cur.To) * g.inv_dx[1], (cur.gxo + cur.gxU) * g.inv_4dx[0],
                (gzo + gzU) * g.inv_4dx[2], 0.5f * (cur.bo[1] + cur.bU[1]), 0.5f * (cur.bo[0] + cur.bU[0]),
                0.5f * (cur.bo[2] + cur.bU[2]), p);
            // +z face
            Fz = face_flux<float, SP, SAT>(
                cur.To, nxt.To, (nxt.To - cur.To) * g.inv_dx[2], (cur.gxo + nxt.gxo) * g.inv_4dx[0],
                (cur.gyo + nxt.gyo) * g.inv_4dx[1], 0.5f * (cur.bo[2] + nxt.bo[2]), 0.5f * (cur.bo[0] + nxt.bo[0]),
                0.5f * (cur.bo[1] + nxt.bo[1]), p);
        }

        const int par = q & 1;
        // faces on the tile's low boundary: y-face below row 0 (warp 0),
        // x-face left of column 0 (warp 1, one row per lane)
        if (iy == 0) {
            sm.Fy[par][0][ix] =
                LIM ? face_lim<SP, SAT, 1>(sm, g, p, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), bslot(q + 1), ix,
                                          -1)
                    : face_y_smem<SP, SAT>(sm, g, p, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), ix, -1);
        } else if (iy == 1 && ix < TY) {
            sm.Fx[par][ix][0] =
                LIM ? face_lim<SP, SAT, 0>(sm, g, p, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), bslot(q + 1), -1,
                                          ix)
                    : face_x_smem<SP, SAT>(sm, g, p, tslot(q - 1), tslot(q), tslot(q + 1), bslot(q), -1, ix);
        }
        float y0v = 0.f, yjm2v = 0.f, my0v = 0.f;
        if (MODE == 2) {
            const int ys = yslot(q);
            y0v = sm.Y[ys][0][tid];
            yjm2v = sm.Y[ys][1][tid];
            my0v = sm.Y[ys][2][tid];
        }
        sm.Fx[par][iy][ix + 1] = Fx;
        sm.Fy[par][iy + 1][ix] = Fy;
        __syncthreads();

        const float div = (sm.Fx[par][iy][ix + 1] - sm.Fx[par][iy][ix]) * g.inv_dx[0] +
                          (sm.Fy[par][iy + 1][ix] - sm.Fy[par][iy][ix]) * g.inv_dx[1] +
                          (Fz - Fz_lo) * g.inv_dx[2];
        const float M = -div;
        if (inside) {
            const int64_t c = ((int64_t)(z0 + q) * ny + (j0 + iy)) * nx + (i0 + ix);
            if (MODE == 0) {
                a.out[c] = M;
            } else if (MODE == 1) {
                if (a.MY0out) a.MY0out[c] = M;
                float y = cur.To + cf.mt * M;
                check_value<float, SP>(y, status);
                a.out[c] = y;
            } else {
                float inc = cf.mu * (cur.To - y0v) + cf.nu * (yjm2v - y0v) + cf.mt * M + cf.gt * my0v;
                float y = y0v + inc;
                check_value<float, SP>(y, status);
                a.out[c] = y;
            }
        }
        Fz_lo = Fz;
        TmO = cur.To;
        TmR = cur.TR;
        TmU = cur.TU;
        cur = nxt;
    }
    cp_wait<0>();
}

template <bool SP, bool SAT, int MODE, bool LIM>
cudaError_t launch3(const KGrid<float>& g, const KPhys<float>& p, const FastArgs& a, const KCoef<float>& cf,
                    unsigned* status, cudaStream_t st)
{
    static bool attr_set = false;
    const int smem = (int)sizeof(Smem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(stage_fast_kernel<SP, SAT, MODE, LIM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + NZC - 1) / NZC);
    stage_fast_kernel<SP, SAT, MODE, LIM><<<grid, NTHREADS, smem, st>>>(g, p, a, cf, status);
    return cudaGetLastError();
}

template <bool SP, bool SAT, bool LIM>
cudaError_t launch_lim(int mode, const KGrid<float>& g, const KPhys<float>& p, const FastArgs& a,
                       const KCoef<float>& cf, unsigned* status, cudaStream_t st)
{
    if (mode == 0) return launch3<SP, SAT, 0, LIM>(g, p, a, cf, status, st);
    if (mode == 1) return launch3<SP, SAT, 1, LIM>(g, p, a, cf, status, st);
    return launch3<SP, SAT, 2, LIM>(g, p, a, cf, status, st);
}

template <bool SP, bool SAT>
cudaError_t launch_mode(bool limiter, int mode, const KGrid<float>& g, const KPhys<float>& p, const FastArgs& a,
                        const KCoef<float>& cf, unsigned* status, cudaStream_t st)
{
    if (limiter) return launch_lim<SP, SAT, true>(mode, g, p, a, cf, status, st);
    return launch_lim<SP, SAT, false>(mode, g, p, a, cf, status, st);
}

}  // namespace

bool fast_stage_supported(const LaunchCfg& c, const KGrid<float>& g)
{
    return c.dtype == 0 && c.ndim == 3 && g.n[0] >= 1 && g.n[1] >= 1 && g.n[2] >= 1;
}

cudaError_t launch_stage_fast(const LaunchCfg& c, const KGrid<float>& g, const KPhys<float>& p,
                              const StageIO& io, const KCoef<float>& coef, unsigned* status, cudaStream_t st)
{
    FastArgs a;
    a.Tin = static_cast<const float*>(io.mode == 1 ? io.Y0 : io.Yjm1);
    a.b = static_cast<const float*>(io.b);
    a.Y0 = static_cast<const float*>(io.Y0);
    a.Yjm2 = static_cast<const float*>(io.Yjm2);
    a.MY0in = static_cast<const float*>(io.MY0);
    a.MY0out = io.mode == 1 ? static_cast<float*>(io.MY0) : nullptr;
    a.out = static_cast<float*>(io.Yj);
    a.coef_tab = static_cast<const float*>(io.coef_tab);
    a.j = io.j;
    if (c.spitzer) {
        if (c.saturate) return launch_mode<true, true>(c.limiter, io.mode, g, p, a, coef, status, st);
        return launch_mode<true, false>(c.limiter, io.mode, g, p, a, coef, status, st);
    }
    if (c.saturate) return launch_mode<false, true>(c.limiter, io.mode, g, p, a, coef, status, st);
    return launch_mode<false, false>(c.limiter, io.mode, g, p, a, coef, status, st);
}

}  // namespace rkl
