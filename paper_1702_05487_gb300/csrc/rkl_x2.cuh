// Layout shared by the paired-cell stage kernel and the persistent ensemble
// kernel: tile geometry, kernel arguments and the shared-memory bundle ring.
#pragma once

#include <cuda.h>

#include "rkl_device.cuh"

namespace rkl {
namespace x2 {

constexpr int TX = 64;                  // tile columns: 32 lanes x 2 cells
constexpr int TY = 4;                   // tile rows: one warp per row
constexpr int NTHREADS = 32 * TY;
// Resident CTAs per SM of the default build: 5 x 4 warps at up to 102
// registers a thread and 5 x 44 KB of shared memory.  Five short CTAs keep
// more warps eligible than four (fewer barrier and dependency stalls).
constexpr int kCtasPerSm = 5;
constexpr int SXS = 72;                 // smem row: halo chunk (4), 64 interior, halo chunk (4)
constexpr int CPR = SXS / 4;            // 16-byte chunks per smem row
constexpr int ROWS = TY + 2;
constexpr int PLANE = ROWS * SXS;
// plane stride of the rings whose slots tensor copies fill: a multiple of
// 128 bytes (a tensor copy's shared-memory destination is 128-byte aligned)
constexpr int PSTR = (PLANE + 31) / 32 * 32;

struct FastArgs {
    const float* Tin;       // field whose M is taken (Y_{j-1}, or Y_0 at stage 1)
    const float* b;         // [3][ncell]
    const float* Y0;
    const float* Yjm2;
    const float* MY0in;
    float* MY0out;          // stage 1 only
    float* out;             // Y_j, or M(T) in mode 0
    const float* coef_tab;  // if non-null: stage coefficients at coef_tab[4 j]
    int j;
};

// Plane rings for a prefetch distance of PD planes: while plane q is
// computed, planes q+1 .. q+PD are in flight and plane q+PD+1 is being
// issued into the slots that plane q-2 (T) or q-1 (b, Y) released.
// Shared-memory plane of a tile TXW columns wide: TXW / 2 lanes per row
// (two cells each), NTHREADS / (TXW / 2) rows, a halo chunk of 4 columns on
// each side and one halo row above and below.
constexpr int plane_of(int txw) { return (NTHREADS / (txw / 2) + 2) * (txw + 8); }

// Geometry and rings of one tile: TXW = 64 (the default, one warp per row)
// or 32 (two rows per warp, for grids whose width is an odd multiple of
// 32).  PS: floats from one ring slot to the next.
template <int PD, int TXW = TX, int PS = plane_of(TXW)>
struct SmemT {
    static constexpr int TX = TXW, LPR = TXW / 2, TY = NTHREADS / LPR;
    static constexpr int SXS = TX + 8, CPR = SXS / 4, ROWS = TY + 2, PLANE = ROWS * SXS;
    static constexpr int NT = 3 + PD, NB = 2 + PD, NY = 2 + PD;
    static constexpr int PSTRIDE = PS;
    static_assert(PS >= PLANE, "ring slot smaller than a plane");
    alignas(128) float T[NT][PS];   // Y_{j-1} planes q-1, q, q+1 and those in flight
    float B[NB][3][PS];             // b planes q, q+1 and those in flight
    alignas(128) float Y[NY][3][TY * TX];   // Y0, Y_{j-2}, M(Y0) of plane q and those in flight
    float Fy[2][TY + 1][TX];        // y-face fluxes (row 0: the tile's lower boundary)
    float FxLo[2][TY];              // x-faces on the tile's left boundary
    alignas(8) unsigned long long bar[PD + 2];    // bundle barriers of the bulk-copy path
    alignas(8) unsigned long long ybar[4];        // Y bundles copied by tensor maps (plane q: ybar[q & 3])
    // offset of cell (row r, column c) of the tile in a plane, halo included
    __device__ static int off(int r, int c) { return (r + 1) * SXS + c + 4; }
};

// Tensor maps of Y0, Y_{j-2} and M(Y0) (3D FP32, boxes of TX x TY x 1) for
// the variant whose Y bundles the TMA engine copies (cp.async.bulk.tensor).
struct YMaps {
    CUtensorMap m[3];
};

// Tensor maps of every bundle for the variant whose plane bundles all come
// from the TMA engine: T (Y_{j-1}) and bx, by, bz with boxes of SXS x
// (TY + 2) x 1 (a tile's rows with their one-cell halo ring, columns from
// i0 - 4), then Y0, Y_{j-2}, M(Y0) with boxes of TX x TY x 1.
struct TMaps {
    CUtensorMap m[7];
};
constexpr int kPD = 2;              // prefetch distance of the default build
using Smem = SmemT<kPD>;

// One problem of an ensemble as the persistent kernel sees it.
struct EnsProb {
    KGrid<float> g;
    KPhys<float> p;
    float* T;               // Y_0 and the result (caller's array)
    const float* b;         // [3][ncell] (caller's array)
    float* buf[3];          // rotating stage buffers (ensemble workspace)
    float* my0;             // M(Y_0)
    const float* coef;      // this super-step's table, stage j at coef[4 j]
    int s;                  // stages this super-step
    int tx, ty, tz, ntiles; // tiles in x, y and z-chunks
    int nzchunk;
    int txw;                // tile width: 64, or 32 (rows of 32 columns, two per warp)
};

// A run of work items: the tiles of stage j of problem p, items
// [first, first + count) in the global order.
struct EnsSeg {
    int first;
    int p;
    int j;
    int count;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The next work item of a persistent ensemble launch, claimed by thread 0
// of the CTA from the global counter in the fixed stage-major order: sets
// (p, j, tile) and returns true once the item may run (every tile of stage
// j - 1 of problem p is done); false when the list is exhausted, another
// CTA gave up, or this CTA's bounded wait ran out (then ST_TIMEOUT and the
// abort flag are set).
__device__ __forceinline__ bool ens_claim(const EnsProb* probs, const EnsSeg* segs, int nseg, int total, int* work,
                                          const unsigned* done, unsigned* status, int* abort_flag,
                                          long long spin_limit, int& p, int& j, int& tile)
{
    const int it = atomicAdd(work, 1);
    if (it >= total || *reinterpret_cast<volatile int*>(abort_flag)) return false;
    int lo = 0, hi = nseg - 1;                 // last segment with first <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first <= it) lo = mid; else hi = mid - 1;
    }
    const EnsSeg sg = segs[lo];
    const unsigned target = (unsigned)((sg.j - 1) * probs[sg.p].ntiles);
    long long n = 0;
    while (ld_acquire(&done[sg.p]) < target) {
        if (++n > spin_limit || *reinterpret_cast<volatile int*>(abort_flag)) {
            atomicOr(status, ST_TIMEOUT);
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(128);
    }
    p = sg.p;
    j = sg.j;
    tile = it - sg.first;
    return true;
}

}  // namespace x2

cudaError_t launch_ensemble_xq(bool spitzer, bool saturate, const x2::EnsProb* probs, const x2::EnsSeg* segs,
                               int nseg, int total, int* work, unsigned* done, unsigned* status, int* abort_flag,
                               long long spin_limit, int grid, cudaStream_t st);

cudaError_t launch_ensemble_x2(bool spitzer, bool saturate, const x2::EnsProb* probs, const x2::EnsSeg* segs,
                               int nseg, int total, int* work, unsigned* done, unsigned* status, int* abort_flag,
                               long long spin_limit, int grid, cudaStream_t st);

}  // namespace rkl
