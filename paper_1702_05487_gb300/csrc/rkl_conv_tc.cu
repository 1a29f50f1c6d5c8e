// Periodic 3x3x3 convolution of the surrogate on the 5th-generation tensor
// cores: tcgen05.mma with operands described in shared memory and the FP32
// accumulator in tensor memory (TMEM).
//
// Implicit GEMM, input-plane major: M = 128 voxels (an 8 x 16 block of a z
// plane, x fastest), K = 9 in-plane offsets x Cin per input plane, and
// N = 3 Cout: one MMA multiplies a shifted copy of input plane q by the
// weights of dz = +1, 0, -1 side by side and so adds q's contribution to
// output planes q - 1, q and q + 1 at once (each output plane owns Cout
// TMEM columns; a chunk of nz planes holds nz + 2 of them).  A resident
// input plane is therefore read by the tensor cores once per in-plane
// offset instead of three times, and a plane needs 9 Cin/16 MMAs instead of
// 27 Cin/16.  Input planes with their one-voxel halo (10 x 18 voxels)
// stream through a 5-slot shared-memory ring, each stored chunk-major
// ([Cin/8][180 voxels][8 channels]): for an offset (dy, dx) the A operand
// is then a plain K-major no-swizzle matrix -- core matrix i (rows y = i,
// x = 0..7) starts at voxel (dx, i + dy) of the halo plane and the next one
// is one halo row (10 voxels) further.  The weights sit in shared memory
// once per persistent CTA as [9][Cin/8][3 Cout][8].  The CTA is a
// pipeline of three roles that meet only at mbarriers: three loader warps
// stream input planes into the ring with cp.async, keeping two planes in
// flight per thread (each thread's 16-byte chunks of the halo plane are
// fixed for a work item, so a plane costs one address add per chunk);
// once a plane's copies have landed each loader fences
// them into the tensor cores' (async) proxy and arrives on the slot's
// "full" barrier.  Thread 0 issues the MMAs of a plane once it is full and
// commits them to the slot's "empty" barrier (the loaders refill the slot
// after it) and to the "done" barrier of the output plane they complete.
// Four drain warps (one TMEM lane quarter each) wait for that, drain the
// plane (bias, ReLU or mask, BF16 or FP32 store), zero its columns for the
// next work item and arrive on its "freed" barrier, which the MMA thread
// waits for before it starts that plane of the next item.  No CTA-wide
// barrier per plane, and no proxy fence on the MMA thread's path.  Every
// wait is bounded and reports ST_TIMEOUT.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rkl_conv.h"
#include "rkl_pair.cuh"

namespace rkl {
namespace conv {
namespace {

using x2::cp16;
using x2::cp_commit;
using x2::cp_wait;
using x2::mbar_init;
using x2::mbar_try_wait;
using x2::smem_u32;

constexpr int QX = 8, QY = 16;                 // output block of a plane: M = 128
constexpr int HX = QX + 2, HY = QY + 2;         // halo plane
constexpr int HP = HX * HY;                     // 180 voxels
constexpr int NSLOT = 5;                        // input-plane ring
constexpr int NLW = 3;                          // loader warps
constexpr int NLOAD = 32 * NLW;                 // loader threads
constexpr int NTHR_TC = 32 * (1 + NLW + 4);     // warp 0 MMA, warps 1 .. NLW loads, the last four drain
constexpr int NZC_TC = 6;                       // output planes per work item
constexpr int TMEM_COLS = 256;                  // 32 (NZC_TC + 2) columns

template <int CIN, int COUT>
struct TcSmem {
    __nv_bfloat16 W[9][CIN / 8][3 * COUT][8];   // B operands: per (dy, dx) the dz = +1, 0, -1 blocks
    __nv_bfloat16 A[NSLOT][CIN / 8][HP][8];     // A operands, one halo plane per slot
    unsigned long long full[NSLOT];             // slot's input plane landed and fenced (one arrival per loader)
    unsigned long long empty[NSLOT];            // MMAs reading the slot completed
    unsigned long long done[NZC_TC];            // output plane r of the current item accumulated
    unsigned long long freed[NZC_TC];           // output plane r drained and its columns zeroed
    unsigned tmem;                              // TMEM base column from tcgen05.alloc
};

// Shared-memory matrix descriptor (no swizzle, K-major): start address,
// leading byte offset (next core matrix along K), stride byte offset (next
// core matrix along M or N), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N given.
template <int N>
__device__ __forceinline__ unsigned idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(unsigned dtmem, uint64_t a, uint64_t b, unsigned id, unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float* v)
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// zero 32 / 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_zero32(unsigned taddr)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr),
        "r"(0u)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_zero16(unsigned taddr)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};\n" ::"r"(taddr),
        "r"(0u)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ int wrapi_tc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// MODE 0: ReLU, bf16 out; 1: linear, f32 out; 2: no bias, times the ReLU
// mask (mask > 0), bf16 out.  Persistent: work item = (8 x 16 column block,
// chunk of NZC_TC output planes); the items of a CTA ascend, so only its
// last one can be short.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NTHR_TC, 1)
conv_tc_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wt,
               const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
               int D, int H, int W, unsigned* status)
{
    using S = TcSmem<CIN, COUT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S& sm = *reinterpret_cast<S*>(smem_raw);
    constexpr int NCH = CIN / 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncolx = W / QX, ncols = ncolx * (H / QY);
    const int nitems = ncols * ((D + NZC_TC - 1) / NZC_TC);
    // output plane r (-1 <= r <= nz of an item) owns columns COUT (r + 1) ...
    auto col_of = [](int r) { return (unsigned)(COUT * (r + 1)); };

    // weights [27][COUT][CIN] (o = (dz+1) 9 + (dy+1) 3 + dx+1) -> [9][CIN/8][3 COUT][8]
    // with block j of the N dimension holding dz = 1 - j
    for (int t = tid; t < 27 * COUT * NCH; t += NTHR_TC) {
        const int e = t / (3 * COUT * NCH), r = t % (3 * COUT * NCH);
        const int jn = r / NCH, ch = r % NCH, j = jn / COUT, n = jn % COUT;
        const int o = (2 - j) * 9 + e;
        cp16(smem_u32(&sm.W[e][ch][jn][0]), wt + ((int64_t)o * COUT + n) * CIN + ch * 8);
    }
    cp_commit();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(smem_u32(&sm.full[i]), NLOAD);
            mbar_init(smem_u32(&sm.empty[i]), 1u);
        }
        for (int i = 0; i < NZC_TC; ++i) {
            mbar_init(smem_u32(&sm.done[i]), 1u);
            mbar_init(smem_u32(&sm.freed[i]), 128u);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    cp_wait<0>();                                // the weights
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tbase = sm.tmem;
    // Bounded waits without a back-off sleep (try_wait itself suspends the
    // thread until the phase completes or a hardware time limit passes; a
    // sleeping waiter would wake late and leave the tensor pipe idle).  A
    // thread whose wait gave up skips its later waits, so a broken pipeline
    // ends after one bounded wait per thread.
    bool ok = true;
    auto wait = [&](unsigned long long& bar, unsigned parity) {
        if (!ok) return;
        for (int it = 0; it < (1 << 24); ++it)
            if (mbar_try_wait(smem_u32(&bar), parity)) return;
        ok = false;
    };

    if (warp == 0) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            const unsigned id3 = idesc<3 * COUT>(), id1 = idesc<COUT>();
            const uint64_t bdesc0 = sdesc(smem_u32(&sm.W[0][0][0][0]), 3 * COUT * 16, 8 * 16);
            unsigned n = 0, k = 0;               // input planes and items of this CTA so far
            for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
                const int z0 = (item / ncols) * NZC_TC, nz = min(NZC_TC, D - z0);
                for (int q = -1; q <= nz; ++q, ++n) {
                    const unsigned sl = n % NSLOT;
                    wait(sm.full[sl], (n / NSLOT) & 1u);
                    // output plane q + 1 is first reached by input plane q: wait
                    // until it is zeroed (phase k: the drain warps' initial pass,
                    // then the drain of each previous item)
                    if (q + 1 < nz) wait(sm.freed[q + 1], k & 1u);
                    fence_after();
                    const uint64_t ab = sdesc(smem_u32(&sm.A[sl][0][0][0]), HP * 16, HX * 16);
                    if (q == -1 || q == nz) {
                        // edge planes reach one output plane: dz = -1 (q = -1 -> r = 0)
                        // or dz = +1 (q = nz -> r = nz - 1)
                        const int j = q == -1 ? 2 : 0;
                        const unsigned dt = tbase + col_of(q == -1 ? 0 : nz - 1);
#pragma unroll
                        for (int e = 0; e < 9; ++e)
#pragma unroll
                            for (int kk = 0; kk < CIN / 16; ++kk) {
                                const uint64_t a =
                                    ab + (uint64_t)((((e / 3) * HX + e % 3) * 16 + 2 * kk * HP * 16) >> 4);
                                const uint64_t b =
                                    bdesc0 + (uint64_t)((((e * NCH + 2 * kk) * 3 * COUT) + j * COUT) * 16 >> 4);
                                mma_f16(dt, a, b, id1, (q == -1 && (e | kk) == 0) ? 0u : 1u);
                            }
                    } else {
                        const unsigned dt = tbase + col_of(q - 1);
#pragma unroll
                        for (int e = 0; e < 9; ++e)
#pragma unroll
                            for (int kk = 0; kk < CIN / 16; ++kk) {
                                const uint64_t a =
                                    ab + (uint64_t)((((e / 3) * HX + e % 3) * 16 + 2 * kk * HP * 16) >> 4);
                                const uint64_t b = bdesc0 + (uint64_t)(((e * NCH + 2 * kk) * 3 * COUT) * 16 >> 4);
                                mma_f16(dt, a, b, id3, 1u);
                            }
                    }
                    mma_commit(smem_u32(&sm.empty[sl]));
                    if (q >= 1) mma_commit(smem_u32(&sm.done[q - 1]));   // output plane q - 1 complete
                }
                // planes a short item does not have: the same one phase per item
                // of "freed" waited and of "done" completed, so that no role
                // gets two phases ahead of another on any barrier
                for (int r = nz; r < NZC_TC; ++r) {
                    wait(sm.freed[r], k & 1u);
                    mbar_arrive(smem_u32(&sm.done[r]));
                }
            }
        }
    } else if (warp <= NLW) {
        // ---------------- loads (warps 1 .. NLW) ----------------
        const int lt = tid - 32;
        // copy tasks of this thread for the current item: 16-byte chunks of
        // the halo plane (element offset within an input plane, byte offset
        // within a ring slot), fixed for the item's planes
        constexpr int NTASK = (HP * NCH + NLOAD - 1) / NLOAD;
        int toff[NTASK];
        unsigned tdst[NTASK];
        const unsigned abase = smem_u32(&sm.A[0][0][0][0]);
        constexpr unsigned kSlotBytes = (unsigned)(NCH * HP * 16);
        const int64_t zstride = (int64_t)H * W * CIN;
        unsigned n = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            const int col = item % ncols, chunk = item / ncols;
            const int x0 = (col % ncolx) * QX, y0 = (col / ncolx) * QY, z0 = chunk * NZC_TC;
            const int nz = min(NZC_TC, D - z0);
#pragma unroll
            for (int i = 0; i < NTASK; ++i) {
                const int t = lt + i * NLOAD;
                const int hv = t / NCH, ch = t % NCH;
                const int gy = wrapi_tc(y0 + hv / HX - 1, H), gx = wrapi_tc(x0 + hv % HX - 1, W);
                toff[i] = t < HP * NCH ? (gy * W + gx) * CIN + ch * 8 : -1;
                tdst[i] = (unsigned)((ch * HP + hv) * 16);
            }
            for (int q = -1; q <= nz; ++q, ++n) {
                const unsigned sl = n % NSLOT;
                // the slot's previous plane (n - NSLOT) has been multiplied
                if (n >= NSLOT) wait(sm.empty[sl], (n / NSLOT - 1) & 1u);
                const __nv_bfloat16* pz = in + (int64_t)wrapi_tc(z0 + q, D) * zstride;
                const unsigned sb = abase + sl * kSlotBytes;
#pragma unroll
                for (int i = 0; i < NTASK; ++i)
                    if (toff[i] >= 0) cp16(sb + tdst[i], pz + toff[i]);
                cp_commit();
                // the previous plane's copies have landed: make them visible to
                // the tensor cores' proxy and report the slot full
                if (n >= 1) {
                    cp_wait<1>();
                    fence_proxy_async();
                    mbar_arrive(smem_u32(&sm.full[(n - 1) % NSLOT]));
                }
            }
        }
        cp_wait<0>();
        if (n >= 1) {
            fence_proxy_async();
            mbar_arrive(smem_u32(&sm.full[(n - 1) % NSLOT]));
        }
    } else {
        // ---------------- drain (the last four warps; a warp reaches TMEM lane quarter warp % 4) ----------------
        const int q4 = warp & 3;
        const unsigned tlane = tbase + ((unsigned)(q4 * 32) << 16);
        float bs[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bs[c] = MODE != 2 ? bias[c] : 0.f;
        auto clear = [&](int r) {
            if (COUT == 32) tmem_zero32(tlane + col_of(r));
            else tmem_zero16(tlane + col_of(r));
        };
        // output planes 1 .. are accumulated from their first MMA on: zero them
        // for the first item (plane 0 starts with an overwriting MMA)
        for (int r = 0; r < NZC_TC; ++r) {
            if (r >= 1) clear(r);
            fence_before();
            mbar_arrive(smem_u32(&sm.freed[r]));
        }
        unsigned k = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
            const int col = item % ncols, chunk = item / ncols;
            const int x0 = (col % ncolx) * QX, y0 = (col / ncolx) * QY, z0 = chunk * NZC_TC;
            const int nz = min(NZC_TC, D - z0);
            for (int r = 0; r < NZC_TC; ++r) {
                wait(sm.done[r], k & 1u);
                if (r < nz) {
                    fence_after();
                    float v[COUT];
                    if (COUT == 32) tmem_ld32(tlane + col_of(r), v);
                    else tmem_ld16(tlane + col_of(r), v);
                    const int m = q4 * 32 + lane;         // TMEM lane = GEMM row = voxel of the block
                    const int64_t gv = ((int64_t)(z0 + r) * H + (y0 + m / QX)) * W + (x0 + m % QX);
                    if (MODE == 1) {
                        float* o = static_cast<float*>(out) + gv * COUT;
#pragma unroll
                        for (int c = 0; c < COUT; c += 4)
                            *reinterpret_cast<float4*>(o + c) = make_float4(v[c] + bs[c], v[c + 1] + bs[c + 1],
                                                                            v[c + 2] + bs[c + 2], v[c + 3] + bs[c + 3]);
                    } else {
                        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + gv * COUT;
#pragma unroll
                        for (int c = 0; c < COUT; c += 8) {
                            float w[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) w[i] = MODE == 0 ? fmaxf(v[c + i] + bs[c + i], 0.f) : v[c + i];
                            if (MODE == 2) {
                                const uint4 mk = *reinterpret_cast<const uint4*>(mask + gv * COUT + c);
                                const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    if (!(__bfloat162float(mb[i]) > 0.f)) w[i] = 0.f;
                            }
                            uint4 pk;
                            __nv_bfloat162* ph = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
                            for (int i = 0; i < 4; ++i) ph[i] = __floats2bfloat162_rn(w[2 * i], w[2 * i + 1]);
                            *reinterpret_cast<uint4*>(o + c) = pk;
                        }
                    }
                }
                // no later MMA of this item writes plane r's columns (for r >= nz
                // all of them are done), so they can be zeroed for the next item
                if (r >= 1) clear(r);
                fence_before();
                mbar_arrive(smem_u32(&sm.freed[r]));
            }
        }
    }
    // every MMA has completed: the drain warps waited for the last plane's
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TMEM_COLS)
                     : "memory");
    }
    if (!ok && status) atomicOr(status, ST_TIMEOUT);
}

int sm_count_tc()
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

template <int CIN, int COUT, int MODE>
cudaError_t conv_tc_t(const void* in, const void* wt, const float* bias, const void* mask, void* out, int D, int H,
                      int W, unsigned* status, cudaStream_t st)
{
    const int smem = (int)sizeof(TcSmem<CIN, COUT>);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<CIN, COUT, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nitems = (W / QX) * (H / QY) * ((D + NZC_TC - 1) / NZC_TC);
    const int per_sm = smem <= 113 * 1024 ? 2 : 1;         // and 2 x 256 TMEM columns
    const int grid = nitems < per_sm * sm_count_tc() ? nitems : per_sm * sm_count_tc();
    conv_tc_kernel<CIN, COUT, MODE><<<grid, NTHR_TC, smem, st>>>(
        static_cast<const __nv_bfloat16*>(in), static_cast<const __nv_bfloat16*>(wt), bias,
        static_cast<const __nv_bfloat16*>(mask), out, D, H, W, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t conv_forward_tc(int cin, int cout, int mode, const void* in, const void* wt, const float* bias,
                            const void* mask, void* out, int D, int H, int W, int nzc, unsigned* status,
                            cudaStream_t st)
{
    (void)nzc;                                   // the chunk length is fixed by the TMEM columns
    if (W % QX || H % QY || D < 1) return cudaErrorInvalidValue;
    if ((int64_t)H * W * cin >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;     // 32-bit in-plane offsets
    if (cin == 16 && cout == 32 && mode == 0)
        return conv_tc_t<16, 32, 0>(in, wt, bias, mask, out, D, H, W, status, st);
    if (cin == 32 && cout == 32 && mode == 0)
        return conv_tc_t<32, 32, 0>(in, wt, bias, mask, out, D, H, W, status, st);
    if (cin == 32 && cout == 16 && mode == 1)
        return conv_tc_t<32, 16, 1>(in, wt, bias, mask, out, D, H, W, status, st);
    if (cin == 32 && cout == 32 && mode == 2)
        return conv_tc_t<32, 32, 2>(in, wt, bias, mask, out, D, H, W, status, st);
    if (cin == 16 && cout == 32 && mode == 2)
        return conv_tc_t<16, 32, 2>(in, wt, bias, mask, out, D, H, W, status, st);
    return cudaErrorInvalidValue;
}

}  // namespace conv
}  // namespace rkl
