// Kernels of the learned surrogate: periodic 3x3x3 convolutions as implicit
// GEMMs on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation), their
// backward passes, the flux-form head, the MSE loss and Adam.
//
// Layouts (voxel v = (z * H + y) * W + x of a periodic D x H x W patch):
//   activations  bf16 [V][C]            (channels last, C = 16 or 32)
//   head output  f32  [V][8]            (channels 0..2 are the face fluxes)
//   weights      bf16 [27][Cout][Cin]   (offset o = ((dz+1) * 3 + dy+1) * 3 + dx+1)
//   masters      f32  [27][Cout][Cin] and bias f32 [Cout]
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rkl_conv.h"

namespace rkl {
namespace conv {
namespace {

constexpr int TZ = 4, TY = 8, TX = 16;                 // output tile
constexpr int TV = TZ * TY * TX;                       // 512 voxels
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;   // halo tile
constexpr int HV = HZ * HY * HX;                       // 1080 voxels
constexpr int NWARP = TV / 32;                         // 16 warps, 32 voxels each
constexpr int NTHR = NWARP * 32;

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(unsigned d, const void* s)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(s));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned addr, unsigned& r0, unsigned& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned& r0, unsigned& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma16816(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// --------------------------------------------------------------------------
// Forward convolution (also the backward-data pass with flipped weights).
//   out[v][co] = act(bias[co] + sum_{o, ci} W[o][co][ci] in[v + off(o)][ci])
// MODE 0: ReLU, bf16 out; 1: linear, f32 out (head); 2: no bias, times the
// ReLU mask (mask[v][co] > 0), bf16 out (backward-data through a ReLU).
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NTHR, 1)
conv_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wt, const float* __restrict__ bias,
            const __nv_bfloat16* __restrict__ mask, void* __restrict__ out, int D, int H, int W)
{
    constexpr int SC = CIN + 8;                 // smem voxel stride (bf16): conflict-free ldmatrix rows
    constexpr int NT = COUT / 8;                // n8 tiles
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem_raw);                  // [27][COUT][SC]
    __nv_bfloat16* sX = sW + 27 * COUT * SC;                                           // [HV][SC]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // weights, once per CTA
    for (int t = tid; t < 27 * COUT * (CIN / 8); t += NTHR) {
        const int row = t / (CIN / 8), ch = t % (CIN / 8);
        cp16(smem_u32(sW + row * SC + ch * 8), wt + (int64_t)row * CIN + ch * 8);
    }
    cp_commit();

    const int tilesx = W / TX, tilesy = H / TY, tilesz = D / TZ;
    const int ntiles = tilesx * tilesy * tilesz;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bx = tile % tilesx, by = (tile / tilesx) % tilesy, bz = tile / (tilesx * tilesy);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        __syncthreads();                        // previous tile's readers are done with sX
        for (int t = tid; t < HV * (CIN / 8); t += NTHR) {
            const int hv = t / (CIN / 8), ch = t % (CIN / 8);
            const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
            const int gz = wrapi(z0 + hz - 1, D), gy = wrapi(y0 + hy - 1, H), gx = wrapi(x0 + hx - 1, W);
            const int64_t gv = ((int64_t)gz * H + gy) * W + gx;
            cp16(smem_u32(sX + hv * SC + ch * 8), in + gv * CIN + ch * 8);
        }
        cp_commit();
        cp_wait_all();
        __syncthreads();

        float acc[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;

        // this lane's A rows: voxel m = warp*32 + mt*16 + (lane%8) + 8*((lane/8)%2)
        int hvb[2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int m = warp * 32 + mt * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
            const int tx = m % TX, ty = (m / TX) % TY, tz = m / (TX * TY);
            hvb[mt] = ((tz + 1) * HY + (ty + 1)) * HX + (tx + 1);
        }
        const int akoff = 8 * (lane >> 4);            // k half supplied by this lane
        for (int o = 0; o < 27; ++o) {
            const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
            const int dhv = (dz * HY + dy) * HX + dx;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    ldsm_x4(smem_u32(sX + (hvb[mt] + dhv) * SC + kc * 16 + akoff), a[mt][0], a[mt][1], a[mt][2],
                            a[mt][3]);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    unsigned b0, b1;
                    const int n = nt * 8 + (lane & 7);
                    const int bk = kc * 16 + 8 * ((lane >> 3) & 1);
                    ldsm_x2(smem_u32(sW + (o * COUT + n) * SC + bk), b0, b1);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
                        mma16816(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                }
            }
        }
        // epilogue: rows lane/4 and lane/4 + 8 of each m16 tile, channels 2(lane%4) + {0, 1}
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = warp * 32 + mt * 16 + (lane >> 2) + 8 * h;
                const int tx = m % TX, ty = (m / TX) % TY, tz = m / (TX * TY);
                const int64_t gv = ((int64_t)(z0 + tz) * H + (y0 + ty)) * W + (x0 + tx);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int c = nt * 8 + 2 * (lane & 3);
                    float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                    if (MODE != 2) {
                        v0 += bias[c];
                        v1 += bias[c + 1];
                    }
                    if (MODE == 0) {
                        v0 = fmaxf(v0, 0.f);
                        v1 = fmaxf(v1, 0.f);
                    }
                    if (MODE == 2) {
                        const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + gv * COUT + c);
                        if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                    }
                    if (MODE == 1) {
                        *reinterpret_cast<float2*>(static_cast<float*>(out) + gv * COUT + c) = make_float2(v0, v1);
                    } else {
                        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(out) + gv * COUT + c) =
                            __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
    }
}

// --------------------------------------------------------------------------
// Weight gradient: dW[o][co][ci] += sum_v dz[v][co] * x[v + off(o)][ci].
// One persistent CTA per SM walks 512-voxel tiles; per tile it stages the
// dz tile and the x tile with its one-cell halo once and serves all 27
// offsets from them.  The work of a tile is split into units (offset o,
// 8-channel ci block nt), each a COUT x 8 block of dW; warp w owns units
// w, w + 16, ... and accumulates them over all its tiles in registers,
// then stores them to the CTA's own slice of part ([gridDim.x][27][COUT]
// [CIN]); sum_partials adds the slices to dW in CTA order, so the result
// does not depend on which CTA finishes first.
// The bias gradient sum_v dz[v][co] rides along: each thread adds up one
// channel's values of every staged dz tile (thread t: channel t % COUT),
// and the CTA stores its per-channel sums to partb[blockIdx.x][COUT].
template <int CIN, int COUT>
__global__ void __launch_bounds__(NTHR, 1)
wgrad_kernel(const __nv_bfloat16* __restrict__ dz, const __nv_bfloat16* __restrict__ x, float* __restrict__ part,
             float* __restrict__ partb, int D, int H, int W)
{
    constexpr int SZ = COUT + 8, SXC = CIN + 8;
    constexpr int MT = COUT / 16;                       // m16 tiles over co
    constexpr int NT = CIN / 8;                         // n8 blocks over ci
    constexpr int NU = 27 * NT;                         // units per tile
    constexpr int UPW = (NU + NWARP - 1) / NWARP;       // units per warp (at most)
    static_assert(COUT % 16 == 0 && CIN % 16 == 0, "channel counts are multiples of 16");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* sZ = reinterpret_cast<__nv_bfloat16*>(smem_raw);        // [TV][SZ]
    __nv_bfloat16* sX = sZ + TV * SZ;                                       // [HV][SXC]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tilesx = W / TX, tilesy = H / TY, tilesz = D / TZ;
    const int ntiles = tilesx * tilesy * tilesz;

    float bacc = 0.f;
    float acc[UPW][MT][4];
#pragma unroll
    for (int i = 0; i < UPW; ++i)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][mt][q] = 0.f;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bx = tile % tilesx, by = (tile / tilesx) % tilesy, bz = tile / (tilesx * tilesy);
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * TZ;
        __syncthreads();
        for (int t = tid; t < TV * (COUT / 8); t += NTHR) {
            const int m = t / (COUT / 8), ch = t % (COUT / 8);
            const int tx = m % TX, ty = (m / TX) % TY, tz = m / (TX * TY);
            const int64_t gv = ((int64_t)(z0 + tz) * H + (y0 + ty)) * W + (x0 + tx);
            cp16(smem_u32(sZ + m * SZ + ch * 8), dz + gv * COUT + ch * 8);
        }
        for (int t = tid; t < HV * (CIN / 8); t += NTHR) {
            const int hv = t / (CIN / 8), ch = t % (CIN / 8);
            const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
            const int gz = wrapi(z0 + hz - 1, D), gy = wrapi(y0 + hy - 1, H), gx = wrapi(x0 + hx - 1, W);
            const int64_t gv = ((int64_t)gz * H + gy) * W + gx;
            cp16(smem_u32(sX + hv * SXC + ch * 8), x + gv * CIN + ch * 8);
        }
        cp_commit();
        cp_wait_all();
        __syncthreads();
#pragma unroll 8
        for (int m = tid / COUT; m < TV; m += NTHR / COUT) bacc += __bfloat162float(sZ[m * SZ + tid % COUT]);
        for (int ks = 0; ks < TV / 16; ++ks) {
            const int v0 = ks * 16;                      // one x-row of the tile
            const int ty = (v0 / TX) % TY, tz = v0 / (TX * TY);
            // A = dz^T (m = co, k = v): transpose-load rows v of sZ
            unsigned a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int q = lane >> 3, r = lane & 7;
                const int vrow = v0 + r + 8 * (q >> 1);
                const int cobase = mt * 16 + 8 * (q & 1);
                ldsm_x4_t(smem_u32(sZ + vrow * SZ + cobase), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
            }
            // B = x shifted by the unit's offset (k = v, n = ci block)
            const int rr = (lane & 7) + 8 * ((lane >> 3) & 1);
            const int hvrow = ((tz + 1) * HY + (ty + 1)) * HX + rr + 1;
#pragma unroll
            for (int i = 0; i < UPW; ++i) {
                const int u = warp + i * NWARP;
                if (u < NU) {
                    const int o = u / NT, nt = u % NT;
                    const int dhv = ((o / 9 - 1) * HY + ((o / 3) % 3 - 1)) * HX + (o % 3 - 1);
                    unsigned b0, b1;
                    ldsm_x2_t(smem_u32(sX + (hvrow + dhv) * SXC + nt * 8), b0, b1);
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
                        mma16816(acc[i][mt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                }
            }
        }
    }
    // rows co = mt*16 + lane/4 (+8), columns ci = nt*8 + 2(lane%4) + {0, 1}
#pragma unroll
    for (int i = 0; i < UPW; ++i) {
        const int u = warp + i * NWARP;
        if (u >= NU) continue;
        const int o = u / NT, nt = u % NT;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = mt * 16 + (lane >> 2) + 8 * h;
                const int ci = nt * 8 + 2 * (lane & 3);
                float* dst = part + (int64_t)blockIdx.x * (27 * COUT * CIN) + ((int64_t)o * COUT + co) * CIN + ci;
                *reinterpret_cast<float2*>(dst) = make_float2(acc[i][mt][2 * h], acc[i][mt][2 * h + 1]);
            }
    }
    // the bias sums: NTHR / COUT threads per channel, added in thread order
    __syncthreads();
    float* red = reinterpret_cast<float*>(smem_raw);
    red[tid] = bacc;
    __syncthreads();
    if (tid < COUT) {
        float t = 0.f;
        for (int k = 0; k < NTHR / COUT; ++k) t += red[k * COUT + tid];
        partb[(int64_t)blockIdx.x * COUT + tid] = t;
    }
}

// --------------------------------------------------------------------------
// Surrogate input features (channels last, 16 channels, 6 or 9 used):
//   T - 1, b_x, b_y, b_z, log10(kappa_par(T) / 0.01), dt/dt_expl / 100, and
//   with F (face fluxes of T, [3][V]) fscale * F_x, F_y, F_z.
__global__ void features_kernel(const float* __restrict__ T, const float* __restrict__ b, int64_t V, float kappa0,
                                int spitzer, float ratio, const float* __restrict__ F, float fscale,
                                __nv_bfloat16* __restrict__ X)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float t = T[v];
        const float kap = spitzer ? kappa0 * t * t * sqrtf(t) : kappa0;
        float f[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) f[c] = 0.f;
        f[0] = t - 1.f;
        f[1] = b[v];
        f[2] = b[V + v];
        f[3] = b[2 * V + v];
        f[4] = log10f(kap) + 2.f;
        f[5] = ratio * 0.01f;
        if (F) {
            f[6] = fscale * F[v];
            f[7] = fscale * F[V + v];
            f[8] = fscale * F[2 * V + v];
        }
        __nv_bfloat162* out = reinterpret_cast<__nv_bfloat162*>(X + v * 16);
#pragma unroll
        for (int c = 0; c < 8; ++c) out[c] = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
    }
}

// Flux-form head: dT[v] = -tau * sum_d (G[v][d] - G[v - e_d][d]) / dx_d (periodic).
__global__ void head_div_kernel(const float* __restrict__ G, int D, int H, int W, float tau, float idx, float idy,
                                float idz, float* __restrict__ dT)
{
    const int64_t V = (int64_t)D * H * W;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        const int64_t vx = ((int64_t)z * H + y) * W + wrapi(x - 1, W);
        const int64_t vy = ((int64_t)z * H + wrapi(y - 1, H)) * W + x;
        const int64_t vz = ((int64_t)wrapi(z - 1, D) * H + y) * W + x;
        const float div = (G[v * 16 + 0] - G[vx * 16 + 0]) * idx + (G[v * 16 + 1] - G[vy * 16 + 1]) * idy +
                          (G[v * 16 + 2] - G[vz * 16 + 2]) * idz;
        dT[v] = -tau * div;
    }
}

// MSE loss 0.5 mean((dT - target)^2): per-block FP64 partial sums of the
// squared residual, and r = (dT - target) / V stored for the adjoint.
__global__ void loss_kernel(const float* __restrict__ dT, const float* __restrict__ target, int64_t V,
                            float* __restrict__ r, double* partial)
{
    double s = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float d = dT[v] - target[v];
        r[v] = d / (float)V;
        s += (double)d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

// Adjoint of the flux-form head: dG[v][d] = -tau * (r[v] - r[v + e_d]) / dx_d
// (bf16, 16 channels, 3 used).
__global__ void head_div_adjoint_kernel(const float* __restrict__ r, int D, int H, int W, float tau, float idx,
                                        float idy, float idz, __nv_bfloat16* __restrict__ dG)
{
    const int64_t V = (int64_t)D * H * W;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        const int64_t vx = ((int64_t)z * H + y) * W + wrapi(x + 1, W);
        const int64_t vy = ((int64_t)z * H + wrapi(y + 1, H)) * W + x;
        const int64_t vz = ((int64_t)wrapi(z + 1, D) * H + y) * W + x;
        const float rv = r[v];
        const float g0 = -tau * (rv - r[vx]) * idx;
        const float g1 = -tau * (rv - r[vy]) * idy;
        const float g2 = -tau * (rv - r[vz]) * idz;
        __nv_bfloat162* out = reinterpret_cast<__nv_bfloat162*>(dG + v * 16);
        out[0] = __floats2bfloat162_rn(g0, g1);
        out[1] = __floats2bfloat162_rn(g2, 0.f);
#pragma unroll
        for (int c = 2; c < 8; ++c) out[c] = __floats2bfloat162_rn(0.f, 0.f);
    }
}

// FP32 masters [27][cout][cin] -> bf16 forward weights (same layout) and
// bf16 backward-data weights wb[o'][ci][co] = w[26 - o'][co][ci] (offset
// reversed: the adjoint gathers from v - off).
__global__ void pack_weights_kernel(const float* __restrict__ w, int cout, int cin, __nv_bfloat16* __restrict__ wf,
                                    __nv_bfloat16* __restrict__ wb)
{
    const int n = 27 * cout * cin;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int o = t / (cout * cin), co = (t / cin) % cout, ci = t % cin;
        const __nv_bfloat16 v = __float2bfloat16_rn(w[t]);
        wf[t] = v;
        if (wb) wb[((26 - o) * cin + ci) * cout + co] = v;
    }
}

// Adam on FP32 masters (bias-corrected moments, step t >= 1).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// out[i] += sum over b = 0 .. nparts - 1 of part[b][i], in that order.
__global__ void sum_partials_kernel(const float* __restrict__ part, int nparts, int n, float* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float t = 0.f;
#pragma unroll 8
        for (int b = 0; b < nparts; ++b) t += part[(int64_t)b * n + i];
        out[i] += t;
    }
}

}  // namespace

// --------------------------------------------------------------------------
// launchers

template <int CIN, int COUT, int MODE>
static cudaError_t conv_t(const void* in, const void* wt, const float* bias, const void* mask, void* out, int D, int H,
                          int W, cudaStream_t st)
{
    constexpr int SC = CIN + 8;
    const int smem = (27 * COUT * SC + HV * SC) * 2;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (D / TZ) * (H / TY) * (W / TX);
    const int grid = ntiles < sms ? ntiles : sms;
    conv_kernel<CIN, COUT, MODE><<<grid, NTHR, smem, st>>>(static_cast<const __nv_bfloat16*>(in),
                                                           static_cast<const __nv_bfloat16*>(wt), bias,
                                                           static_cast<const __nv_bfloat16*>(mask), out, D, H, W);
    return cudaGetLastError();
}

cudaError_t conv_forward(int cin, int cout, int mode, const void* in, const void* wt, const float* bias,
                         const void* mask, void* out, int D, int H, int W, cudaStream_t st)
{
    if (D % TZ || H % TY || W % TX) return cudaErrorInvalidValue;
    if (cin == 16 && cout == 32 && mode == 0) return conv_t<16, 32, 0>(in, wt, bias, mask, out, D, H, W, st);
    if (cin == 32 && cout == 32 && mode == 0) return conv_t<32, 32, 0>(in, wt, bias, mask, out, D, H, W, st);
    if (cin == 32 && cout == 16 && mode == 1) return conv_t<32, 16, 1>(in, wt, bias, mask, out, D, H, W, st);
    if (cin == 32 && cout == 32 && mode == 2) return conv_t<32, 32, 2>(in, wt, bias, mask, out, D, H, W, st);
    if (cin == 16 && cout == 32 && mode == 2) return conv_t<16, 32, 2>(in, wt, bias, mask, out, D, H, W, st);
    return cudaErrorInvalidValue;
}

static int grid_for(int64_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

cudaError_t features(const float* T, const float* b, int64_t V, float kappa0, int spitzer, float ratio, const float* F,
                     float fscale, void* X, cudaStream_t st)
{
    features_kernel<<<grid_for(V), 256, 0, st>>>(T, b, V, kappa0, spitzer, ratio, F, fscale,
                                                 static_cast<__nv_bfloat16*>(X));
    return cudaGetLastError();
}

cudaError_t head_div(const float* G, int D, int H, int W, float tau, const float inv_dx[3], float* dT, cudaStream_t st)
{
    head_div_kernel<<<grid_for((int64_t)D * H * W), 256, 0, st>>>(G, D, H, W, tau, inv_dx[0], inv_dx[1], inv_dx[2], dT);
    return cudaGetLastError();
}

cudaError_t loss_and_adjoint(const float* dT, const float* target, int D, int H, int W, float tau,
                             const float inv_dx[3], float* r, double* partial, int npartial, void* dG, cudaStream_t st)
{
    const int64_t V = (int64_t)D * H * W;
    loss_kernel<<<npartial, 256, 0, st>>>(dT, target, V, r, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    head_div_adjoint_kernel<<<grid_for(V), 256, 0, st>>>(r, D, H, W, tau, inv_dx[0], inv_dx[1], inv_dx[2],
                                                         static_cast<__nv_bfloat16*>(dG));
    return cudaGetLastError();
}

cudaError_t pack_weights(const float* w, int cout, int cin, void* wf, void* wb, cudaStream_t st)
{
    pack_weights_kernel<<<grid_for(27 * cout * cin), 256, 0, st>>>(w, cout, cin, static_cast<__nv_bfloat16*>(wf),
                                                                    static_cast<__nv_bfloat16*>(wb));
    return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, int t,
                 cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t wgrad_t(const void* dz, const void* x, float* dW, float* db, float* part, int D, int H, int W,
                           cudaStream_t st)
{
    constexpr int SZ = COUT + 8, SXC = CIN + 8;
    const int smem = (TV * SZ + HV * SXC) * 2;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = (D / TZ) * (H / TY) * (W / TX);
    const int sms = wgrad_max_ctas();
    const int grid = ntiles < sms ? ntiles : sms;
    float* partb = part + (size_t)grid * 27 * COUT * CIN;
    wgrad_kernel<CIN, COUT><<<grid, NTHR, smem, st>>>(static_cast<const __nv_bfloat16*>(dz),
                                                     static_cast<const __nv_bfloat16*>(x), part, partb, D, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<grid_for(27 * COUT * CIN), 256, 0, st>>>(part, grid, 27 * COUT * CIN, dW);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sum_partials_kernel<<<1, 32, 0, st>>>(partb, grid, COUT, db);
    return cudaGetLastError();
}

int wgrad_max_ctas()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    return sms;
}

size_t wgrad_workspace_floats() { return (size_t)wgrad_max_ctas() * (27 * 32 * 32 + 32); }

cudaError_t conv_wgrad(int cin, int cout, const void* dz, const void* x, float* dW, float* db, float* part, int D,
                       int H, int W, cudaStream_t st)
{
    if (D % TZ || H % TY || W % TX) return cudaErrorInvalidValue;
    if (cin == 16 && cout == 32) return wgrad_t<16, 32>(dz, x, dW, db, part, D, H, W, st);
    if (cin == 32 && cout == 32) return wgrad_t<32, 32>(dz, x, dW, db, part, D, H, W, st);
    if (cin == 32 && cout == 16) return wgrad_t<32, 16>(dz, x, dW, db, part, D, H, W, st);
    return cudaErrorInvalidValue;
}


}  // namespace conv
}  // namespace rkl
