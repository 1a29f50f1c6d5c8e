// dt_expl and energy without any device allocation.
//
// rkl_dt_expl and rkl_energy need a plan, and creating a plan allocates
// device memory.  Some callers cannot allocate at the point where they need
// these two numbers: a host code that hands the library a fixed device
// memory budget up front, or a time-step loop that must not stall on
// cudaMalloc / cudaFree (both may synchronise the whole device).  This file
// gives them one entry point that reduces a caller-owned temperature array
// using only a fixed scratch array that lives in the library image.
//
// The scratch is a file-scope __device__ array sized for grids of up to
// kNoAllocMaxCells cells (2^27, one 512^3 grid): 65536 partial results of
// three doubles plus the final three, about 1.5 MB.  Every GPU that loads
// the library holds it until the process exits.  All calls on a device share
// it; each call overwrites every partial it later reads, so nothing needs
// clearing, but two calls whose work overlaps on the GPU (different streams,
// no ordering between them) race on it.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/rkl.h"

namespace rkl {
void set_unplanned_error(const std::string& msg);   // defined in rkl_api.cu
}

namespace {

constexpr int64_t kNoAllocMaxCells = (int64_t)1 << 27;
constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;                 // 2048
constexpr int kMaxPartials = (int)(kNoAllocMaxCells / kCellsPerBlock);     // 65536
constexpr int kMaxDevices = 64;

// [3 * kMaxPartials] partials (max, min, sum per block) then [3] results.
__device__ __align__(256) double g_noalloc_scratch[3 * kMaxPartials + 3];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ void fold(double v, double& mx, double& mn, double& sm)
{
    mx = (v > mx || v != v) ? v : mx;
    mn = (v < mn || v != v) ? v : mn;
    sm += v;
}

__device__ __forceinline__ void warp_fold(double& mx, double& mn, double& sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double a = __shfl_xor_sync(0xffffffffu, mx, o);
        double b = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = (a > mx || a != a) ? a : mx;
        mn = (b < mn || b != b) ? b : mn;
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
}

// Block b folds cells [b * 2048, (b + 1) * 2048) into scratch[3 b .. 3 b + 2].
template <typename R>
__global__ void __launch_bounds__(kThreads) partial_kernel(const R* __restrict__ T, int64_t n, double* scratch)
{
    double mx = -INFINITY, mn = INFINITY, sm = 0.0;
    int64_t base = (int64_t)blockIdx.x * kCellsPerBlock + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kCellsPerThread; ++k) {
        int64_t c = base + (int64_t)k * kThreads;
        if (c < n) fold((double)T[c], mx, mn, sm);
    }
    warp_fold(mx, mn, sm);
    __shared__ double s[3][kThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = mx; s[1][w] = mn; s[2][w] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kThreads / 32; ++q) {
            mx = (s[0][q] > mx || s[0][q] != s[0][q]) ? s[0][q] : mx;
            mn = (s[1][q] < mn || s[1][q] != s[1][q]) ? s[1][q] : mn;
            sm += s[2][q];
        }
        scratch[3 * blockIdx.x + 0] = mx;
        scratch[3 * blockIdx.x + 1] = mn;
        scratch[3 * blockIdx.x + 2] = sm;
    }
}

// One block folds the nblk partials (fixed order) into scratch[3 kMaxPartials ..].
__global__ void __launch_bounds__(kThreads) final_kernel(double* scratch, int nblk)
{
    double mx = -INFINITY, mn = INFINITY, sm = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kThreads) {
        double a = scratch[3 * q], b = scratch[3 * q + 1];
        mx = (a > mx || a != a) ? a : mx;
        mn = (b < mn || b != b) ? b : mn;
        sm += scratch[3 * q + 2];
    }
    warp_fold(mx, mn, sm);
    __shared__ double s[3][kThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s[0][w] = mx; s[1][w] = mn; s[2][w] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kThreads / 32; ++q) {
            mx = (s[0][q] > mx || s[0][q] != s[0][q]) ? s[0][q] : mx;
            mn = (s[1][q] < mn || s[1][q] != s[1][q]) ? s[1][q] : mn;
            sm += s[2][q];
        }
        double* out = scratch + 3 * kMaxPartials;
        out[0] = mx;
        out[1] = mn;
        out[2] = sm;
    }
}

rkl_status err(rkl_status st, const std::string& msg)
{
    rkl::set_unplanned_error(msg);
    return st;
}

// Device address of the scratch array for the current device, looked up
// once per device (host code cannot use the array's name as an address).
rkl_status scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(RKL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(RKL_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(RKL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return RKL_OK;
}

}  // namespace

extern "C" rkl_status rkl_dt_expl_energy_noalloc(const rkl_grid* grid, const rkl_phys* phys, const void* T,
                                                 void* cuda_stream, double* dt_out, double* energy_out)
{
    if (!grid || !phys || !T || !dt_out || !energy_out) return err(RKL_ERR_INVALID_ARG, "null argument");
    const rkl_grid& g = *grid;
    const rkl_phys& ph = *phys;
    if (g.ndim < 1 || g.ndim > 3) return err(RKL_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
    if (g.dtype != RKL_F32 && g.dtype != RKL_F64) return err(RKL_ERR_INVALID_ARG, "bad dtype");
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
        if (g.n[d] < 1) return err(RKL_ERR_INVALID_ARG, "bad n");
        if (d >= g.ndim && g.n[d] != 1) return err(RKL_ERR_INVALID_ARG, "inactive axis must have n = 1");
        if (d < g.ndim && !(g.dx[d] > 0.0 && std::isfinite(g.dx[d])))
            return err(RKL_ERR_INVALID_ARG, "dx must be finite and > 0");
        if (g.n[d] > kNoAllocMaxCells) return err(RKL_ERR_INVALID_ARG, "grid larger than the no-allocation limit");
        n *= g.n[d];
        if (n > kNoAllocMaxCells) break;
    }
    if (n > kNoAllocMaxCells)
        return err(RKL_ERR_INVALID_ARG, "grid has more than 134217728 cells, the most the no-allocation "
                                        "scratch (static, 1.5 MB) can reduce; use rkl_dt_expl / rkl_energy");
    if (ph.kappa_model != RKL_KAPPA_CONST && ph.kappa_model != RKL_KAPPA_SPITZER)
        return err(RKL_ERR_INVALID_ARG, "bad kappa_model");
    if (!(ph.kappa_par0 > 0.0) || !std::isfinite(ph.kappa_par0) || !(ph.kappa_perp_ratio >= 0.0) ||
        !std::isfinite(ph.kappa_perp_ratio))
        return err(RKL_ERR_INVALID_ARG, "bad conductivity");
    if (!(ph.cp > 0.0 && ph.cp <= 0.5)) return err(RKL_ERR_INVALID_ARG, "cp must be in (0, 1/2]");

    double* scratch = nullptr;
    rkl_status st = scratch_for_current_device(&scratch);
    if (st != RKL_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblk = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    if (g.dtype == RKL_F64)
        partial_kernel<double><<<nblk, kThreads, 0, s>>>(static_cast<const double*>(T), n, scratch);
    else
        partial_kernel<float><<<nblk, kThreads, 0, s>>>(static_cast<const float*>(T), n, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(RKL_ERR_CUDA, std::string("partial_kernel: ") + cudaGetErrorString(e));
    final_kernel<<<1, kThreads, 0, s>>>(scratch, nblk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(RKL_ERR_CUDA, std::string("final_kernel: ") + cudaGetErrorString(e));
    double res[3] = {0.0, 0.0, 0.0};
    e = cudaMemcpyAsync(res, scratch + 3 * kMaxPartials, sizeof(res), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(RKL_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    if (!std::isfinite(res[0]) || !std::isfinite(res[1])) return err(RKL_ERR_NONFINITE, "T holds NaN or Inf");

    double Tmax = 1.0;
    if (ph.kappa_model == RKL_KAPPA_SPITZER) {
        if (!(res[1] > 0.0)) return err(RKL_ERR_NONPOSITIVE_T, "T must be > 0 under Spitzer kappa");
        Tmax = res[0];
    }
    double inv = 0.0, dV = 1.0;
    for (int d = 0; d < g.ndim; ++d) {
        inv += 1.0 / (g.dx[d] * g.dx[d]);
        dV *= g.dx[d];
    }
    double kpar = ph.kappa_model == RKL_KAPPA_SPITZER ? ph.kappa_par0 * Tmax * Tmax * std::sqrt(Tmax)
                                                       : ph.kappa_par0;
    *dt_out = ph.cp / (kpar * (1.0 + ph.kappa_perp_ratio) * inv);
    *energy_out = res[2] * dV;
    return RKL_OK;
}
