// The learned surrogate of one RKL2 super-step (host side of the C ABI's
// rkl_sur_* entry points): a 6-layer periodic 3x3x3 convolutional network
// (6 -> 32 -> 32 -> 32 -> 32 -> 32 -> 3 face-flux channels, ReLU between
// layers, BF16 weights and activations, FP32 accumulation) whose output
// fluxes G give the increment dT = -head_scale * sum_d (G_d - G_d(-e_d)) / dx_d,
// a conservative divergence (exact energy conservation).  Training runs on
// the GPU with the library's own forward, backward and Adam kernels.  A
// super-step with the surrogate checks the prediction with one residual of
// the trapezoidal rule built from two M evaluations and falls back to the
// plain RKL2 super-step when the check fails.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rkl.h"
#include "rkl_conv.h"
#include "rkl_launch.h"

namespace rkl {
void set_unplanned_error(const std::string& msg);
const rkl_grid* plan_grid(const rkl_plan* p);
const rkl_phys* plan_phys(const rkl_plan* p);
cudaStream_t plan_stream(const rkl_plan* p);
}  // namespace rkl

using namespace rkl;

namespace {
constexpr int kLayers = 6;
constexpr int kCout[kLayers] = {32, 32, 32, 32, 32, 16};
constexpr int kCin[kLayers] = {16, 32, 32, 32, 32, 32};
constexpr int kPartials = 1024;

__global__ void axpy_kernel(const float* a, const float* b, float* out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// M = -sum_d (F_d(c) - F_d(c - e_d)) / dx_d on the periodic patch from the
// face fluxes of rkl_flux (the flux at face c + e_d / 2 stored at c): the
// conservative divergence, without evaluating the fluxes again
__global__ void div3_kernel(const float* __restrict__ F, int D, int H, int W, float ix, float iy, float iz,
                            float* __restrict__ M)
{
    const int64_t V = (int64_t)D * H * W;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < V; c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % W), y = (int)((c / W) % H), z = (int)(c / ((int64_t)W * H));
        const int64_t cx = c - x + (x == 0 ? W - 1 : x - 1);
        const int64_t cy = c + (int64_t)((y == 0 ? H - 1 : y - 1) - y) * W;
        const int64_t cz = c + (int64_t)((z == 0 ? D - 1 : z - 1) - z) * W * H;
        M[c] = -((F[c] - F[cx]) * ix + (F[V + c] - F[V + cy]) * iy + (F[2 * V + c] - F[2 * V + cz]) * iz);
    }
}

// sums of (dT - h (M0 + Mp))^2 and dT^2 in FP64, per block
__global__ void residual_kernel(const float* dT, const float* M0, const float* Mp, float h, int64_t n, double* part)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = dT[i];
        const double r = d - (double)h * ((double)M0[i] + (double)Mp[i]);
        s1 += r * r;
        s2 += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    __shared__ double sh[2][8];
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s1; sh[1][threadIdx.x >> 5] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += sh[0][w]; b += sh[1][w]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}
}  // namespace

struct rkl_surrogate {
    int D = 0, H = 0, W = 0;
    int64_t V = 0;
    double dx[3] = {1, 1, 1};
    float inv_dx[3] = {1, 1, 1};
    cudaStream_t stream = nullptr;
    int device = 0;
    // parameters: FP32 masters, gradients, Adam moments, packed BF16 copies
    float* w[kLayers] = {};
    float* b[kLayers] = {};
    float* gw[kLayers] = {};
    float* gb[kLayers] = {};
    float* mw[kLayers] = {};
    float* vw[kLayers] = {};
    float* mb[kLayers] = {};
    float* vb[kLayers] = {};
    void* wf[kLayers] = {};
    void* wb[kLayers] = {};
    int adam_t = 0;
    // activations
    void* X0 = nullptr;            // bf16 [V][16]
    void* A[kLayers - 1] = {};     // bf16 [V][32]
    float* G = nullptr;            // f32 [V][16]
    float* dT = nullptr;           // f32 [V]
    float* r = nullptr;            // f32 [V]
    void* dG = nullptr;            // bf16 [V][16]
    void* dZ[2] = {};              // bf16 [V][32]
    float* gpart = nullptr;        // per-CTA partial weight / bias gradients (fixed-order sums)
    float* F3 = nullptr;           // f32 [3][V] face fluxes of T (flux features)
    double flux_c = 0.0;           // > 0: rkl_sur_super_step feeds flux features, scale flux_c dt / head_scale
    float* Yp = nullptr;
    float* M0 = nullptr;
    float* Mp = nullptr;
    int backend = 0;               // 0: warp-level mma.sync convolutions, 1: tcgen05
    unsigned* d_tcst = nullptr;    // status word of the tcgen05 kernels' bounded waits
    double* d_part = nullptr;
    double* h_part = nullptr;      // pinned
    bool forward_done = false;
    double head_scale = 0.0;
    std::string err;
};

namespace {

rkl_status sfail(rkl_surrogate* s, rkl_status st, const std::string& m)
{
    if (s) s->err = m;
    else rkl::set_unplanned_error(m);
    return st;
}

#define SUR_CK(s, call)                                                                                   \
    do {                                                                                                  \
        cudaError_t c_ = (call);                                                                          \
        if (c_ != cudaSuccess) return sfail((s), RKL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(c_)); \
    } while (0)

size_t wcount(int l) { return (size_t)27 * kCout[l] * kCin[l]; }

// Forward (and backward-data) convolution on the selected backend.
cudaError_t conv_fwd(rkl_surrogate* s, int cin, int cout, int mode, const void* in, const void* wt, const float* bias,
                     const void* mask, void* out)
{
    if (s->backend == 1)
        return conv::conv_forward_tc(cin, cout, mode, in, wt, bias, mask, out, s->D, s->H, s->W, 8, s->d_tcst,
                                     s->stream);
    return conv::conv_forward(cin, cout, mode, in, wt, bias, mask, out, s->D, s->H, s->W, s->stream);
}

rkl_status forward_impl(rkl_surrogate* s, double head_scale)
{
    const int D = s->D, H = s->H, W = s->W;
    const void* in = s->X0;
    for (int l = 0; l < kLayers - 1; ++l) {
        SUR_CK(s, conv_fwd(s, kCin[l], kCout[l], 0, in, s->wf[l], s->b[l], nullptr, s->A[l]));
        in = s->A[l];
    }
    SUR_CK(s, conv_fwd(s, 32, 16, 1, in, s->wf[kLayers - 1], s->b[kLayers - 1], nullptr, s->G));
    SUR_CK(s, conv::head_div(s->G, D, H, W, (float)head_scale, s->inv_dx, s->dT, s->stream));
    s->forward_done = true;
    s->head_scale = head_scale;
    return RKL_OK;
}

rkl_status backward_impl(rkl_surrogate* s, const float* target, double* loss)
{
    const int D = s->D, H = s->H, W = s->W;
    SUR_CK(s, conv::loss_and_adjoint(s->dT, target, D, H, W, (float)s->head_scale, s->inv_dx, s->r, s->d_part,
                                     kPartials, s->dG, s->stream));
    SUR_CK(s, cudaMemcpyAsync(s->h_part, s->d_part, sizeof(double) * kPartials, cudaMemcpyDeviceToHost, s->stream));
    for (int l = 0; l < kLayers; ++l) {
        SUR_CK(s, cudaMemsetAsync(s->gw[l], 0, sizeof(float) * wcount(l), s->stream));
        SUR_CK(s, cudaMemsetAsync(s->gb[l], 0, sizeof(float) * kCout[l], s->stream));
    }
    // head
    const void* dz = s->dG;
    SUR_CK(s, conv::conv_wgrad(32, 16, dz, s->A[4], s->gw[5], s->gb[5], s->gpart, D, H, W, s->stream));
    SUR_CK(s, conv_fwd(s, 16, 32, 2, dz, s->wb[5], nullptr, s->A[4], s->dZ[0]));
    int cur = 0;
    for (int l = kLayers - 2; l >= 0; --l) {
        dz = s->dZ[cur];
        const void* x = l > 0 ? s->A[l - 1] : s->X0;
        SUR_CK(s, conv::conv_wgrad(kCin[l], 32, dz, x, s->gw[l], s->gb[l], s->gpart, D, H, W, s->stream));
        if (l > 0) {
            SUR_CK(s, conv_fwd(s, 32, 32, 2, dz, s->wb[l], nullptr, s->A[l - 1], s->dZ[1 - cur]));
            cur = 1 - cur;
        }
    }
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    double acc = 0.0;
    for (int k = 0; k < kPartials; ++k) acc += s->h_part[k];
    if (loss) *loss = 0.5 * acc / (double)s->V;
    return RKL_OK;
}

rkl_status pack_impl(rkl_surrogate* s, int l)
{
    SUR_CK(s, conv::pack_weights(s->w[l], kCout[l], kCin[l], s->wf[l], s->wb[l], s->stream));
    return RKL_OK;
}

}  // namespace

extern "C" {

rkl_status rkl_sur_layer_shape(int layer, int* cout, int* cin)
{
    if (layer < 0 || layer >= kLayers || !cout || !cin) return RKL_ERR_INVALID_ARG;
    *cout = kCout[layer];
    *cin = kCin[layer];
    return RKL_OK;
}

rkl_status rkl_sur_create(int D, int H, int W, const double* dx, void* cuda_stream, rkl_surrogate** out)
{
    if (!out || !dx) return sfail(nullptr, RKL_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (D < 4 || H < 8 || W < 16 || D % 4 || H % 8 || W % 16 || (int64_t)D * H * W > ((int64_t)1 << 28))
        return sfail(nullptr, RKL_ERR_INVALID_ARG, "patch must be D % 4 == H % 8 == W % 16 == 0, at most 2^28 cells");
    for (int d = 0; d < 3; ++d)
        if (!(dx[d] > 0.0) || !std::isfinite(dx[d])) return sfail(nullptr, RKL_ERR_INVALID_ARG, "bad dx");
    rkl_surrogate* s = new rkl_surrogate();
    s->D = D; s->H = H; s->W = W;
    s->backend = (W % 8 == 0 && H % 16 == 0) ? 1 : 0;     // tcgen05 where the blocks tile the patch
    s->V = (int64_t)D * H * W;
    for (int d = 0; d < 3; ++d) {
        s->dx[d] = dx[d];
        s->inv_dx[d] = (float)(1.0 / dx[d]);
    }
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&s->device);
    auto bail = [&](cudaError_t c, const char* w) {
        std::string m = std::string(w) + ": " + cudaGetErrorString(c);
        rkl_sur_destroy(s);
        return sfail(nullptr, c == cudaErrorMemoryAllocation ? RKL_ERR_NOMEM : RKL_ERR_CUDA, m);
    };
    cudaError_t c;
    for (int l = 0; l < kLayers; ++l) {
        const size_t n = wcount(l), nb = kCout[l];
        float** f[] = {&s->w[l], &s->gw[l], &s->mw[l], &s->vw[l]};
        for (auto p : f) {
            if ((c = cudaMalloc(p, sizeof(float) * n)) != cudaSuccess) return bail(c, "params");
            if ((c = cudaMemsetAsync(*p, 0, sizeof(float) * n, s->stream)) != cudaSuccess) return bail(c, "params");
        }
        float** fb[] = {&s->b[l], &s->gb[l], &s->mb[l], &s->vb[l]};
        for (auto p : fb) {
            if ((c = cudaMalloc(p, sizeof(float) * nb)) != cudaSuccess) return bail(c, "bias");
            if ((c = cudaMemsetAsync(*p, 0, sizeof(float) * nb, s->stream)) != cudaSuccess) return bail(c, "bias");
        }
        if ((c = cudaMalloc(&s->wf[l], 2 * n)) != cudaSuccess) return bail(c, "packed");
        if ((c = cudaMalloc(&s->wb[l], 2 * n)) != cudaSuccess) return bail(c, "packed");
    }
    const int64_t V = s->V;
    if ((c = cudaMalloc(&s->X0, (size_t)V * 16 * 2)) != cudaSuccess) return bail(c, "activations");
    for (int l = 0; l < kLayers - 1; ++l)
        if ((c = cudaMalloc(&s->A[l], (size_t)V * 32 * 2)) != cudaSuccess) return bail(c, "activations");
    if ((c = cudaMalloc(&s->G, (size_t)V * 16 * 4)) != cudaSuccess) return bail(c, "head");
    if ((c = cudaMalloc(&s->dT, (size_t)V * 4)) != cudaSuccess) return bail(c, "dT");
    if ((c = cudaMalloc(&s->r, (size_t)V * 4)) != cudaSuccess) return bail(c, "r");
    if ((c = cudaMalloc(&s->dG, (size_t)V * 16 * 2)) != cudaSuccess) return bail(c, "dG");
    for (int k = 0; k < 2; ++k)
        if ((c = cudaMalloc(&s->dZ[k], (size_t)V * 32 * 2)) != cudaSuccess) return bail(c, "dZ");
    if ((c = cudaMalloc(&s->Yp, (size_t)V * 4)) != cudaSuccess) return bail(c, "Yp");
    if ((c = cudaMalloc(&s->M0, (size_t)V * 4)) != cudaSuccess) return bail(c, "M0");
    if ((c = cudaMalloc(&s->Mp, (size_t)V * 4)) != cudaSuccess) return bail(c, "Mp");
    if ((c = cudaMalloc(&s->F3, (size_t)V * 12)) != cudaSuccess) return bail(c, "flux features");
    if ((c = cudaMalloc(&s->d_part, sizeof(double) * 2 * kPartials)) != cudaSuccess) return bail(c, "partials");
    if ((c = cudaMalloc(&s->gpart, sizeof(float) * conv::wgrad_workspace_floats())) != cudaSuccess)
        return bail(c, "gradient partials");
    if ((c = cudaMalloc(&s->d_tcst, sizeof(unsigned))) != cudaSuccess) return bail(c, "status");
    if ((c = cudaMemsetAsync(s->d_tcst, 0, sizeof(unsigned), s->stream)) != cudaSuccess) return bail(c, "status");
    if ((c = cudaMallocHost(&s->h_part, sizeof(double) * 2 * kPartials)) != cudaSuccess) return bail(c, "partials");
    if ((c = cudaStreamSynchronize(s->stream)) != cudaSuccess) return bail(c, "sync");
    for (int l = 0; l < kLayers; ++l)
        if (pack_impl(s, l) != RKL_OK) return bail(cudaGetLastError(), "pack");
    *out = s;
    return RKL_OK;
}

rkl_status rkl_sur_destroy(rkl_surrogate* s)
{
    if (!s) return RKL_ERR_INVALID_ARG;
    cudaStreamSynchronize(s->stream);
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(s->w[l]); cudaFree(s->b[l]); cudaFree(s->gw[l]); cudaFree(s->gb[l]);
        cudaFree(s->mw[l]); cudaFree(s->vw[l]); cudaFree(s->mb[l]); cudaFree(s->vb[l]);
        cudaFree(s->wf[l]); cudaFree(s->wb[l]);
    }
    cudaFree(s->X0);
    for (int l = 0; l < kLayers - 1; ++l) cudaFree(s->A[l]);
    cudaFree(s->G); cudaFree(s->dT); cudaFree(s->r); cudaFree(s->dG);
    cudaFree(s->dZ[0]); cudaFree(s->dZ[1]);
    cudaFree(s->Yp); cudaFree(s->M0); cudaFree(s->Mp); cudaFree(s->F3);
    cudaFree(s->d_part);
    cudaFree(s->gpart);
    cudaFree(s->d_tcst);
    if (s->h_part) cudaFreeHost(s->h_part);
    delete s;
    return RKL_OK;
}

const char* rkl_sur_last_error(const rkl_surrogate* s) { return s ? s->err.c_str() : ""; }

rkl_status rkl_sur_set_params(rkl_surrogate* s, int layer, const float* w_host, const float* b_host)
{
    if (!s || layer < 0 || layer >= kLayers || !w_host || !b_host) return RKL_ERR_INVALID_ARG;
    SUR_CK(s, cudaMemcpyAsync(s->w[layer], w_host, sizeof(float) * wcount(layer), cudaMemcpyHostToDevice, s->stream));
    SUR_CK(s, cudaMemcpyAsync(s->b[layer], b_host, sizeof(float) * kCout[layer], cudaMemcpyHostToDevice, s->stream));
    rkl_status st = pack_impl(s, layer);
    if (st != RKL_OK) return st;
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    return RKL_OK;
}

rkl_status rkl_sur_get_params(rkl_surrogate* s, int layer, float* w_host, float* b_host)
{
    if (!s || layer < 0 || layer >= kLayers || !w_host || !b_host) return RKL_ERR_INVALID_ARG;
    SUR_CK(s, cudaMemcpyAsync(w_host, s->w[layer], sizeof(float) * wcount(layer), cudaMemcpyDeviceToHost, s->stream));
    SUR_CK(s, cudaMemcpyAsync(b_host, s->b[layer], sizeof(float) * kCout[layer], cudaMemcpyDeviceToHost, s->stream));
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    return RKL_OK;
}

rkl_status rkl_sur_get_grads(rkl_surrogate* s, int layer, float* gw_host, float* gb_host)
{
    if (!s || layer < 0 || layer >= kLayers || !gw_host || !gb_host) return RKL_ERR_INVALID_ARG;
    SUR_CK(s, cudaMemcpyAsync(gw_host, s->gw[layer], sizeof(float) * wcount(layer), cudaMemcpyDeviceToHost, s->stream));
    SUR_CK(s, cudaMemcpyAsync(gb_host, s->gb[layer], sizeof(float) * kCout[layer], cudaMemcpyDeviceToHost, s->stream));
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    return RKL_OK;
}

rkl_status rkl_sur_features(rkl_surrogate* s, const void* T, const void* b, double kappa0, int spitzer, double ratio)
{
    if (!s || !T || !b) return RKL_ERR_INVALID_ARG;
    if (!(kappa0 > 0.0) || !(ratio > 0.0)) return sfail(s, RKL_ERR_INVALID_ARG, "kappa0 and ratio must be > 0");
    SUR_CK(s, conv::features(static_cast<const float*>(T), static_cast<const float*>(b), s->V, (float)kappa0,
                             spitzer ? 1 : 0, (float)ratio, nullptr, 0.f, s->X0, s->stream));
    s->forward_done = false;
    return RKL_OK;
}

namespace {
rkl_status check_patch_plan(rkl_surrogate* s, rkl_plan* plan)
{
    const rkl_grid& g = *plan_grid(plan);
    if (g.ndim != 3 || g.dtype != RKL_F32 || g.bc != RKL_PERIODIC || g.n[0] != s->W || g.n[1] != s->H ||
        g.n[2] != s->D)
        return sfail(s, RKL_ERR_INVALID_ARG, "plan must be the surrogate's periodic 3D FP32 patch");
    return RKL_OK;
}
}  // namespace

rkl_status rkl_sur_features_flux(rkl_surrogate* s, rkl_plan* plan, const void* T, const void* b, double ratio,
                                 double flux_scale)
{
    if (!s || !plan || !T || !b) return RKL_ERR_INVALID_ARG;
    if (!(ratio > 0.0) || !std::isfinite(flux_scale)) return sfail(s, RKL_ERR_INVALID_ARG, "bad ratio or scale");
    rkl_status st = check_patch_plan(s, plan);
    if (st != RKL_OK) return st;
    const rkl_phys& ph = *plan_phys(plan);
    st = rkl_flux(plan, T, b, s->F3, s->F3 + s->V, s->F3 + 2 * s->V);
    if (st != RKL_OK) return sfail(s, st, "flux of the plan failed");
    SUR_CK(s, conv::features(static_cast<const float*>(T), static_cast<const float*>(b), s->V, (float)ph.kappa_par0,
                             ph.kappa_model == RKL_KAPPA_SPITZER ? 1 : 0, (float)ratio, s->F3, (float)flux_scale,
                             s->X0, s->stream));
    s->forward_done = false;
    return RKL_OK;
}

rkl_status rkl_sur_set_flux_features(rkl_surrogate* s, double c)
{
    if (!s || !(c >= 0.0) || !std::isfinite(c)) return RKL_ERR_INVALID_ARG;
    s->flux_c = c;
    return RKL_OK;
}

rkl_status rkl_sur_set_backend(rkl_surrogate* s, int backend)
{
    if (!s) return RKL_ERR_INVALID_ARG;
    if (backend != 0 && backend != 1) return sfail(s, RKL_ERR_INVALID_ARG, "backend must be 0 or 1");
    if (backend == 1 && (s->W % 8 != 0 || s->H % 16 != 0))
        return sfail(s, RKL_ERR_UNSUPPORTED, "the tcgen05 convolutions need W % 8 == 0 and H % 16 == 0");
    s->backend = backend;
    return RKL_OK;
}

rkl_status rkl_sur_check(rkl_surrogate* s)
{
    if (!s) return RKL_ERR_INVALID_ARG;
    unsigned w = 0;
    SUR_CK(s, cudaMemcpyAsync(&w, s->d_tcst, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    SUR_CK(s, cudaMemsetAsync(s->d_tcst, 0, sizeof(unsigned), s->stream));
    if (w & ST_TIMEOUT) return sfail(s, RKL_ERR_TIMEOUT, "a bounded wait of a tensor-core convolution gave up");
    return RKL_OK;
}

rkl_status rkl_sur_forward(rkl_surrogate* s, double head_scale, void* dT_out)
{
    if (!s) return RKL_ERR_INVALID_ARG;
    rkl_status st = forward_impl(s, head_scale);
    if (st != RKL_OK) return st;
    if (dT_out) SUR_CK(s, cudaMemcpyAsync(dT_out, s->dT, sizeof(float) * s->V, cudaMemcpyDeviceToDevice, s->stream));
    return RKL_OK;
}

rkl_status rkl_sur_backward(rkl_surrogate* s, const void* target, double* loss)
{
    if (!s || !target) return RKL_ERR_INVALID_ARG;
    if (!s->forward_done) return sfail(s, RKL_ERR_INVALID_ARG, "run rkl_sur_forward first");
    return backward_impl(s, static_cast<const float*>(target), loss);
}

rkl_status rkl_sur_adam(rkl_surrogate* s, double lr, double beta1, double beta2, double eps)
{
    if (!s || !(lr > 0.0)) return RKL_ERR_INVALID_ARG;
    s->adam_t += 1;
    for (int l = 0; l < kLayers; ++l) {
        SUR_CK(s, conv::adam(s->w[l], s->gw[l], s->mw[l], s->vw[l], (int)wcount(l), (float)lr, (float)beta1,
                             (float)beta2, (float)eps, s->adam_t, s->stream));
        SUR_CK(s, conv::adam(s->b[l], s->gb[l], s->mb[l], s->vb[l], kCout[l], (float)lr, (float)beta1, (float)beta2,
                             (float)eps, s->adam_t, s->stream));
        rkl_status st = pack_impl(s, l);
        if (st != RKL_OK) return st;
    }
    return RKL_OK;
}

rkl_status rkl_sur_train_step(rkl_surrogate* s, double head_scale, const void* target, double lr, double* loss)
{
    if (!s || !target) return RKL_ERR_INVALID_ARG;
    rkl_status st = forward_impl(s, head_scale);
    if (st != RKL_OK) return st;
    st = backward_impl(s, static_cast<const float*>(target), loss);
    if (st != RKL_OK) return st;
    return rkl_sur_adam(s, lr, 0.9, 0.999, 1e-8);
}

rkl_status rkl_sur_layer_forward(rkl_surrogate* s, int layer, const void* in, void* out)
{
    if (!s || layer < 0 || layer >= kLayers || !in || !out) return RKL_ERR_INVALID_ARG;
    const int mode = layer == kLayers - 1 ? 1 : 0;
    SUR_CK(s, conv_fwd(s, kCin[layer], kCout[layer], mode, in, s->wf[layer], s->b[layer], nullptr, out));
    return RKL_OK;
}

rkl_status rkl_sur_layer_backward_data(rkl_surrogate* s, int layer, const void* dz, const void* mask, void* out)
{
    if (!s || layer < 1 || layer >= kLayers || !dz || !mask || !out) return RKL_ERR_INVALID_ARG;
    SUR_CK(s, conv_fwd(s, kCout[layer], kCin[layer], 2, dz, s->wb[layer], nullptr, mask, out));
    return RKL_OK;
}

rkl_status rkl_sur_layer_weight_grad(rkl_surrogate* s, int layer, const void* dz, const void* x)
{
    if (!s || layer < 0 || layer >= kLayers || !dz || !x) return RKL_ERR_INVALID_ARG;
    SUR_CK(s, cudaMemsetAsync(s->gw[layer], 0, sizeof(float) * wcount(layer), s->stream));
    SUR_CK(s, cudaMemsetAsync(s->gb[layer], 0, sizeof(float) * kCout[layer], s->stream));
    SUR_CK(s, conv::conv_wgrad(kCin[layer], kCout[layer], dz, x, s->gw[layer], s->gb[layer], s->gpart, s->D, s->H,
                               s->W, s->stream));
    return RKL_OK;
}

rkl_status rkl_sur_super_step(rkl_surrogate* s, rkl_plan* plan, double dt, void* T, const void* b,
                              double head_scale, double threshold, int* accepted, double* residual, int* s_used)
{
    if (!s || !plan || !T || !b || !accepted) return RKL_ERR_INVALID_ARG;
    const rkl_phys& ph = *plan_phys(plan);
    rkl_status st = check_patch_plan(s, plan);
    if (st != RKL_OK) return st;
    double dte = 0.0;
    st = rkl_dt_expl(plan, T, &dte);
    if (st != RKL_OK) return st;
    if (s->flux_c > 0.0 && !(head_scale > 0.0))
        return sfail(s, RKL_ERR_INVALID_ARG, "flux features need head_scale > 0");
    if (s->flux_c > 0.0)
        st = rkl_sur_features_flux(s, plan, T, b, dt / dte, s->flux_c * dt / head_scale);
    else
        st = rkl_sur_features(s, T, b, ph.kappa_par0, ph.kappa_model == RKL_KAPPA_SPITZER, dt / dte);
    if (st != RKL_OK) return st;
    st = forward_impl(s, head_scale);
    if (st != RKL_OK) return st;
    // residual of the trapezoidal rule: dT - (dt / 2) (M(Y0) + M(Y0 + dT)), relative to dT
    axpy_kernel<<<1024, 256, 0, s->stream>>>(static_cast<const float*>(T), s->dT, s->Yp, s->V);
    SUR_CK(s, cudaGetLastError());
    if (s->flux_c > 0.0) {
        // the flux features left T's face fluxes in F3: M(Y0) is their
        // divergence, so the check evaluates M only once, at Y0 + dT
        div3_kernel<<<1024, 256, 0, s->stream>>>(s->F3, s->D, s->H, s->W, s->inv_dx[0], s->inv_dx[1], s->inv_dx[2],
                                                 s->M0);
        SUR_CK(s, cudaGetLastError());
    } else {
        st = rkl_apply_M(plan, T, b, s->M0);
        if (st != RKL_OK) return st;
    }
    st = rkl_apply_M(plan, s->Yp, b, s->Mp);
    if (st != RKL_OK) return st;
    residual_kernel<<<kPartials, 256, 0, s->stream>>>(s->dT, s->M0, s->Mp, (float)(0.5 * dt), s->V, s->d_part);
    SUR_CK(s, cudaGetLastError());
    SUR_CK(s, cudaMemcpyAsync(s->h_part, s->d_part, sizeof(double) * 2 * kPartials, cudaMemcpyDeviceToHost,
                              s->stream));
    SUR_CK(s, cudaStreamSynchronize(s->stream));
    double n1 = 0.0, n2 = 0.0;
    for (int k = 0; k < kPartials; ++k) {
        n1 += s->h_part[2 * k];
        n2 += s->h_part[2 * k + 1];
    }
    const double rho = n2 > 0.0 ? std::sqrt(n1 / n2) : INFINITY;
    if (residual) *residual = rho;
    if (rho <= threshold && std::isfinite(rho)) {
        SUR_CK(s, cudaMemcpyAsync(T, s->Yp, sizeof(float) * s->V, cudaMemcpyDeviceToDevice, s->stream));
        *accepted = 1;
        if (s_used) *s_used = 0;
        return RKL_OK;
    }
    *accepted = 0;
    return rkl_super_step(plan, dt, T, b, s_used, nullptr, nullptr);
}

}  // extern "C"
