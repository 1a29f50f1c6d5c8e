// Host launchers of the surrogate's kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rkl {
namespace conv {

// out = act(bias + conv3x3x3_periodic(in, wt)); patch D x H x W with D % 4,
// H % 8, W % 16 == 0.  (cin, cout, mode) in {(16,32,0), (32,32,0),
// (32,16,1), (32,32,2), (16,32,2)}; mode 0 ReLU bf16 out, 1 linear f32 out,
// 2 no bias, result times (mask > 0), bf16 out.
cudaError_t conv_forward(int cin, int cout, int mode, const void* in, const void* wt, const float* bias,
                         const void* mask, void* out, int D, int H, int W, cudaStream_t st);
// The same convolutions on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in TMEM): W % 8 == 0, H % 16 == 0, nzc planes per CTA.  A
// bounded wait that gives up sets ST_TIMEOUT in *status (may be NULL).
cudaError_t conv_forward_tc(int cin, int cout, int mode, const void* in, const void* wt, const float* bias,
                            const void* mask, void* out, int D, int H, int W, int nzc, unsigned* status,
                            cudaStream_t st);
// dW[27][cout][cin] += sum_v dz[v][cout] x[v + off][cin] and db[cout] +=
// sum_v dz[v][cout]; (cin, cout) in {(16,32), (32,32), (32,16)}.  Each CTA
// writes its partial sums to its own slice of part
// (wgrad_workspace_floats() floats), which are then added to dW and db in
// a fixed order: the result is the same from run to run.
int wgrad_max_ctas();
size_t wgrad_workspace_floats();
cudaError_t conv_wgrad(int cin, int cout, const void* dz, const void* x, float* dW, float* db, float* part, int D,
                       int H, int W, cudaStream_t st);

cudaError_t features(const float* T, const float* b, int64_t V, float kappa0, int spitzer, float ratio, const float* F,
                     float fscale, void* X, cudaStream_t st);
cudaError_t head_div(const float* G, int D, int H, int W, float tau, const float inv_dx[3], float* dT,
                     cudaStream_t st);
cudaError_t loss_and_adjoint(const float* dT, const float* target, int D, int H, int W, float tau,
                             const float inv_dx[3], float* r, double* partial, int npartial, void* dG,
                             cudaStream_t st);
cudaError_t pack_weights(const float* w, int cout, int cin, void* wf, void* wb, cudaStream_t st);
cudaError_t adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, int t,
                 cudaStream_t st);

}  // namespace conv
}  // namespace rkl
