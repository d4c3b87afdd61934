// FP64 arithmetic rate of the device (no counterpart in the paper): the bound of the FP64
// products here is GB300's FP64 pipe, not HBM, so their roofline needs its rate measured on
// the device at hand.  Every thread runs eight independent fused multiply-add chains in
// registers (enough to cover the pipe latency), one resident wave of CTAs, CUDA events around
// the launch; the chains' results are stored so the work cannot be dropped.
#include <algorithm>

#include "omen_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma64_kernel(double* __restrict__ out, int iters, double a, double b) {
  double c[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) c[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) c[i] = fma(c[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += c[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" omen_status omen_probe_fp64_rate(omen_ctx* ctx, double* tflops) {
  if (!ctx || !tflops) return set_err(ctx, OMEN_EINVAL, "null argument");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  int sms = 0, per_sm = 0;
  OMEN_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  OMEN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma64_kernel, 256, 0));
  const int blocks = sms * std::max(1, per_sm);
  const int iters = 4096;
  double* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(double) * blocks * 256, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "probe buffer");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, ctx->stream);
    fma64_kernel<<<blocks, 256, 0, ctx->stream>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, ctx->stream);
  const cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return set_err(ctx, OMEN_ECUDA, "FP64 probe: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  *tflops = 2.0 * (double)blocks * 256 * kChains * iters / (best * 1e-3) / 1e12;
  return OMEN_OK;
}
