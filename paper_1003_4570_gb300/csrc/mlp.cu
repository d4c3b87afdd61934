// Learned warm start for the self-consistent loop: a 3-layer perceptron that maps the doping
// profile to the self-consistent electrostatic potential (no counterpart in the paper, whose
// Section III-A loop starts from a given potential; here the network's output is that start,
// and the zero-field start remains the fallback).
//
//   x (n_in)  -> h1 = tanh(W1 x + b1) -> h2 = tanh(W2 h1 + b2) -> y = W3 h2 + b3 (n_out)
//
// Weights are used as BF16 copies in the forward and backward products with FP32
// accumulation; FP32 master weights take the Adam update (Kingma & Ba 2015) and are rounded to
// the BF16 copies after every step.  Loss: mean squared error over batch and outputs.
// The layers are small (under 0.6 GFLOP per batch of 256), so the products are tiled SIMT
// kernels; their cost is launch latency, not tensor throughput.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "omen_internal.h"

struct omen_mlp {
  int d[4];
  double x_shift, x_scale, y_scale;
  float* W32[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16* W16[3] = {nullptr, nullptr, nullptr};
  float* b[3] = {nullptr, nullptr, nullptr};
  float* mW[3] = {nullptr, nullptr, nullptr};
  float* vW[3] = {nullptr, nullptr, nullptr};
  float* mb[3] = {nullptr, nullptr, nullptr};
  float* vb[3] = {nullptr, nullptr, nullptr};
  float* gW[3] = {nullptr, nullptr, nullptr};
  float* gb[3] = {nullptr, nullptr, nullptr};
  long long step = 0;
  int cap = 0;                              // batch capacity of the activation buffers
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *G1 = nullptr, *G2 = nullptr, *G3 = nullptr;
  float* part = nullptr;                    // loss partial sums
};

static constexpr int TM = 64, TN = 64, TK = 16;

template <typename TB> __device__ __forceinline__ float ld(const TB* p) { return (float)(*p); }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C(m, n) = sum_k A(m, k) B(k, n) with A(m,k) = A[m*ars + k*acs], B(k,n) = B[k*brs + n*bcs].
// EPI 0: store; 1: + bias[n], tanh; 2: + bias[n].
template <typename TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, long long ars,
                                                   long long acs, const TB* __restrict__ B, long long brs, long long bcs,
                                                   float* __restrict__ C, long long crs, const float* __restrict__ bias) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int mm = e % TM, kk = e / TM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(size_t)m * ars + (size_t)k * acs] : 0.f;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      const int nn = e % TN, kk = e / TN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? ld<TB>(B + (size_t)k * brs + (size_t)n * bcs) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI >= 1) v += bias[n];
      if (EPI == 1) v = tanhf(v);
      C[(size_t)m * crs + n] = v;
    }
  }
}

// dY = 2 (Y - T) / (B n); per-block partial sums of (Y - T)^2
__global__ void mse_kernel(const float* __restrict__ Y, const float* __restrict__ T, long long total, float scale,
                           float* __restrict__ dY, float* __restrict__ part) {
  float s = 0.f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.f * d * scale;
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    part[blockIdx.x] = t;
  }
}

// G <- G * (1 - H^2)  (derivative of tanh through its output)
__global__ void tanh_back_kernel(float* __restrict__ G, const float* __restrict__ H, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    G[i] *= 1.f - H[i] * H[i];
}

// db[o] = sum_b G[b][o]
__global__ void colsum_kernel(const float* __restrict__ G, int B, int n, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += G[(size_t)b * n + o];
  db[o] = s;
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                            __nv_bfloat16* __restrict__ w16, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16_rn(w[i]);
}

__global__ void from_bf16_kernel(const __nv_bfloat16* __restrict__ w16, float* __restrict__ w, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w[i] = __bfloat162float(w16[i]);
}

// Profile on the grid's interior planes (lateral mean) sampled at z_j = (j + 1/2) Lz / n by linear
// interpolation, with 0 on the z = 0 and z = Lz planes.
__device__ __forceinline__ double plane_mean(const double* f, int nx, int ny, int k) {
  double s = 0.0;
  for (int i = 0; i < nx * ny; ++i) s += f[(size_t)(k - 1) * nx * ny + i];
  return s / (nx * ny);
}
__device__ __forceinline__ double sample_profile(const double* f, int nx, int ny, int nz, double t) {
  // t in plane units (0..nz)
  int k0 = (int)floor(t);
  k0 = max(0, min(k0, nz - 1));
  const double w = t - k0;
  const double a = (k0 >= 1 && k0 <= nz - 1) ? plane_mean(f, nx, ny, k0) : 0.0;
  const double b = (k0 + 1 >= 1 && k0 + 1 <= nz - 1) ? plane_mean(f, nx, ny, k0 + 1) : 0.0;
  return (1.0 - w) * a + w * b;
}

__global__ void features_kernel(const double* __restrict__ rho, int nx, int ny, int nz, int n, double shift, double scale,
                                float* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double t = (j + 0.5) * nz / n;
  const double nd = sample_profile(rho, nx, ny, nz, t) / 1.602176634e-19;   // donors per m^3
  x[j] = (float)((log10(fmax(nd, 1e15)) - shift) / scale);
}

__global__ void targets_kernel(const double* __restrict__ phi, int nx, int ny, int nz, int n, double scale,
                               float* __restrict__ t_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double t = (j + 0.5) * nz / n;
  t_out[j] = (float)(sample_profile(phi, nx, ny, nz, t) / scale);
}

// phi on the interior planes from the n-point network output (linear interpolation between the
// sample points, extended to 0 V at the two grounded planes), broadcast laterally.
__global__ void inject_kernel(const float* __restrict__ y, int n, int nx, int ny, int nz, double scale,
                              double* __restrict__ phi) {
  const long long total = (long long)nx * ny * (nz - 1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / ((long long)nx * ny)) + 1;      // plane index 1..nz-1
    const double u = (double)k * n / nz - 0.5;              // position in sample units
    double v;
    if (u <= 0.0) {
      const double w = (u + 0.5) / 0.5;                     // from 0 V at z = 0 to sample 0
      v = w * y[0];
    } else if (u >= n - 1) {
      const double w = (n - 0.5 - u) / 0.5;
      v = w * y[n - 1];
    } else {
      const int j = (int)floor(u);
      const double w = u - j;
      v = (1.0 - w) * y[j] + w * y[j + 1];
    }
    phi[i] = v * scale;
  }
}

static unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

template <typename TB, int EPI>
static void gemm(cudaStream_t st, int M, int N, int K, const float* A, long long ars, long long acs, const TB* B,
                 long long brs, long long bcs, float* C, long long crs, const float* bias) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, ars, acs, B, brs, bcs, C, crs, bias);
}

static void free_mlp(omen_mlp* m) {
  for (int l = 0; l < 3; ++l) {
    cudaFree(m->W32[l]); cudaFree(m->W16[l]); cudaFree(m->b[l]);
    cudaFree(m->mW[l]); cudaFree(m->vW[l]); cudaFree(m->mb[l]); cudaFree(m->vb[l]);
    cudaFree(m->gW[l]); cudaFree(m->gb[l]);
  }
  cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->Y); cudaFree(m->G1); cudaFree(m->G2); cudaFree(m->G3); cudaFree(m->part);
}

extern "C" void omen_mlp_free(omen_mlp* m) {
  if (!m) return;
  free_mlp(m);
  delete m;
}

extern "C" long long omen_mlp_param_count(const omen_mlp* m) {
  if (!m) return 0;
  long long n = 0;
  for (int l = 0; l < 3; ++l) n += (long long)m->d[l + 1] * m->d[l] + m->d[l + 1];
  return n;
}

extern "C" omen_status omen_mlp_create(omen_ctx* ctx, const omen_mlp_desc* desc, const float* params, omen_mlp** out) {
  if (!ctx || !desc || !params || !out) return set_err(ctx, OMEN_EINVAL, "null argument");
  *out = nullptr;
  const int d[4] = {desc->n_in, desc->n_hidden1, desc->n_hidden2, desc->n_out};
  for (int i = 0; i < 4; ++i)
    if (d[i] < 1 || d[i] > 8192) return set_err(ctx, OMEN_EINVAL, "layer width out of range");
  if (!(desc->feat_log10_scale > 0) || !(desc->target_scale > 0)) return set_err(ctx, OMEN_EINVAL, "scales must be > 0");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* m = new omen_mlp();
  for (int i = 0; i < 4; ++i) m->d[i] = d[i];
  m->x_shift = desc->feat_log10_shift;
  m->x_scale = desc->feat_log10_scale;
  m->y_scale = desc->target_scale;
  bool ok = true;
  size_t off = 0;
  for (int l = 0; l < 3 && ok; ++l) {
    const size_t nw = (size_t)d[l + 1] * d[l], nb = d[l + 1];
    ok = cudaMalloc(&m->W32[l], nw * 4) == cudaSuccess && cudaMalloc(&m->W16[l], nw * 2) == cudaSuccess &&
         cudaMalloc(&m->b[l], nb * 4) == cudaSuccess && cudaMalloc(&m->mW[l], nw * 4) == cudaSuccess &&
         cudaMalloc(&m->vW[l], nw * 4) == cudaSuccess && cudaMalloc(&m->mb[l], nb * 4) == cudaSuccess &&
         cudaMalloc(&m->vb[l], nb * 4) == cudaSuccess && cudaMalloc(&m->gW[l], nw * 4) == cudaSuccess &&
         cudaMalloc(&m->gb[l], nb * 4) == cudaSuccess;
    if (!ok) break;
    cudaMemcpyAsync(m->W32[l], params + off, nw * 4, cudaMemcpyHostToDevice, ctx->stream);
    off += nw;
    cudaMemcpyAsync(m->b[l], params + off, nb * 4, cudaMemcpyHostToDevice, ctx->stream);
    off += nb;
    cudaMemsetAsync(m->mW[l], 0, nw * 4, ctx->stream);
    cudaMemsetAsync(m->vW[l], 0, nw * 4, ctx->stream);
    cudaMemsetAsync(m->mb[l], 0, nb * 4, ctx->stream);
    cudaMemsetAsync(m->vb[l], 0, nb * 4, ctx->stream);
    to_bf16_kernel<<<grid_for(nw), 256, 0, ctx->stream>>>(m->W32[l], m->W16[l], nw);
  }
  if (!ok || cudaMalloc(&m->part, 4096 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    omen_mlp_free(m);
    return set_err(ctx, OMEN_ENOMEM, "network parameters");
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    omen_mlp_free(m);
    return set_err(ctx, OMEN_ECUDA, "network upload: %s", cudaGetErrorString(e));
  }
  *out = m;
  return OMEN_OK;
}

static omen_status ensure_batch(omen_ctx* ctx, omen_mlp* m, int B) {
  if (B <= m->cap) return OMEN_OK;
  cudaFree(m->H1); cudaFree(m->H2); cudaFree(m->Y); cudaFree(m->G1); cudaFree(m->G2); cudaFree(m->G3);
  m->H1 = m->H2 = m->Y = m->G1 = m->G2 = m->G3 = nullptr;
  m->cap = 0;
  const size_t b = (size_t)B;
  if (cudaMalloc(&m->H1, b * m->d[1] * 4) != cudaSuccess || cudaMalloc(&m->H2, b * m->d[2] * 4) != cudaSuccess ||
      cudaMalloc(&m->Y, b * m->d[3] * 4) != cudaSuccess || cudaMalloc(&m->G1, b * m->d[1] * 4) != cudaSuccess ||
      cudaMalloc(&m->G2, b * m->d[2] * 4) != cudaSuccess || cudaMalloc(&m->G3, b * m->d[3] * 4) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "activation buffers for batch %d", B);
  }
  m->cap = B;
  return OMEN_OK;
}

static void forward(cudaStream_t st, omen_mlp* m, const float* X, int B, float* Y) {
  const int* d = m->d;
  gemm<__nv_bfloat16, 1>(st, B, d[1], d[0], X, d[0], 1, m->W16[0], 1, d[0], m->H1, d[1], m->b[0]);
  gemm<__nv_bfloat16, 1>(st, B, d[2], d[1], m->H1, d[1], 1, m->W16[1], 1, d[1], m->H2, d[2], m->b[1]);
  gemm<__nv_bfloat16, 2>(st, B, d[3], d[2], m->H2, d[2], 1, m->W16[2], 1, d[2], Y, d[3], m->b[2]);
}

// forward + loss + gradients into m->gW/gb; loss (mean squared error) to *loss
static omen_status backward(omen_ctx* ctx, omen_mlp* m, const float* X, const float* T, int B, float* loss) {
  cudaStream_t st = ctx->stream;
  const int* d = m->d;
  forward(st, m, X, B, m->Y);
  const long long ny = (long long)B * d[3];
  const unsigned gm = std::min<unsigned>(grid_for(ny), 4096u);
  mse_kernel<<<gm, 256, 0, st>>>(m->Y, T, ny, 1.f / (float)ny, m->G3, m->part);
  // layer 3: dW3 = G3^T H2, db3 = colsum G3, G2 = G3 W3
  gemm<float, 0>(st, d[3], d[2], B, m->G3, 1, d[3], m->H2, d[2], 1, m->gW[2], d[2], nullptr);
  colsum_kernel<<<(d[3] + 255) / 256, 256, 0, st>>>(m->G3, B, d[3], m->gb[2]);
  gemm<__nv_bfloat16, 0>(st, B, d[2], d[3], m->G3, d[3], 1, m->W16[2], d[2], 1, m->G2, d[2], nullptr);
  tanh_back_kernel<<<grid_for((long long)B * d[2]), 256, 0, st>>>(m->G2, m->H2, (long long)B * d[2]);
  // layer 2
  gemm<float, 0>(st, d[2], d[1], B, m->G2, 1, d[2], m->H1, d[1], 1, m->gW[1], d[1], nullptr);
  colsum_kernel<<<(d[2] + 255) / 256, 256, 0, st>>>(m->G2, B, d[2], m->gb[1]);
  gemm<__nv_bfloat16, 0>(st, B, d[1], d[2], m->G2, d[2], 1, m->W16[1], d[1], 1, m->G1, d[1], nullptr);
  tanh_back_kernel<<<grid_for((long long)B * d[1]), 256, 0, st>>>(m->G1, m->H1, (long long)B * d[1]);
  // layer 1
  gemm<float, 0>(st, d[1], d[0], B, m->G1, 1, d[1], X, d[0], 1, m->gW[0], d[0], nullptr);
  colsum_kernel<<<(d[1] + 255) / 256, 256, 0, st>>>(m->G1, B, d[1], m->gb[0]);
  OMEN_CHECK_LAUNCH(ctx);
  if (loss) {
    std::vector<float> hp(gm);
    OMEN_CUDA(ctx, cudaMemcpyAsync(hp.data(), m->part, gm * sizeof(float), cudaMemcpyDeviceToHost, st));
    OMEN_CUDA(ctx, cudaStreamSynchronize(st));
    double s = 0.0;
    for (float v : hp) s += v;
    *loss = (float)(s / (double)ny);
  }
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_forward(omen_ctx* ctx, omen_mlp* m, const float* X, int B, float* Y) {
  if (!ctx || !m || !X || !Y || B < 1) return set_err(ctx, OMEN_EINVAL, "null argument or batch < 1");
  omen_status s = ensure_batch(ctx, m, B);
  if (s != OMEN_OK) return s;
  forward(ctx->stream, m, X, B, Y);
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_gradients(omen_ctx* ctx, omen_mlp* m, const float* X, const float* T, int B,
                                          float* grad_host, float* loss_host) {
  if (!ctx || !m || !X || !T || B < 1) return set_err(ctx, OMEN_EINVAL, "null argument or batch < 1");
  omen_status s = ensure_batch(ctx, m, B);
  if (s != OMEN_OK) return s;
  s = backward(ctx, m, X, T, B, loss_host);
  if (s != OMEN_OK) return s;
  if (grad_host) {
    size_t off = 0;
    for (int l = 0; l < 3; ++l) {
      const size_t nw = (size_t)m->d[l + 1] * m->d[l], nb = m->d[l + 1];
      OMEN_CUDA(ctx, cudaMemcpyAsync(grad_host + off, m->gW[l], nw * 4, cudaMemcpyDeviceToHost, ctx->stream));
      off += nw;
      OMEN_CUDA(ctx, cudaMemcpyAsync(grad_host + off, m->gb[l], nb * 4, cudaMemcpyDeviceToHost, ctx->stream));
      off += nb;
    }
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_train_step(omen_ctx* ctx, omen_mlp* m, const float* X, const float* T, int B, double lr,
                                           float* loss_host) {
  if (!ctx || !m || !X || !T || B < 1 || !(lr > 0)) return set_err(ctx, OMEN_EINVAL, "invalid training arguments");
  omen_status s = ensure_batch(ctx, m, B);
  if (s != OMEN_OK) return s;
  s = backward(ctx, m, X, T, B, loss_host);
  if (s != OMEN_OK) return s;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
  for (int l = 0; l < 3; ++l) {
    const long long nw = (long long)m->d[l + 1] * m->d[l], nb = m->d[l + 1];
    adam_kernel<<<grid_for(nw), 256, 0, ctx->stream>>>(m->W32[l], m->mW[l], m->vW[l], m->gW[l], m->W16[l], nw, (float)lr, b1, b2, eps, c1, c2);
    adam_kernel<<<grid_for(nb), 256, 0, ctx->stream>>>(m->b[l], m->mb[l], m->vb[l], m->gb[l], nullptr, nb, (float)lr, b1, b2, eps, c1, c2);
  }
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_get_params(omen_ctx* ctx, const omen_mlp* m, float* params, int bf16_rounded) {
  if (!ctx || !m || !params) return set_err(ctx, OMEN_EINVAL, "null argument");
  size_t off = 0;
  float* tmp = nullptr;
  for (int l = 0; l < 3; ++l) {
    const size_t nw = (size_t)m->d[l + 1] * m->d[l], nb = m->d[l + 1];
    if (bf16_rounded) {
      if (cudaMallocAsync(&tmp, nw * 4, ctx->stream) != cudaSuccess) { cudaGetLastError(); return set_err(ctx, OMEN_ENOMEM, "copy buffer"); }
      from_bf16_kernel<<<grid_for(nw), 256, 0, ctx->stream>>>(m->W16[l], tmp, nw);
      OMEN_CUDA(ctx, cudaMemcpyAsync(params + off, tmp, nw * 4, cudaMemcpyDeviceToHost, ctx->stream));
      cudaFreeAsync(tmp, ctx->stream);
    } else {
      OMEN_CUDA(ctx, cudaMemcpyAsync(params + off, m->W32[l], nw * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    off += nw;
    OMEN_CUDA(ctx, cudaMemcpyAsync(params + off, m->b[l], nb * 4, cudaMemcpyDeviceToHost, ctx->stream));
    off += nb;
  }
  OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return OMEN_OK;
}

static omen_status check_grid2(omen_ctx* ctx, const omen_grid* g) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 2) return set_err(ctx, OMEN_EINVAL, "invalid grid");
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_features(omen_ctx* ctx, const omen_mlp* m, const omen_grid* g, const double* rho,
                                         float* x) {
  if (!ctx || !m || !rho || !x) return set_err(ctx, OMEN_EINVAL, "null argument");
  omen_status s = check_grid2(ctx, g);
  if (s != OMEN_OK) return s;
  features_kernel<<<(m->d[0] + 255) / 256, 256, 0, ctx->stream>>>(rho, g->nx, g->ny, g->nz, m->d[0], m->x_shift, m->x_scale, x);
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_targets(omen_ctx* ctx, const omen_mlp* m, const omen_grid* g, const double* phi, float* t) {
  if (!ctx || !m || !phi || !t) return set_err(ctx, OMEN_EINVAL, "null argument");
  omen_status s = check_grid2(ctx, g);
  if (s != OMEN_OK) return s;
  targets_kernel<<<(m->d[3] + 255) / 256, 256, 0, ctx->stream>>>(phi, g->nx, g->ny, g->nz, m->d[3], m->y_scale, t);
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

extern "C" omen_status omen_mlp_warm_start(omen_ctx* ctx, omen_mlp* m, const omen_grid* g, const double* rho,
                                           double* phi) {
  if (!ctx || !m || !rho || !phi) return set_err(ctx, OMEN_EINVAL, "null argument");
  omen_status s = check_grid2(ctx, g);
  if (s != OMEN_OK) return s;
  s = ensure_batch(ctx, m, 1);
  if (s != OMEN_OK) return s;
  float* xy = nullptr;
  if (cudaMallocAsync(&xy, sizeof(float) * (m->d[0] + m->d[3]), ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "warm-start buffers");
  }
  features_kernel<<<(m->d[0] + 255) / 256, 256, 0, ctx->stream>>>(rho, g->nx, g->ny, g->nz, m->d[0], m->x_shift, m->x_scale, xy);
  forward(ctx->stream, m, xy, 1, xy + m->d[0]);
  const long long total = (long long)g->nx * g->ny * (g->nz - 1);
  inject_kernel<<<grid_for(total), 256, 0, ctx->stream>>>(xy + m->d[0], m->d[3], g->nx, g->ny, g->nz, m->y_scale, phi);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(xy, ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "warm start: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

// The learned start with the zero-field start as fallback and judge: the network's potential
// starts omen_scf; if that loop fails (iteration limit, or a start so far off that the states it
// produces cannot hold the electrons), phi is reset to zero field and the loop runs again from
// there.  info covers the run that produced phi; *fallback tells which start that was.
extern "C" omen_status omen_scf_learned(omen_ctx* ctx, const omen_scf_desc* d, omen_mlp* m, double* phi,
                                        omen_scf_info* info, int* fallback) {
  if (!ctx || !d || !m || !phi || !d->grid || !d->donor_rho_dev) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (fallback) *fallback = 0;
  omen_status s = omen_mlp_warm_start(ctx, m, d->grid, d->donor_rho_dev, phi);
  if (s != OMEN_OK) return s;
  omen_scf_info first{};
  s = omen_scf(ctx, d, phi, &first);
  if (s == OMEN_OK || (s != OMEN_ENOCONV && s != OMEN_ENUMERIC)) {
    if (info) *info = first;
    return s;
  }
  const long long ng = (long long)d->grid->nx * d->grid->ny * (d->grid->nz - 1);
  OMEN_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * ng, ctx->stream));
  if (fallback) *fallback = 1;
  omen_scf_info second{};
  s = omen_scf(ctx, d, phi, &second);
  second.seconds += first.seconds;          // the failed learned run is part of the cost
  second.eig_seconds += first.eig_seconds;
  second.poisson_seconds += first.poisson_seconds;
  second.hx_count += first.hx_count;
  if (info) *info = second;
  return s;
}
