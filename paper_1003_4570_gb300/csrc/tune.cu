// Launch-shape tuner for the H·X kernels.  The tile shape of a product (CTA width; block rows
// per register batch, or wave vectors per thread in the k batch) trades memory-level
// parallelism against registers and occupancy, and the best choice moves with the basis,
// precision and structure.  The tuner times every compiled shape on the Hamiltonian itself
// (CUDA events on the context's stream, after warm-up launches) and keeps the fastest.  No
// shape changes the result: each accumulator sums its terms in the same order.
#include <vector>

#include "omen_internal.h"

bool hx_tile_valid(const omen_ham* h, int vec_precision, int threads, int rb);
bool hx_kbatch_tile_valid(int vec_precision, int threads, int kb);

namespace {

__global__ void tune_fill_kernel(float* p, long long nwords) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (long long)gridDim.x * blockDim.x)
    p[i] = 1.0f / (float)(1 + (i % 13));
}

int prec_slot(int vec_precision) { return vec_precision == OMEN_F64 ? 0 : 1; }

bool has_blocks(const omen_ham* h, int vec_precision) {
  if (h->matrix_free) return true;
  return vec_precision == OMEN_F64 ? h->d_blk64 != nullptr : h->d_blk32 != nullptr;
}

struct Scratch {
  omen_ctx* ctx;
  void* p = nullptr;
  ~Scratch() { if (p) cudaFreeAsync(p, ctx->stream); }
};

// average milliseconds of `reps` launches after two warm-up launches
template <typename F>
omen_status time_launches(omen_ctx* ctx, int reps, F&& launch, double& ms) {
  for (int i = 0; i < 2; ++i) {
    omen_status s = launch();
    if (s != OMEN_OK) return s;
  }
  cudaEvent_t e0, e1;
  OMEN_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_err(ctx, OMEN_ECUDA, "event creation failed");
  }
  omen_status s = OMEN_OK;
  cudaEventRecord(e0, ctx->stream);
  for (int i = 0; i < reps && s == OMEN_OK; ++i) s = launch();
  cudaEventRecord(e1, ctx->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != OMEN_OK) return s;
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "tuner timing: %s", cudaGetErrorString(e));
  ms = t / reps;
  return OMEN_OK;
}

// Time every candidate (threads, rb) with `launch`, set the fastest through `set`.
template <typename L, typename S>
omen_status tune_loop(omen_ctx* ctx, const std::vector<HxTile>& cand, int reps, L&& launch, S&& set,
                      omen_tune_result* out) {
  double best = 0.0, dflt = 0.0;
  HxTile pick;
  int timed = 0;
  for (const HxTile& t : cand) {
    set(t);
    double ms = 0.0;
    omen_status s = time_launches(ctx, reps, launch, ms);
    if (s != OMEN_OK) {
      set(HxTile{});
      return s;
    }
    if (t.threads == 0 && t.rb == 0) dflt = ms;
    if (timed == 0 || ms < best) {
      best = ms;
      pick = t;
    }
    ++timed;
  }
  set(pick);
  if (out) {
    out->threads = pick.threads ? pick.threads : 128;
    out->rows_per_batch = pick.rb;
    out->candidates = timed;
    out->ms_best = best;
    out->ms_default = dflt;
  }
  return OMEN_OK;
}

}  // namespace

extern "C" omen_status omen_hx_set_tile(omen_ctx* ctx, omen_ham* h, int vec_precision, int threads, int rb) {
  if (!ctx || !h) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "the effective-mass product has one launch shape");
  if (vec_precision != OMEN_F64 && vec_precision != OMEN_F32) return set_err(ctx, OMEN_EINVAL, "vector precision must be F64 or F32");
  if (!hx_tile_valid(h, vec_precision, threads, rb))
    return set_err(ctx, OMEN_EINVAL, "launch shape (%d threads, %d rows per batch) is not compiled for this Hamiltonian", threads, rb);
  h->tile[prec_slot(vec_precision)] = HxTile{threads, rb};
  return OMEN_OK;
}

extern "C" omen_status omen_hx_kbatch_set_tile(omen_ctx* ctx, omen_ham* h, int vec_precision, int threads, int kb) {
  if (!ctx || !h) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs on tight-binding Hamiltonians");
  if (vec_precision != OMEN_F64 && vec_precision != OMEN_F32) return set_err(ctx, OMEN_EINVAL, "vector precision must be F64 or F32");
  if (!hx_kbatch_tile_valid(vec_precision, threads, kb))
    return set_err(ctx, OMEN_EINVAL, "k-batch launch shape (%d threads, %d wave vectors per thread) is not compiled", threads, kb);
  h->ktile[prec_slot(vec_precision)] = HxTile{threads, kb};
  return OMEN_OK;
}

extern "C" omen_status omen_tune_hx(omen_ctx* ctx, omen_ham* h, int vec_precision, int nvec, int reps,
                                    omen_tune_result* out) {
  if (!ctx || !h || nvec < 1 || nvec > 65535 || reps < 1) return set_err(ctx, OMEN_EINVAL, "null argument, nvec or reps out of range");
  if (vec_precision != OMEN_F64 && vec_precision != OMEN_F32) return set_err(ctx, OMEN_EINVAL, "vector precision must be F64 or F32");
  if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "the effective-mass product has one launch shape");
  if (!has_blocks(h, vec_precision)) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no blocks of that precision");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t bytes = vec_elem_bytes(h, vec_precision) * (size_t)h->nrows * nvec;
  Scratch sx{ctx}, sy{ctx};
  if (cudaMallocAsync(&sx.p, bytes, ctx->stream) != cudaSuccess || cudaMallocAsync(&sy.p, bytes, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "tuner vectors (%zu bytes each)", bytes);
  }
  tune_fill_kernel<<<1216, 256, 0, ctx->stream>>>(static_cast<float*>(sx.p), (long long)(bytes / 4));
  OMEN_CHECK_LAUNCH(ctx);
  std::vector<HxTile> cand{HxTile{}};
  for (int thr : {32, 64, 96, 128})
    for (int rb : {0, 1, 2, 5, 10})
      if (hx_tile_valid(h, vec_precision, thr, rb)) cand.push_back(HxTile{thr, rb});
  const int slot = prec_slot(vec_precision);
  return tune_loop(
      ctx, cand, reps, [&]() { return launch_hx(ctx, h, sx.p, sy.p, nvec, 0.0, vec_precision); },
      [&](HxTile t) { h->tile[slot] = t; }, out);
}

extern "C" omen_status omen_tune_hx_kbatch(omen_ctx* ctx, omen_ham* h, int nk, int reps, omen_tune_result* out) {
  if (!ctx || !h || nk < 1 || nk > 65535 || reps < 1) return set_err(ctx, OMEN_EINVAL, "null argument, nk or reps out of range");
  if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs on tight-binding Hamiltonians");
  if (!h->bloch || h->spin_orbit || h->matrix_free) return set_err(ctx, OMEN_EINVAL, "k batch needs a Bloch Hamiltonian with stored blocks and no spin-orbit");
  const int prec = h->precision == OMEN_F32 ? OMEN_F32 : OMEN_F64;
  if (!has_blocks(h, prec)) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no blocks of its precision");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t bytes = vec_elem_bytes(h, prec) * (size_t)h->nrows * nk;
  Scratch sx{ctx}, sy{ctx};
  if (cudaMallocAsync(&sx.p, bytes, ctx->stream) != cudaSuccess || cudaMallocAsync(&sy.p, bytes, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "tuner vectors (%zu bytes each)", bytes);
  }
  tune_fill_kernel<<<1216, 256, 0, ctx->stream>>>(static_cast<float*>(sx.p), (long long)(bytes / 4));
  OMEN_CHECK_LAUNCH(ctx);
  std::vector<double> k((size_t)nk * 3);
  for (int q = 0; q < nk; ++q) {
    k[(size_t)q * 3 + 0] = 0.37 * q / nk;
    k[(size_t)q * 3 + 1] = -0.21 * q / nk;
    k[(size_t)q * 3 + 2] = 0.0;
  }
  double2* ph = nullptr;
  omen_status s = make_phases(ctx, h, nk, k.data(), &ph);
  if (s != OMEN_OK) return s;
  std::vector<HxTile> cand{HxTile{}};
  for (int thr : {32, 64, 96, 128})
    for (int kb : {1, 2, 4})
      if (hx_kbatch_tile_valid(prec, thr, kb)) cand.push_back(HxTile{thr, kb});
  const int slot = prec_slot(prec);
  s = tune_loop(
      ctx, cand, reps, [&]() { return launch_hx_kbatch(ctx, h, nk, ph, sx.p, sy.p, 0.0, prec); },
      [&](HxTile t) { h->ktile[slot] = t; }, out);
  cudaFreeAsync(ph, ctx->stream);
  return s;
}
