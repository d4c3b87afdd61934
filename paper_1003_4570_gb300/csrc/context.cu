// Context: device, stream, last error, small work buffers.
#include "omen_internal.h"

extern "C" omen_status omen_create(omen_ctx** out, int device, void* stream) {
  if (!out) return OMEN_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return OMEN_ECUDA;
  }
  if (device < 0 || device >= ndev) return OMEN_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OMEN_ECUDA;
  auto* c = new omen_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->work_bytes = 1 << 20;
  if (cudaMalloc(&c->d_work, c->work_bytes) != cudaSuccess || cudaMalloc(&c->d_status, 64 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    omen_destroy(c);
    return OMEN_ENOMEM;
  }
  *out = c;
  return OMEN_OK;
}

extern "C" void omen_destroy(omen_ctx* c) {
  if (!c) return;
  cudaFree(c->d_work);
  cudaFree(c->d_status);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaStream_t st : c->copy_stream)
    if (st) cudaStreamDestroy(st);
  if (c->host_scratch) cudaFree(c->host_scratch);
  for (cudaEvent_t e : c->host_events) cudaEventDestroy(e);
  delete c;
}

extern "C" omen_status omen_set_reorthogonalization(omen_ctx* c, int policy) {
  if (!c) return OMEN_EINVAL;
  if (policy != OMEN_REORTH_FULL && policy != OMEN_REORTH_SEMI && policy != OMEN_REORTH_PARTIAL)
    return set_err(c, OMEN_EINVAL, "unknown policy %d", policy);
  c->reorth = policy;
  return OMEN_OK;
}

extern "C" omen_status omen_set_locking_check(omen_ctx* c, int enable) {
  if (!c) return OMEN_EINVAL;
  c->lock_check = enable != 0;
  return OMEN_OK;
}

extern "C" omen_status omen_set_graph_capture(omen_ctx* c, int enable) {
  if (!c) return OMEN_EINVAL;
  c->use_graphs = enable != 0;
  return OMEN_OK;
}

extern "C" const char* omen_last_error(const omen_ctx* c) { return c ? c->err.c_str() : "null context"; }
