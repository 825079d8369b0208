// peak.cu -- FMA issue-rate microbenchmark. The step kernels are bound by the
// FP32 (or, for FP64 rows, the FP64) arithmetic pipe, so their roofline needs
// that pipe's peak. Besides the figure derived from the unit counts and the
// clock (SMs x lanes x clock), the library measures what a register-resident
// FMA loop sustains on every SM at the clock the GPU runs at that moment.
#include <cuda_runtime.h>

#include <cstdint>

#include "api_internal.h"
#include "common.cuh"

namespace burgers {

// Each thread runs CH independent FMA chains for `iters` iterations; the
// chains' sum is stored only under a condition no run meets, which keeps them
// live. x <- x * a + b with a < 1 stays bounded.
template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_peak(T* __restrict__ sink, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + 7 * c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = tfma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == T(-1)) sink[blockIdx.x] = s;
}

}  // namespace burgers

using namespace burgers;

extern "C" burgers_status burgers_fma_peak(burgers_ctx* ctx, int32_t dtype, double* lane_fmas_per_s) {
  if (!ctx) return set_error(BURGERS_EINVAL, "ctx is NULL");
  if (!lane_fmas_per_s) return set_error(BURGERS_EINVAL, "NULL pointer");
  if (dtype != BURGERS_F32 && dtype != BURGERS_F64) return set_error(BURGERS_EINVAL, "bad dtype");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
  constexpr int CH = 8, NT = 256, PER_SM = 8;  // 2048 threads per SM
  const int grid = sms * PER_SM;
  // FP64 runs on a far narrower pipe: fewer iterations for a similar duration
  const int iters = dtype == BURGERS_F32 ? 1 << 16 : 1 << 10;
  void* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  float ms = 0.f;
  e = cudaMalloc(&sink, size_t(grid) * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
    e = cudaEventRecord(ev[0], s);
    if (e != cudaSuccess) break;
    if (dtype == BURGERS_F32)
      k_fma_peak<float, CH><<<grid, NT, 0, s>>>(static_cast<float*>(sink), iters, 0.999999f, 1e-6f);
    else
      k_fma_peak<double, CH><<<grid, NT, 0, s>>>(static_cast<double*>(sink), iters, 0.999999, 1e-6);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ctx->launches += 1;
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_error(e, "fma_peak");
  if (!(ms > 0.f)) return set_error(BURGERS_ECUDA, "fma_peak: no elapsed time");
  const double fmas = double(grid) * NT * CH * double(iters);
  *lane_fmas_per_s = fmas / (double(ms) * 1e-3);
  return BURGERS_OK;
}
