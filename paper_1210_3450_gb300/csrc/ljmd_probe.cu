// Pipe-rate probe: the FP64 and FP32 fused multiply-add throughput of the current
// GPU, measured rather than taken from a data sheet, for the denominators of the
// FP64 force kernel's roofline (its bound is the FP64 pipe, not HBM). Not part of
// the paper's method.
//
// Every thread runs eight independent multiply-add chains (enough to keep the pipe
// busy between dependent instructions) for a run-time number of iterations, so
// the compiler can neither fold nor shorten them; the result is written only under
// a condition that never holds, so the chains are not removed either.
#include <cuda_runtime.h>

#include <string>

#include "ljmd.h"
#include "ljmd_engine.h"

namespace ljmd {
namespace {

__device__ double g_probe_sink;

template <class T>
__global__ void __launch_bounds__(256) k_probe_fma(int64_t iters, T m, T c) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)0.1, a2 = a0 + (T)0.2, a3 = a0 + (T)0.3;
  T a4 = a0 + (T)0.4, a5 = a0 + (T)0.5, a6 = a0 + (T)0.6, a7 = a0 + (T)0.7;
#pragma unroll 4
  for (int64_t k = 0; k < iters; ++k) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == (T)-1.2345) g_probe_sink = (double)s;
}

}  // namespace
}  // namespace ljmd

extern "C" int md_probe_fma_rate(int kind, int64_t iters, double* fma_per_s) {
  using namespace ljmd;
  set_error("");
  if ((kind != 0 && kind != 1) || iters < 1 || !fma_per_s) {
    set_error("md_probe_fma_rate: kind 0 (FP64) or 1 (FP32), iters >= 1, non-null output");
    return MD_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const unsigned blocks = (unsigned)sms * 8u;  // 64 warps per SM
  float ms = 0.f;
  if (e == cudaSuccess) {
    // one short launch to load the module, then the timed one
    if (kind == 0) k_probe_fma<double><<<blocks, 256>>>(1, 0.9999999, 1e-7);
    else k_probe_fma<float><<<blocks, 256>>>(1, 0.9999999f, 1e-7f);
    cudaEventRecord(t0);
    if (kind == 0) k_probe_fma<double><<<blocks, 256>>>(iters, 0.9999999, 1e-7);
    else k_probe_fma<float><<<blocks, 256>>>(iters, 0.9999999f, 1e-7f);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess || !(ms > 0.f)) {
    set_error(std::string("md_probe_fma_rate: ") + cudaGetErrorString(e));
    return MD_ERR_CUDA;
  }
  *fma_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
  return MD_OK;
}
