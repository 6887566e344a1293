// Throughput probe for the arithmetic pipes that bound the small-block trace
// (FP64 and FP32 fused multiply-add).  Used to state the ALU roofline of the
// FP64 path; it computes nothing of the trace itself.
#include <cuda_runtime.h>

#include "ctq_internal.h"

namespace ctq {
namespace {

template <typename T>
__global__ void k_fma_rate(T* out, int iters, T x, T y) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], x, y);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == T(-12345.0)) out[blockIdx.x] = s;  // keeps the loop alive
}

template <typename T>
int run_probe(int device, int iters, double* flops_per_s) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (device != prev && cudaSetDevice(device) != cudaSuccess) return CTQ_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int threads = 256, blocks = sms * 8;
  T* out = nullptr;
  int st = CTQ_OK;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&out, blocks * sizeof(T)) != cudaSuccess) st = CTQ_ERR_NOMEM;
  if (st == CTQ_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_rate<T><<<blocks, threads>>>(out, iters / 10 + 1, T(0.999), T(1e-4));  // warm-up
    cudaEventRecord(e0);
    k_fma_rate<T><<<blocks, threads>>>(out, iters, T(0.999), T(1e-4));
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = CTQ_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *flops_per_s = 2.0 * 8.0 * double(iters) * threads * blocks / (double(ms) * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
  }
  if (device != prev) cudaSetDevice(prev);
  return st;
}

}  // namespace
}  // namespace ctq

extern "C" int ctq_probe_fma_rate(int device, int kind, int iters, double* flops_per_s) {
  if (!flops_per_s || iters < 1 || (kind != 0 && kind != 1)) return CTQ_ERR_ARG;
  return kind == 0 ? ctq::run_probe<double>(device, iters, flops_per_s)
                   : ctq::run_probe<float>(device, iters, flops_per_s);
}
