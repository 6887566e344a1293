// Throughput probes for the arithmetic pipes that bound the small-block trace
// (FP64 and FP32 fused multiply-add, and the FP64 warp-level MMA
// mma.sync.m8n8k4.f64), and an accuracy hook for the propagators' table
// exponential.  Used to state the ALU roofline of the FP64 path; they compute
// nothing of the trace itself.
#include <cuda_runtime.h>

#include <vector>

#include "ctq_internal.h"
#include "exp_tang.cuh"

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

// 8 independent accumulator chains per warp of D(8x8) += A(8x4) B(4x8) in
// float64 (256 multiply-adds per instruction).
__global__ void k_dmma_rate(double* out, int iters, double x) {
  const double a = x * double(threadIdx.x + 1), b = x;
  double d[8][2];
#pragma unroll
  for (int j = 0; j < 8; ++j) d[j][0] = d[j][1] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[j][0]), "+d"(d[j][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += d[j][0] + d[j][1];
  if (s == -12345.0) out[blockIdx.x] = s;
}

__global__ void k_exp_check(const double* x, double* y_table, double* y_lib, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    y_table[i] = dev::exp_nonpos(x[i]);
    y_lib[i] = exp(x[i]);
  }
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

namespace ctq {
namespace {

int run_dmma_probe(int device, int iters, double* flops_per_s) {
  int prev = 0;
  cudaGetDevice(&prev);
  if (device != prev && cudaSetDevice(device) != cudaSuccess) return CTQ_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int threads = 256, blocks = sms * 8;
  double* out = nullptr;
  int st = CTQ_OK;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) st = CTQ_ERR_NOMEM;
  if (st == CTQ_OK) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dmma_rate<<<blocks, threads>>>(out, iters / 10 + 1, 1e-3);  // warm-up
    cudaEventRecord(e0);
    k_dmma_rate<<<blocks, threads>>>(out, iters, 1e-3);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = CTQ_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    // per warp and instruction: 8 x 8 x 4 multiply-adds
    *flops_per_s = 2.0 * 256.0 * 8.0 * double(iters) * (threads / 32) * blocks / (double(ms) * 1e-3);
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
  if (!flops_per_s || iters < 1 || kind < 0 || kind > 2) return CTQ_ERR_ARG;
  if (kind == 2) return ctq::run_dmma_probe(device, iters, flops_per_s);
  return kind == 0 ? ctq::run_probe<double>(device, iters, flops_per_s)
                   : ctq::run_probe<float>(device, iters, flops_per_s);
}

extern "C" int ctq_probe_exp(int device, int n, const double* x, double* y_table, double* y_lib) {
  if (n < 0 || (n > 0 && (!x || !y_table || !y_lib))) return CTQ_ERR_ARG;
  if (n == 0) return CTQ_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (device != prev && cudaSetDevice(device) != cudaSuccess) return CTQ_ERR_CUDA;
  double* d = nullptr;
  int st = CTQ_OK;
  const size_t b = size_t(n) * sizeof(double);
  if (cudaMalloc(&d, 3 * b) != cudaSuccess) st = CTQ_ERR_NOMEM;
  if (st == CTQ_OK) {
    if (cudaMemcpy(d, x, b, cudaMemcpyHostToDevice) != cudaSuccess) st = CTQ_ERR_CUDA;
    if (st == CTQ_OK) {
      ctq::k_exp_check<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256>>>(d, d + n, d + 2 * size_t(n), n);
      if (cudaGetLastError() != cudaSuccess || cudaMemcpy(y_table, d + n, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(y_lib, d + 2 * size_t(n), b, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = CTQ_ERR_CUDA;
    }
    cudaFree(d);
  }
  if (device != prev) cudaSetDevice(prev);
  return st;
}
