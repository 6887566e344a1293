// Device helpers shared by the trace kernels (warp / block reductions,
// compensated sums).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ctq_internal.h"

namespace ctq {
namespace dev {

constexpr double LN2 = 0.69314718055994530942;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// log(sum exp(x_i)) over a warp, every lane holding a (max, scaled-sum) pair.
__device__ __forceinline__ double warp_logsumexp(double m, double s) {
  const double gm = warp_max(m);
  double t = (m == -INFINITY) ? 0.0 : s * exp(m - gm);
  t = warp_sum(t);
  return (gm == -INFINITY || t == 0.0) ? -INFINITY : gm + log(t);
}

// Compensated (Neumaier) sum of float64 terms.
struct KSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double val() const { return s + c; }
};


// Block-wide reduction of (max, sum) pairs; every thread gets the result.
// red: 64 doubles of shared memory.
__device__ __forceinline__ void block_max_sum(double& mx, double& sm, double* red) {
  mx = warp_max(mx);
  sm = warp_sum(sm);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // red[] may still be read from the previous reduction
  if ((threadIdx.x & 31) == 0) {
    red[w] = mx;
    red[32 + w] = sm;
  }
  __syncthreads();
  mx = red[0];
  sm = red[32];
  for (int i = 1; i < nw; ++i) {
    mx = fmax(mx, red[i]);
    sm += red[32 + i];
  }
}

// Block-wide sum; every thread gets the result.  red: 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double sm, double* red) {
  sm = warp_sum(sm);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nw == 1) return sm;
  __syncthreads();  // red[] may still be read from the previous reduction
  if ((threadIdx.x & 31) == 0) red[w] = sm;
  __syncthreads();
  sm = red[0];
  for (int i = 1; i < nw; ++i) sm += red[i];
  return sm;
}

}  // namespace dev

// Kernels shared by every precision (plan_combine.cu).
int prepare_plan(int optin);
int launch_plan(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, cudaStream_t st);
int launch_combine(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, const ctq_result* R,
                   cudaStream_t st);

}  // namespace ctq
