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

// 2^e as a float64 built from its exponent field, -1022 <= e <= 1023.
__device__ __forceinline__ double pow2i(int e) { return __hiloint2double((e + 1023) << 20, 0); }

// h + l += x with the rounding error of h + x kept in l (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_acc(double& h, double& l, double x) {
  const double s = h + x;
  const double bp = s - h;
  l += (h - (s - bp)) + (x - bp);
  h = s;
}

// Log scale of one sector string, computed by one warp with lanes over
// chunks of operators (Sec. 3.3.1 propagators: every time step dtau_j in
// sector q_j contributes -dtau_j (E_min(q_j) - E_ref) to the log of the
// product).  The chunk sums are compensated and combined by a compensated
// inclusive scan over lanes, so the total keeps the accuracy of a
// compensated sequential sum.  With tracking, every segment end (a multiple
// of S operators) is a chunk end and the scan also yields the log scale segL
// and the applied log-norm prefix segP there.
__device__ __forceinline__ void chain_log_scale(const DevModel& M, const BatchView& B, const EvalCfg& cfg, int a0, int n, int q0,
                                double t_first, double t_last, bool track, const short* path, const short* opsm,
                                double* segL, double* segP, double* out_L) {
  const int lane = threadIdx.x & 31;
  const int ns = M.n_sec;
  const double emr0 = M.E_min[q0] - M.E_ref;
  // chunk length over j = 1 .. n-1: with tracking the smallest divisor of S
  // that covers the string in one pass of 32 lanes (segment ends stay chunk
  // ends), else S; without tracking ceil((n - 1) / 32)
  int CH = max(1, (n + 30) / 32);
  if (track) {
    CH = cfg.S;
    for (int d = 1; d < cfg.S; ++d)
      if (cfg.S % d == 0 && 32 * d >= n - 1) {
        CH = d;
        break;
      }
  }
  const int nch = (n - 1 + CH - 1) / CH;
  double ch = -t_first * emr0, cl = 0.0, cp = 0.0;  // running carry (compensated) and log-norm prefix
  two_sum_acc(ch, cl, -t_last * emr0);
  for (int base = 0; base < nch; base += 32) {
    const int t = base + lane;
    double h = 0.0, l = 0.0, ps = 0.0;
    if (t < nch) {
      const int j2 = min((t + 1) * CH, n - 1);
      for (int j = t * CH + 1; j <= j2; ++j) {
        const double term = -(B.tau[a0 + j] - B.tau[a0 + j - 1]) * (M.E_min[path[j]] - M.E_ref);
        two_sum_acc(h, l, term);
        if (track) ps += term + M.log_norm[opsm[j - 1] * ns + path[j - 1]];
      }
    }
    for (int o = 1; o < 32; o <<= 1) {  // inclusive scan over the lanes
      const double oh = __shfl_up_sync(FULL, h, o), ol = __shfl_up_sync(FULL, l, o);
      const double op = __shfl_up_sync(FULL, ps, o);
      if (lane >= o) {
        two_sum_acc(h, l, oh);
        l += ol;
        ps += op;
      }
    }
    double H = ch, Lo = cl + l;
    two_sum_acc(H, Lo, h);
    const double P = cp + ps;
    if (track && t < nch && (t + 1) * CH < n && ((t + 1) * CH) % cfg.S == 0) {
      segL[(t + 1) * CH / cfg.S] = H + Lo;
      segP[(t + 1) * CH / cfg.S] = P;
    }
    ch = __shfl_sync(FULL, H, 31);
    cl = __shfl_sync(FULL, Lo, 31);
    cp = __shfl_sync(FULL, P, 31);
  }
  if (lane == 0) *out_L = ch + cl;
}

}  // namespace dev

// Kernels shared by every precision (plan_combine.cu).
int prepare_plan(int optin);
int launch_plan(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, cudaStream_t st);
int launch_combine(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, const ctq_result* R,
                   cudaStream_t st);

}  // namespace ctq
