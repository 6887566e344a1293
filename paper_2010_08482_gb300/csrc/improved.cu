// Static part of the improved estimator for the self-energy
// (Sec. 2.4, Eq. PImprovedEstimatorStatic): h^st = w^U / w_loc, the local
// weight with one annihilator c_f(tau) replaced by the Bulla operator
// [c_f, U](tau) over the plain local weight, from two evaluated batches.
#include <cuda_runtime.h>

#include <cmath>

#include "ctq_internal.h"

namespace ctq {
namespace {

// One thread per replaced sequence i: w^U_i = phase_u e^{log_abs_u},
// w = phase e^{log_abs} (|phase| = 1), so h = e^{log_abs_u - log_abs}
// phase_u conj(phase).
__global__ void k_static_ratios(int m, int n_chains, const int* __restrict__ chain,
                                const double* __restrict__ log_abs, const double* __restrict__ phase,
                                const double* __restrict__ log_abs_u, const double* __restrict__ phase_u,
                                double* __restrict__ h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int c = chain[i];
  double hr = NAN, hi = NAN;
  if (c >= 0 && c < n_chains) {
    const double la = log_abs[c], lu = log_abs_u[i];
    const bool w_ok = !isnan(la) && la != -INFINITY;
    if (w_ok && lu == -INFINITY) {
      hr = 0.0;
      hi = 0.0;
    } else if (w_ok && !isnan(lu)) {
      const double r = exp(lu - la);
      const double ar = phase[2 * c], ai = phase[2 * c + 1];
      const double br = phase_u[2 * size_t(i)], bi = phase_u[2 * size_t(i) + 1];
      hr = r * (br * ar + bi * ai);
      hi = r * (bi * ar - br * ai);
    }
  }
  h[2 * size_t(i)] = hr;
  h[2 * size_t(i) + 1] = hi;
}

}  // namespace

int launch_static_ratios(int m, const int* chain, int n_chains, const double* log_abs, const double* phase,
                         const double* log_abs_u, const double* phase_u, double* h, void* stream) {
  if (m == 0) return CTQ_OK;
  const int threads = 256;
  const int grid = (m + threads - 1) / threads;
  k_static_ratios<<<grid, threads, 0, static_cast<cudaStream_t>(stream)>>>(m, n_chains, chain, log_abs, phase,
                                                                           log_abs_u, phase_u, h);
  return cudaGetLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

}  // namespace ctq
