// Sector-string local trace on the GPU: the FP64 chain-product kernel.
//
// One evaluation of a batch runs three kernels on the caller's stream:
// k_plan (plan_combine.cu), k_trace (here) and k_combine (plan_combine.cu).
//
//   k_trace    persistent CTAs pull (chain, q0) items.  The product
//                Y_1 = P_1 F_1 P_wrap,  Y_i = P_i F_i Y_{i-1},
//                w_q0 = Tr(F_n Y_{n-1}) (diagonal only)
//              runs with Y resident in shared memory; P_i = diag(e^{-dtau (E - E_min)})
//              rows are applied in the GEMM epilogue (the "time-evolution
//              kernel" of Sec. 3.3.2), the wrap-around propagators of q0
//              (times tau_1 and beta - tau_n) scale the columns of the first
//              block (trace cyclicity).  After every product the max |Y| is
//              reduced across the CTA and the next product absorbs the exact
//              power-of-two rescale; the log scale (energy shifts and
//              exponents) stays in float64, relative to e^{-beta E_gs} (the
//              propagation times sum to beta) and summed with compensation,
//              so that log|w| ~ 10^3 loses no accuracy before the final
//              -beta E_gs is added.  Every `segment` operators the refined bound
//                ub = sqrt(r) ||Y||_F prod_{rest} ||F||_2 e^{-dtau E_min}
//              is recorded and, with lazy evaluation, the chain's live bound
//              sum is compared with its threshold (stop early if below).
#include "device_common.cuh"

namespace ctq {
namespace {

using namespace dev;

// ----------------------------------------------------------------------- trace

template <bool CPLX>
struct Scalar;
template <>
struct Scalar<false> {
  using T = double;
};
template <>
struct Scalar<true> {
  using T = double2;
};

__device__ __forceinline__ double mag(double v) { return fabs(v); }
__device__ __forceinline__ double mag(double2 v) { return fmax(fabs(v.x), fabs(v.y)); }
__device__ __forceinline__ double sq(double v) { return v * v; }
__device__ __forceinline__ double sq(double2 v) { return v.x * v.x + v.y * v.y; }
__device__ __forceinline__ double2 operator*(double a, double2 b) { return make_double2(a * b.x, a * b.y); }

__device__ __forceinline__ double load_blk(const double* blk, int64_t i, double) { return __ldg(blk + i); }
__device__ __forceinline__ double2 load_blk(const double* blk, int64_t i, double2) {
  return __ldg(reinterpret_cast<const double2*>(blk) + i);
}
__device__ __forceinline__ void fma_acc(double& acc, double f, double y) { acc = fma(f, y, acc); }
__device__ __forceinline__ void fma_acc(double2& acc, double2 f, double2 y) {
  acc.x = fma(f.x, y.x, acc.x);
  acc.x = fma(-f.y, y.y, acc.x);
  acc.y = fma(f.x, y.y, acc.y);
  acc.y = fma(f.y, y.x, acc.y);
}
__device__ __forceinline__ void zero(double& v) { v = 0.0; }
__device__ __forceinline__ void zero(double2& v) { v = make_double2(0.0, 0.0); }

template <bool CPLX>
__global__ void __launch_bounds__(256) k_trace(DevModel M, BatchView B, EvalCfg cfg, Work W) {
  using T = typename Scalar<CPLX>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int D = M.max_dim;
  T* Ybuf0 = reinterpret_cast<T*>(smem_raw);
  T* Ybuf1 = Ybuf0 + size_t(D) * D;
  double* p = reinterpret_cast<double*>(Ybuf1 + size_t(D) * D);  // [D] row propagators
  double* p0 = p + D;                                            // [D] wrap propagator (columns)
  double* red = p0 + D;                                          // [64] reductions
  __shared__ int s_item;
  __shared__ int s_abort;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ns = M.n_sec;
  const int n_items = W.counters[0];
  const Item* items = W.items + size_t(B.n_chains) * ns;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(&W.counters[1], 1);
    __syncthreads();
    const int it_idx = s_item;
    if (it_idx >= n_items) break;
    const Item it = items[it_idx];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);

    if (n == 0) {  // empty sequence: Tr e^{-beta H(q0)}
      double sm = 0.0, mx = 0.0;
      for (int j = tid; j < d0; j += nt) sm += exp(-B.beta * E0[j]);
      block_max_sum(mx, sm, red);
      if (tid == 0) {
        const double l = -B.beta * (M.E_min[q0] - M.E_ref);
        W.res_val[2 * slot] = sm;
        W.res_val[2 * slot + 1] = 0.0;
        W.res_log[slot] = l;
        if (track) segp[0] = log(sm) + l;
      }
      continue;
    }

    // The wrap-around propagators P_{beta - tau_n}(q0) and P_{tau_1}(q0) scale
    // the columns of the first block (trace cyclicity); the two time
    // arguments are kept separate so that no extra rounding enters them.
    const double t_first = B.tau[a0], t_last = B.beta - B.tau[a0 + n - 1];
    KSum L;                            // log scale (energy shifts, relative to E_ref)
    L.add(-t_first * (M.E_min[q0] - M.E_ref));
    L.add(-t_last * (M.E_min[q0] - M.E_ref));
    long long Eacc = 0;                // power-of-two exponent: true = stored * 2^Eacc
    for (int j = tid; j < d0; j += nt) p0[j] = exp(-t_first * E0[j]) * exp(-t_last * E0[j]);

    if (n == 1) {  // only reachable with user tables where s_alpha(q0) = q0
      __syncthreads();
      const int alpha = B.op[a0];
      const int64_t off = M.blk_off[alpha * ns + q0];
      double vr = 0.0, vi = 0.0, mx = 0.0;
      for (int j = tid; j < d0; j += nt) {
        const T f = load_blk(M.blk, off + int64_t(j) * d0 + j, T());
        if constexpr (CPLX) {
          vr += f.x * p0[j];
          vi += f.y * p0[j];
        } else {
          vr += f * p0[j];
        }
      }
      block_max_sum(mx, vr, red);
      mx = 0.0;
      block_max_sum(mx, vi, red);
      if (tid == 0) {
        const bool zero_v = (vr == 0.0 && vi == 0.0);
        W.res_val[2 * slot] = vr;
        W.res_val[2 * slot + 1] = vi;
        W.res_log[slot] = zero_v ? -INFINITY : L.val();
        if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(vr * vr + vi * vi)) + L.val();
      }
      continue;
    }

    // ---- operator 1: Y1[m][j] = p1[m] F1[m][j] p0[j]
    int qa = q0;
    int alpha = B.op[a0];
    int qb = M.s[alpha * ns + qa];
    double prefix = M.log_norm[alpha * ns + qa];  // log-norm + propagator sums of applied ops
    {
      const double dt = B.tau[a0 + 1] - B.tau[a0];
      const double* Eb = M.E_rel + M.E_off[qb];
      const int db = M.dims[qb];
      for (int m = tid; m < db; m += nt) p[m] = exp(-dt * Eb[m]);
      L.add(-dt * (M.E_min[qb] - M.E_ref));
      prefix -= dt * (M.E_min[qb] - M.E_ref);
    }
    __syncthreads();
    T* Y = Ybuf0;
    T* Yn = Ybuf1;
    int dcur = M.dims[qb];
    double mx = 0.0, fr = 0.0;
    {
      const int64_t off = M.blk_off[alpha * ns + qa];
      const int tot = dcur * d0;
      for (int idx = tid; idx < tot; idx += nt) {
        const int m = idx / d0, j = idx - m * d0;
        const T f = load_blk(M.blk, off + idx, T());
        const T v = (p[m] * p0[j]) * f;
        Y[idx] = v;
        mx = fmax(mx, mag(v));
        fr += sq(v);
      }
    }
    block_max_sum(mx, fr, red);
    qa = qb;
    int applied = 1;
    bool dead = false;
    bool aborted = false;

    // ---- operators 2 .. n-1: Y <- P F Y, previous rescale folded into P
    for (int i = 1; i < n; ++i) {
      // bookkeeping for the product that has just been stored in Y (after `applied` operators)
      if (mx == 0.0) { dead = true; break; }
      int e = ilogb(mx);
      if (track && applied % cfg.S == 0 && applied < n) {
        const double ub = 0.5 * log(double(it.r)) + 0.5 * log(fr) + double(Eacc) * LN2 + L.val() +
                          (it.t_all - prefix);
        if (tid == 0) {
          segp[applied / cfg.S] = ub;
          if (cfg.lazy) {
            W.live[slot] = fmin(W.live[slot], ub);
            __threadfence();
          }
        }
        if (cfg.lazy) {
          // chain bound from the live slots of every q0 (warp 0)
          if (tid < 32) {
            double lm = -INFINITY, lsum = 0.0;
            for (int q = tid; q < ns; q += 32) {
              const double v = __ldcg(&W.live[size_t(c) * ns + q]);
              if (v > lm) { lsum = lsum * exp(lm - v) + 1.0; lm = v; }
              else if (v != -INFINITY) lsum += exp(v - lm);
            }
            const double lub = warp_logsumexp(lm, lsum);
            if (tid == 0) {
              int flag = atomicAdd(&W.chain_flag[c], 0);
              if (!(flag & FLAG_REJECTED) && lub + cfg.margin < B.log_threshold[c] + B.beta * M.E_ref) {
                atomicOr(&W.chain_flag[c], FLAG_REJECTED);
                flag |= FLAG_REJECTED;
              }
              s_abort = (flag & FLAG_REJECTED) ? 1 : 0;
            }
          }
          __syncthreads();
          if (s_abort) { aborted = true; break; }
        }
      }
      alpha = B.op[a0 + i];
      const int idx_a = alpha * ns + qa;
      qb = M.s[idx_a];
      const int64_t off = M.blk_off[idx_a];
      prefix += M.log_norm[idx_a];
      const double scale = ldexp(1.0, -e);
      Eacc += e;

      if (i == n - 1) {  // final operator: only the diagonal of F_n Y is needed
        // qb == q0; F_n is d0 x dcur
        double vr = 0.0, vi = 0.0;
        const int tot = d0 * dcur;
        for (int idx = tid; idx < tot; idx += nt) {
          const int j = idx / dcur, k = idx - j * dcur;
          const T f = load_blk(M.blk, off + idx, T());
          const T y = Y[k * d0 + j];
          if constexpr (CPLX) {
            vr += f.x * y.x - f.y * y.y;
            vi += f.x * y.y + f.y * y.x;
          } else {
            vr += f * y;
          }
        }
        double dm = 0.0;
        block_max_sum(dm, vr, red);
        if constexpr (CPLX) {
          dm = 0.0;
          block_max_sum(dm, vi, red);
        }
        if (tid == 0) {
          W.res_val[2 * slot] = vr * scale;
          W.res_val[2 * slot + 1] = vi * scale;
          const bool zero_v = (vr == 0.0 && vi == 0.0);
          W.res_log[slot] = zero_v ? -INFINITY : L.val() + double(Eacc) * LN2;
          if (track) {
            const double a = sqrt(vr * vr + vi * vi) * scale;
            segp[it.n_seg] = zero_v ? -INFINITY : log(a) + L.val() + double(Eacc) * LN2;
          }
        }
        applied = n;
        break;
      }

      const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
      const double* Eb = M.E_rel + M.E_off[qb];
      const int db = M.dims[qb];
      for (int m = tid; m < db; m += nt) p[m] = exp(-dt * Eb[m]) * scale;
      L.add(-dt * (M.E_min[qb] - M.E_ref));
      prefix -= dt * (M.E_min[qb] - M.E_ref);
      __syncthreads();
      // Yn[m][j] = p[m] * sum_k F[m][k] Y[k][j]
      mx = 0.0;
      fr = 0.0;
      const int tot = db * d0;
      for (int idx = tid; idx < tot; idx += nt) {
        const int m = idx / d0, j = idx - m * d0;
        T acc;
        zero(acc);
        const int64_t frow = off + int64_t(m) * dcur;
        for (int k = 0; k < dcur; ++k) fma_acc(acc, load_blk(M.blk, frow + k, T()), Y[k * d0 + j]);
        const T v = p[m] * acc;
        Yn[idx] = v;
        mx = fmax(mx, mag(v));
        fr += sq(v);
      }
      block_max_sum(mx, fr, red);
      T* tmp = Y;
      Y = Yn;
      Yn = tmp;
      dcur = db;
      qa = qb;
      ++applied;
    }
    if (dead && tid == 0) {
      W.res_val[2 * slot] = 0.0;
      W.res_val[2 * slot + 1] = 0.0;
      W.res_log[slot] = -INFINITY;
      if (track)
        for (int s = (applied + cfg.S - 1) / cfg.S; s <= it.n_seg; ++s)
          if (s > 0) segp[s] = -INFINITY;
    }
    if (aborted && tid == 0) W.res_log[slot] = NAN;
  }
}

}  // namespace

static int trace_threads(int max_dim) {
  if (max_dim <= 12) return 32;
  if (max_dim <= 32) return 128;
  return 256;
}

static size_t trace_smem(int max_dim, bool cplx) {
  const size_t el = cplx ? 16 : 8;
  return 2 * size_t(max_dim) * max_dim * el + 2 * size_t(max_dim) * 8 + 64 * 8;
}

int prepare_eval_fp64(const DevModel& M, int num_sms, LaunchCfg* lc) {
  lc->threads = trace_threads(M.max_dim);
  lc->smem = trace_smem(M.max_dim, M.is_complex != 0);
  lc->num_sms = num_sms;
  lc->per_sm = 0;
  if (lc->smem > 227 * 1024) return CTQ_OK;  // needs the large-block path
  int per_sm = 0;
  if (M.is_complex) {
    if (cudaFuncSetAttribute(k_trace<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem)) !=
        cudaSuccess)
      return CTQ_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<true>, lc->threads, lc->smem) != cudaSuccess)
      return CTQ_ERR_CUDA;
  } else {
    if (cudaFuncSetAttribute(k_trace<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem)) !=
        cudaSuccess)
      return CTQ_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<false>, lc->threads, lc->smem) != cudaSuccess)
      return CTQ_ERR_CUDA;
  }
  lc->per_sm = per_sm;
  return CTQ_OK;
}

int launch_eval_fp64(const DevModel& M, const LaunchCfg& lc, const BatchView& B, const EvalCfg& cfg,
                     const Work& W, const ctq_result* R, void* stream, void* const* events) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (lc.per_sm < 1) return CTQ_ERR_UNSUPPORTED;
  auto mark = [&](int i) {
    if (events) cudaEventRecord(static_cast<cudaEvent_t>(events[i]), st);
  };
  if (cudaMemsetAsync(W.counters, 0, 256, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(0);
  const int warps_per_block = 4;
  const int grid_c = (B.n_chains + warps_per_block - 1) / warps_per_block;
  k_plan<<<grid_c, 32 * warps_per_block, 0, st>>>(M, B, cfg, W);
  if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
  mark(1);
  long long max_items = (long long)B.n_chains * M.n_sec;
  long long grid = (long long)lc.num_sms * lc.per_sm;
  if (grid > max_items) grid = max_items;
  if (M.is_complex)
    k_trace<true><<<int(grid), lc.threads, lc.smem, st>>>(M, B, cfg, W);
  else
    k_trace<false><<<int(grid), lc.threads, lc.smem, st>>>(M, B, cfg, W);
  if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
  mark(2);
  k_combine<<<grid_c, 32 * warps_per_block, 0, st>>>(M, B, cfg, W, *R);
  if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
  mark(3);
  return CTQ_OK;
}

}  // namespace ctq
