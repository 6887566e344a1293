// Sector-string local trace on the GPU: plan, FP64 chain products, combine.
//
// One evaluation of a batch runs three kernels on the caller's stream:
//
//   k_plan     one warp per chain.  Validates the sequence, follows the sector
//              map s_alpha(q) for every q0 without any matrix work (Sec. 3.3.1,
//              the string q0 -> q1 -> ... must return to q0 and never visit the
//              zero sector), computes the level-0 lazy bound per surviving q0
//                b(q0) = r * prod ||F_i||_2 * prod e^{-dtau E_min(q)}
//              (Sec. 3.3.1, lazy-trace paragraph: submultiplicative norms, the
//              spectral norm of a propagator is e^{-dtau E_min}), decides an
//              early reject when log sum_q0 b < T, and appends the surviving
//              (chain, q0) strings to the work list.
//   k_trace    persistent CTAs pull (chain, q0) items.  The product
//                Y_1 = P_1 F_1 P_wrap,  Y_i = P_i F_i Y_{i-1},
//                w_q0 = Tr(F_n Y_{n-1}) (diagonal only)
//              runs with Y resident in shared memory; P_i = diag(e^{-dtau (E - E_min)})
//              rows are applied in the GEMM epilogue (the "time-evolution
//              kernel"), the wrap-around propagator of q0 for beta - tau_n +
//              tau_1 scales the columns of the first block (trace cyclicity).
//              After every product the max |Y| is reduced across the CTA and
//              the next product absorbs the exact power-of-two rescale; the
//              log scale (energy shifts and exponents) stays in float64,
//              relative to e^{-beta E_gs} (the propagation times sum to beta)
//              and summed with compensation, so that log|w| ~ 10^3 loses no
//              accuracy before the final -beta E_gs is added.  Every
//              `segment` operators the refined bound
//                ub = sqrt(r) ||Y||_F prod_{rest} ||F||_2 e^{-dtau E_min}
//              is recorded and, with lazy evaluation, the chain's live bound
//              sum is compared with its threshold (stop early if below).
//   k_combine  one warp per chain: w = sum_q0 w_q0 in log space with sign or
//              phase (Sec. 3.1.4, Eqs. PSignRewrite / Sign: the sampled weight is
//              |w| with phase w/|w|), the Metropolis decision (App. B, Eq.
//              decide) and the per-segment chain bounds.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ctq_internal.h"

namespace ctq {
namespace {

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

// ----------------------------------------------------------------------- plan

__global__ void k_plan(DevModel M, BatchView B, EvalCfg cfg, Work W) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= B.n_chains) return;
  const int a0 = B.offsets[c];
  const int n = B.offsets[c + 1] - a0;
  const int ns = M.n_sec;

  bool bad = n < 0 || n > cfg.max_ops;
  for (int i = lane; !bad && i < n; i += 32) {
    const int alpha = B.op[a0 + i];
    const double t = B.tau[a0 + i];
    if (alpha < 0 || alpha >= M.n_alpha || !(t >= 0.0) || !(t < B.beta)) bad = true;
    if (i > 0 && !(t > B.tau[a0 + i - 1])) bad = true;
  }
  bad = __any_sync(FULL, bad);
  if (bad) {
    for (int q0 = lane; q0 < ns; q0 += 32) {
      W.lvl0[size_t(c) * ns + q0] = -INFINITY;
      W.live[size_t(c) * ns + q0] = -INFINITY;
      W.res_log[size_t(c) * ns + q0] = -INFINITY;
    }
    if (lane == 0) W.chain_flag[c] = FLAG_INVALID;
    return;
  }
  const double t_wrap = (n > 0) ? (B.beta - B.tau[a0 + n - 1] + B.tau[a0]) : B.beta;

  // walk every q0 (lanes stride over sectors)
  double lm = -INFINITY, ls = 0.0;  // running logsumexp of b over this lane's q0
  for (int q0 = lane; q0 < ns; q0 += 32) {
    int q = q0, r = M.dims[q0];
    double lb = 0.0;
    bool alive = true;
    for (int i = 0; i < n; ++i) {
      const int alpha = B.op[a0 + i];
      const int idx = alpha * ns + q;
      lb += M.log_norm[idx];
      q = M.s[idx];
      if (q < 0) { alive = false; break; }
      r = min(r, M.dims[q]);
      if (i + 1 < n) lb -= (B.tau[a0 + i + 1] - B.tau[a0 + i]) * (M.E_min[q] - M.E_ref);
    }
    alive = alive && (q == q0);
    const size_t slot = size_t(c) * ns + q0;
    double b = -INFINITY;
    if (alive) {
      b = (n == 0) ? (log(double(M.dims[q0])) - B.beta * (M.E_min[q0] - M.E_ref))
                   : (log(double(r)) - t_wrap * (M.E_min[q0] - M.E_ref) + lb);
      Item it;
      it.c = c;
      it.q0 = q0;
      it.r = r;
      it.n_seg = (n + cfg.S - 1) / cfg.S;
      it.t_all = lb;
      // the item is appended below unless the chain is rejected at level 0
      W.items[slot] = it;  // staging copy in the (c, q0) slot
    }
    W.lvl0[slot] = b;
    W.live[slot] = b;
    W.res_log[slot] = -INFINITY;
    W.res_val[2 * slot] = 0.0;
    W.res_val[2 * slot + 1] = 0.0;
    if (b > lm) {
      ls = ls * exp(lm - b) + 1.0;
      lm = b;
    } else if (b != -INFINITY) {
      ls += exp(b - lm);
    }
  }
  const double logB = warp_logsumexp(lm, ls);  // relative to -beta E_ref
  const double shift = -B.beta * M.E_ref;
  if (cfg.bounds && lane == 0) cfg.bounds[size_t(c) * (cfg.n_seg_max + 1)] = logB + shift;
  bool reject = false;
  if (cfg.lazy && logB != -INFINITY) reject = (logB + cfg.margin < B.log_threshold[c] - shift);
  if (lane == 0) W.chain_flag[c] = reject ? FLAG_REJECTED : 0;
  if (reject) return;
  // append the surviving strings (warp-aggregated atomic)
  for (int base = 0; base < ns; base += 32) {
    const int q0 = base + lane;
    const bool alive = q0 < ns && W.lvl0[size_t(c) * ns + q0] != -INFINITY;
    const unsigned mask = __ballot_sync(FULL, alive);
    if (!mask) continue;
    int first = 0;
    if (lane == 0) first = atomicAdd(&W.counters[0], __popc(mask));
    first = __shfl_sync(FULL, first, 0);
    if (alive) {
      const int pos = first + __popc(mask & ((1u << lane) - 1u));
      // items[pos] may alias a staging slot of another chain that is already
      // consumed: staging copies live in a separate region (see Work).
      W.items[size_t(B.n_chains) * ns + pos] = W.items[size_t(c) * ns + q0];
    }
  }
}

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

// Block-wide reduction of (max, sum) pairs; every thread gets the result.
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

// ----------------------------------------------------------------------- combine

__global__ void k_combine(DevModel M, BatchView B, EvalCfg cfg, Work W, ctq_result R) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= B.n_chains) return;
  const int ns = M.n_sec;
  const int flag = W.chain_flag[c];
  const int nb = cfg.n_seg_max + 1;
  if (flag & (FLAG_INVALID | FLAG_REJECTED)) {
    if (lane == 0) {
      R.log_abs[c] = NAN;
      R.phase[2 * c] = 0.0;
      R.phase[2 * c + 1] = 0.0;
      R.status[c] = (flag & FLAG_INVALID) ? CTQ_CHAIN_ERR_ARG : CTQ_CHAIN_REJECTED_EARLY;
    }
    if (cfg.bounds)
      for (int s = lane; s < nb; s += 32)
        if (s > 0 || (flag & FLAG_INVALID)) cfg.bounds[size_t(c) * nb + s] = NAN;
    return;
  }
  // sum_q0 w_q0 = sum val * e^{log}, with a common max log
  double lm = -INFINITY;
  for (int q = lane; q < ns; q += 32) {
    const size_t slot = size_t(c) * ns + q;
    const double lg = W.res_log[slot];
    if (lg == -INFINITY) continue;
    const double a = hypot(W.res_val[2 * slot], W.res_val[2 * slot + 1]);
    if (a > 0.0) lm = fmax(lm, lg + log(a));
  }
  lm = warp_max(lm);
  double sr = 0.0, si = 0.0;
  if (lm != -INFINITY) {
    for (int q = lane; q < ns; q += 32) {
      const size_t slot = size_t(c) * ns + q;
      const double lg = W.res_log[slot];
      if (lg == -INFINITY) continue;
      const double f = exp(lg - lm);
      sr += W.res_val[2 * slot] * f;
      si += W.res_val[2 * slot + 1] * f;
    }
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  const double a = hypot(sr, si);
  const double shift = -B.beta * M.E_ref;  // logs above are relative to e^{-beta E_ref}
  if (lane == 0) {
    int st = CTQ_CHAIN_OK;
    if (lm == -INFINITY || a == 0.0) {
      R.log_abs[c] = -INFINITY;
      R.phase[2 * c] = 0.0;
      R.phase[2 * c + 1] = 0.0;
      st = CTQ_CHAIN_ZERO;
    } else {
      const double la = (lm + log(a)) + shift;
      R.log_abs[c] = la;
      R.phase[2 * c] = sr / a;
      R.phase[2 * c + 1] = si / a;
      if (cfg.has_thr) st = (la >= B.log_threshold[c]) ? CTQ_CHAIN_ACCEPTED : CTQ_CHAIN_REJECTED;
    }
    R.status[c] = st;
  }
  if (cfg.bounds) {
    for (int s = 1; s < nb; ++s) {
      double m2 = -INFINITY, s2 = 0.0;
      for (int q = lane; q < ns; q += 32) {
        const size_t slot = size_t(c) * ns + q;
        if (W.lvl0[slot] == -INFINITY) continue;
        // items finish at their own last segment; later columns repeat the exact value
        const int n = B.offsets[c + 1] - B.offsets[c];
        const int nseg = (n + cfg.S - 1) / cfg.S;
        const double v = W.seg[slot * size_t(nb) + min(s, nseg)];
        if (v > m2) { s2 = s2 * exp(m2 - v) + 1.0; m2 = v; }
        else if (v != -INFINITY) s2 += exp(v - m2);
      }
      const double lb = warp_logsumexp(m2, s2);
      if (lane == 0) cfg.bounds[size_t(c) * nb + s] = lb + shift;
    }
  }
}

}  // namespace

size_t workspace_layout(int n_chains, int n_sec, int n_seg_max, void* base, Work* w) {
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t cs = size_t(n_chains) * n_sec;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    char* p = b ? b + off : nullptr;
    off += align(bytes);
    return p;
  };
  char* counters = take(256);
  char* items = take(2 * cs * sizeof(Item));  // staging slots + compacted list
  char* res_val = take(2 * cs * sizeof(double));
  char* res_log = take(cs * sizeof(double));
  char* live = take(cs * sizeof(double));
  char* lvl0 = take(cs * sizeof(double));
  char* seg = take(cs * size_t(n_seg_max + 1) * sizeof(double));
  char* flags = take(size_t(n_chains) * sizeof(int));
  if (w) {
    w->counters = reinterpret_cast<int*>(counters);
    w->items = reinterpret_cast<Item*>(items);
    w->res_val = reinterpret_cast<double*>(res_val);
    w->res_log = reinterpret_cast<double*>(res_log);
    w->live = reinterpret_cast<double*>(live);
    w->lvl0 = reinterpret_cast<double*>(lvl0);
    w->seg = reinterpret_cast<double*>(seg);
    w->chain_flag = reinterpret_cast<int*>(flags);
  }
  return off;
}

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
