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
//              -beta E_gs is added (one warp, lanes over chunks of
//              operators).  Every `segment` operators the refined bound
//                ub = sqrt(r) ||Y||_F prod_{rest} ||F||_2 e^{-dtau E_min}
//              is recorded and, with lazy evaluation, the chain's live bound
//              sum is compared with its threshold (stop early if below);
//              without lazy evaluation the logarithms of all segments are
//              taken at the end, lanes over segments.  For short strings the
//              propagators of the whole string are computed in one dense
//              pass, once per distinct energy level of each visited sector,
//              by the table-driven exponential of exp_tang.cuh, and the
//              power-of-two rescale enters them by an exponent add.
#include <algorithm>

#include "device_common.cuh"
#include "exp_tang.cuh"
#include "two_float.cuh"

namespace ctq {
namespace {

using namespace dev;
using namespace tf2;

// ----------------------------------------------------------------------- trace

template <bool CPLX, bool X2>
struct Scalar;
template <>
struct Scalar<false, false> {
  using T = double;
  using PT = double;  // propagator entry
};
template <>
struct Scalar<true, false> {
  using T = double2;
  using PT = double;
};
template <>
struct Scalar<false, true> {
  using T = DF;
  using PT = DF;
};
template <>
struct Scalar<true, true> {
  using T = CDF;
  using PT = DF;
};

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

// Largest exponent field of |v| (integer; 0 for +-0 and subnormals).
__device__ __forceinline__ int exp_key(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ int exp_key(double2 v) { return max(exp_key(v.x), exp_key(v.y)); }

__device__ __forceinline__ double df_val(double a) { return a; }
__device__ __forceinline__ double2 df_val(double2 a) { return a; }

// block element i: float64 blocks, or their two-float copy
__device__ __forceinline__ double load_el(const DevModel& M, int64_t i, double) { return __ldg(M.blk + i); }
__device__ __forceinline__ double2 load_el(const DevModel& M, int64_t i, double2) {
  return __ldg(reinterpret_cast<const double2*>(M.blk) + i);
}
__device__ __forceinline__ DF load_el(const DevModel& M, int64_t i, DF) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(M.blk_x2) + i);
  return DF{v.x, v.y};
}
__device__ __forceinline__ CDF load_el(const DevModel& M, int64_t i, CDF) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(M.blk_x2) + i);
  return CDF{DF{v.x, v.y}, DF{v.z, v.w}};
}
__device__ __forceinline__ double to_prop(double x, double) { return x; }
__device__ __forceinline__ DF to_prop(double x, DF) { return df_split(x); }

// Block-wide max of an int; every thread gets the result.  redi: 32 ints.
__device__ __forceinline__ int block_max_int(int v, int* redi) {
  v = __reduce_max_sync(0xffffffffu, v);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nw == 1) return v;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) redi[w] = v;
  __syncthreads();
  v = redi[0];
  for (int i = 1; i < nw; ++i) v = max(v, redi[i]);
  return v;
}

// PRE: every propagator value of the chain is computed in one dense pass at
// the start of an item (lanes over all (operator, state) pairs), which keeps
// the FP64 pipe busy with full warps; used when max_ops * max_dim fits.
// X2: two-float products (CTQ_F32X2); propagators, log scale and the
// final diagonal stay in float64.  SMALL: a one-warp build held to 64
// registers so that 32 CTAs fit an SM (used for the two-float products of
// blocks of at most 12 states, whose FP32 add chains are latency bound).
template <bool CPLX, bool PRE, bool X2, bool SMALL>
__global__ void __launch_bounds__(SMALL ? 32 : 512, SMALL ? 32 : 1)
    k_trace(DevModel M, BatchView B, EvalCfg cfg, Work W) {
  using T = typename Scalar<CPLX, X2>::T;
  using T64 = typename Scalar<CPLX, false>::T;
  using PT = typename Scalar<CPLX, X2>::PT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int D = M.max_dim;
  const int MO = max(cfg.max_ops, 1);
  const int NS = cfg.n_seg_max + 1;
  T* Ybuf0 = reinterpret_cast<T*>(smem_raw);
  T* Ybuf1 = Ybuf0 + size_t(D) * D;
  double* p = reinterpret_cast<double*>(Ybuf1 + size_t(D) * D);  // [D] propagator of the current step
  PT* pp = reinterpret_cast<PT*>(p);  // the same, in the product's format (8 bytes either way)
  double* p0 = p + D;                                            // [D] wrap-around propagator (columns)
  double* red = p0 + D;                                          // [64] reductions
  double* segL = red + 64;                                       // [NS] log scale at segment ends
  double* segP = segL + NS;                                      // [NS] applied log-norm sums
  double* segF = segP + NS;                                      // [NS] ||Y||^2 at segment ends (deferred)
  double* segE = segF + NS;                                      // [NS] exponent sums at segment ends
  double* pall = segE + NS;                                      // [MO * max_lev] (PRE)
  int* poff = reinterpret_cast<int*>(pall + (PRE ? size_t(MO) * M.max_lev : 0));  // [MO + 1] (PRE)
  short* path = reinterpret_cast<short*>(poff + (PRE ? MO + 1 : 0));     // [MO + 1] sectors q_0..q_n
  short* opsm = path + (MO + 1);                                          // [MO] operator codes
  __shared__ int s_item;
  __shared__ int s_abort;
  __shared__ int redi[32];
  __shared__ double s_L;  // total log scale of the chain (thread 0 writes)
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
    const Item it = items[W.order[it_idx]];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);
    const double ub_const = (track && n > 1) ? 0.5 * it.log_r : 0.0;  // sqrt(r) of the refined bound

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

    if (n == 1) {  // only reachable with user tables where s_alpha(q0) = q0
      const double t1 = B.tau[a0], t2 = B.beta - B.tau[a0];
      const int64_t off = M.blk_off[B.op[a0] * ns + q0];
      double vr = 0.0, vi = 0.0, mx = 0.0;
      for (int j = tid; j < d0; j += nt) {
        const double pj = exp(-t1 * E0[j]) * exp(-t2 * E0[j]);
        const T64 f = load_blk(M.blk, off + int64_t(j) * d0 + j, T64());
        if constexpr (CPLX) {
          vr += f.x * pj;
          vi += f.y * pj;
        } else {
          vr += f * pj;
        }
      }
      block_max_sum(mx, vr, red);
      mx = 0.0;
      block_max_sum(mx, vi, red);
      if (tid == 0) {
        const double l = -B.beta * (M.E_min[q0] - M.E_ref);
        const bool zero_v = (vr == 0.0 && vi == 0.0);
        W.res_val[2 * slot] = vr;
        W.res_val[2 * slot + 1] = vi;
        W.res_log[slot] = zero_v ? -INFINITY : l;
        if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(vr * vr + vi * vi)) + l;
      }
      continue;
    }

    // ---- walk the string once: sectors, operator codes, log scale and the
    // applied log-norm sums at every segment end.  The wrap-around
    // propagators P_{beta - tau_n}(q0) and P_{tau_1}(q0) scale the columns of
    // the first block (trace cyclicity); their two time arguments are kept
    // separate so that no extra rounding enters them.
    const double t_first = B.tau[a0], t_last = B.beta - B.tau[a0 + n - 1];
    for (int i = tid; i < n; i += nt) opsm[i] = short(B.op[a0 + i]);
    __syncthreads();
    if (tid == 0) {  // integer walk only
      int q = q0;
      path[0] = short(q0);
      if (PRE) poff[0] = 0;
      for (int i = 0; i < n; ++i) {
        q = M.s[opsm[i] * ns + q];
        path[i + 1] = short(q);
        if (PRE && i + 1 < n) poff[i + 1] = poff[i] + (M.lev_off[q + 1] - M.lev_off[q]);
      }
    }
    __syncthreads();
    if (tid < 32) chain_log_scale(M, B, cfg, a0, n, q0, t_first, t_last, track, path, opsm, segL, segP, &s_L);
    __syncthreads();
    for (int j = tid; j < d0; j += nt) p0[j] = exp_nonpos(-t_first * E0[j]) * exp_nonpos(-t_last * E0[j]);
    if (PRE) {
      // all propagators of the chain, one per distinct level of each visited
      // sector: flat index j -> (operator i, level l)
      const int total = poff[n - 1];
      for (int j = tid; j < total; j += nt) {
        int lo = 0, hi = n - 2;  // largest i with poff[i] <= j
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (poff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int q = path[lo + 1];
        const double dt = B.tau[a0 + lo + 1] - B.tau[a0 + lo];
        pall[j] = exp_nonpos(-dt * M.lev_E[M.lev_off[q] + (j - poff[lo])]);
      }
    }

    // ---- operator 1: Y1[m][j] = p1[m] F1[m][j] p0[j]
    int qa = q0;
    int alpha = opsm[0];
    int qb = path[1];
    const double* p1 = p;
    if (!PRE) {
      const double dt = B.tau[a0 + 1] - B.tau[a0];
      const double* Eb = M.E_rel + M.E_off[qb];
      for (int m = tid; m < M.dims[qb]; m += nt) p[m] = exp_nonpos(-dt * Eb[m]);
    } else {
      __syncthreads();  // pall complete
      const int* lv = M.lev_idx + M.E_off[qb];
      for (int m = tid; m < M.dims[qb]; m += nt) p[m] = pall[lv[m]];  // poff[0] = 0
    }
    __syncthreads();
    T* Y = Ybuf0;
    T* Yn = Ybuf1;
    int dcur = M.dims[qb];
    int ekey = 0;
    {
      const int64_t off = M.blk_off[alpha * ns + qa];
      const int tot = dcur * d0;
      for (int idx = tid; idx < tot; idx += nt) {
        const int m = idx / d0, j = idx - m * d0;
        const T v = (p1[m] * p0[j]) * load_el(M, off + idx, T());
        Y[idx] = v;
        ekey = max(ekey, exp_key(v));
      }
    }
    ekey = block_max_int(ekey, redi);
    qa = qb;
    int applied = 1;
    long long Eacc = 0;  // power-of-two exponent: true = stored * 2^Eacc
    bool dead = false;
    bool aborted = false;
    double fr = 0.0;     // ||Y||^2 of the stored product (segment steps only)
    bool have_fr = false;
    int k_rec = 0;       // segments recorded for the deferred bounds

    // ---- operators 2 .. n: Y <- P F Y, the previous rescale folded into P
    for (int i = 1; i < n; ++i) {
      if (ekey == 0) { dead = true; break; }
      const int e = min(ekey - 1023, 1022);  // floor(log2 max|Y|) for normal values
      if (track && applied % cfg.S == 0 && applied < n) {
        if (!have_fr) {  // only after the first operator (segment length 1)
          double f = 0.0;
          for (int idx = tid; idx < dcur * d0; idx += nt) f += sq(Y[idx]);
          fr = block_sum(f, red);
        }
        if (!cfg.lazy) {  // bounds output only: the logarithms are taken for all segments at the end
          if (tid == 0) {
            segF[applied / cfg.S] = fr;
            segE[applied / cfg.S] = double(Eacc);
          }
          ++k_rec;
        } else if (tid == 0) {
          const double ub = ub_const + 0.5 * log(fr) + double(Eacc) * LN2 +
                            segL[applied / cfg.S] + (it.t_all - segP[applied / cfg.S]);
          segp[applied / cfg.S] = ub;
          W.live[slot] = fmin(W.live[slot], ub);
          __threadfence();
        }
        if (cfg.lazy) {
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
      alpha = opsm[i];
      const int idx_a = alpha * ns + qa;
      qb = path[i + 1];
      const int64_t off = M.blk_off[idx_a];
      const double scale = pow2i(-e);
      Eacc += e;

      if (i == n - 1) {  // final operator: only the diagonal of F_n Y is needed
        double vr = 0.0, vi = 0.0;
        const int tot = d0 * dcur;
        for (int idx = tid; idx < tot; idx += nt) {
          const int j = idx / dcur, k = idx - j * dcur;
          const T64 f = load_blk(M.blk, off + idx, T64());
          const T64 y = df_val(Y[k * d0 + j]);
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
          const double Lv = s_L;
          W.res_val[2 * slot] = vr * scale;
          W.res_val[2 * slot + 1] = vi * scale;
          const bool zero_v = (vr == 0.0 && vi == 0.0);
          W.res_log[slot] = zero_v ? -INFINITY : Lv + double(Eacc) * LN2;
          if (track) {
            const double a = sqrt(vr * vr + vi * vi) * scale;
            segp[it.n_seg] = zero_v ? -INFINITY : log(a) + Lv + double(Eacc) * LN2;
          }
        }
        applied = n;
        break;
      }

      const int db = M.dims[qb];
      if (PRE) {
        const double* pi = pall + poff[i];
        const int* lv = M.lev_idx + M.E_off[qb];
        for (int m = tid; m < db; m += nt) pp[m] = to_prop(scale_pow2(pi[lv[m]], -e), PT());
      } else {
        const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
        const double* Eb = M.E_rel + M.E_off[qb];
        for (int m = tid; m < db; m += nt) pp[m] = to_prop(scale_pow2(exp_nonpos(-dt * Eb[m]), -e), PT());
      }
      __syncthreads();
      // Yn[m][j] = p[m] * sum_k F[m][k] Y[k][j]
      const bool seg_next = track && (applied + 1) % cfg.S == 0 && (applied + 1) < n;
      ekey = 0;
      double f2 = 0.0;
      const int tot = db * d0;
      for (int idx = tid; idx < tot; idx += nt) {
        const int m = idx / d0, j = idx - m * d0;
        T acc;
        zero(acc);
        const int64_t frow = off + int64_t(m) * dcur;
        if constexpr (X2) {
          // two independent accumulators (even and odd terms: the FP32 add
          // chains of one output overlap), each renormalised every
          // X2_RENORM terms so that its low word holds a few ulps of the
          // high word and rounds at ~2^-48 of the sum per term
          T acc2;
          zero(acc2);
          int k = 0;
          for (; k + 2 * X2_RENORM <= dcur; k += 2 * X2_RENORM) {
#pragma unroll
            for (int u = 0; u < 2 * X2_RENORM; u += 2) {
              fma_acc(acc, load_el(M, frow + k + u, T()), Y[(k + u) * d0 + j]);
              fma_acc(acc2, load_el(M, frow + k + u + 1, T()), Y[(k + u + 1) * d0 + j]);
            }
            finish(acc);
            finish(acc2);
          }
          for (; k < dcur; ++k) fma_acc(acc, load_el(M, frow + k, T()), Y[k * d0 + j]);
          finish(acc);
          add_into(acc, acc2);
        } else {
          for (int k = 0; k < dcur; ++k) fma_acc(acc, load_el(M, frow + k, T()), Y[k * d0 + j]);
        }
        const T v = pp[m] * acc;
        Yn[idx] = v;
        ekey = max(ekey, exp_key(v));
        if (seg_next) f2 += sq(v);
      }
      ekey = block_max_int(ekey, redi);
      if (seg_next) fr = block_sum(f2, red);
      have_fr = seg_next;
      T* tmp = Y;
      Y = Yn;
      Yn = tmp;
      dcur = db;
      qa = qb;
      ++applied;
    }
    if (k_rec > 0) {  // deferred refined bounds, lanes over segments
      __syncthreads();
      for (int k = 1 + tid; k <= k_rec; k += nt)
        segp[k] = ub_const + 0.5 * log(segF[k]) + segE[k] * LN2 + segL[k] + (it.t_all - segP[k]);
      __syncthreads();
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

// Dynamic shared memory of k_trace: two Y buffers, p, p0, reductions, the
// segment bookkeeping, and (PRE) the chain's propagators (one per distinct
// level of each visited sector) and offsets, then the path and operator codes.
static size_t trace_smem(int max_dim, bool cplx, int max_ops, int n_seg_max, bool pre, int max_lev = 0) {
  const size_t el = cplx ? 16 : 8;
  const size_t mo = size_t(std::max(max_ops, 1));
  size_t b = 2 * size_t(max_dim) * max_dim * el + 2 * size_t(max_dim) * 8 + 64 * 8 + 4 * size_t(n_seg_max + 1) * 8;
  if (pre) b += mo * size_t(max_lev) * 8 + (mo + 1) * 4;
  b += (mo + 1) * 2 + mo * 2;
  return (b + 15) & ~size_t(15);
}

// Whole-chain propagator precompute when it fits comfortably.
static bool use_pre(int max_lev, int max_ops) { return size_t(std::max(max_ops, 1)) * max_lev * 8 <= 48 * 1024; }

// Raise the dynamic shared-memory cap to the opt-in maximum minus the
// kernel's static shared memory.
template <bool CPLX, bool PRE, bool X2, bool SMALL>
static int set_attr(int optin, int* regs) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_trace<CPLX, PRE, X2, SMALL>) != cudaSuccess) return CTQ_ERR_CUDA;
  *regs = std::max(*regs, fa.numRegs);
  const int cap = optin - int(fa.sharedSizeBytes);
  return cudaFuncSetAttribute(k_trace<CPLX, PRE, X2, SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) ==
                 cudaSuccess
             ? CTQ_OK
             : CTQ_ERR_CUDA;
}

template <bool SMALL>
static int set_attrs(int optin, int* regs) {
  int st;
  if ((st = set_attr<false, false, false, SMALL>(optin, regs)) || (st = set_attr<false, true, false, SMALL>(optin, regs)) ||
      (st = set_attr<true, false, false, SMALL>(optin, regs)) || (st = set_attr<true, true, false, SMALL>(optin, regs)) ||
      (st = set_attr<false, false, true, SMALL>(optin, regs)) || (st = set_attr<false, true, true, SMALL>(optin, regs)) ||
      (st = set_attr<true, false, true, SMALL>(optin, regs)) || (st = set_attr<true, true, true, SMALL>(optin, regs)))
    return st;
  return CTQ_OK;
}

template <bool SMALL>
static void launch_trace(bool x2, bool cplx, bool pre, dim3 g, dim3 b, size_t smem, cudaStream_t st, const DevModel& M,
                         const BatchView& B, const EvalCfg& cfg, const Work& W) {
  if (x2 && cplx) {
    if (pre) k_trace<true, true, true, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
    else k_trace<true, false, true, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
  } else if (x2) {
    if (pre) k_trace<false, true, true, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
    else k_trace<false, false, true, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
  } else if (cplx) {
    if (pre) k_trace<true, true, false, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
    else k_trace<true, false, false, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
  } else {
    if (pre) k_trace<false, true, false, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
    else k_trace<false, false, false, SMALL><<<g, b, smem, st>>>(M, B, cfg, W);
  }
}

// Whether the shared-memory FP64 kernel can hold two blocks of the largest
// sector (shortest strings); otherwise the float64 large-block kernel runs.
bool fp64_shared_kernel_fits(const DevModel& M, int optin) {
  return trace_smem(M.max_dim, M.is_complex != 0, 1, 1, false) + 2048 <= size_t(optin);
}

int prepare_eval_fp64(const DevModel& M, int num_sms, LaunchCfg* lc) {
  lc->threads = trace_threads(M.max_dim);
  lc->num_sms = num_sms;
  lc->smem = trace_smem(M.max_dim, M.is_complex != 0, 1, 1, false);
  lc->per_sm = (lc->smem > 200 * 1024) ? 0 : 1;  // feasibility at the smallest max_ops
  int st, dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return CTQ_ERR_CUDA;
  lc->smem_optin = optin;
  if ((st = prepare_plan(optin)) != CTQ_OK) return st;
  int regs = 0, regs_small = 0;  // the largest of the variants sizes the resident CTAs
  if ((st = set_attrs<false>(optin, &regs)) || (st = set_attrs<true>(optin, &regs_small))) return st;
  lc->regs = regs;
  lc->regs_small = regs_small;
  return CTQ_OK;
}

int launch_eval_fp64(const DevModel& M, const LaunchCfg& lc, const BatchView& B, const EvalCfg& cfg,
                     const Work& W, const ctq_result* R, void* stream, void* const* events, bool x2) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (x2 && M.blk_x2 == nullptr) return CTQ_ERR_UNSUPPORTED;
  if (lc.per_sm < 1) return CTQ_ERR_UNSUPPORTED;
  const bool pre = use_pre(M.max_lev, cfg.max_ops);
  const size_t smem = trace_smem(M.max_dim, M.is_complex != 0, cfg.max_ops, cfg.n_seg_max, pre, M.max_lev);
  if (smem + 1024 > size_t(lc.smem_optin)) return CTQ_ERR_UNSUPPORTED;
  // resident CTAs per SM from shared memory, registers and the 32-CTA
  // limit, optionally capped by the caller's launch tuning
  // the two-float products are FP32 add chains: blocks above 32 states get
  // 16 warps per CTA to hide their latency (float64 needs no more than 8)
  const int threads = cfg.threads > 0 ? cfg.threads : (x2 && lc.threads == 256 ? 512 : lc.threads);
  // the one-warp two-float variant at 64 registers (32 CTAs per SM: its FP32
  // add chains need the latency hiding; measured on t2g, 4 % faster); the
  // float64 products are FP64-pipe bound, and the register cap only added
  // instructions there (3 % slower), so they keep the 512-thread build
  const bool small = threads == 32 && x2;
  int per_sm = int((228 * 1024) / (smem + 1024));
  per_sm = std::min(per_sm, 65536 / std::max(1, (small ? lc.regs_small : lc.regs) * threads));
  per_sm = std::min(per_sm, std::min(32, 2048 / threads));
  if (cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, cfg.ctas_per_sm);
  if (per_sm < 1) return CTQ_ERR_UNSUPPORTED;
  auto mark = [&](int i) {
    if (events) record_timing_event(events[i], st);
  };
  if (cudaMemsetAsync(W.counters, 0, COUNTER_BYTES, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(0);
  {
    const int ps = launch_plan(M, B, cfg, W, st);
    if (ps != CTQ_OK) return ps;
  }
  mark(1);
  long long max_items = (long long)B.n_chains * M.n_sec;
  long long grid = (long long)lc.num_sms * per_sm;
  if (grid > max_items) grid = max_items;
  const dim3 g{unsigned(grid)}, b{unsigned(threads)};
  if (small) launch_trace<true>(x2, M.is_complex != 0, pre, g, b, smem, st, M, B, cfg, W);
  else launch_trace<false>(x2, M.is_complex != 0, pre, g, b, smem, st, M, B, cfg, W);
  if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
  mark(2);
  {
    const int cs = launch_combine(M, B, cfg, W, R, st);
    if (cs != CTQ_OK) return cs;
  }
  mark(3);
  return CTQ_OK;
}

}  // namespace ctq
