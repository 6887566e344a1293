// Plan and combine kernels of the local-trace evaluation (every precision).
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
//   k_combine  one warp per chain: w = sum_q0 w_q0 in log space with sign or
//              phase (Sec. 3.1.4, Eqs. PSignRewrite / Sign: the sampled weight is
//              |w| with phase w/|w|), the Metropolis decision (App. B, Eq.
//              decide) and the per-segment chain bounds.
#include "device_common.cuh"

namespace ctq {

using namespace dev;

// ----------------------------------------------------------------------- plan

// One warp per chain; the lanes walk different q0 with integer table lookups
// only and keep the visited sectors in shared memory (one byte per operator,
// PLAN_MAX_OPS per lane), so that the float64 sums of a surviving string are
// then taken by the whole warp with lanes over operators.
// Work of one operator besides its block product (rescale, propagators,
// reductions), in multiply-adds, for the ordering of the work list.
constexpr float PLAN_OP_COST = 200.f;

// Cost class of a string, 0 = most expensive: 1/8-octave steps of the float
// cost (its exponent and top three mantissa bits) from 2^7 upward.
__device__ __forceinline__ int order_class(float cost) {
  const int key = (__float_as_int(fmaxf(cost, 1.f)) >> 20) - ((127 + 7) << 3);
  return ORDER_CLASSES - 1 - min(ORDER_CLASSES - 1, max(0, key));
}

__device__ void plan_chain(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W) {
  extern __shared__ unsigned char plan_paths[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= B.n_chains) return;
  const int a0 = B.offsets[c];
  const int n = B.offsets[c + 1] - a0;
  const int ns = M.n_sec;
  const int MO = max(cfg.max_ops, 1);

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
  unsigned char* mine = plan_paths + size_t(wib * 32 + lane) * MO;

  double lm = -INFINITY, ls = 0.0;  // running logsumexp of b over this lane's q0
  for (int base = 0; base < ns; base += 32) {
    const int q0 = base + lane;
    bool alive = q0 < ns;
    int q = q0, r = alive ? M.dims[q0] : 0, qr = q0;  // qr: a sector of the smallest dimension r
    float cw = 0.f;  // sum over the block products of d_i d_{i+1}
    if (alive) {
      int dprev = r;
      for (int i = 0; i < n; ++i) {
        q = M.s[B.op[a0 + i] * ns + q];
        if (q < 0) { alive = false; break; }
        const int dq = M.dims[q];
        if (dq < r) { r = dq; qr = q; }
        if (i >= 1 && i <= n - 2) cw += float(dprev) * float(dq);
        dprev = dq;
        mine[i] = static_cast<unsigned char>(q);
      }
      alive = alive && (q == q0);
    }
    if (q0 < ns) {
      const size_t slot = size_t(c) * ns + q0;
      W.lvl0[slot] = -INFINITY;
      W.live[slot] = -INFINITY;
      W.res_log[slot] = -INFINITY;
      W.res_val[2 * slot] = 0.0;
      W.res_val[2 * slot + 1] = 0.0;
    }
    unsigned mask = __ballot_sync(FULL, alive);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int qs = base + src;
      const unsigned char* path = plan_paths + size_t(wib * 32 + src) * MO;
      double acc = 0.0;  // sum of log ||F_i|| - dtau_i (E_min(q_{i+1}) - E_ref)
      for (int i = lane; i < n; i += 32) {
        const int qi = (i == 0) ? qs : path[i - 1];
        acc += M.log_norm[B.op[a0 + i] * ns + qi];
        if (i + 1 < n) acc -= (B.tau[a0 + i + 1] - B.tau[a0 + i]) * (M.E_min[path[i]] - M.E_ref);
      }
      acc = warp_sum(acc);
      const int rs = __shfl_sync(FULL, r, src);
      const float cws = __shfl_sync(FULL, cw, src);
      if (lane == src) {
        const double b = (n == 0) ? (M.log_dim[qs] - B.beta * (M.E_min[qs] - M.E_ref))
                                  : (M.log_dim[qr] - t_wrap * (M.E_min[qs] - M.E_ref) + acc);
        const size_t slot = size_t(c) * ns + qs;
        Item it;
        it.c = c;
        it.q0 = qs;
        it.r = rs;
        it.log_r = M.log_dim[qr];
        it.n_seg = (n + cfg.S - 1) / cfg.S;
        it.t_all = acc;
        it.cost = float(M.dims[qs]) * cws + PLAN_OP_COST * float(n);
        W.items[slot] = it;  // staging copy in the (c, q0) slot
        W.lvl0[slot] = b;
        W.live[slot] = b;
        if (lm == -INFINITY) {  // first surviving string of this lane
          ls = 1.0;
          lm = b;
        } else if (b > lm) {
          ls = ls * exp(lm - b) + 1.0;
          lm = b;
        } else {
          ls += exp(b - lm);
        }
      }
    }
  }
  // relative to -beta E_ref; one lane with one surviving string needs no exp / log
  const unsigned has = __ballot_sync(FULL, lm != -INFINITY);
  double logB;
  if (has == 0u) {
    logB = -INFINITY;
  } else if ((has & (has - 1u)) == 0u) {
    const int src = __ffs(has) - 1;
    const double l1 = __shfl_sync(FULL, lm, src), s1 = __shfl_sync(FULL, ls, src);
    logB = (s1 == 1.0) ? l1 : l1 + log(s1);
  } else {
    logB = warp_logsumexp(lm, ls);
  }
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
      W.items[size_t(B.n_chains) * ns + pos] = W.items[size_t(c) * ns + q0];
    }
  }
}

// Orders the compacted work list by decreasing cost estimate (a counting
// sort over the cost classes, done by one CTA: histogram in shared memory,
// prefix, scatter of the list positions): the persistent trace kernels pull
// strings through W.order, so the longest start first and the short ones fill
// the tail.  (Histogram atomics in global memory from every plan CTA cost more
// than this pass: the classes of one workload crowd into a few counters.)
// CTA size of k_plan: 512 threads (16 chains) while the per-lane sector
// buffers fit, 128 for the longest strings.
constexpr int PLAN_THREADS_MAX = 512, PLAN_THREADS_MIN = 128;
static_assert(ORDER_CLASSES % PLAN_THREADS_MIN == 0 && ORDER_CLASSES % PLAN_THREADS_MAX == 0, "classes per thread");

__device__ void order_items(const Work& W, size_t cs) {
  __shared__ int off_s[ORDER_CLASSES];
  __shared__ int warp_s[PLAN_THREADS_MAX / 32];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int cpt = ORDER_CLASSES / nt;  // classes per thread in the prefix sum
  const int n = *((volatile int*)&W.counters[0]);
  const Item* list = W.items + cs;
  constexpr int U = 8;  // independent loads in flight per thread
  for (int k = tid; k < ORDER_CLASSES; k += nt) off_s[k] = 0;
  __syncthreads();
  for (int i0 = tid; i0 < n; i0 += U * nt) {  // histogram of the classes
    float cst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nt;
      cst[u] = (i < n) ? __ldcg(&list[i].cost) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * nt < n) atomicAdd(&off_s[order_class(cst[u])], 1);
  }
  __syncthreads();
  int loc[ORDER_CLASSES / PLAN_THREADS_MIN];
  int sum = 0;
  for (int u = 0; u < cpt; ++u) {
    loc[u] = off_s[cpt * tid + u];
    sum += loc[u];
  }
  // exclusive prefix over the threads: a warp scan, then the warp totals
  int inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_s[wid] = inc;
  __syncthreads();
  int base = 0;
  for (int w = 0; w < wid; ++w) base += warp_s[w];
  int acc = base + inc - sum;
  for (int u = 0; u < cpt; ++u) {
    off_s[cpt * tid + u] = acc;
    acc += loc[u];
  }
  __syncthreads();
  for (int i0 = tid; i0 < n; i0 += U * nt) {  // scatter of the list positions
    float cst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nt;
      cst[u] = (i < n) ? __ldcg(&list[i].cost) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nt;
      if (i < n) W.order[atomicAdd(&off_s[order_class(cst[u])], 1)] = i;
    }
  }
}

__global__ void __launch_bounds__(PLAN_THREADS_MAX) k_plan(DevModel M, BatchView B, EvalCfg cfg, Work W) {
  plan_chain(M, B, cfg, W);
  // the last CTA to finish orders the work list (no wait: it is simply the
  // one whose arrival completes the count).  One thread per CTA fences: the
  // barrier orders the CTA's writes before its fence, which is cumulative,
  // and the last CTA's fence orders every CTA's writes before its reads.
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&W.counters[4], 1) == int(gridDim.x) - 1) ? 1 : 0;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  order_items(W, size_t(B.n_chains) * M.n_sec);
}

// ----------------------------------------------------------------------- combine

// GB300 runs float64 at 1/64 of the float32 rate, so the per-chain
// bookkeeping below avoids float64 work that integer operations can do:
// -inf tests on the bit pattern, exponents from the exponent field.
__device__ __forceinline__ bool is_neg_inf(double x) {
  return __double_as_longlong(x) == static_cast<long long>(0xFFF0000000000000ull);
}
// floor(log2 a) for a > 0 (ilogb for subnormal a)
__device__ __forceinline__ int exp_of(double a) {
  const int f = int((__double_as_longlong(a) >> 52) & 0x7ff);
  return f ? f - 1023 : ilogb(a);
}

__global__ void k_combine(DevModel M, BatchView B, EvalCfg cfg, Work W, ctq_result R) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= B.n_chains) return;
  const int ns = M.n_sec;
  const int flag = W.chain_flag[c];
  const int nb = cfg.n_seg_max + 1;
  if (W.counters[2] != 0) {  // a bounded wait expired in the trace kernel
    if (lane == 0) {
      R.log_abs[c] = NAN;
      R.phase[2 * c] = 0.0;
      R.phase[2 * c + 1] = 0.0;
      R.status[c] = (flag & FLAG_INVALID) ? CTQ_CHAIN_ERR_ARG : CTQ_CHAIN_ERR_TIMEOUT;
    }
    if (cfg.bounds)
      for (int s = lane; s < nb; s += 32) cfg.bounds[size_t(c) * nb + s] = NAN;
    return;
  }
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
  // w = sum_q0 val * e^{log} with a common scale lm = max_q0 (log + exponent
  // of |val|): the dominant string's factor is the exact power of two
  // 2^{-exponent}; only the others need an exponential (lanes over q0)
  double lm = -INFINITY;
  for (int q = lane; q < ns; q += 32) {
    const size_t slot = size_t(c) * ns + q;
    const double lg = W.res_log[slot];
    if (is_neg_inf(lg)) continue;
    const double a = fabs(W.res_val[2 * slot]) + fabs(W.res_val[2 * slot + 1]);
    if (a > 0.0) lm = fmax(lm, lg + double(exp_of(a)) * LN2);
  }
  lm = warp_max(lm);
  double sr = 0.0, si = 0.0;
  if (lm != -INFINITY) {
    for (int q = lane; q < ns; q += 32) {
      const size_t slot = size_t(c) * ns + q;
      const double lg = W.res_log[slot];
      if (is_neg_inf(lg)) continue;
      const double vr = W.res_val[2 * slot], vi = W.res_val[2 * slot + 1];
      const double a = fabs(vr) + fabs(vi);
      if (a == 0.0) continue;
      const int ea = exp_of(a);
      const double f = (lg + double(ea) * LN2 == lm) ? scalbn(1.0, -ea) : exp(lg - lm);
      sr += vr * f;
      si += vi * f;
    }
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  const double shift = -B.beta * M.E_ref;  // logs above are relative to e^{-beta E_ref}
  if (lane == 0) {
    const double a = M.is_complex ? hypot(sr, si) : fabs(sr);
    int st = CTQ_CHAIN_OK;
    if (lm == -INFINITY || a == 0.0) {
      R.log_abs[c] = -INFINITY;
      R.phase[2 * c] = 0.0;
      R.phase[2 * c + 1] = 0.0;
      st = CTQ_CHAIN_ZERO;
    } else {
      const double la = (lm + log(a)) + shift;
      R.log_abs[c] = la;
      if (M.is_complex) {
        R.phase[2 * c] = sr / a;
        R.phase[2 * c + 1] = si / a;
      } else {  // the sign, without a float64 division
        R.phase[2 * c] = copysign(1.0, sr);
        R.phase[2 * c + 1] = 0.0;
      }
      if (cfg.has_thr) st = (la >= B.log_threshold[c]) ? CTQ_CHAIN_ACCEPTED : CTQ_CHAIN_REJECTED;
    }
    R.status[c] = st;
  }
  if (cfg.bounds) {
    // lanes over segments; each lane sums over the surviving q0 serially
    const int n = B.offsets[c + 1] - B.offsets[c];
    const int nseg = (n + cfg.S - 1) / cfg.S;
    for (int s = 1 + lane; s < nb; s += 32) {
      const int ss = min(s, nseg);
      double m2 = -INFINITY, s2 = 0.0;
      int cnt = 0;
      for (int q = 0; q < ns; ++q) {
        const size_t slot = size_t(c) * ns + q;
        if (is_neg_inf(W.lvl0[slot])) continue;
        const double v = W.seg[slot * size_t(nb) + ss];
        if (is_neg_inf(v)) continue;
        ++cnt;
        if (v > m2) { s2 = (cnt == 1) ? 1.0 : s2 * exp(m2 - v) + 1.0; m2 = v; }
        else s2 += exp(v - m2);
      }
      const double lb = (cnt == 0) ? -INFINITY : (cnt == 1 ? m2 : m2 + log(s2));
      cfg.bounds[size_t(c) * nb + s] = lb + shift;
    }
  }
}

int prepare_plan(int optin) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_plan) != cudaSuccess) return CTQ_ERR_CUDA;
  return cudaFuncSetAttribute(k_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - int(fa.sharedSizeBytes)) == cudaSuccess
             ? CTQ_OK
             : CTQ_ERR_CUDA;
}

// k_plan keeps one byte per operator per lane (16 or 4 warps of 32 lanes per CTA).
int launch_plan(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, cudaStream_t st) {
  if (M.n_sec > 255) return CTQ_ERR_UNSUPPORTED;
  const size_t mo = size_t(cfg.max_ops > 0 ? cfg.max_ops : 1);
  // one byte per operator per lane: the largest CTA whose buffers fit 200 KB
  const int threads = (size_t(PLAN_THREADS_MAX) * mo <= 200 * 1024) ? PLAN_THREADS_MAX : PLAN_THREADS_MIN;
  const size_t smem = size_t(threads) * mo;
  if (smem > 200 * 1024) return CTQ_ERR_UNSUPPORTED;  // max_ops <= 1600
  const int warps = threads / 32;
  const int grid = (B.n_chains + warps - 1) / warps;
  k_plan<<<grid, threads, smem, st>>>(M, B, cfg, W);
  return cudaGetLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

int launch_combine(const DevModel& M, const BatchView& B, const EvalCfg& cfg, const Work& W, const ctq_result* R,
                   cudaStream_t st) {
  const int grid = (B.n_chains + 3) / 4;
  k_combine<<<grid, 128, 0, st>>>(M, B, cfg, W, *R);
  return cudaGetLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

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
  char* counters = take(COUNTER_BYTES);
  char* items = take(2 * cs * sizeof(Item));  // staging slots + compacted list
  char* res_val = take(2 * cs * sizeof(double));
  char* res_log = take(cs * sizeof(double));
  char* live = take(cs * sizeof(double));
  char* lvl0 = take(cs * sizeof(double));
  char* seg = take(cs * size_t(n_seg_max + 1) * sizeof(double));
  char* flags = take(size_t(n_chains) * sizeof(int));
  char* order = take(cs * sizeof(int));
  if (w) {
    w->counters = reinterpret_cast<int*>(counters);
    w->items = reinterpret_cast<Item*>(items);
    w->res_val = reinterpret_cast<double*>(res_val);
    w->res_log = reinterpret_cast<double*>(res_log);
    w->live = reinterpret_cast<double*>(live);
    w->lvl0 = reinterpret_cast<double*>(lvl0);
    w->seg = reinterpret_cast<double*>(seg);
    w->chain_flag = reinterpret_cast<int*>(flags);
    w->order = reinterpret_cast<int*>(order);
  }
  return off;
}

}  // namespace ctq
