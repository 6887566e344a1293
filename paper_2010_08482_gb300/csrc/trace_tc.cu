// Sector-string local trace on the 5th-generation tensor cores (tcgen05).
//
// Same mathematics as k_trace (trace_fp64.cu), with the block products in
// TF32 or in three-term split TF32 (hi*hi + hi*lo + lo*hi) with FP32
// accumulation; the log scale, the renormalisation exponents, the segment
// bounds and the final trace sum stay in float64 (mixed-precision reading of
// Sec. 3.3.2, which anticipates mixed-precision products).
//
// Layout (one (chain, q0) item per CTA at a time, 4 warps):
//   The chain runs transposed, Z_i = Y_i^T (d0 x d_i):
//       Z_{i+1} = Z_i F_{i+1}^T P_{i+1}
//   so that the running product is the MMA's A operand and stays in tensor
//   memory (TMEM) for the whole chain: A = Z_i (128 lanes = rows of Z, one
//   32-bit column per K element), B = F_{i+1}^T, whose K-major form is F's own
//   row-major layout, staged from a pre-formatted global copy into shared
//   memory by cp.async.bulk (double-buffered: the next block is prefetched
//   while the current MMA runs), D accumulates in TMEM.  The epilogue reads
//   D with tcgen05.ld (thread = row), applies the propagator column scale
//   p_j = e^{-dtau (E_j - E_min)} times the power-of-two rescale of the
//   previous step, reduces max|Z| and ||Z||_F, splits hi/lo and writes the
//   next A with tcgen05.st.  The first product only scales F_1 (elementwise);
//   the last one needs only the diagonal of F_n Y (FP32 products, FP64 sum).
//
// Every wait on an mbarrier is bounded by the caller's timeout; on expiry
// the kernel records CTQ_ERR_TIMEOUT in the workspace, waits (bounded) for
// its own copies in flight, frees its TMEM and returns.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ctq {
namespace {

using namespace dev;
using namespace ptx;

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;

// Block-wide (max, sum) of floats; all threads get the result.  red: 8 floats.
__device__ __forceinline__ void block_max_sum_f(float& mx, float& sm, float* red) {
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sm += __shfl_xor_sync(0xffffffffu, sm, o);
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[w] = mx;
    red[4 + w] = sm;
  }
  __syncthreads();
  mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
  sm = (red[4] + red[5]) + (red[6] + red[7]);
}

__device__ __forceinline__ int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Shared state of one CTA.
struct TcShared {
  uint64_t bar_load[2];
  uint64_t bar_mma;
  uint64_t bar_never;  // never arrived on: CTQ_DEBUG_STALL_WAIT waits on it
  uint32_t tmem_base;
  int item;
  int abort_flag;
  int fail;
  float red[8];
  double redd[64];
};

}  // namespace


namespace {

template <int SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_trace_tc(DevModel M, BatchView B, EvalCfg cfg, Work W, TcParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* stage[2];
  stage[0] = reinterpret_cast<float*>(smem_raw);
  stage[1] = stage[0] + P.stage_floats;
  float* p_s = stage[1] + P.stage_floats;  // [128] column scales of the current step
  float* p0_s = p_s + TC_M;                // [128] wrap-around propagator of q0
  __shared__ TcShared S;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid;  // TMEM lane owned by this thread
  const int ns = M.n_sec;

  if (tid == 0) {
    mbar_init(&S.bar_load[0], 1);
    mbar_init(&S.bar_load[1], 1);
    mbar_init(&S.bar_mma, 1);
    mbar_init(&S.bar_never, 1);
    S.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(P.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((cfg.debug & CTQ_DEBUG_STALL_WAIT) && tid == 0 && !mbar_wait(&S.bar_never, 0, P.timeout_ns)) {
    S.fail = 1;  // expected: nothing arrives on bar_never
    atomicOr(&W.counters[2], 1);
  }
  __syncthreads();
  const uint32_t tbase = S.tmem_base;
  const uint32_t lane_off = uint32_t(32 * warp) << 16;
  const uint32_t tD = tbase;          // D: columns [0, 128)
  const uint32_t tAh = tbase + 128;   // A hi: [128, 256)
  const uint32_t tAl = tbase + 256;   // A lo: [256, 384) (split mode)

  uint32_t ph_load[2] = {0, 0};   // next parity to wait for, per stage (thread 0)
  int pending[2] = {0, 0};        // loads issued and not yet waited for (thread 0)
  uint32_t ph_mma = 0;            // next parity of bar_mma (all threads)
  const int n_items = W.counters[0];
  const Item* items = W.items + size_t(B.n_chains) * ns;

  for (;;) {
    __syncthreads();
    if (tid == 0) S.item = atomicAdd(&W.counters[1], 1);
    __syncthreads();
    const int it_idx = S.item;
    if (it_idx >= n_items || S.fail) break;
    const Item it = items[it_idx];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);

    if (n < 2) {  // empty sequence (Tr e^{-beta H(q0)}) or a one-operator string
      double sm = 0.0, si = 0.0, mx = 0.0;
      if (n == 0) {
        for (int j = tid; j < d0; j += TC_THREADS) sm += exp(-B.beta * E0[j]);
      } else {
        const double t1 = B.tau[a0], t2 = B.beta - B.tau[a0];
        const int64_t off = M.blk_off[B.op[a0] * ns + q0];
        for (int j = tid; j < d0; j += TC_THREADS) {
          const double pj = exp(-t1 * E0[j]) * exp(-t2 * E0[j]);
          if (M.is_complex) {
            sm += M.blk[2 * (off + int64_t(j) * d0 + j)] * pj;
            si += M.blk[2 * (off + int64_t(j) * d0 + j) + 1] * pj;
          } else {
            sm += M.blk[off + int64_t(j) * d0 + j] * pj;
          }
        }
      }
      block_max_sum(mx, sm, S.redd);
      mx = 0.0;
      block_max_sum(mx, si, S.redd);
      if (tid == 0) {
        const double l = (n == 0) ? -B.beta * (M.E_min[q0] - M.E_ref)
                                  : -B.beta * (M.E_min[q0] - M.E_ref);
        const bool zero_v = (sm == 0.0 && si == 0.0);
        W.res_val[2 * slot] = sm;
        W.res_val[2 * slot + 1] = si;
        W.res_log[slot] = zero_v ? -INFINITY : l;
        if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(sm * sm + si * si)) + l;
      }
      continue;
    }

    // ---- operator 1 (elementwise): Z_1[j][m] = p0[j] F_1[m][j] p1[m]
    int qa = q0;
    int alpha = B.op[a0];
    int qb = M.s[alpha * ns + qa];
    const double t_first = B.tau[a0], t_last = B.beta - B.tau[a0 + n - 1];
    KSum L;  // thread 0 only (log scale relative to E_ref)
    long long Eacc = 0;
    double prefix = 0.0;
    if (tid == 0) {
      L.add(-t_first * (M.E_min[q0] - M.E_ref));
      L.add(-t_last * (M.E_min[q0] - M.E_ref));
      prefix = M.log_norm[alpha * ns + qa];
    }
    {
      const double dt = B.tau[a0 + 1] - B.tau[a0];
      const float* Eb = M.E_relf + M.E_off[qb];
      const float* E0f = M.E_relf + M.E_off[q0];
      const int db = M.dims[qb];
      for (int j = tid; j < TC_M; j += TC_THREADS) {
        // FP32 exponentials: an absolute argument error of ~1e-7 x changes
        // e^{-x} by at most max(x e^{-x}) 1e-7 < 4e-8 relative to the largest
        // entry, below the resolution of the products.
        p_s[j] = (j < db) ? __expf(-float(dt) * Eb[j]) : 0.0f;
        p0_s[j] = (j < d0) ? __expf(-float(t_first) * E0f[j]) * __expf(-float(t_last) * E0f[j]) : 0.0f;
      }
      if (tid == 0) {
        L.add(-dt * (M.E_min[qb] - M.E_ref));
        prefix -= dt * (M.E_min[qb] - M.E_ref);
      }
    }
    // prefetch the block of operator 2 (the first tensor-core product)
    if (tid == 0 && n > 2) {
      const int alpha2 = B.op[a0 + 1];
      const int qn = M.s[alpha2 * ns + qb];
      const int np = round_up(M.dims[qn], 16), kp = round_up(M.dims[qb], 8);
      const uint32_t bytes = uint32_t(SPLIT == 3 ? 2 : 1) * np * kp * 4;
      mbar_arrive_expect_tx(&S.bar_load[0], bytes);
      bulk_g2s(stage[0], P.blk + P.off[alpha2 * ns + qb], bytes, &S.bar_load[0]);
      pending[0] = 1;
    }
    __syncthreads();
    int dcur = M.dims[qb];
    float mx = 0.f, fr = 0.f;
    {
      const int64_t off = M.blk_off[alpha * ns + qa];
      const int kp = round_up(dcur, 16);
      const float p0r = p0_s[row];
      for (int c0 = 0; c0 < kp; c0 += 16) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int m = c0 + t;
          float x = 0.f;
          if (row < d0 && m < dcur) x = float(M.blk[off + int64_t(m) * d0 + row]) * p0r * p_s[m];
          mx = fmaxf(mx, fabsf(x));
          fr += x * x;
          hi[t] = to_tf32(x);
          lo[t] = to_tf32(x - __uint_as_float(hi[t]));
        }
        tmem_st16(tAh + lane_off + c0, hi);
        if (SPLIT == 3) tmem_st16(tAl + lane_off + c0, lo);
      }
      tmem_wait_st();
    }
    tc_fence_before();
    block_max_sum_f(mx, fr, S.red);
    qa = qb;
    int applied = 1;
    bool dead = false, aborted = false;
    int cur_stage = 0;

    for (int i = 1; i < n; ++i) {
      if (mx == 0.f) { dead = true; break; }
      const int e = ilogbf(mx);
      if (track && applied % cfg.S == 0 && applied < n) {
        if (tid == 0) {
          const double ub = 0.5 * log(double(it.r)) + 0.5 * log(double(fr)) + double(Eacc) * LN2 + L.val() +
                            (it.t_all - prefix);
          segp[applied / cfg.S] = ub;
          if (cfg.lazy) {
            W.live[slot] = fmin(W.live[slot], ub);
            __threadfence();
          }
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
              S.abort_flag = (flag & FLAG_REJECTED) ? 1 : 0;
            }
          }
          __syncthreads();
          if (S.abort_flag) { aborted = true; break; }
        }
      }
      alpha = B.op[a0 + i];
      const int idx_a = alpha * ns + qa;
      qb = M.s[idx_a];
      const float scale = ldexpf(1.0f, -e);
      if (tid == 0) prefix += M.log_norm[idx_a];
      Eacc += e;

      if (i == n - 1) {  // final operator: diagonal of F_n Y = sum_{j,k} F_n[j][k] Z[j][k]
        const int64_t off = M.blk_off[idx_a];
        double vr = 0.0, vi = 0.0;
        float acc = 0.f;
        tc_fence_after();
        for (int c0 = 0; c0 < round_up(dcur, 16); c0 += 16) {
          uint32_t hi[16], lo[16];
          tmem_ld16(tAh + lane_off + c0, hi);
          if (SPLIT == 3) tmem_ld16(tAl + lane_off + c0, lo);
          tmem_wait_ld();
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int k = c0 + t;
            if (row < d0 && k < dcur) {
              float z = __uint_as_float(hi[t]);
              if (SPLIT == 3) z += __uint_as_float(lo[t]);
              acc = fmaf(float(M.blk[off + int64_t(row) * dcur + k]), z, acc);
            }
          }
        }
        vr = double(acc) * double(scale);
        double dm = 0.0;
        block_max_sum(dm, vr, S.redd);
        if (tid == 0) {
          W.res_val[2 * slot] = vr;
          W.res_val[2 * slot + 1] = vi;
          const bool zero_v = (vr == 0.0);
          W.res_log[slot] = zero_v ? -INFINITY : L.val() + double(Eacc) * LN2;
          if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(fabs(vr)) + L.val() + double(Eacc) * LN2;
        }
        applied = n;
        break;
      }

      // ---- tensor-core product Z <- Z F^T, then column scale
      const int db = M.dims[qb];
      const int np = round_up(db, 16), kp = round_up(dcur, 8);
      if (tid == 0) {
        // prefetch the next block into the other stage (its last reader has completed)
        if (i + 1 < n - 1) {
          const int alpha_n = B.op[a0 + i + 1];
          const int qn = M.s[alpha_n * ns + qb];
          const int np2 = round_up(M.dims[qn], 16), kp2 = round_up(db, 8);
          const uint32_t bytes = uint32_t(SPLIT == 3 ? 2 : 1) * np2 * kp2 * 4;
          const int st2 = cur_stage ^ 1;
          mbar_arrive_expect_tx(&S.bar_load[st2], bytes);
          bulk_g2s(stage[st2], P.blk + P.off[alpha_n * ns + qb], bytes, &S.bar_load[st2]);
          pending[st2] = 1;
        }
        // operand of this product
        bool ok = mbar_wait(&S.bar_load[cur_stage], ph_load[cur_stage], P.timeout_ns);
        if (ok) {
          ph_load[cur_stage] ^= 1u;
          pending[cur_stage] = 0;
          tc_fence_after();
          const uint32_t sb = smem_u32(stage[cur_stage]);
          const uint32_t lbo = uint32_t(np / 8) * 128u, sbo = 128u;
          const uint32_t lo_off = uint32_t(np) * kp * 4u;
          const uint32_t id = idesc_tf32(TC_M, np);
          for (int kk = 0; kk < kp / 8; ++kk) {
            const uint32_t kb = uint32_t(2 * kk) * lbo;
            mma_tf32_ts(tD, tAh + 8 * kk, sdesc(sb + kb, lbo, sbo), id, kk > 0 ? 1u : 0u);
            if (SPLIT == 3) {
              mma_tf32_ts(tD, tAh + 8 * kk, sdesc(sb + lo_off + kb, lbo, sbo), id, 1u);
              mma_tf32_ts(tD, tAl + 8 * kk, sdesc(sb + kb, lbo, sbo), id, 1u);
            }
          }
          mma_commit(&S.bar_mma);
        } else {
          S.fail = 1;
        }
      }
      // column scales of this step (overlaps the MMA)
      {
        const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
        const float* Eb = M.E_relf + M.E_off[qb];
        const float dtf = float(dt);
        for (int j = tid; j < TC_M; j += TC_THREADS) p_s[j] = (j < db) ? __expf(-dtf * Eb[j]) * scale : 0.0f;
        if (tid == 0) {
          L.add(-dt * (M.E_min[qb] - M.E_ref));
          prefix -= dt * (M.E_min[qb] - M.E_ref);
        }
      }
      __syncthreads();
      bool ok = (S.fail == 0) && mbar_wait(&S.bar_mma, ph_mma, P.timeout_ns);
      ph_mma ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) S.fail = 1;
        break;
      }
      tc_fence_after();
      // epilogue: Z_next[row][j] = D[row][j] * p_s[j]
      mx = 0.f;
      fr = 0.f;
      for (int c0 = 0; c0 < np; c0 += 16) {
        uint32_t v[16], hi[16], lo[16];
        tmem_ld16(tD + lane_off + c0, v);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const float x = __uint_as_float(v[t]) * p_s[c0 + t];
          mx = fmaxf(mx, fabsf(x));
          fr += x * x;
          hi[t] = to_tf32(x);
          lo[t] = to_tf32(x - __uint_as_float(hi[t]));
        }
        tmem_st16(tAh + lane_off + c0, hi);
        if (SPLIT == 3) tmem_st16(tAl + lane_off + c0, lo);
      }
      tmem_wait_st();
      tc_fence_before();
      block_max_sum_f(mx, fr, S.red);
      cur_stage ^= 1;
      dcur = db;
      qa = qb;
      ++applied;
    }
    // drain prefetches that this item no longer needs
    if (tid == 0) {
      for (int st = 0; st < 2; ++st)
        if (pending[st]) {
          if (mbar_wait(&S.bar_load[st], ph_load[st], P.timeout_ns)) ph_load[st] ^= 1u;
          else S.fail = 1;
          pending[st] = 0;
        }
    }
    if (tid == 0) {
      if (dead) {
        W.res_val[2 * slot] = 0.0;
        W.res_val[2 * slot + 1] = 0.0;
        W.res_log[slot] = -INFINITY;
        if (track)
          for (int s = (applied + cfg.S - 1) / cfg.S; s <= it.n_seg; ++s)
            if (s > 0) segp[s] = -INFINITY;
      }
      if (aborted) W.res_log[slot] = NAN;
      if (S.fail) {
        W.res_log[slot] = NAN;
        atomicOr(&W.counters[2], 1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(P.tmem_cols));
  }
}

// One D = A B^T product (M = 128) with the same operand layouts as k_trace_tc:
// A (128 x K, row-major floats) written to TMEM with tcgen05.st, B (N x K,
// row-major) formatted by the threads into K-major core matrices in shared
// memory, D read back with tcgen05.ld.  Diagnostic for the descriptor and
// layout conventions.
template <int SPLIT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm_check(const float* A, const float* Bm, float* D, int N,
                                                                 int K, uint64_t timeout_ns, int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sb = reinterpret_cast<float*>(smem_raw);
  __shared__ TcShared S;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&S.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // B: hi at 0, lo at N*K (core matrix (nb, kb) at ((kb * N/8) + nb) * 32 floats)
  const int cnt = N * K;
  for (int idx = tid; idx < cnt; idx += TC_THREADS) {
    const int nn = idx / K, k = idx - nn * K;
    const int pos = ((k / 4) * (N / 8) + nn / 8) * 32 + (nn % 8) * 4 + (k % 4);
    const float f = Bm[idx];
    const uint32_t hi = to_tf32(f);
    sb[pos] = __uint_as_float(hi);
    sb[cnt + pos] = __uint_as_float(to_tf32(f - __uint_as_float(hi)));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tmem_base;
  const uint32_t lane_off = uint32_t(32 * warp) << 16;
  const uint32_t tD = tbase, tAh = tbase + 128, tAl = tbase + 256;
  for (int c0 = 0; c0 < K; c0 += 16) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const float x = (c0 + t < K) ? A[tid * K + c0 + t] : 0.f;
      hi[t] = to_tf32(x);
      lo[t] = to_tf32(x - __uint_as_float(hi[t]));
    }
    tmem_st16(tAh + lane_off + c0, hi);
    tmem_st16(tAl + lane_off + c0, lo);
  }
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    const uint32_t base = smem_u32(sb);
    const uint32_t lbo = uint32_t(N / 8) * 128u, sbo = 128u;
    const uint32_t id = idesc_tf32(TC_M, N);
    for (int kk = 0; kk < K / 8; ++kk) {
      const uint32_t kb = uint32_t(2 * kk) * lbo;
      mma_tf32_ts(tD, tAh + 8 * kk, sdesc(base + kb, lbo, sbo), id, kk > 0 ? 1u : 0u);
      if (SPLIT == 3) {
        mma_tf32_ts(tD, tAh + 8 * kk, sdesc(base + uint32_t(cnt) * 4u + kb, lbo, sbo), id, 1u);
        mma_tf32_ts(tD, tAl + 8 * kk, sdesc(base + kb, lbo, sbo), id, 1u);
      }
    }
    mma_commit(&S.bar_mma);
  }
  const bool ok = mbar_wait(&S.bar_mma, 0, timeout_ns);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) *status = CTQ_ERR_TIMEOUT;
  } else {
    tc_fence_after();
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tD + lane_off + c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int t = 0; t < 16; ++t) D[tid * N + c0 + t] = __uint_as_float(v[t]);
    }
    if (tid == 0) *status = CTQ_OK;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
  }
}

}  // namespace

// ----------------------------------------------------------------- host side

// Pre-formats every real block F_alpha(q) (d_{q'} x d_q) as the B operand of
// Z F^T: N = d_{q'} rows padded to 16, K = d_q padded to 8, K-major core
// matrices of 8 rows x 4 floats, core (nb, kb) at ((kb * N/8) + nb) * 32
// floats; hi = tf32(F) and, for split mode, lo = tf32(F - hi) after it.
int build_tc_blocks(const HostModel& h, int split, std::vector<float>& out, std::vector<int64_t>& off,
                    int* stage_floats) {
  if (h.is_complex) return CTQ_ERR_UNSUPPORTED;
  const int na = h.n_alpha();
  off.assign(size_t(na) * h.n_sec, -1);
  out.clear();
  int max_stage = 0;
  auto tf32 = [](float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {  // round half away from zero on the magnitude
      u += 0x1000u;
      u &= 0xffffe000u;
    }
    float r;
    std::memcpy(&r, &u, 4);
    return r;
  };
  for (int a = 0; a < na; ++a)
    for (int q = 0; q < h.n_sec; ++q) {
      const size_t i = size_t(a) * h.n_sec + q;
      const int qp = h.s[i];
      if (qp < 0) continue;
      const int dn = h.dims[qp], dk = h.dims[q];
      const int np = (dn + 15) / 16 * 16, kp = (dk + 7) / 8 * 8;
      const size_t base = (out.size() + 31) / 32 * 32;  // 128-byte aligned
      const size_t cnt = size_t(np) * kp;
      out.resize(base + (split == 3 ? 2 : 1) * cnt, 0.0f);
      off[i] = int64_t(base);
      max_stage = std::max(max_stage, int((split == 3 ? 2 : 1) * cnt));
      const double* F = &h.blk_re[h.blk_off[i]];
      for (int nn = 0; nn < dn; ++nn)
        for (int k = 0; k < dk; ++k) {
          const size_t pos = (size_t(k / 4) * (np / 8) + nn / 8) * 32 + (nn % 8) * 4 + (k % 4);
          const double f = F[size_t(nn) * dk + k];
          const float hi = tf32(float(f));
          out[base + pos] = hi;
          if (split == 3) out[base + cnt + pos] = tf32(float(f - double(hi)));
        }
    }
  *stage_floats = max_stage;
  return CTQ_OK;
}

int prepare_eval_tc(const DevModel& M, int split, int stage_floats, int num_sms, LaunchCfg* lc) {
  lc->threads = TC_THREADS;
  lc->smem = size_t(2) * stage_floats * 4 + 2 * TC_M * 4;
  // At most 512 / tmem_cols CTAs may share an SM (each holds its TMEM for the
  // whole kernel): request enough shared memory to enforce that.
  lc->smem = std::max(lc->smem, size_t(split == 3 ? 116 * 1024 : 76 * 1024));
  lc->num_sms = num_sms;
  lc->per_sm = 0;
  if (M.is_complex || M.max_dim > TC_M || lc->smem > 227 * 1024) return CTQ_OK;  // not supported
  cudaError_t e = (split == 3)
                      ? cudaFuncSetAttribute(k_trace_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem))
                      : cudaFuncSetAttribute(k_trace_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem));
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  int per_sm = 0;
  e = (split == 3) ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tc<3>, TC_THREADS, lc->smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_tc<1>, TC_THREADS, lc->smem);
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  lc->per_sm = std::min(per_sm, split == 3 ? 1 : 2);  // TMEM: 512 or 256 columns per CTA
  return CTQ_OK;
}

int launch_eval_tc(const DevModel& M, const LaunchCfg& lc, const TcParams& P, const BatchView& B,
                   const EvalCfg& cfg, const Work& W, const ctq_result* R, void* stream, void* const* events) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (lc.per_sm < 1) return CTQ_ERR_UNSUPPORTED;
  auto mark = [&](int i) {
    if (events) cudaEventRecord(static_cast<cudaEvent_t>(events[i]), st);
  };
  if (cudaMemsetAsync(W.counters, 0, 256, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(0);
  {
    const int ps = launch_plan(M, B, cfg, W, st);
    if (ps != CTQ_OK) return ps;
  }
  mark(1);
  long long max_items = (long long)B.n_chains * M.n_sec;
  long long grid = (long long)lc.num_sms * lc.per_sm;
  if (grid > max_items) grid = max_items;
  if (P.split == 3)
    k_trace_tc<3><<<int(grid), TC_THREADS, lc.smem, st>>>(M, B, cfg, W, P);
  else
    k_trace_tc<1><<<int(grid), TC_THREADS, lc.smem, st>>>(M, B, cfg, W, P);
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

extern "C" int ctq_tc_gemm_check(int device, const float* A, const float* Bm, float* D, int N, int K, int split) {
  using namespace ctq;
  if (!A || !Bm || !D || N < 16 || N > 112 || N % 16 || K < 16 || K > 112 || K % 16 || (split != 1 && split != 3))
    return CTQ_ERR_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return CTQ_ERR_CUDA;
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dS = nullptr;
  int st = CTQ_OK, hs = CTQ_ERR_CUDA;
  // hi + lo operands, with as much again of slack behind them
  const size_t smem = size_t(4) * N * K * 4;
  if (cudaMalloc(&dA, size_t(128) * K * 4) || cudaMalloc(&dB, size_t(N) * K * 4) ||
      cudaMalloc(&dD, size_t(128) * N * 4) || cudaMalloc(&dS, 4)) {
    st = CTQ_ERR_NOMEM;
  } else {
    cudaMemcpy(dA, A, size_t(128) * K * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, Bm, size_t(N) * K * 4, cudaMemcpyHostToDevice);
    cudaMemset(dS, 0xff, 4);
    if (split == 3) {
      cudaFuncSetAttribute(k_tc_gemm_check<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_tc_gemm_check<3><<<1, TC_THREADS, smem>>>(dA, dB, dD, N, K, 2000000000ull, dS);
    } else {
      cudaFuncSetAttribute(k_tc_gemm_check<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_tc_gemm_check<1><<<1, TC_THREADS, smem>>>(dA, dB, dD, N, K, 2000000000ull, dS);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) st = CTQ_ERR_CUDA;
    if (st == CTQ_OK) {
      cudaMemcpy(D, dD, size_t(128) * N * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(&hs, dS, 4, cudaMemcpyDeviceToHost);
      st = hs;
    }
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dS);
  if (prev != device) cudaSetDevice(prev);
  return st;
}
