// Sector-string local trace on the 5th-generation tensor cores (tcgen05).
//
// Same mathematics as k_trace (trace_fp64.cu), with the block products in
// TF32, in three-term split TF32 (hi*hi + hi*lo + lo*hi) or in three-term
// split bf16 (bf16 hi / lo operands, kind::f16 MMAs), all with FP32
// accumulation; the log scale, the renormalisation exponents, the segment
// bounds and the final trace sum stay in float64 (mixed-precision reading of
// Sec. 3.3.2, which anticipates mixed-precision products).
//
// Layout (one (chain, q0) item per CTA at a time, 4 warps):
//   The chain runs transposed, Z_i = Y_i^T (d0 x d_i):
//       Z_{i+1} = Z_i F_{i+1}^T P_{i+1}
//   so that the running product is the MMA's A operand and stays in tensor
//   memory (TMEM) for the whole chain: A = Z_i (128 lanes = rows of Z, one
//   32-bit column per tf32 K element, or two bf16 K elements packed per
//   column), B = F_{i+1}^T, whose K-major form is F's own
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
constexpr int TC_MAX_DIM = 112;  // largest sector of the small-block kernel (A, D <= 128 columns)
constexpr int TC_META_BYTES = 8192;  // staged string of one item: see k_trace_tc

// Bytes of the staged string for max_ops operators and n_seg_max segments.
__host__ __device__ constexpr size_t tc_meta_bytes(int max_ops, int n_seg_max) {
  return size_t(4) * (n_seg_max + 1) * 8 + size_t(max_ops > 1 ? max_ops : 1) * (4 + 2 + 2) + 2;
}

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

// K padding of a block: one MMA takes 8 tf32 or 16 bf16 K elements.
__host__ __device__ constexpr int tc_kstep(int prec) { return prec == CTQ_BF16X3 ? 16 : 8; }

// Writes 16 consecutive K elements (from column element c0) of this
// thread's row of the A operand into tensor memory, split as PREC needs.
template <int PREC>
__device__ __forceinline__ void store_a16(uint32_t tAh, uint32_t tAl, int c0, const float (&x)[16]) {
  if constexpr (PREC == CTQ_BF16X3) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) split_bf16x2(x[2 * t], x[2 * t + 1], hi[t], lo[t]);
    tmem_st8(tAh + uint32_t(c0 / 2), hi);
    tmem_st8(tAl + uint32_t(c0 / 2), lo);
  } else {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      hi[t] = to_tf32(x[t]);
      lo[t] = to_tf32(x[t] - __uint_as_float(hi[t]));
    }
    tmem_st16(tAh + uint32_t(c0), hi);
    if (PREC == CTQ_TF32X3) tmem_st16(tAl + uint32_t(c0), lo);
  }
}

// Reads back 16 K elements of this thread's row of A (hi + lo).
template <int PREC>
__device__ __forceinline__ void load_a16(uint32_t tAh, uint32_t tAl, int c0, float (&z)[16]) {
  if constexpr (PREC == CTQ_BF16X3) {
    uint32_t hi[8], lo[8];
    tmem_ld8(tAh + uint32_t(c0 / 2), hi);
    tmem_ld8(tAl + uint32_t(c0 / 2), lo);
    tmem_wait_ld();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      z[2 * t] = bf16_val(hi[t] & 0xffffu) + bf16_val(lo[t] & 0xffffu);
      z[2 * t + 1] = bf16_val(hi[t] >> 16) + bf16_val(lo[t] >> 16);
    }
  } else {
    uint32_t hi[16], lo[16];
    tmem_ld16(tAh + uint32_t(c0), hi);
    if (PREC == CTQ_TF32X3) tmem_ld16(tAl + uint32_t(c0), lo);
    tmem_wait_ld();
#pragma unroll
    for (int t = 0; t < 16; ++t) z[t] = __uint_as_float(hi[t]) + (PREC == CTQ_TF32X3 ? __uint_as_float(lo[t]) : 0.f);
  }
}

// D = A B^T for one block: A in tensor memory (hi at tAh, lo at tAl), B in
// shared memory at sb (hi plane, then lo plane at lo_off bytes), np x kp.
template <int PREC>
__device__ __forceinline__ void mma_block(uint32_t tD, uint32_t tAh, uint32_t tAl, uint32_t sb, int np, int kp,
                                          uint32_t lo_off) {
  const uint32_t lbo = uint32_t(np / 8) * 128u, sbo = 128u;
  const uint32_t id = (PREC == CTQ_BF16X3) ? idesc_bf16(TC_M, np) : idesc_tf32(TC_M, np);
  // one MMA: 32 bytes of K (two core matrices of B, 8 tensor-memory columns of A)
  for (int kk = 0; kk < kp / tc_kstep(PREC); ++kk) {
    const uint32_t kb = uint32_t(2 * kk) * lbo;
    const uint32_t ah = tAh + 8u * kk, al = tAl + 8u * kk;
    if constexpr (PREC == CTQ_BF16X3) {
      mma_bf16_ts(tD, ah, sdesc(sb + kb, lbo, sbo), id, kk > 0 ? 1u : 0u);
      mma_bf16_ts(tD, ah, sdesc(sb + lo_off + kb, lbo, sbo), id, 1u);
      mma_bf16_ts(tD, al, sdesc(sb + kb, lbo, sbo), id, 1u);
    } else {
      mma_tf32_ts(tD, ah, sdesc(sb + kb, lbo, sbo), id, kk > 0 ? 1u : 0u);
      if (PREC == CTQ_TF32X3) {
        mma_tf32_ts(tD, ah, sdesc(sb + lo_off + kb, lbo, sbo), id, 1u);
        mma_tf32_ts(tD, al, sdesc(sb + kb, lbo, sbo), id, 1u);
      }
    }
  }
}

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
  double L;  // log scale of the current string (warp 0 writes)
};

}  // namespace


namespace {

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_trace_tc(DevModel M, BatchView B, EvalCfg cfg, Work W, TcParams P) {
  constexpr int EB = PREC == CTQ_BF16X3 ? 2 : 4;  // bytes per staged B element
  constexpr bool SPLIT = PREC != CTQ_TF32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* stage[2];
  stage[0] = smem_raw;
  stage[1] = stage[0] + P.stage_bytes;
  float* p_s = reinterpret_cast<float*>(stage[1] + P.stage_bytes);  // [128] column scales of the current step
  float* p0_s = p_s + TC_M;                // [128] wrap-around propagator of q0
  // the item's string, staged once (TC_META_BYTES): log scale and applied
  // log-norm sums at segment ends, operator codes, sectors, time steps
  const int MO = max(cfg.max_ops, 1), NS = cfg.n_seg_max + 1;
  double* segL = reinterpret_cast<double*>(p0_s + TC_M);  // [NS]
  double* segP = segL + NS;                                // [NS]
  double* segF = segP + NS;                                // [NS] ||Z||^2 at segment ends (deferred bounds)
  double* segE = segF + NS;                                // [NS] exponent sums at segment ends
  float* dtf = reinterpret_cast<float*>(segE + NS);        // [MO] tau_{i+1} - tau_i
  short* opsm = reinterpret_cast<short*>(dtf + MO);        // [MO]
  short* path = opsm + MO;                                 // [MO + 1]
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
  // D: columns [0, 128); A hi from 128; A lo from 256 (3xTF32) or 192 (bf16,
  // two K elements per column).  Addresses include this warp's lane quarter.
  const uint32_t tD = tbase;
  const uint32_t tAh = tbase + 128 + lane_off;
  const uint32_t tAl = tbase + (PREC == CTQ_BF16X3 ? 192 : 256) + lane_off;

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
    const Item it = items[W.order[it_idx]];
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

    // ---- the string once: operator codes and time steps (all threads),
    // sectors (thread 0, integer walk), log scale and segment sums (warp 0,
    // compensated, lanes over chunks of operators)
    const double t_first = B.tau[a0], t_last = B.beta - B.tau[a0 + n - 1];
    for (int i = tid; i < n; i += TC_THREADS) {
      opsm[i] = short(B.op[a0 + i]);
      if (i + 1 < n) dtf[i] = float(B.tau[a0 + i + 1] - B.tau[a0 + i]);
    }
    __syncthreads();
    if (tid == 0) {
      int q = q0;
      path[0] = short(q0);
      for (int i = 0; i < n; ++i) {
        q = M.s[opsm[i] * ns + q];
        path[i + 1] = short(q);
      }
    }
    __syncthreads();
    if (tid < 32) chain_log_scale(M, B, cfg, a0, n, q0, t_first, t_last, track, path, opsm, segL, segP, &S.L);
    const double ub_const = track ? 0.5 * it.log_r + it.t_all : 0.0;  // sqrt(r), all log-norms

    // ---- operator 1 (elementwise): Z_1[j][m] = p0[j] F_1[m][j] p1[m]
    int qa = q0;
    int alpha = opsm[0];
    int qb = path[1];
    long long Eacc = 0;
    {
      const float dt1 = dtf[0];
      const float* Eb = M.E_relf + M.E_off[qb];
      const float* E0f = M.E_relf + M.E_off[q0];
      const int db = M.dims[qb];
      for (int j = tid; j < TC_M; j += TC_THREADS) {
        // FP32 exponentials: an absolute argument error of ~1e-7 x changes
        // e^{-x} by at most max(x e^{-x}) 1e-7 < 4e-8 relative to the largest
        // entry, below the resolution of the products.
        p_s[j] = (j < db) ? __expf(-dt1 * Eb[j]) : 0.0f;
        p0_s[j] = (j < d0) ? __expf(-float(t_first) * E0f[j]) * __expf(-float(t_last) * E0f[j]) : 0.0f;
      }
    }
    // prefetch the block of operator 2 (the first tensor-core product)
    if (tid == 0 && n > 2) {
      const int alpha2 = opsm[1];
      const int qn = path[2];
      const int np = round_up(M.dims[qn], 16), kp = round_up(M.dims[qb], tc_kstep(PREC));
      const uint32_t bytes = uint32_t(SPLIT ? 2 : 1) * np * kp * EB;
      mbar_arrive_expect_tx(&S.bar_load[0], bytes);
      bulk_g2s(stage[0], static_cast<const unsigned char*>(P.blk) + P.off[alpha2 * ns + qb], bytes, &S.bar_load[0]);
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
        float x[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const int m = c0 + t;
          x[t] = 0.f;
          if (row < d0 && m < dcur) x[t] = float(M.blk[off + int64_t(m) * d0 + row]) * p0r * p_s[m];
          mx = fmaxf(mx, fabsf(x[t]));
          fr += x[t] * x[t];
        }
        store_a16<PREC>(tAh, tAl, c0, x);
      }
      tmem_wait_st();
    }
    tc_fence_before();
    block_max_sum_f(mx, fr, S.red);
    qa = qb;
    int applied = 1;
    int k_rec = 0;  // segments recorded for the deferred bounds
    bool dead = false, aborted = false;
    int cur_stage = 0;

    for (int i = 1; i < n; ++i) {
      if (mx == 0.f) { dead = true; break; }
      const int e = ilogbf(mx);
      if (track && applied % cfg.S == 0 && applied < n) {
        if (!cfg.lazy) {  // bounds output only: the logarithms are taken for all segments at the end
          if (tid == 0) {
            segF[applied / cfg.S] = double(fr);
            segE[applied / cfg.S] = double(Eacc);
          }
          k_rec = applied / cfg.S;
        } else if (tid == 0) {
          const double ub = ub_const + 0.5 * log(double(fr)) + double(Eacc) * LN2 + segL[applied / cfg.S] -
                            segP[applied / cfg.S];
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
              S.abort_flag = (flag & FLAG_REJECTED) ? 1 : 0;
            }
          }
          __syncthreads();
          if (S.abort_flag) { aborted = true; break; }
        }
      }
      alpha = opsm[i];
      const int idx_a = alpha * ns + qa;
      qb = path[i + 1];
      const float scale = ldexpf(1.0f, -e);
      Eacc += e;

      if (i == n - 1) {  // final operator: diagonal of F_n Y = sum_{j,k} F_n[j][k] Z[j][k]
        const int64_t off = M.blk_off[idx_a];
        double vr = 0.0, vi = 0.0;
        float acc = 0.f;
        tc_fence_after();
        for (int c0 = 0; c0 < round_up(dcur, 16); c0 += 16) {
          float z[16];
          load_a16<PREC>(tAh, tAl, c0, z);
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int k = c0 + t;
            if (row < d0 && k < dcur) acc = fmaf(float(M.blk[off + int64_t(row) * dcur + k]), z[t], acc);
          }
        }
        vr = double(acc) * double(scale);
        double dm = 0.0;
        block_max_sum(dm, vr, S.redd);
        if (tid == 0) {
          W.res_val[2 * slot] = vr;
          W.res_val[2 * slot + 1] = vi;
          const bool zero_v = (vr == 0.0);
          W.res_log[slot] = zero_v ? -INFINITY : S.L + double(Eacc) * LN2;
          if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(fabs(vr)) + S.L + double(Eacc) * LN2;
        }
        applied = n;
        break;
      }

      // ---- tensor-core product Z <- Z F^T, then column scale
      const int db = M.dims[qb];
      const int np = round_up(db, 16), kp = round_up(dcur, tc_kstep(PREC));
      if (tid == 0) {
        // prefetch the next block into the other stage (its last reader has completed)
        if (i + 1 < n - 1) {
          const int alpha_n = opsm[i + 1];
          const int qn = path[i + 2];
          const int np2 = round_up(M.dims[qn], 16), kp2 = round_up(db, tc_kstep(PREC));
          const uint32_t bytes = uint32_t(SPLIT ? 2 : 1) * np2 * kp2 * EB;
          const int st2 = cur_stage ^ 1;
          mbar_arrive_expect_tx(&S.bar_load[st2], bytes);
          bulk_g2s(stage[st2], static_cast<const unsigned char*>(P.blk) + P.off[alpha_n * ns + qb], bytes,
                   &S.bar_load[st2]);
          pending[st2] = 1;
        }
        // operand of this product
        bool ok = mbar_wait(&S.bar_load[cur_stage], ph_load[cur_stage], P.timeout_ns);
        if (ok) {
          ph_load[cur_stage] ^= 1u;
          pending[cur_stage] = 0;
          tc_fence_after();
          // thread 0 is lane 0 of warp 0: its A addresses are the operand's base
          mma_block<PREC>(tD, tAh, tAl, smem_u32(stage[cur_stage]), np, kp, uint32_t(np) * kp * EB);
          mma_commit(&S.bar_mma);
        } else {
          S.fail = 1;
        }
      }
      // column scales of this step (overlaps the MMA)
      {
        const float* Eb = M.E_relf + M.E_off[qb];
        const float dti = dtf[i];
        for (int j = tid; j < TC_M; j += TC_THREADS) p_s[j] = (j < db) ? __expf(-dti * Eb[j]) * scale : 0.0f;
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
      for (int g0 = 0; g0 < np; g0 += 64) {  // four tensor-memory loads in flight, one wait
        uint32_t v[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (g0 + 16 * u < np) tmem_ld16(tD + lane_off + g0 + 16 * u, v[u]);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (g0 + 16 * u >= np) break;
          const int c0 = g0 + 16 * u;
          float x[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            x[t] = __uint_as_float(v[u][t]) * p_s[c0 + t];
            mx = fmaxf(mx, fabsf(x[t]));
            fr += x[t] * x[t];
          }
          store_a16<PREC>(tAh, tAl, c0, x);
        }
      }
      tmem_wait_st();
      tc_fence_before();
      block_max_sum_f(mx, fr, S.red);
      cur_stage ^= 1;
      dcur = db;
      qa = qb;
      ++applied;
    }
    if (k_rec > 0) {  // deferred bounds, lanes over segments
      __syncthreads();
      for (int k = 1 + tid; k <= k_rec; k += TC_THREADS)
        segp[k] = ub_const + 0.5 * log(segF[k]) + segE[k] * LN2 + segL[k] - segP[k];
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
// layout conventions of each precision.
template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gemm_check(const float* A, const float* Bm, float* D, int N,
                                                                 int K, uint64_t timeout_ns, int* status) {
  constexpr int EB = PREC == CTQ_BF16X3 ? 2 : 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
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
  // B: hi plane at 0, lo plane at N*K elements; core matrix (nb, kb) of 8 rows
  // x 16 bytes at ((kb * N/8) + nb) * 128 bytes
  const int cnt = N * K;
  constexpr int EPC = 16 / EB;
  for (int idx = tid; idx < cnt; idx += TC_THREADS) {
    const int nn = idx / K, k = idx - nn * K;
    const int pos = ((k / EPC) * (N / 8) + nn / 8) * (8 * EPC) + (nn % 8) * EPC + (k % EPC);
    const float f = Bm[idx];
    if constexpr (PREC == CTQ_BF16X3) {
      uint16_t* sb = reinterpret_cast<uint16_t*>(smem_raw);
      const uint32_t h = bf16_bits(f);
      sb[pos] = uint16_t(h);
      sb[cnt + pos] = uint16_t(bf16_bits(f - bf16_val(h)));
    } else {
      float* sb = reinterpret_cast<float*>(smem_raw);
      const uint32_t h = to_tf32(f);
      sb[pos] = __uint_as_float(h);
      sb[cnt + pos] = __uint_as_float(to_tf32(f - __uint_as_float(h)));
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tmem_base;
  const uint32_t lane_off = uint32_t(32 * warp) << 16;
  const uint32_t tD = tbase;
  const uint32_t tAh = tbase + 128 + lane_off;
  const uint32_t tAl = tbase + (PREC == CTQ_BF16X3 ? 192 : 256) + lane_off;
  for (int c0 = 0; c0 < K; c0 += 16) {
    float x[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) x[t] = (c0 + t < K) ? A[tid * K + c0 + t] : 0.f;
    store_a16<PREC>(tAh, tAl, c0, x);
  }
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    mma_block<PREC>(tD, tAh, tAl, smem_u32(smem_raw), N, K, uint32_t(cnt) * EB);
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
// Z F^T: N = d_{q'} rows padded to 16, K = d_q padded to 8 (tf32) or 16
// (bf16), K-major core matrices of 8 rows x 16 bytes, core (nb, kb) at
// ((kb * N/8) + nb) * 128 bytes; the hi plane (tf32(F) or bf16(F)) and, for
// the split precisions, the lo plane (of F - hi) after it.  Offsets and
// stage sizes in bytes; every block starts on a 128-byte boundary.
int build_tc_blocks(const HostModel& h, int prec, std::vector<unsigned char>& out, std::vector<int64_t>& off,
                    int* stage_bytes) {
  if (h.is_complex) return CTQ_ERR_UNSUPPORTED;
  const bool bf = prec == CTQ_BF16X3;
  const bool split = prec != CTQ_TF32;
  const int eb = bf ? 2 : 4, epc = 16 / eb, kstep = tc_kstep(prec);
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
  auto bf16 = [](float x) -> uint16_t {  // round to nearest even (finite x)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return uint16_t((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
  };
  auto bf16_value = [](uint16_t b) {
    const uint32_t u = uint32_t(b) << 16;
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
      const int np = (dn + 15) / 16 * 16, kp = (dk + kstep - 1) / kstep * kstep;
      const size_t base = (out.size() + 127) / 128 * 128;
      const size_t cnt = size_t(np) * kp;  // elements of one plane
      const size_t bytes = (split ? 2 : 1) * cnt * eb;
      out.resize(base + bytes, 0);
      off[i] = int64_t(base);
      max_stage = std::max(max_stage, int(bytes));
      const double* F = &h.blk_re[h.blk_off[i]];
      for (int nn = 0; nn < dn; ++nn)
        for (int k = 0; k < dk; ++k) {
          const size_t pos = (size_t(k / epc) * (np / 8) + nn / 8) * (8 * epc) + (nn % 8) * epc + (k % epc);
          const double f = F[size_t(nn) * dk + k];
          if (bf) {
            const uint16_t hi = bf16(float(f));
            const uint16_t lo = bf16(float(f - double(bf16_value(hi))));
            std::memcpy(&out[base + pos * 2], &hi, 2);
            std::memcpy(&out[base + (cnt + pos) * 2], &lo, 2);
          } else {
            const float hi = tf32(float(f));
            std::memcpy(&out[base + pos * 4], &hi, 4);
            if (split) {
              const float lo = tf32(float(f - double(hi)));
              std::memcpy(&out[base + (cnt + pos) * 4], &lo, 4);
            }
          }
        }
    }
  *stage_bytes = max_stage;
  return CTQ_OK;
}

template <int PREC>
static cudaError_t tc_attr(size_t smem) {
  const cudaError_t e = cudaFuncSetAttribute(k_trace_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  // all of the SM's unified L1 / shared storage as shared memory, so that two
  // CTAs of the 256-column precisions can be resident together
  return cudaFuncSetAttribute(k_trace_tc<PREC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              int(cudaSharedmemCarveoutMaxShared));
}

int prepare_eval_tc(const DevModel& M, int prec, int stage_bytes, int num_sms, LaunchCfg* lc) {
  lc->threads = TC_THREADS;
  lc->smem = size_t(2) * stage_bytes + 2 * TC_M * 4 + TC_META_BYTES;
  // At most 512 / tmem_cols CTAs may share an SM (each holds its TMEM for the
  // whole kernel): request enough shared memory to enforce that.
  lc->smem = std::max(lc->smem, size_t(prec == CTQ_TF32X3 ? 116 * 1024 : 76 * 1024));
  lc->num_sms = num_sms;
  lc->per_sm = 0;
  if (M.is_complex || M.max_dim > TC_MAX_DIM || lc->smem > 227 * 1024) return CTQ_OK;  // not supported
  cudaError_t e = prec == CTQ_TF32     ? tc_attr<CTQ_TF32>(lc->smem)
                  : prec == CTQ_BF16X3 ? tc_attr<CTQ_BF16X3>(lc->smem)
                                       : tc_attr<CTQ_TF32X3>(lc->smem);
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  // resident CTAs per SM: shared memory (with the 1 KB per CTA the CUDA runtime reserves),
  // registers, and tensor memory (512 or 256 of the SM's 512 columns)
  cudaFuncAttributes fa;
  e = prec == CTQ_TF32     ? cudaFuncGetAttributes(&fa, k_trace_tc<CTQ_TF32>)
      : prec == CTQ_BF16X3 ? cudaFuncGetAttributes(&fa, k_trace_tc<CTQ_BF16X3>)
                           : cudaFuncGetAttributes(&fa, k_trace_tc<CTQ_TF32X3>);
  int dev = 0, sm_smem = 0;
  if (e != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return CTQ_ERR_CUDA;
  const int by_smem = int(size_t(sm_smem) / (lc->smem + fa.sharedSizeBytes + 1024));
  const int regs = (fa.numRegs + 7) / 8 * 8;
  const int by_regs = 65536 / std::max(1, regs * TC_THREADS);
  const int by_tmem = prec == CTQ_TF32X3 ? 1 : 2;
  lc->regs = fa.numRegs;
  lc->per_sm = std::max(0, std::min(by_smem, std::min(by_regs, by_tmem)));
  return CTQ_OK;
}

int launch_eval_tc(const DevModel& M, const LaunchCfg& lc, const TcParams& P, const BatchView& B,
                   const EvalCfg& cfg, const Work& W, const ctq_result* R, void* stream, void* const* events) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (lc.per_sm < 1) return CTQ_ERR_UNSUPPORTED;
  if (tc_meta_bytes(cfg.max_ops, cfg.n_seg_max) > size_t(TC_META_BYTES)) return CTQ_ERR_UNSUPPORTED;
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
  const int per_sm = cfg.ctas_per_sm > 0 ? std::min(lc.per_sm, cfg.ctas_per_sm) : lc.per_sm;
  long long grid = (long long)lc.num_sms * per_sm;
  if (grid > max_items) grid = max_items;
  if (P.prec == CTQ_TF32)
    k_trace_tc<CTQ_TF32><<<int(grid), TC_THREADS, lc.smem, st>>>(M, B, cfg, W, P);
  else if (P.prec == CTQ_BF16X3)
    k_trace_tc<CTQ_BF16X3><<<int(grid), TC_THREADS, lc.smem, st>>>(M, B, cfg, W, P);
  else
    k_trace_tc<CTQ_TF32X3><<<int(grid), TC_THREADS, lc.smem, st>>>(M, B, cfg, W, P);
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
  if (!A || !Bm || !D || N < 16 || N > 112 || N % 16 || K < 16 || K > 112 || K % 16 ||
      (split != CTQ_TF32 && split != CTQ_TF32X3 && split != CTQ_BF16X3))
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
    if (split == CTQ_TF32X3) {
      cudaFuncSetAttribute(k_tc_gemm_check<CTQ_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_tc_gemm_check<CTQ_TF32X3><<<1, TC_THREADS, smem>>>(dA, dB, dD, N, K, 2000000000ull, dS);
    } else if (split == CTQ_BF16X3) {
      cudaFuncSetAttribute(k_tc_gemm_check<CTQ_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_tc_gemm_check<CTQ_BF16X3><<<1, TC_THREADS, smem>>>(dA, dB, dD, N, K, 2000000000ull, dS);
    } else {
      cudaFuncSetAttribute(k_tc_gemm_check<CTQ_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_tc_gemm_check<CTQ_TF32><<<1, TC_THREADS, smem>>>(dA, dB, dD, N, K, 2000000000ull, dS);
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
