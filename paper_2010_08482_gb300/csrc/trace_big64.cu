// Large-block sector-string trace in float64: the plain FP64 path for
// impurities whose blocks are too large for the shared-memory kernel k_trace
// (trace_fp64.cu), e.g. a complex d shell or the f shell with blocks of
// 1001 / 2002 / 3003 states.
//
// Same schedule as the tensor-core large-block kernel (trace_big.cu): a
// persistent cooperative kernel, one CTA per SM, evaluates one (chain, q0)
// string at a time on the whole GPU, with a bounded grid barrier between
// operators.  The chain runs transposed, Z_i = Y_i^T (d0 x d_i),
//     Z_{i+1} = Z_i F_{i+1}^T P_{i+1},
// complex numbers in the real embedding
//     [Re Z' | Im Z'] = [Re Z | Im Z] [[Re F, -Im F], [Im F, Re F]]^T,
// so every product is a real GEMM C = Z B'^T, here on the CUDA cores in
// float64: 128 x 128 tiles of C, K chunks of 16 staged in shared memory, an
// 8 x 8 register tile per thread.  The epilogue applies the column
// propagators e^{-dtau (E - E_min)} (float64 exponentials, times the exact
// power-of-two rescale of the previous product), reduces the exponent
// maximum and ||Z||_F over the grid, and writes Z_{i+1} row-major.  The first
// operator only scales F_1, the last one needs only the diagonal of F_n Y.
// Log scale, exponents, segment bounds and the trace follow k_trace_big.
//
// Every wait is bounded (the grid barrier) by the caller's timeout: on expiry
// the kernel records CTQ_ERR_TIMEOUT in the workspace and returns.
#include <algorithm>

#include "big_common.cuh"
#include "device_common.cuh"
#include "two_float.cuh"

namespace ctq {
namespace {

using namespace dev;
using namespace bigc;
using namespace tf2;

constexpr int B64_THREADS = 256;
constexpr int TM = 128, TN = 128, TK = 16;  // C tile and K chunk (float64 elements)
constexpr int PAD64 = 32;                   // sector dimensions padded to multiples of PAD64
constexpr int PVEC64 = 3072;                // largest sector dimension of this path
constexpr uint32_t BAR_TIMEOUT_FLAG = 1u;

struct Big64Shared {
  double As[TK][TM];  // A chunk, transposed: As[k][row]
  double Bs[TK][TN];  // B' chunk, transposed: Bs[k][row of B']
  double redd[64];
  uint64_t never;     // never arrived on: CTQ_DEBUG_STALL_WAIT waits on it
  int fail;
};

__device__ __forceinline__ int exp_key64(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// Operand element of the product: float64, or (X2, CTQ_F32X2) a two-float
// pair of the same 8 bytes.  Staging copies bytes; only the arithmetic
// differs.
template <bool X2>
struct Op64;
template <>
struct Op64<false> {
  using E = double;
  static __device__ __forceinline__ E make(double x) { return x; }
  static __device__ __forceinline__ double val(E x) { return x; }
};
template <>
struct Op64<true> {
  using E = DF;
  static __device__ __forceinline__ E make(double x) { return df_split(x); }
  static __device__ __forceinline__ double val(E x) { return df_val(x); }
};

// X2: the products in two-float arithmetic on the FP32 pipe (accumulators
// renormalised every X2_RENORM K terms); propagators, log scale, bounds and
// the final trace in float64.
template <bool CPLX, bool X2>
__global__ void __launch_bounds__(B64_THREADS, 1)
    k_trace_big64(DevModel M, BatchView B, EvalCfg cfg, Work W, Big64Params P) {
  using E = typename Op64<X2>::E;
  // C tiles of TM x TNV: the two-float accumulators take two registers each,
  // so that variant keeps an 8 x 4 tile per thread on 128 x 64 C tiles
  constexpr int TNV = X2 ? TN / 2 : TN;
  constexpr int CB = TNV / 16;                // columns of the register tile (rows: 8)
  constexpr int EPB = TNV * TK / B64_THREADS;  // staged B elements per thread
  static_assert(sizeof(E) == 8, "operand elements are 8 bytes in both forms");
  extern __shared__ __align__(16) double dsm[];
  double* p_s = dsm;           // [PVEC64] column scales of the current product
  double* q_s = dsm + PVEC64;  // [PVEC64] wrap-around propagator of q0
  __shared__ Big64Shared S;
  const int tid = threadIdx.x;
  const int ns = M.n_sec;
  const int tx = tid & 15, ty = tid >> 4;

  if (tid == 0) {
    ptx::mbar_init(&S.never, 1);
    S.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool alive = true;
  if (cfg.debug & CTQ_DEBUG_STALL_WAIT) {
    // CTA 0 waits on an event that never happens; the others then time out
    // in the first grid barrier.
    if (blockIdx.x == 0 && tid == 0 && !ptx::mbar_wait(&S.never, 0, P.timeout_ns)) S.fail = 1;
    __syncthreads();
    if (S.fail) alive = false;
  }

  const int n_items = W.counters[0];
  const Item* items = W.items + size_t(B.n_chains) * ns;
  E* Z[2] = {reinterpret_cast<E*>(P.zbuf), reinterpret_cast<E*>(P.zbuf) + P.zelems};

  for (int it_idx = 0; it_idx < n_items && alive; ++it_idx) {
    const Item it = items[W.order[it_idx]];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const int dp0 = rup(d0, TM);
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);
    if (blockIdx.x == 0)
      for (int i = tid; i <= n; i += B64_THREADS) {
        P.ekey[i] = 0;
        P.fr[i] = 0.0;
      }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }

    if (n < 2) {  // tiny strings: one CTA
      if (blockIdx.x == 0) {
        double sm = 0.0, si = 0.0, mx = 0.0;
        if (n == 0) {
          for (int j = tid; j < d0; j += B64_THREADS) sm += exp(-B.beta * E0[j]);
        } else {
          const double t1 = B.tau[a0], t2 = B.beta - B.tau[a0];
          const int64_t off = M.blk_off[B.op[a0] * ns + q0];
          for (int j = tid; j < d0; j += B64_THREADS) {
            const double pj = exp(-t1 * E0[j]) * exp(-t2 * E0[j]);
            const int64_t e = off + int64_t(j) * d0 + j;
            sm += (CPLX ? M.blk[2 * e] : M.blk[e]) * pj;
            if (CPLX) si += M.blk[2 * e + 1] * pj;
          }
        }
        block_max_sum(mx, sm, S.redd);
        mx = 0.0;
        block_max_sum(mx, si, S.redd);
        if (tid == 0) {
          const double l = -B.beta * (M.E_min[q0] - M.E_ref);
          const bool zero_v = (sm == 0.0 && si == 0.0);
          W.res_val[2 * slot] = sm;
          W.res_val[2 * slot + 1] = si;
          W.res_log[slot] = zero_v ? -INFINITY : l;
          if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(sm * sm + si * si)) + l;
        }
      }
      continue;
    }

    // ---- operator 1 (elementwise): Z_1[j][m] = p0[j] F_1[m][j] p1[m]
    const double t_first = B.tau[a0], t_last = B.beta - B.tau[a0 + n - 1];
    int qa = q0;
    int alpha = B.op[a0];
    int qb = M.s[alpha * ns + qa];
    KSum L;
    long long Eacc = 0;
    double prefix = M.log_norm[alpha * ns + qa];
    L.add(-t_first * (M.E_min[q0] - M.E_ref));
    L.add(-t_last * (M.E_min[q0] - M.E_ref));
    {
      const double dt = B.tau[a0 + 1] - B.tau[a0];
      L.add(-dt * (M.E_min[qb] - M.E_ref));
      prefix -= dt * (M.E_min[qb] - M.E_ref);
      const int d1 = M.dims[qb];
      const int dpk = rup(d1, PAD64), K2 = 2 * dpk;
      const double* Eb = M.E_rel + M.E_off[qb];
      for (int j = tid; j < d0; j += B64_THREADS) q_s[j] = exp(-t_first * E0[j]) * exp(-t_last * E0[j]);
      for (int m = tid; m < d1; m += B64_THREADS) p_s[m] = exp(-dt * Eb[m]);
      __syncthreads();
      const int64_t off = M.blk_off[alpha * ns + qa];
      int ek = 0;
      double f2 = 0.0;
      const long long total = (long long)dp0 * dpk;
      for (long long e = (long long)blockIdx.x * B64_THREADS + tid; e < total;
           e += (long long)gridDim.x * B64_THREADS) {
        const int j = int(e / dpk), m = int(e - (long long)j * dpk);
        double xr = 0.0, xi = 0.0;
        if (j < d0 && m < d1) {
          const double pj = q_s[j] * p_s[m];
          const int64_t fe = off + int64_t(m) * d0 + j;
          xr = (CPLX ? M.blk[2 * fe] : M.blk[fe]) * pj;
          xi = CPLX ? M.blk[2 * fe + 1] * pj : 0.0;
        }
        ek = max(ek, max(exp_key64(xr), exp_key64(xi)));
        f2 += xr * xr + xi * xi;
        Z[0][size_t(j) * K2 + m] = Op64<X2>::make(xr);
        Z[0][size_t(j) * K2 + dpk + m] = Op64<X2>::make(xi);
      }
      ek = __reduce_max_sync(0xffffffffu, ek);
      const double f2d = warp_sum(f2);
      if ((tid & 31) == 0) {
        atomicMax(&P.ekey[1], ek);
        atomicAdd(&P.fr[1], f2d);
      }
    }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
    int cur = 0;
    int dcur = M.dims[qb];
    qa = qb;
    int applied = 1;
    bool dead = false, aborted = false;

    for (int i = 1; i < n; ++i) {
      const int ekey = *((volatile int*)&P.ekey[applied]);
      if (ekey == 0) { dead = true; break; }
      const int e = min(ekey - 1023, 1022);  // floor(log2 max|Z|) of the stored product
      if (track && applied % cfg.S == 0 && applied < n) {
        const double frv = *((volatile double*)&P.fr[applied]);
        const double ub = 0.5 * it.log_r + 0.5 * log(frv) + double(Eacc) * LN2 + L.val() +
                          (it.t_all - prefix);
        if (blockIdx.x == 0 && tid == 0) {
          segp[applied / cfg.S] = ub;
          if (cfg.lazy) {
            W.live[slot] = fmin(W.live[slot], ub);
            double lm = -INFINITY, lsum = 0.0;
            for (int q = 0; q < ns; ++q) {
              const double v = W.live[size_t(c) * ns + q];
              if (v > lm) { lsum = lsum * exp(lm - v) + 1.0; lm = v; }
              else if (v != -INFINITY) lsum += exp(v - lm);
            }
            const double lub = (lm == -INFINITY) ? lm : lm + log(lsum);
            int flag = W.chain_flag[c];
            if (!(flag & FLAG_REJECTED) && lub + cfg.margin < B.log_threshold[c] + B.beta * M.E_ref) {
              flag |= FLAG_REJECTED;
              W.chain_flag[c] = flag;
            }
            *P.abort_flag = (flag & FLAG_REJECTED) ? 1 : 0;
            __threadfence();
          }
        }
        if (cfg.lazy) {
          if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
          if (*((volatile int*)P.abort_flag)) { aborted = true; break; }
        }
      }
      alpha = B.op[a0 + i];
      const int idx_a = alpha * ns + qa;
      qb = M.s[idx_a];
      const double scale = pow2i(-e);
      prefix += M.log_norm[idx_a];
      Eacc += e;
      const int dpk = rup(dcur, PAD64), K2 = 2 * dpk;  // K of this product

      if (i == n - 1) {  // final operator: sum_{j,k} F_n[j][k] Z[j][k]
        const int64_t off = M.blk_off[idx_a];
        double vr = 0.0, vi = 0.0;
        const long long total = (long long)d0 * dcur;
        for (long long e2 = (long long)blockIdx.x * B64_THREADS + tid; e2 < total;
             e2 += (long long)gridDim.x * B64_THREADS) {
          const int j = int(e2 / dcur), k = int(e2 - (long long)j * dcur);
          const double zr = Op64<X2>::val(Z[cur][size_t(j) * K2 + k]);
          const double zi = Op64<X2>::val(Z[cur][size_t(j) * K2 + dpk + k]);
          const int64_t fe = off + int64_t(j) * dcur + k;
          const double fr_ = CPLX ? M.blk[2 * fe] : M.blk[fe];
          const double fi_ = CPLX ? M.blk[2 * fe + 1] : 0.0;
          vr += fr_ * zr - fi_ * zi;
          vi += fr_ * zi + fi_ * zr;
        }
        double dm = 0.0;
        block_max_sum(dm, vr, S.redd);
        dm = 0.0;
        block_max_sum(dm, vi, S.redd);
        if (tid == 0) {
          P.part[2 * blockIdx.x] = vr;
          P.part[2 * blockIdx.x + 1] = vi;
        }
        if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
        if (blockIdx.x == 0 && tid == 0) {
          double sr = 0.0, si = 0.0;
          for (int b = 0; b < int(gridDim.x); ++b) {
            sr += P.part[2 * b];
            si += P.part[2 * b + 1];
          }
          sr *= scale;
          si *= scale;
          const bool zero_v = (sr == 0.0 && si == 0.0);
          W.res_val[2 * slot] = sr;
          W.res_val[2 * slot + 1] = si;
          W.res_log[slot] = zero_v ? -INFINITY : L.val() + double(Eacc) * LN2;
          if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(sr * sr + si * si)) + L.val() + double(Eacc) * LN2;
        }
        applied = n;
        break;
      }

      // ---- float64 product: Z_next = Z F^T, columns scaled by p * 2^-e
      const int db = M.dims[qb];
      const int dpn = rup(db, PAD64), N2 = 2 * dpn;  // columns of C = K of the next product
      {
        const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
        const double* Eb = M.E_rel + M.E_off[qb];
        for (int j = tid; j < dpn; j += B64_THREADS) p_s[j] = (j < db) ? exp(-dt * Eb[j]) * scale : 0.0;
        L.add(-dt * (M.E_min[qb] - M.E_ref));
        prefix -= dt * (M.E_min[qb] - M.E_ref);
      }
      __syncthreads();
      // rup(N2, TN) x K2, row-major
      const E* Bt = (X2 ? reinterpret_cast<const E*>(P.bt_x2) : reinterpret_cast<const E*>(P.bt)) + P.bt_off[idx_a];
      const E* A = Z[cur];
      E* C = Z[cur ^ 1];
      const int n_mt = dp0 / TM, n_nt = rup(N2, TN) / TNV;
      const int n_tiles = n_mt * n_nt;
      int ek = 0;
      double f2 = 0.0;
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        int mt, nt;
        tile_coords(t, n_mt, n_nt, P.order, mt, nt);
        E acc[8][CB];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < CB; ++b) acc[a][b] = Op64<X2>::make(0.0);
        const E* Ab = A + size_t(mt) * TM * K2;
        const E* Bb = Bt + size_t(nt) * TNV * K2;
        const int lr = tid >> 1, lk = (tid & 1) * 8;  // this thread's staging row and K half of A
        const int lrb = tid / (TK / EPB), lkb = (tid % (TK / EPB)) * EPB;  // and of B
        for (int k0 = 0; k0 < K2; k0 += TK) {
          {
            // 16-byte copies of the operand bytes (two elements of either form)
            const double2* sa = reinterpret_cast<const double2*>(Ab + size_t(lr) * K2 + k0 + lk);
            const double2* sb = reinterpret_cast<const double2*>(Bb + size_t(lrb) * K2 + k0 + lkb);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const double2 va = __ldg(sa + u);
              S.As[lk + 2 * u][lr] = va.x;
              S.As[lk + 2 * u + 1][lr] = va.y;
            }
#pragma unroll
            for (int u = 0; u < EPB / 2; ++u) {
              const double2 vb = __ldg(sb + u);
              S.Bs[lkb + 2 * u][lrb] = vb.x;
              S.Bs[lkb + 2 * u + 1][lrb] = vb.y;
            }
          }
          __syncthreads();
#pragma unroll
          for (int k = 0; k < TK; ++k) {
            E av[8], bv[CB];
            const E* as = reinterpret_cast<const E*>(&S.As[k][0]);
            const E* bs = reinterpret_cast<const E*>(&S.Bs[k][0]);
#pragma unroll
            for (int a = 0; a < 8; ++a) av[a] = as[ty + 16 * a];
#pragma unroll
            for (int b = 0; b < CB; ++b) bv[b] = bs[tx + 16 * b];
            if constexpr (X2) {
#pragma unroll
              for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < CB; ++b) fma_acc(acc[a][b], av[a], bv[b]);
              if (k % X2_RENORM == X2_RENORM - 1) {
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                  for (int b = 0; b < CB; ++b) finish(acc[a][b]);
              }
            } else {
#pragma unroll
              for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < CB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
          }
          __syncthreads();
        }
        // epilogue: rows mt*TM + ty + 16a, columns nt*TNV + tx + 16b
#pragma unroll
        for (int b = 0; b < CB; ++b) {
          const int col = nt * TNV + tx + 16 * b;  // embedded column
          if (col >= N2) continue;
          const double ps = p_s[(col < dpn) ? col : col - dpn];
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const int row = mt * TM + ty + 16 * a;
            if constexpr (X2) {
              const DF x = df_split(ps) * acc[a][b];
              ek = max(ek, exp_key(x));
              f2 += sq(x);
              C[size_t(row) * N2 + col] = x;
            } else {
              const double x = acc[a][b] * ps;
              ek = max(ek, exp_key64(x));
              f2 = fma(x, x, f2);
              C[size_t(row) * N2 + col] = x;
            }
          }
        }
      }
      ek = __reduce_max_sync(0xffffffffu, ek);
      const double f2d = warp_sum(f2);
      if ((tid & 31) == 0) {
        atomicMax(&P.ekey[applied + 1], ek);
        atomicAdd(&P.fr[applied + 1], f2d);
      }
      if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
      cur ^= 1;
      dcur = db;
      qa = qb;
      ++applied;
    }
    if (blockIdx.x == 0 && tid == 0) {
      if (dead) {
        W.res_val[2 * slot] = 0.0;
        W.res_val[2 * slot + 1] = 0.0;
        W.res_log[slot] = -INFINITY;
        if (track)
          for (int s2 = (applied + cfg.S - 1) / cfg.S; s2 <= it.n_seg; ++s2)
            if (s2 > 0) segp[s2] = -INFINITY;
      }
      if (aborted) W.res_log[slot] = NAN;
    }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) alive = false;
  }
  if (!alive && tid == 0) atomicOr(&W.counters[2], int(BAR_TIMEOUT_FLAG));
}

// Embedded float64 copy of a block, row-major B'[n][k] (n < rup(2 dpn, TN),
// k < 2 dpk) with
//   n < dpn:  [Re F[n][k],  -Im F[n][k - dpk]]
//   n >= dpn: [Im F[n - dpn][k], Re F[n - dpn][k - dpk]].
template <typename OUT>
__global__ void k_format_big64(const double* blk, int cplx, int dn, int dk, OUT* out) {
  const int dpn = rup(dn, PAD64), dpk = rup(dk, PAD64);
  const int N2 = rup(2 * dpn, TN), K2 = 2 * dpk;
  const long long total = (long long)N2 * K2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = int(e / K2), k = int(e - (long long)n * K2);
    const int nn = (n < dpn) ? n : n - dpn;
    const int kk = (k < dpk) ? k : k - dpk;
    double v = 0.0;
    if (n < 2 * dpn && nn < dn && kk < dk) {
      const size_t f = size_t(nn) * dk + kk;
      const double re = cplx ? blk[2 * f] : blk[f];
      const double im = cplx ? blk[2 * f + 1] : 0.0;
      if (n < dpn) v = (k < dpk) ? re : -im;
      else v = (k < dpk) ? im : re;
    }
    if constexpr (sizeof(OUT) == 8 && alignof(OUT) == 4) {  // two-float pair
      const float hi = __double2float_rn(v);
      out[e] = OUT{hi, __double2float_rn(v - double(hi))};
    } else {
      out[e] = v;
    }
  }
}

}  // namespace

size_t big64_block_elems(int dn, int dk) {
  const int dpn = (dn + PAD64 - 1) / PAD64 * PAD64, dpk = (dk + PAD64 - 1) / PAD64 * PAD64;
  return size_t((2 * dpn + TN - 1) / TN * TN) * size_t(2 * dpk);
}

// x2: the two-float copy (float hi, lo per element) for CTQ_F32X2.
int format_big64_blocks(const HostModel& h, const double* d_blk, void* out, const std::vector<int64_t>& off, bool x2) {
  const int na = h.n_alpha();
  for (int a = 0; a < na; ++a)
    for (int q = 0; q < h.n_sec; ++q) {
      const size_t i = size_t(a) * h.n_sec + q;
      const int qp = h.s[i];
      if (qp < 0) continue;
      const double* src = d_blk + (h.is_complex ? 2 : 1) * h.blk_off[i];
      if (x2)
        k_format_big64<DF><<<1024, 256>>>(src, h.is_complex, h.dims[qp], h.dims[q], static_cast<DF*>(out) + off[i]);
      else
        k_format_big64<double><<<1024, 256>>>(src, h.is_complex, h.dims[qp], h.dims[q],
                                              static_cast<double*>(out) + off[i]);
      if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
    }
  return cudaDeviceSynchronize() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

static size_t z64_elems(int dmax) {
  return size_t((dmax + TM - 1) / TM * TM) * size_t(2 * ((dmax + PAD64 - 1) / PAD64 * PAD64));
}

size_t big64_scratch_bytes(const HostModel& h, int max_ops, int grid) {
  return 2 * z64_elems(h.max_dim) * 8 + 256 + size_t(max_ops + 2) * (4 + 8) + size_t(2 * grid) * 8 + 1024;
}

int prepare_eval_big64(int num_sms, LaunchCfg* lc) {
  lc->threads = B64_THREADS;
  lc->num_sms = num_sms;
  lc->smem = 2 * PVEC64 * sizeof(double);
  const int sm = int(lc->smem);
  if (cudaFuncSetAttribute(k_trace_big64<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_trace_big64<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_trace_big64<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_trace_big64<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
    return CTQ_ERR_CUDA;
  lc->per_sm = 1;
  return CTQ_OK;
}

int launch_eval_big64(const DevModel& M, const LaunchCfg& lc, Big64Params P, const BatchView& B, const EvalCfg& cfg,
                      const Work& W, const ctq_result* R, void* scratch, void* stream, void* const* events, bool x2) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (M.max_dim > PVEC64 || (x2 && P.bt_x2 == nullptr)) return CTQ_ERR_UNSUPPORTED;
  auto mark = [&](int i) {
    if (events) record_timing_event(events[i], st);
  };
  const int grid = lc.num_sms;
  char* s = static_cast<char*>(scratch);
  P.zelems = z64_elems(M.max_dim);
  P.zbuf = reinterpret_cast<double*>(s);
  s += 2 * P.zelems * 8;
  P.bar = reinterpret_cast<unsigned*>(s);
  s += 256;
  P.ekey = reinterpret_cast<int*>(s);
  s += size_t(cfg.max_ops + 2) * 4;
  s = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s) + 7) & ~uintptr_t(7));
  P.fr = reinterpret_cast<double*>(s);
  s += size_t(cfg.max_ops + 2) * 8;
  P.part = reinterpret_cast<double*>(s);
  s += size_t(2 * grid) * 8;
  P.abort_flag = reinterpret_cast<int*>(s);
  P.order = cfg.tile_order == 0 ? 0 : cfg.tile_order - 1;  // tile_coords codes; column-major by default
  if (cudaMemsetAsync(W.counters, 0, COUNTER_BYTES, st) != cudaSuccess) return CTQ_ERR_CUDA;
  if (cudaMemsetAsync(P.bar, 0, 256, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(0);
  {
    const int ps = launch_plan(M, B, cfg, W, st);
    if (ps != CTQ_OK) return ps;
  }
  mark(1);
  void* args[] = {const_cast<DevModel*>(&M), const_cast<BatchView*>(&B), const_cast<EvalCfg*>(&cfg),
                  const_cast<Work*>(&W), &P};
  void* fn = x2 ? (M.is_complex ? (void*)k_trace_big64<true, true> : (void*)k_trace_big64<false, true>)
               : (M.is_complex ? (void*)k_trace_big64<true, false> : (void*)k_trace_big64<false, false>);
  if (cudaLaunchCooperativeKernel(fn, grid, B64_THREADS, args, lc.smem, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(2);
  {
    const int cs = launch_combine(M, B, cfg, W, R, st);
    if (cs != CTQ_OK) return cs;
  }
  mark(3);
  return CTQ_OK;
}

}  // namespace ctq
