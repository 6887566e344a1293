// Large-block sector-string trace on the tensor cores (blocks of hundreds to
// thousands of states, e.g. an f shell with N in {4, 5, 6}: 1001 / 2002 / 3003).
//
// One (chain, q0) item is evaluated at a time by the whole GPU: a persistent
// cooperative kernel (one CTA per SM) walks the items of the work list and,
// for each, the operators of its string; a bounded grid barrier separates
// the operators.  The chain runs transposed, Z_i = Y_i^T (d0 x d_i),
//     Z_{i+1} = Z_i F_{i+1}^T P_{i+1},
// with complex numbers in the real embedding
//     [Re Z' | Im Z'] = [Re Z | Im Z] [[Re F, -Im F], [Im F, Re F]]^T,
// so every product is a real GEMM C = A B^T with both operands K-major:
//   A = Z_i in global memory as 128 x 32 tiles of K-major core matrices
//       (8 rows x 16 bytes) so that one cp.async.bulk stages a tile,
//   B = the embedded block, pre-formatted once per impurity as 256 x 32 tiles,
// in TF32 or three-term split TF32 (hi*hi + hi*lo + lo*hi) with FP32
// accumulation in tensor memory.  The epilogue applies the propagator
// column scale e^{-dtau (E - E_min)} (times the power-of-two rescale of the
// previous operator), reduces max|Z| and ||Z||_F over the grid, splits
// hi/lo and writes Z_{i+1} tiles.  Tiles are visited column-major so that a
// B tile is read from HBM once per product and reused from L2 by all row
// tiles.  The first operator only scales F_1; the last one needs only the
// diagonal of F_n Y (FP32 products, FP64 sum).  Log scale, exponents,
// segment bounds and the trace stay in float64.
//
// Every wait is bounded (mbarriers and the grid barrier) by the caller's
// timeout: on expiry the kernel records CTQ_ERR_TIMEOUT in the workspace,
// stops, frees its tensor memory and returns.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace ctq {
namespace {

using namespace dev;
using namespace ptx;

constexpr int BG_THREADS = 128;
constexpr int BM = 128;       // rows of a C tile (rows of Z)
constexpr int BN = 128;       // columns of a C tile (embedded output states)
constexpr int BK = 32;        // K elements (floats) per staged chunk
constexpr int A_TILE = BM * BK;  // floats
constexpr int B_TILE = BN * BK;  // floats
constexpr uint32_t BAR_TIMEOUT_FLAG = 1u;

__device__ __forceinline__ int rup(int x, int m) { return (x + m - 1) / m * m; }

// Offset (floats) of element (row r, column k) of a matrix stored as tiles
// of `rows_per_tile` x BK, tile (rt, kc) at ((rt * n_kc) + kc) * tile size,
// core matrix (nb, kb) at (kb * rows_per_tile/8 + nb) * 32 floats.
__device__ __forceinline__ size_t tiled_off(int r, int k, int rows_per_tile, int n_kc) {
  const int rt = r / rows_per_tile, rr = r - rt * rows_per_tile;
  const int kc = k / BK, kk = k - kc * BK;
  return (size_t(rt) * n_kc + kc) * size_t(rows_per_tile) * BK +
         size_t((kk >> 2) * (rows_per_tile >> 3) + (rr >> 3)) * 32 + (rr & 7) * 4 + (kk & 3);
}

// Grid barrier with a bounded wait (sense reversal on a generation word).
__device__ __forceinline__ bool grid_sync(unsigned* count, volatile unsigned* gen, uint64_t timeout_ns) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    ok_s = 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd(const_cast<unsigned*>(gen), 1u);
    } else {
      const uint64_t t0 = globaltimer();
      while (*gen == g) {
        if (globaltimer() - t0 > timeout_ns) {
          ok_s = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok_s != 0;
}

constexpr int MAX_NST = 6;
// The K loop of a product is spread over NACC tensor-memory accumulators
// (chunk kc into accumulator kc % NACC) that the epilogue adds in FP32: each
// accumulator then sums 1/NACC of the K' terms, which divides the
// accumulation error of long products (K' up to ~6000) by about NACC.
constexpr int NACC = 4;
constexpr int PVEC = 3072;    // largest sector dimension of this path

struct BigShared {
  uint64_t full[MAX_NST];
  uint64_t empty[MAX_NST];
  uint64_t done;
  uint64_t never;  // never arrived on: CTQ_DEBUG_STALL_WAIT waits on it
  uint32_t tmem_base;
  int fail;
  float red[8];
  double redd[64];
};

}  // namespace

namespace {

template <int SPLIT>
__global__ void __launch_bounds__(BG_THREADS, 1)
    k_trace_big(DevModel M, BatchView B, EvalCfg cfg, Work W, BigParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ BigShared S;
  const int NST = P.nst;
  const int stage_floats = (SPLIT == 3 ? 2 : 1) * (A_TILE + B_TILE);
  float* stage0 = reinterpret_cast<float*>(smem_raw);
  float* p_s = stage0 + size_t(NST) * stage_floats;  // [PVEC] column scales of the current product
  float* q_s = p_s + PVEC;                            // [PVEC] wrap-around propagator of q0 (first product)
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ns = M.n_sec;
  const int cplx = M.is_complex;

  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    mbar_init(&S.done, 1);
    mbar_init(&S.never, 1);
    S.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&S.tmem_base, NACC * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = S.tmem_base;
  const uint32_t lane_off = uint32_t(32 * warp) << 16;
  uint32_t ph_full[MAX_NST] = {0, 0, 0, 0, 0, 0}, ph_empty[MAX_NST] = {0, 0, 0, 0, 0, 0};
  uint32_t ph_done = 0;
  bool alive = true;
  if (cfg.debug & CTQ_DEBUG_STALL_WAIT) {
    // CTA 0 waits on an event that never happens; the others then time out
    // in the first grid barrier.
    if (blockIdx.x == 0 && tid == 0 && !mbar_wait(&S.never, 0, P.timeout_ns)) S.fail = 1;
    __syncthreads();
    if (S.fail) alive = false;
  }

  const int n_items = W.counters[0];
  const Item* items = W.items + size_t(B.n_chains) * ns;
  float* Zh[2] = {P.zbuf, P.zbuf + 2 * P.zfloats};
  float* Zl[2] = {P.zbuf + P.zfloats, P.zbuf + 3 * P.zfloats};

  for (int it_idx = 0; it_idx < n_items && alive; ++it_idx) {
    const Item it = items[it_idx];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const int dp0 = rup(d0, BM);
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);
    if (blockIdx.x == 0 && tid <= n) {
      for (int i = tid; i <= n; i += BG_THREADS) {
        P.ekey[i] = 0;
        P.fr[i] = 0.0;
      }
    }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }

    if (n < 2) {  // tiny strings: one CTA does it in float64
      if (blockIdx.x == 0) {
        double sm = 0.0, si = 0.0, mx = 0.0;
        if (n == 0) {
          for (int j = tid; j < d0; j += BG_THREADS) sm += exp(-B.beta * E0[j]);
        } else {
          const double t1 = B.tau[a0], t2 = B.beta - B.tau[a0];
          const int64_t off = M.blk_off[B.op[a0] * ns + q0];
          for (int j = tid; j < d0; j += BG_THREADS) {
            const double pj = exp(-t1 * E0[j]) * exp(-t2 * E0[j]);
            const int64_t e = off + int64_t(j) * d0 + j;
            sm += (cplx ? M.blk[2 * e] : M.blk[e]) * pj;
            if (cplx) si += M.blk[2 * e + 1] * pj;
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
      const int dpk = rup(d1, BK);
      const int nkc = 2 * dpk / BK;
      const double* Eb = M.E_rel + M.E_off[qb];
      for (int j = tid; j < d0; j += BG_THREADS)
        q_s[j] = expf(float(-t_first * E0[j])) * expf(float(-t_last * E0[j]));
      for (int m = tid; m < d1; m += BG_THREADS) p_s[m] = expf(float(-dt * Eb[m]));
      __syncthreads();
      const int64_t off = M.blk_off[alpha * ns + qa];
      int ek = 0;
      float f2 = 0.f;
      const long long total = (long long)dp0 * dpk;
      for (long long e = (long long)blockIdx.x * BG_THREADS + tid; e < total; e += (long long)gridDim.x * BG_THREADS) {
        const int j = int(e / dpk), m = int(e - (long long)j * dpk);
        float xr = 0.f, xi = 0.f;
        if (j < d0 && m < d1) {
          const float pj = q_s[j] * p_s[m];
          const int64_t fe = off + int64_t(m) * d0 + j;
          xr = float(cplx ? M.blk[2 * fe] : M.blk[fe]) * pj;
          xi = cplx ? float(M.blk[2 * fe + 1]) * pj : 0.f;
        }
        ek = max(ek, max((__float_as_int(xr) >> 23) & 0xff, (__float_as_int(xi) >> 23) & 0xff));
        f2 += xr * xr + xi * xi;
        const size_t o_r = tiled_off(j, m, BM, nkc), o_i = tiled_off(j, dpk + m, BM, nkc);
        const uint32_t hr = to_tf32(xr), hi_ = to_tf32(xi);
        Zh[0][o_r] = __uint_as_float(hr);
        Zh[0][o_i] = __uint_as_float(hi_);
        if (SPLIT == 3) {
          Zl[0][o_r] = __uint_as_float(to_tf32(xr - __uint_as_float(hr)));
          Zl[0][o_i] = __uint_as_float(to_tf32(xi - __uint_as_float(hi_)));
        }
      }
      ek = __reduce_max_sync(0xffffffffu, ek);
      double f2d = warp_sum(double(f2));
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
      const int e = ekey - 127;  // floor(log2 max|Z|) of the stored product (float exponent)
      if (track && applied % cfg.S == 0 && applied < n) {
        const double frv = *((volatile double*)&P.fr[applied]);
        const double ub = 0.5 * log(double(it.r)) + 0.5 * log(frv) + double(Eacc) * LN2 + L.val() +
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
      const float scale = ldexpf(1.0f, -e);
      prefix += M.log_norm[idx_a];
      Eacc += e;

      if (i == n - 1) {  // final operator: sum_{j,k} F_n[j][k] Z[j][k]
        const int64_t off = M.blk_off[idx_a];
        const int dpk = rup(dcur, BK), nkc = 2 * dpk / BK;
        double vr = 0.0, vi = 0.0;
        const long long total = (long long)d0 * dcur;
        for (long long e2 = (long long)blockIdx.x * BG_THREADS + tid; e2 < total;
             e2 += (long long)gridDim.x * BG_THREADS) {
          const int j = int(e2 / dcur), k = int(e2 - (long long)j * dcur);
          const size_t o_r = tiled_off(j, k, BM, nkc), o_i = tiled_off(j, dpk + k, BM, nkc);
          float zr = Zh[cur][o_r], zi = Zh[cur][o_i];
          if (SPLIT == 3) {
            zr += Zl[cur][o_r];
            zi += Zl[cur][o_i];
          }
          const int64_t fe = off + int64_t(j) * dcur + k;
          const float fr_ = float(cplx ? M.blk[2 * fe] : M.blk[fe]);
          const float fi_ = cplx ? float(M.blk[2 * fe + 1]) : 0.f;
          vr += double(fr_ * zr - fi_ * zi);
          vi += double(fr_ * zi + fi_ * zr);
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
          sr *= double(scale);
          si *= double(scale);
          const bool zero_v = (sr == 0.0 && si == 0.0);
          W.res_val[2 * slot] = sr;
          W.res_val[2 * slot + 1] = si;
          W.res_log[slot] = zero_v ? -INFINITY : L.val() + double(Eacc) * LN2;
          if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(sr * sr + si * si)) + L.val() + double(Eacc) * LN2;
        }
        applied = n;
        break;
      }

      // ---- tensor-core product: Z_next = Z F^T, columns scaled by p * 2^-e
      const int db = M.dims[qb];
      const int dpk = rup(dcur, BK), nkc = 2 * dpk / BK;   // K of this product
      const int dpn = rup(db, BK), nkc_n = 2 * dpn / BK;   // K of the next one
      {
        const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
        const double* Eb = M.E_rel + M.E_off[qb];
        for (int j = tid; j < dpn; j += BG_THREADS) p_s[j] = (j < db) ? expf(float(-dt * Eb[j])) * scale : 0.f;
        __syncthreads();
        L.add(-dt * (M.E_min[qb] - M.E_ref));
        prefix -= dt * (M.E_min[qb] - M.E_ref);
      }
      __syncthreads();
      const float* Bt = P.bt + P.bt_off[idx_a];
      const size_t b_plane = size_t(rup(2 * dpn, BN) / BN) * nkc * B_TILE;  // floats of one B plane
      const int n_mt = dp0 / BM, n_nt = (2 * dpn + BN - 1) / BN;
      const int n_tiles = n_mt * n_nt;
      const int nxt = cur ^ 1;
      int ek = 0;
      float f2 = 0.f;
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int mt = t % n_mt, nt = t / n_mt;  // column-major: B tiles reused across rows
        const int ncols = min(BN, 2 * dpn - nt * BN);
        const uint32_t idesc = idesc_tf32(BM, ncols);
        const float* Asrc = Zh[cur] + size_t(mt) * nkc * A_TILE;
        const float* Alo = Zl[cur] + size_t(mt) * nkc * A_TILE;
        const float* Bsrc = Bt + size_t(nt) * nkc * B_TILE;
        const float* Blo = Bsrc + b_plane;
        const uint32_t a_bytes = A_TILE * 4, b_bytes = B_TILE * 4;
        const uint32_t st_bytes = (SPLIT == 3 ? 2 : 1) * (a_bytes + b_bytes);
        if (tid == 0) {
          auto issue = [&](int kc) {
            const int st = kc % NST;
            float* sb = stage0 + size_t(st) * stage_floats;
            mbar_arrive_expect_tx(&S.full[st], st_bytes);
            bulk_g2s(sb, Asrc + size_t(kc) * A_TILE, a_bytes, &S.full[st]);
            bulk_g2s(sb + A_TILE, Bsrc + size_t(kc) * B_TILE, b_bytes, &S.full[st]);
            if (SPLIT == 3) {
              bulk_g2s(sb + A_TILE + B_TILE, Alo + size_t(kc) * A_TILE, a_bytes, &S.full[st]);
              bulk_g2s(sb + 2 * A_TILE + B_TILE, Blo + size_t(kc) * B_TILE, b_bytes, &S.full[st]);
            }
          };
          // Chunk kc lives in stage kc % NST.  After the products of chunk kc
          // are queued, the stage of chunk kc - 1 is refilled with chunk
          // kc - 1 + NST as soon as its products have completed, so loads run
          // NST - 1 chunks ahead of the tensor core.
          for (int kc = 0; kc < min(NST, nkc); ++kc) issue(kc);
          int waited_upto = 0;  // chunks [0, waited_upto) have had their empty barrier waited
          for (int kc = 0; kc < nkc && !S.fail; ++kc) {
            const int st = kc % NST;
            if (!mbar_wait(&S.full[st], ph_full[st], P.timeout_ns)) { S.fail = 1; break; }
            ph_full[st] ^= 1u;
            tc_fence_after();
            const uint32_t sa = smem_u32(stage0 + size_t(st) * stage_floats);
            const uint32_t sbh = sa + a_bytes, sal = sbh + b_bytes, sbl = sal + a_bytes;
            for (int kk = 0; kk < BK / 8; ++kk) {
              const uint64_t da = sdesc(sa + kk * 2 * 2048, 2048, 128);
              const uint64_t dbh = sdesc(sbh + kk * 2 * 2048, 2048, 128);
              const uint32_t tacc = tD + uint32_t(kc % NACC) * BN;
              mma_tf32_ss(tacc, da, dbh, idesc, (kc >= NACC || kk > 0) ? 1u : 0u);
              if (SPLIT == 3) {
                mma_tf32_ss(tacc, da, sdesc(sbl + kk * 2 * 2048, 2048, 128), idesc, 1u);
                mma_tf32_ss(tacc, sdesc(sal + kk * 2 * 2048, 2048, 128), dbh, idesc, 1u);
              }
            }
            mma_commit(&S.empty[st]);
            if (kc >= 1) {
              const int pk = kc - 1, ps = pk % NST;
              if (!mbar_wait(&S.empty[ps], ph_empty[ps], P.timeout_ns)) { S.fail = 1; break; }
              ph_empty[ps] ^= 1u;
              waited_upto = kc;
              if (pk + NST < nkc) issue(pk + NST);
            }
          }
          // keep the empty-barrier phases in step for the next tile
          for (int kc = waited_upto; kc < nkc && !S.fail; ++kc) {
            const int st = kc % NST;
            if (!mbar_wait(&S.empty[st], ph_empty[st], P.timeout_ns)) { S.fail = 1; break; }
            ph_empty[st] ^= 1u;
          }
          mma_commit(&S.done);
        }
        __syncthreads();
        const bool ok = (S.fail == 0) && mbar_wait(&S.done, ph_done, P.timeout_ns);
        ph_done ^= 1u;
        if (__syncthreads_or(!ok)) { alive = false; break; }
        tc_fence_after();
        // epilogue: thread = row of the tile
        const int row = mt * BM + tid;
        const int nacc = min(NACC, nkc);
        for (int c0 = 0; c0 < ncols; c0 += 16) {
          float acc[16];
          {
            uint32_t v[16];
            tmem_ld16(tD + lane_off + c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2) acc[t2] = __uint_as_float(v[t2]);
          }
          for (int a = 1; a < nacc; ++a) {
            uint32_t v[16];
            tmem_ld16(tD + uint32_t(a * BN) + lane_off + c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int t2 = 0; t2 < 16; ++t2) acc[t2] += __uint_as_float(v[t2]);
          }
          float hi[16], lo[16];
#pragma unroll
          for (int t2 = 0; t2 < 16; ++t2) {
            const int col = nt * BN + c0 + t2;  // embedded column
            const int j = (col < dpn) ? col : col - dpn;
            const float x = acc[t2] * p_s[j];
            ek = max(ek, (__float_as_int(x) >> 23) & 0xff);
            f2 += x * x;
            const uint32_t h = to_tf32(x);
            hi[t2] = __uint_as_float(h);
            lo[t2] = __uint_as_float(to_tf32(x - hi[t2]));
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const size_t o = tiled_off(row, nt * BN + c0 + 4 * g, BM, nkc_n);
            *reinterpret_cast<float4*>(Zh[nxt] + o) = make_float4(hi[4 * g], hi[4 * g + 1], hi[4 * g + 2], hi[4 * g + 3]);
            if (SPLIT == 3)
              *reinterpret_cast<float4*>(Zl[nxt] + o) = make_float4(lo[4 * g], lo[4 * g + 1], lo[4 * g + 2], lo[4 * g + 3]);
          }
        }
        tc_fence_before();
        __syncthreads();
      }
      if (!alive) break;
      ek = __reduce_max_sync(0xffffffffu, ek);
      const double f2d = warp_sum(double(f2));
      if ((tid & 31) == 0) {
        atomicMax(&P.ekey[applied + 1], ek);
        atomicAdd(&P.fr[applied + 1], f2d);
      }
      if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
      cur = nxt;
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
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tD, NACC * BN);
  }
}

// Embedded, tiled, tf32-split copy of every block (one CTA per output tile row
// chunk): B'[n][k] for n < 2 dpn, k < 2 dpk with
//   n < dpn:  [Re F[n][k],  -Im F[n][k - dpk]]
//   n >= dpn: [Im F[n - dpn][k], Re F[n - dpn][k - dpk]].
__global__ void k_format_big(const double* blk, int cplx, int dn, int dk, float* out, int split) {
  const int dpn = rup(dn, BK), dpk = rup(dk, BK);
  const int N2 = rup(2 * dpn, BN), K2 = 2 * dpk, nkc = K2 / BK;
  const size_t plane = size_t(N2) * K2;
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
    const size_t o = tiled_off(n, k, BN, nkc);
    const uint32_t h = to_tf32(float(v));
    out[o] = __uint_as_float(h);
    if (split == 3) out[plane + o] = __uint_as_float(to_tf32(float(v - double(__uint_as_float(h)))));
  }
}

}  // namespace

size_t big_block_floats(int dn, int dk) {
  const int dpn = (dn + BK - 1) / BK * BK, dpk = (dk + BK - 1) / BK * BK;
  return size_t((2 * dpn + BN - 1) / BN * BN) * size_t(2 * dpk) * 2;  // hi and lo planes
}

// Lays out and fills the embedded blocks on the device (d_blk: the float64
// blocks already on the device).  out/off: device buffer and host offsets.
int format_big_blocks(const HostModel& h, const double* d_blk, float* out, const std::vector<int64_t>& off) {
  const int na = h.n_alpha();
  for (int a = 0; a < na; ++a)
    for (int q = 0; q < h.n_sec; ++q) {
      const size_t i = size_t(a) * h.n_sec + q;
      const int qp = h.s[i];
      if (qp < 0) continue;
      const double* src = d_blk + (h.is_complex ? 2 : 1) * h.blk_off[i];
      k_format_big<<<1024, 256>>>(src, h.is_complex, h.dims[qp], h.dims[q], out + off[i], 3);
      if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
    }
  return cudaDeviceSynchronize() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

size_t big_scratch_bytes(const HostModel& h, int max_ops, int grid) {
  int dmax = h.max_dim;
  const size_t zf = size_t((dmax + BM - 1) / BM * BM) * size_t(2 * ((dmax + BK - 1) / BK * BK));
  return 4 * zf * 4 + 256 + size_t(max_ops + 2) * (4 + 8) + size_t(2 * grid) * 8 + 1024;
}

int prepare_eval_big(int split, int num_sms, LaunchCfg* lc) {
  lc->threads = BG_THREADS;
  lc->num_sms = num_sms;
  const int nst = split == 3 ? 3 : 6;
  lc->smem = size_t(nst) * (split == 3 ? 2 : 1) * (A_TILE + B_TILE) * 4 + 2 * PVEC * 4;
  const cudaError_t e = (split == 3)
                            ? cudaFuncSetAttribute(k_trace_big<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem))
                            : cudaFuncSetAttribute(k_trace_big<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(lc->smem));
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  lc->per_sm = 1;
  return CTQ_OK;
}

int launch_eval_big(const DevModel& M, const LaunchCfg& lc, BigParams P, const BatchView& B, const EvalCfg& cfg,
                    const Work& W, const ctq_result* R, void* scratch, void* stream, void* const* events) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (B.n_chains == 0) return CTQ_OK;
  if (M.max_dim > PVEC) return CTQ_ERR_UNSUPPORTED;
  auto mark = [&](int i) {
    if (events) cudaEventRecord(static_cast<cudaEvent_t>(events[i]), st);
  };
  const int grid = lc.num_sms;
  // carve the scratch
  char* s = static_cast<char*>(scratch);
  const int dmax = M.max_dim;
  P.zfloats = size_t((dmax + BM - 1) / BM * BM) * size_t(2 * ((dmax + BK - 1) / BK * BK));
  P.zbuf = reinterpret_cast<float*>(s);
  s += 4 * P.zfloats * 4;
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
  P.nst = P.split == 3 ? 3 : 6;
  if (cudaMemsetAsync(W.counters, 0, 256, st) != cudaSuccess) return CTQ_ERR_CUDA;
  if (cudaMemsetAsync(P.bar, 0, 256, st) != cudaSuccess) return CTQ_ERR_CUDA;
  if (cudaMemsetAsync(P.zbuf, 0, 4 * P.zfloats * 4, st) != cudaSuccess) return CTQ_ERR_CUDA;
  mark(0);
  {
    const int ps = launch_plan(M, B, cfg, W, st);
    if (ps != CTQ_OK) return ps;
  }
  mark(1);
  void* args[] = {const_cast<DevModel*>(&M), const_cast<BatchView*>(&B), const_cast<EvalCfg*>(&cfg),
                  const_cast<Work*>(&W), &P};
  const cudaError_t e = (P.split == 3)
                            ? cudaLaunchCooperativeKernel((void*)k_trace_big<3>, grid, BG_THREADS, args, lc.smem, st)
                            : cudaLaunchCooperativeKernel((void*)k_trace_big<1>, grid, BG_THREADS, args, lc.smem, st);
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  mark(2);
  {
    const int cs = launch_combine(M, B, cfg, W, R, st);
    if (cs != CTQ_OK) return cs;
  }
  mark(3);
  return CTQ_OK;
}

}  // namespace ctq
