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
//   A = Z_i in global memory as 128-row tiles of K-major core matrices
//       (8 rows x 16 bytes), 128 bytes of K per staged chunk, so that one
//       cp.async.bulk stages a chunk,
//   B = the embedded block, pre-formatted once per impurity as 256-row tiles
//       of the same form,
// in TF32, three-term split TF32 (hi*hi + hi*lo + lo*hi) or three-term split
// bf16, with FP32 accumulation in tensor memory (a 128 x 256 tile: two
// accumulators fill the 512 columns, chunks alternate between them).  The
// epilogue applies the propagator column scale e^{-dtau (E - E_min)} (times
// the power-of-two rescale of the previous operator), reduces max|Z| and
// ||Z||_F over the grid, splits hi/lo and writes Z_{i+1} tiles.  Tiles are
// visited column-major by default so that a B tile is read from HBM once
// per product and reused from L2 by all row tiles.  The first operator only
// scales F_1; the last one needs only the diagonal of F_n Y (FP32 products,
// FP64 sum).  Log scale, exponents, segment bounds and the trace stay in
// float64.
//
// Every wait is bounded (mbarriers and the grid barrier) by the caller's
// timeout: on expiry the kernel records CTQ_ERR_TIMEOUT in the workspace,
// stops, frees its tensor memory and returns.
#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "tc_ptx.cuh"
#include "big_common.cuh"

namespace ctq {
namespace {

using namespace dev;
using namespace ptx;
using namespace bigc;

constexpr int N_DRAIN = 8;                       // drain / epilogue warps (N_DRAIN / 4 per lane quarter)
constexpr int BG_THREADS = 32 * (2 + N_DRAIN);   // warp 0: MMA issuer, warp 1: producer
constexpr int BM = 128;       // rows of a C tile (rows of Z)
constexpr int BN = 256;       // columns of a C tile (embedded output states)
constexpr int BK = 32;        // sector dimensions are padded to multiples of BK
constexpr int ROWB = 128;     // bytes of one tile row in a staged K chunk
constexpr uint32_t A_BYTES = BM * ROWB;  // one staged A tile (16 KB)
constexpr uint32_t B_BYTES = BN * ROWB;  // one staged B tile (32 KB)
// Descriptor strides of a staged tile: core matrices (8 rows x 16 bytes)
// adjacent in K are rows/8 x 128 bytes apart, adjacent in M/N 128 bytes.
constexpr uint32_t LBO_A = (BM / 8) * 128, LBO_B = (BN / 8) * 128;
constexpr uint32_t BAR_TIMEOUT_FLAG = 1u;

// Operand elements: TF32 and 3xTF32 stage float tiles (tf32-rounded), BF16X3
// stages bf16 hi / lo tiles.  A staged chunk row is always ROWB bytes (32
// floats or 64 bf16), so tile geometry and descriptors in bytes are shared.
template <int PREC>
struct Elt {
  using T = float;
};
template <>
struct Elt<CTQ_BF16X3> {
  using T = uint16_t;
};


// Offset (elements of EB bytes) of element (row r, column k) of a matrix
// stored as tiles of `rows_per_tile` rows x 128 bytes of K, tile (rt, kc) at
// ((rt * n_kc) + kc) * tile size, core matrix (nb, kb) of 8 rows x 16 bytes at
// (kb * rows_per_tile/8 + nb) * 128 bytes.
template <int EB>
__host__ __device__ __forceinline__ size_t tiled_off(int r, int k, int rows_per_tile, int n_kc) {
  constexpr int EPC = 16 / EB;    // elements per core-matrix row
  constexpr int BKE = ROWB / EB;  // elements per chunk row
  const int rt = r / rows_per_tile, rr = r - rt * rows_per_tile;
  const int kc = k / BKE, kk = k - kc * BKE;
  return (size_t(rt) * n_kc + kc) * size_t(rows_per_tile) * BKE +
         size_t((kk / EPC) * (rows_per_tile >> 3) + (rr >> 3)) * (8 * EPC) + (rr & 7) * EPC + (kk % EPC);
}


// hi / lo split of x in the operand format of PREC.
template <int PREC>
__device__ __forceinline__ void split_store(float x, typename Elt<PREC>::T& hi, typename Elt<PREC>::T& lo) {
  if constexpr (PREC == CTQ_BF16X3) {
    const uint32_t h = bf16_bits(x);
    hi = uint16_t(h);
    lo = uint16_t(bf16_bits(x - bf16_val(h)));
  } else {
    const uint32_t h = to_tf32(x);
    hi = __uint_as_float(h);
    lo = __uint_as_float(to_tf32(x - __uint_as_float(h)));
  }
}
template <int PREC>
__device__ __forceinline__ float elt_val(typename Elt<PREC>::T v) {
  if constexpr (PREC == CTQ_BF16X3) return bf16_val(v);
  else return v;
}

// 16 bytes of consecutive operand elements as one vector.
template <int PREC>
__device__ __forceinline__ uint4 pack16(const typename Elt<PREC>::T* v) {
  if constexpr (PREC == CTQ_BF16X3) {
    return make_uint4(uint32_t(v[0]) | (uint32_t(v[1]) << 16), uint32_t(v[2]) | (uint32_t(v[3]) << 16),
                      uint32_t(v[4]) | (uint32_t(v[5]) << 16), uint32_t(v[6]) | (uint32_t(v[7]) << 16));
  } else {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
  }
}

// D[tmem] (+)= A[smem] * B[smem] in the operand format of PREC.
template <int PREC>
__device__ __forceinline__ void mma_big(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (PREC == CTQ_BF16X3) mma_bf16_ss(d, a, b, idesc, acc);
  else mma_tf32_ss(d, a, b, idesc, acc);
}


constexpr int MAX_NST = 12;
// The K loop of a product is cut into groups of GRP chunks accumulated in
// alternating tensor-memory banks and added into FP32 registers (round to
// nearest) by the N_DRAIN drain warps, so the tensor core's own FP32 accumulation
// spans at most GRP chunks (128 or 256 K' terms) of a product whose K' reaches
// ~6000.
constexpr int NBANK = 512 / BN;  // accumulator banks filling the 512 tensor-memory columns
constexpr int GRP = 4;            // K chunks accumulated in a bank before it is drained
constexpr int PVEC = 3072;    // largest sector dimension of this path

struct BigShared {
  uint64_t full[MAX_NST];
  uint64_t empty[MAX_NST];
  uint64_t bank_full[2];  // MMAs of a group have completed in the bank
  uint64_t bank_free[2];  // the drain warps have read the bank
  uint64_t never;  // never arrived on: CTQ_DEBUG_STALL_WAIT waits on it
  uint32_t issued;    // chunks issued by the producer (sequence numbers [0, issued))
  uint32_t consumed;  // chunks whose data the MMA issuer has waited for
  uint32_t tmem_base;
  int fail;
  float red[8];
  double redd[64];
};

}  // namespace

namespace {

template <int PREC>
__global__ void __launch_bounds__(BG_THREADS, 1)
    k_trace_big(DevModel M, BatchView B, EvalCfg cfg, Work W, BigParams P) {
  using T = typename Elt<PREC>::T;
  constexpr bool SPLIT = PREC != CTQ_TF32;   // hi and lo operand planes
  constexpr int EB = int(sizeof(T));
  constexpr int BKE = ROWB / EB;             // K elements per staged chunk
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ BigShared S;
  const int NST = P.nst;
  const uint32_t stage_bytes = (SPLIT ? 2u : 1u) * (A_BYTES + B_BYTES);
  unsigned char* stage0 = smem_raw;
  float* p_s = reinterpret_cast<float*>(stage0 + size_t(NST) * stage_bytes);  // [PVEC] column scales
  // [PVEC] wrap-around propagator of q0: only the first, elementwise product
  // of a string reads it, when no copy or MMA uses the stages
  float* q_s = reinterpret_cast<float*>(stage0);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ns = M.n_sec;
  const int cplx = M.is_complex;

  if (tid == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.bank_full[b], 1);
      mbar_init(&S.bank_free[b], N_DRAIN);  // one arrival per drain warp
    }
    mbar_init(&S.never, 1);
    S.fail = 0;
    S.issued = 0;
    S.consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&S.tmem_base, NBANK * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = S.tmem_base;
  const int lane = tid & 31;
  uint32_t seq_base = 0;  // sequence number of chunk 0 of the current tile (all threads)
  uint32_t grp_base = 0;  // sequence number of the current tile's first accumulation group
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
  T* zb = reinterpret_cast<T*>(P.zbuf);
  T* Zh[2] = {zb, zb + 2 * P.zfloats};
  T* Zl[2] = {zb + P.zfloats, zb + 3 * P.zfloats};

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
      const int nkc = 2 * dpk / BKE;
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
        const size_t o_r = tiled_off<EB>(j, m, BM, nkc), o_i = tiled_off<EB>(j, dpk + m, BM, nkc);
        T hr, lr, hi_, li;
        split_store<PREC>(xr, hr, lr);
        split_store<PREC>(xi, hi_, li);
        Zh[0][o_r] = hr;
        Zh[0][o_i] = hi_;
        if (SPLIT) {
          Zl[0][o_r] = lr;
          Zl[0][o_i] = li;
        }
      }
      // q_s lives in the stages: order these generic accesses before the
      // bulk copies that will refill them
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
        const int dpk = rup(dcur, BK), nkc = 2 * dpk / BKE;
        double vr = 0.0, vi = 0.0;
        const long long total = (long long)d0 * dcur;
        for (long long e2 = (long long)blockIdx.x * BG_THREADS + tid; e2 < total;
             e2 += (long long)gridDim.x * BG_THREADS) {
          const int j = int(e2 / dcur), k = int(e2 - (long long)j * dcur);
          const size_t o_r = tiled_off<EB>(j, k, BM, nkc), o_i = tiled_off<EB>(j, dpk + k, BM, nkc);
          float zr = elt_val<PREC>(Zh[cur][o_r]), zi = elt_val<PREC>(Zh[cur][o_i]);
          if (SPLIT) {
            zr += elt_val<PREC>(Zl[cur][o_r]);
            zi += elt_val<PREC>(Zl[cur][o_i]);
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
      const int dpk = rup(dcur, BK), nkc = 2 * dpk / BKE;   // K chunks of this product
      const int dpn = rup(db, BK), nkc_n = 2 * dpn / BKE;   // K chunks of the next one
      {
        const double dt = B.tau[a0 + i + 1] - B.tau[a0 + i];
        const double* Eb = M.E_rel + M.E_off[qb];
        for (int j = tid; j < dpn; j += BG_THREADS) p_s[j] = (j < db) ? expf(float(-dt * Eb[j])) * scale : 0.f;
        __syncthreads();
        L.add(-dt * (M.E_min[qb] - M.E_ref));
        prefix -= dt * (M.E_min[qb] - M.E_ref);
      }
      __syncthreads();
      const T* Bt = reinterpret_cast<const T*>(P.bt) + P.bt_off[idx_a];
      const size_t b_tile = B_BYTES / EB, a_tile = A_BYTES / EB;      // elements per staged tile
      const size_t b_plane = size_t(rup(2 * dpn, BN) / BN) * nkc * b_tile;  // elements of one B plane
      const int n_mt = dp0 / BM, n_nt = (2 * dpn + BN - 1) / BN;
      const int n_tiles = n_mt * n_nt;
      const int nxt = cur ^ 1;
      int ek = 0;
      float f2 = 0.f;
      // Warp-specialised pipeline.  Chunks carry a per-CTA sequence number q
      // (q = seq_base + kc within a tile), live in stage q % NST and complete
      // phase q / NST of that stage's full / empty barriers.  Thread 32 (the
      // producer) refills a stage as soon as the products reading it have
      // completed and, at the end of a tile, issues the first chunks of the
      // CTA's next tile of the same product; thread 0 (the MMA issuer) only
      // waits for data.  The K loop is cut into groups of GRP chunks with
      // sequence numbers g (g = grp_base + kc / GRP); group g accumulates in
      // tensor-memory bank g % 2, which the N_DRAIN drain warps add into FP32
      // registers (round to nearest) while the tensor core fills the other
      // bank.  After a tile's last group the drain warps run the epilogue
      // from registers and the issuer and producer go on with the next tile.
      volatile int* fail_v = &S.fail;
      auto produce = [&](uint32_t q, int tt, int kc) -> bool {
        int mt_, nt_;
        tile_coords(tt, n_mt, n_nt, P.order, mt_, nt_);
        const int st = int(q % uint32_t(NST));
        if (q >= uint32_t(NST) && !mbar_wait(&S.empty[st], ((q / NST) - 1u) & 1u, P.timeout_ns)) return false;
        unsigned char* sb = stage0 + size_t(st) * stage_bytes;
        const size_t ao = (size_t(mt_) * nkc + kc) * a_tile, bo = (size_t(nt_) * nkc + kc) * b_tile;
        mbar_arrive_expect_tx(&S.full[st], stage_bytes);
        bulk_g2s(sb, Zh[cur] + ao, A_BYTES, &S.full[st]);
        bulk_g2s(sb + A_BYTES, Bt + bo, B_BYTES, &S.full[st]);
        if (SPLIT) {
          bulk_g2s(sb + A_BYTES + B_BYTES, Zl[cur] + ao, A_BYTES, &S.full[st]);
          bulk_g2s(sb + 2 * A_BYTES + B_BYTES, Bt + b_plane + bo, B_BYTES, &S.full[st]);
        }
        S.issued = q + 1;
        return true;
      };
      const int ngrp = (nkc + GRP - 1) / GRP;
      int pre = 0;  // (producer) chunks of the current tile already issued
      for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        int mt, nt;
        tile_coords(t, n_mt, n_nt, P.order, mt, nt);
        const int ncols = min(BN, 2 * dpn - nt * BN);
        if (tid == 32) {
          bool okp = true;
          for (int kc = pre; kc < nkc && okp && !*fail_v; ++kc) okp = produce(seq_base + kc, t, kc);
          pre = 0;
          const int tn = t + int(gridDim.x);
          if (okp && tn < n_tiles) {
            const int np = min(NST, nkc);
            for (int j = 0; j < np && okp && !*fail_v; ++j) okp = produce(seq_base + nkc + j, tn, j);
            pre = np;
          }
          if (!okp) *fail_v = 1;
        } else if (tid == 0) {
          const uint32_t idesc = (PREC == CTQ_BF16X3) ? idesc_bf16(BM, ncols) : idesc_tf32(BM, ncols);
          for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t q = seq_base + kc;
            const uint32_t g = grp_base + uint32_t(kc / GRP);
            const int st = int(q % uint32_t(NST));
            const uint32_t bank = g & 1u;
            if (kc % GRP == 0 && g >= 2u &&
                (*fail_v || !mbar_wait(&S.bank_free[bank], ((g >> 1) - 1u) & 1u, P.timeout_ns))) {
              *fail_v = 1;
              break;
            }
            if (*fail_v || !mbar_wait(&S.full[st], (q / NST) & 1u, P.timeout_ns)) {
              *fail_v = 1;
              break;
            }
            S.consumed = q + 1;
            tc_fence_after();
            const uint32_t sa = smem_u32(stage0 + size_t(st) * stage_bytes);
            const uint32_t sbh = sa + A_BYTES, sal = sbh + B_BYTES, sbl = sal + A_BYTES;
            const uint32_t tacc = tD + bank * uint32_t(BN);
            // one MMA covers 32 bytes of K (8 tf32 or 16 bf16): two core matrices
            for (int kk = 0; kk < ROWB / 32; ++kk) {
              const uint64_t da = sdesc(sa + kk * 2 * LBO_A, LBO_A, 128);
              const uint64_t dbh = sdesc(sbh + kk * 2 * LBO_B, LBO_B, 128);
              mma_big<PREC>(tacc, da, dbh, idesc, (kc % GRP != 0 || kk > 0) ? 1u : 0u);
              if (SPLIT) {
                mma_big<PREC>(tacc, da, sdesc(sbl + kk * 2 * LBO_B, LBO_B, 128), idesc, 1u);
                mma_big<PREC>(tacc, sdesc(sal + kk * 2 * LBO_A, LBO_A, 128), dbh, idesc, 1u);
              }
            }
            mma_commit(&S.empty[st]);
            if (kc % GRP == GRP - 1 || kc == nkc - 1) mma_commit(&S.bank_full[bank]);
          }
        } else if (warp >= 2) {
          // drain warps: lane quarter warp % 4, column slice (warp - 2) / 4 of
          // COLS columns
          constexpr int COLS = BN / (N_DRAIN / 4);
          const int slice = (warp - 2) >> 2;
          const uint32_t tl = uint32_t(32 * (warp & 3)) << 16;
          float acc[COLS];
#pragma unroll
          for (int c = 0; c < COLS; ++c) acc[c] = 0.f;
          bool okd = true;
          for (int gi = 0; gi < ngrp; ++gi) {
            const uint32_t g = grp_base + uint32_t(gi);
            const uint32_t bank = g & 1u;
            if (*fail_v || !mbar_wait(&S.bank_full[bank], (g >> 1) & 1u, P.timeout_ns)) {
              okd = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < COLS / 32; ++h) {  // 32 columns per tensor-memory wait
              uint32_t v[2][16];
#pragma unroll
              for (int u = 0; u < 2; ++u)
                tmem_ld16(tD + bank * uint32_t(BN) + tl + uint32_t(slice * COLS + h * 32 + u * 16), v[u]);
              tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[h * 32 + u * 16 + c] += __uint_as_float(v[u][c]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.bank_free[bank]);
          }
          if (!okd) *fail_v = 1;
          // epilogue from registers: this thread's row, COLS columns
          const int row = mt * BM + 32 * (warp & 3) + lane;
#pragma unroll
          for (int c0 = 0; c0 < COLS; c0 += 16) {
            const int cb = slice * COLS + c0;  // column within the tile
            if (!okd || cb >= ncols) break;
            // 16 consecutive K elements of the next product, written as
            // 16-byte vectors of PER16 elements
            constexpr int PER16 = 16 / EB;
#pragma unroll
            for (int g = 0; g < 16 / PER16; ++g) {
              T hi[PER16], lo[PER16];
#pragma unroll
              for (int t2 = 0; t2 < PER16; ++t2) {
                const int col = nt * BN + cb + PER16 * g + t2;  // embedded column
                const int j = (col < dpn) ? col : col - dpn;
                const float x = acc[c0 + PER16 * g + t2] * p_s[j];
                ek = max(ek, (__float_as_int(x) >> 23) & 0xff);
                f2 += x * x;
                split_store<PREC>(x, hi[t2], lo[t2]);
              }
              const size_t o = tiled_off<EB>(row, nt * BN + cb + PER16 * g, BM, nkc_n);
              *reinterpret_cast<uint4*>(Zh[nxt] + o) = pack16<PREC>(hi);
              if (SPLIT) *reinterpret_cast<uint4*>(Zl[nxt] + o) = pack16<PREC>(lo);
            }
          }
        }
        seq_base += uint32_t(nkc);
        grp_base += uint32_t(ngrp);
      }
      // the running product is read by bulk copies (async proxy) next
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __syncthreads();
      if (S.fail) {
        if (tid == 32)  // let issued copies that were never consumed land before leaving
          for (uint32_t q = S.consumed; q < S.issued; ++q)
            mbar_wait(&S.full[q % uint32_t(NST)], (q / NST) & 1u, P.timeout_ns);
        alive = false;
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
    tmem_dealloc(tD, NBANK * BN);
  }
}

// Embedded, tiled, split copy of every block (grid-stride over elements):
// B'[n][k] for n < 2 dpn, k < 2 dpk with
//   n < dpn:  [Re F[n][k],  -Im F[n][k - dpk]]
//   n >= dpn: [Im F[n - dpn][k], Re F[n - dpn][k - dpk]],
// hi plane then lo plane in the operand format of PREC.
template <int PREC>
__global__ void k_format_big(const double* blk, int cplx, int dn, int dk, typename Elt<PREC>::T* out) {
  using T = typename Elt<PREC>::T;
  constexpr int EB = int(sizeof(T));
  const int dpn = rup(dn, BK), dpk = rup(dk, BK);
  const int N2 = rup(2 * dpn, BN), K2 = 2 * dpk, nkc = K2 / (ROWB / EB);
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
    const size_t o = tiled_off<EB>(n, k, BN, nkc);
    if constexpr (PREC == CTQ_BF16X3) {
      const uint32_t h = bf16_bits(float(v));
      out[o] = uint16_t(h);
      out[plane + o] = uint16_t(bf16_bits(float(v - double(bf16_val(h)))));
    } else {
      const uint32_t h = to_tf32(float(v));
      out[o] = __uint_as_float(h);
      out[plane + o] = __uint_as_float(to_tf32(float(v - double(__uint_as_float(h)))));
    }
  }
}

// Diagnostic GEMM with the operand conventions of k_trace_big: D = A B^T for
// one 128 x N tile, A (128 x K) and B (N x K) split and tiled on the device
// exactly like Z and the embedded blocks, staged chunk by chunk with bulk
// copies and multiplied with the same descriptors and instruction kinds.
constexpr int CHK_THREADS = 128;  // one thread per row of the tile

template <int PREC>
__global__ void __launch_bounds__(CHK_THREADS, 1)
    k_big_gemm_check(const float* A, const float* Bm, typename Elt<PREC>::T* ws, float* D, int N, int K,
                     uint64_t timeout_ns, int* status) {
  using T = typename Elt<PREC>::T;
  constexpr bool SPLIT = PREC != CTQ_TF32;
  constexpr int EB = int(sizeof(T));
  constexpr int BKE = ROWB / EB;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar_full, bar_done;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nkc = K / BKE;
  const size_t a_tile = A_BYTES / EB, b_tile = B_BYTES / EB;
  T* Ah = ws;
  T* Al = Ah + size_t(nkc) * a_tile;
  T* Bh = Al + size_t(nkc) * a_tile;
  T* Bl = Bh + size_t(nkc) * b_tile;
  for (int e = tid; e < 128 * K; e += CHK_THREADS) {
    const int r = e / K, k = e - r * K;
    T h, l;
    split_store<PREC>(A[e], h, l);
    Ah[tiled_off<EB>(r, k, BM, nkc)] = h;
    Al[tiled_off<EB>(r, k, BM, nkc)] = l;
  }
  for (int e = tid; e < BN * K; e += CHK_THREADS) {
    const int r = e / K, k = e - r * K;
    T h, l;
    split_store<PREC>(r < N ? Bm[size_t(r) * K + k] : 0.f, h, l);
    Bh[tiled_off<EB>(r, k, BN, nkc)] = h;
    Bl[tiled_off<EB>(r, k, BN, nkc)] = l;
  }
  __threadfence();
  asm volatile("fence.proxy.async.global;" ::: "memory");
  if (tid == 0) {
    mbar_init(&bar_full, 1);
    mbar_init(&bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = tmem_base;
  bool ok = true;
  if (tid == 0) {
    const uint32_t idesc = (PREC == CTQ_BF16X3) ? idesc_bf16(BM, N) : idesc_tf32(BM, N);
    const uint32_t bytes = (SPLIT ? 2u : 1u) * (A_BYTES + B_BYTES);
    for (int kc = 0; kc < nkc && ok; ++kc) {
      mbar_arrive_expect_tx(&bar_full, bytes);
      bulk_g2s(smem_raw, Ah + size_t(kc) * a_tile, A_BYTES, &bar_full);
      bulk_g2s(smem_raw + A_BYTES, Bh + size_t(kc) * b_tile, B_BYTES, &bar_full);
      if (SPLIT) {
        bulk_g2s(smem_raw + A_BYTES + B_BYTES, Al + size_t(kc) * a_tile, A_BYTES, &bar_full);
        bulk_g2s(smem_raw + 2 * A_BYTES + B_BYTES, Bl + size_t(kc) * b_tile, B_BYTES, &bar_full);
      }
      ok = mbar_wait(&bar_full, uint32_t(kc & 1), timeout_ns);
      if (!ok) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem_raw), sbh = sa + A_BYTES, sal = sbh + B_BYTES, sbl = sal + A_BYTES;
      for (int kk = 0; kk < ROWB / 32; ++kk) {
        const uint64_t da = sdesc(sa + kk * 2 * LBO_A, LBO_A, 128);
        const uint64_t dbh = sdesc(sbh + kk * 2 * LBO_B, LBO_B, 128);
        mma_big<PREC>(tD, da, dbh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
        if (SPLIT) {
          mma_big<PREC>(tD, da, sdesc(sbl + kk * 2 * LBO_B, LBO_B, 128), idesc, 1u);
          mma_big<PREC>(tD, sdesc(sal + kk * 2 * LBO_A, LBO_A, 128), dbh, idesc, 1u);
        }
      }
      mma_commit(&bar_done);
      ok = mbar_wait(&bar_done, uint32_t(kc & 1), timeout_ns);  // the stage is reused by the next chunk
    }
    if (!ok) *status = CTQ_ERR_TIMEOUT;
  }
  __syncthreads();
  if (*status == 0) {
    tc_fence_after();
    const uint32_t lane_off = uint32_t(32 * warp) << 16;
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tD + lane_off + c0, v);
      tmem_wait_ld();
      for (int t = 0; t < 16; ++t) D[size_t(tid) * N + c0 + t] = __uint_as_float(v[t]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tD, BN);
  }
}

}  // namespace

size_t big_block_elems(int dn, int dk) {
  const int dpn = (dn + BK - 1) / BK * BK, dpk = (dk + BK - 1) / BK * BK;
  return size_t((2 * dpn + BN - 1) / BN * BN) * size_t(2 * dpk) * 2;  // hi and lo planes
}

// Lays out and fills the embedded blocks on the device (d_blk: the float64
// blocks already on the device) in the operand format of prec (CTQ_TF32X3
// planes also serve CTQ_TF32).  out/off: device buffer and element offsets.
int format_big_blocks(const HostModel& h, const double* d_blk, void* out, const std::vector<int64_t>& off, int prec) {
  const int na = h.n_alpha();
  for (int a = 0; a < na; ++a)
    for (int q = 0; q < h.n_sec; ++q) {
      const size_t i = size_t(a) * h.n_sec + q;
      const int qp = h.s[i];
      if (qp < 0) continue;
      const double* src = d_blk + (h.is_complex ? 2 : 1) * h.blk_off[i];
      if (prec == CTQ_BF16X3)
        k_format_big<CTQ_BF16X3><<<1024, 256>>>(src, h.is_complex, h.dims[qp], h.dims[q],
                                                static_cast<uint16_t*>(out) + off[i]);
      else
        k_format_big<CTQ_TF32X3><<<1024, 256>>>(src, h.is_complex, h.dims[qp], h.dims[q],
                                                static_cast<float*>(out) + off[i]);
      if (cudaGetLastError() != cudaSuccess) return CTQ_ERR_CUDA;
    }
  return cudaDeviceSynchronize() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

size_t big_scratch_bytes(const HostModel& h, int max_ops, int grid) {
  int dmax = h.max_dim;
  const size_t zf = size_t((dmax + BM - 1) / BM * BM) * size_t(2 * ((dmax + BK - 1) / BK * BK));
  return 4 * zf * 4 + 256 + size_t(max_ops + 2) * (4 + 8) + size_t(2 * grid) * 8 + 1024;
}

static int big_stages(int prec) { return prec == CTQ_TF32 ? 4 : 2; }

static size_t big_smem(int prec, int nst) {
  const size_t stages = size_t(nst) * (prec == CTQ_TF32 ? 1 : 2) * (A_BYTES + B_BYTES);
  return std::max(stages, size_t(PVEC) * 4) + PVEC * 4;  // the stages also hold q_s
}

template <int PREC>
static cudaError_t big_attr(size_t smem) {
  return cudaFuncSetAttribute(k_trace_big<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

// The kernel may be launched with up to lc->smem_optin bytes of dynamic shared
// memory (more pipeline stages through the caller's launch tuning); lc->smem
// is the default stage count's need.
int prepare_eval_big(int prec, int num_sms, LaunchCfg* lc) {
  lc->threads = BG_THREADS;
  lc->num_sms = num_sms;
  lc->smem = big_smem(prec, big_stages(prec));
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return CTQ_ERR_CUDA;
  cudaFuncAttributes fa;
  cudaError_t e = prec == CTQ_TF32     ? cudaFuncGetAttributes(&fa, k_trace_big<CTQ_TF32>)
                  : prec == CTQ_BF16X3 ? cudaFuncGetAttributes(&fa, k_trace_big<CTQ_BF16X3>)
                                       : cudaFuncGetAttributes(&fa, k_trace_big<CTQ_TF32X3>);
  if (e != cudaSuccess) return CTQ_ERR_CUDA;
  lc->smem_optin = optin - int(fa.sharedSizeBytes);
  e = prec == CTQ_TF32     ? big_attr<CTQ_TF32>(lc->smem_optin)
      : prec == CTQ_BF16X3 ? big_attr<CTQ_BF16X3>(lc->smem_optin)
                           : big_attr<CTQ_TF32X3>(lc->smem_optin);
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
  P.nst = cfg.stages > 0 ? cfg.stages : big_stages(P.prec);
  P.order = cfg.tile_order;
  const size_t smem = big_smem(P.prec, P.nst);
  if (P.nst < 2 || P.nst > MAX_NST || smem > size_t(lc.smem_optin)) return CTQ_ERR_UNSUPPORTED;
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
  void* fn = P.prec == CTQ_TF32     ? (void*)k_trace_big<CTQ_TF32>
             : P.prec == CTQ_BF16X3 ? (void*)k_trace_big<CTQ_BF16X3>
                                    : (void*)k_trace_big<CTQ_TF32X3>;
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, grid, BG_THREADS, args, smem, st);
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

extern "C" int ctq_big_gemm_check(int device, const float* A, const float* Bm, float* D, int N, int K, int precision) {
  using namespace ctq;
  auto fail = [](int code, const char* msg) {
    set_last_error(msg);
    return code;
  };
  if (!A || !Bm || !D) return fail(CTQ_ERR_ARG, "null argument");
  if (precision != CTQ_TF32 && precision != CTQ_TF32X3 && precision != CTQ_BF16X3)
    return fail(CTQ_ERR_ARG, "precision must be CTQ_TF32, CTQ_TF32X3 or CTQ_BF16X3");
  if (N < 16 || N > BN || N % 16 != 0) return fail(CTQ_ERR_ARG, "N must be a multiple of 16 in [16, 128]");
  if (K < 64 || K > 4096 || K % 64 != 0) return fail(CTQ_ERR_ARG, "K must be a multiple of 64 in [64, 4096]");
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return fail(CTQ_ERR_CUDA, "cudaSetDevice failed");
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  void* ws = nullptr;
  int* dS = nullptr;
  int st = CTQ_OK;
  const size_t ws_bytes = size_t(2) * (128 + BN) * K * 4;
  if (cudaMalloc(&dA, size_t(128) * K * 4) || cudaMalloc(&dB, size_t(N) * K * 4) ||
      cudaMalloc(&dD, size_t(128) * N * 4) || cudaMalloc(&ws, ws_bytes) || cudaMalloc(&dS, 4)) {
    st = CTQ_ERR_NOMEM;
  } else {
    cudaMemcpy(dA, A, size_t(128) * K * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, Bm, size_t(N) * K * 4, cudaMemcpyHostToDevice);
    cudaMemset(dS, 0, 4);
    const size_t smem = 2 * size_t(A_BYTES + B_BYTES);
    const uint64_t tmo = 2000000000ull;
    if (precision == CTQ_BF16X3) {
      cudaFuncSetAttribute(k_big_gemm_check<CTQ_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_big_gemm_check<CTQ_BF16X3><<<1, CHK_THREADS, smem>>>(dA, dB, static_cast<uint16_t*>(ws), dD, N, K, tmo, dS);
    } else if (precision == CTQ_TF32X3) {
      cudaFuncSetAttribute(k_big_gemm_check<CTQ_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_big_gemm_check<CTQ_TF32X3><<<1, CHK_THREADS, smem>>>(dA, dB, static_cast<float*>(ws), dD, N, K, tmo, dS);
    } else {
      cudaFuncSetAttribute(k_big_gemm_check<CTQ_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      k_big_gemm_check<CTQ_TF32><<<1, CHK_THREADS, smem>>>(dA, dB, static_cast<float*>(ws), dD, N, K, tmo, dS);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) st = CTQ_ERR_CUDA;
    if (st == CTQ_OK) {
      int hs = 0;
      cudaMemcpy(D, dD, size_t(128) * N * 4, cudaMemcpyDeviceToHost);
      cudaMemcpy(&hs, dS, 4, cudaMemcpyDeviceToHost);
      st = hs;
    }
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(ws);
  cudaFree(dS);
  if (prev != device) cudaSetDevice(prev);
  return st == CTQ_OK ? CTQ_OK : fail(st, "big-path GEMM check failed");
}
