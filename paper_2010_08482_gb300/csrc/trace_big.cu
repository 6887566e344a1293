// Large-block sector-string trace on the tensor cores (blocks of hundreds to
// thousands of states, e.g. an f shell with N in {4, 5, 6}: 1001 / 2002 / 3003).
//
// One (chain, q0) item is evaluated at a time by the whole GPU: a persistent
// cooperative kernel (one CTA per SM) walks the items of the work list and,
// for each, the operators of its string.  The chain runs transposed,
// Z_i = Y_i^T (d0 x d_i),
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
// the power-of-two rescale of the previous operator, one per 128-row tile),
// reduces max|Z| and ||Z||_F per row tile, splits hi/lo and writes Z_{i+1}
// tiles.  A row of Z belongs to one initial state and rows never mix, so the
// products of a string are scheduled tile by tile with row-tile
// dependencies instead of a grid barrier per operator (see k_trace_big).
// The first operator only scales F_1; the last one needs only the diagonal
// of F_n Y (FP32 products, FP64 sum).  Log scale, exponents, segment bounds
// and the trace stay in float64.
//
// Every wait is bounded (mbarriers, row-tile flags and the grid barrier) by
// the caller's timeout: on expiry the kernel records CTQ_ERR_TIMEOUT in the
// workspace, stops, frees its tensor memory and returns.
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
constexpr int PVEC = 3072;        // largest sector dimension of this path
constexpr int RT_MAX = PVEC / BM; // row tiles of the largest running product
constexpr int DR = 4;             // tile descriptors the producer may announce ahead

// One tile of the product schedule: stage s (Z_{s+1} = Z_s F_{s+1}^T P_{s+1}),
// row tile mt, column tile nt; s < 0 ends the products of the string.
struct Unit {
  int s, mt, nt, skip;
};

struct BigShared {
  uint64_t full[MAX_NST];
  uint64_t empty[MAX_NST];
  uint64_t bank_full[2];   // MMAs of a group have completed in the bank
  uint64_t bank_free[2];   // the drain warps have read the bank
  uint64_t unit_full[DR];  // the producer has announced the tile in slot i
  uint64_t unit_empty[DR]; // the MMA issuer and the drain warps have read it
  uint64_t never;  // never arrived on: CTQ_DEBUG_STALL_WAIT waits on it
  Unit unit[DR];
  uint32_t issued;    // chunks issued by the producer (sequence numbers [0, issued))
  uint32_t consumed;  // chunks whose data the MMA issuer has waited for
  uint32_t tmem_base;
  int fail;
  double redd[64];
};

// Per-string state of the product schedule in global memory, two copies that
// alternate between consecutive strings.  Entry s * RT_MAX + r belongs to row
// tile r of the stored product Z_s:
//   ekey   max float exponent field over the row tile,
//   cnt    reports of drain warps (N_DRAIN per column tile) for the row tile,
//   ready  the row tile is complete (set once, by the tile that completes it),
//   ecum   sum over t <= s of the power-of-two exponents e_r(t) taken out of
//          row tile r (every row tile carries its own rescale),
//   fr     squared Frobenius norm of the stored row tile;
// rows[s]: row tiles of Z_s complete; part[2 r]: partial trace of row tile r
// (re, im); abort[0]: the string was rejected early.
struct RowState {
  int *ekey, *cnt, *ready, *ecum, *rows, *abort;
  double *fr, *part;
};

__host__ __device__ __forceinline__ size_t row_state_int_bytes(int max_ops) {
  return ((4 * size_t(max_ops + 2) * RT_MAX + size_t(max_ops + 2) + 2) * 4 + 15) / 16 * 16;
}
__host__ __device__ __forceinline__ size_t row_state_bytes(int max_ops) {
  return (row_state_int_bytes(max_ops) + 8 * (size_t(max_ops + 2) * RT_MAX + 2 * RT_MAX) + 255) / 256 * 256;
}
__device__ __forceinline__ RowState row_state(unsigned char* base, int max_ops) {
  const size_t ne = size_t(max_ops + 2) * RT_MAX;
  int* ip = reinterpret_cast<int*>(base);
  RowState R;
  R.ekey = ip;
  R.cnt = ip + ne;
  R.ready = ip + 2 * ne;
  R.ecum = ip + 3 * ne;
  R.rows = ip + 4 * ne;
  R.abort = R.rows + (max_ops + 2);
  R.fr = reinterpret_cast<double*>(base + row_state_int_bytes(max_ops));
  R.part = R.fr + ne;
  return R;
}

// Shared-memory tables of the current string, after the stages: tau, log
// scale and bound prefix (float64), operator, sector path and first tile of
// every product stage (int), max_ops + 1 entries each.
__host__ __device__ __forceinline__ size_t big_table_bytes(int max_ops) {
  return size_t(max_ops + 1) * (3 * 8 + 3 * 4);
}

// Warp-uniform bounded wait: every lane waits, the warp goes on only if all
// lanes saw the phase complete and nobody has failed.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit, volatile int* fail) {
  const bool ok = !*fail && mbar_wait(bar, parity, limit);
  return __all_sync(0xffffffffu, ok) != 0;
}

}  // namespace

namespace {

// Products are scheduled tile by tile: all tiles of all product stages of a
// string form one sequence (stage by stage, tile order P.order inside a
// stage) dealt round-robin to the persistent CTAs.  A tile of stage s only
// needs row tile mt of Z_s (a row of Z is one initial state: rows never mix),
// so instead of a grid barrier per operator the producer waits for that row
// tile's ready flag, and a CTA whose share of stage s runs out goes on with
// stage s + 1 while others finish stage s.  Each row tile is rescaled by its
// own power of two; the lazy bound of a checkpoint is computed by the tile
// that completes the stage, and a rejected string's remaining tiles are
// skipped.  Deadlock freedom: every tile depends only on tiles earlier in the
// sequence, each CTA takes its tiles in sequence order, and all CTAs are
// co-resident, so the earliest unfinished tile can always run.
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
  // [PVEC] column propagator of the first, elementwise product: lives in the
  // stages, which no copy or MMA uses at that time
  float* p_s = reinterpret_cast<float*>(stage0);
  const int TBL = cfg.max_ops + 1;
  double* tau_s = reinterpret_cast<double*>(stage0 + size_t(NST) * stage_bytes);
  double* L_s = tau_s + TBL;    // log scale after k propagators (compensated sum)
  double* pre_s = L_s + TBL;    // bound prefix after k propagators
  int* op_s = reinterpret_cast<int*>(pre_s + TBL);
  int* path_s = op_s + TBL;     // sector after k operators
  int* ustart_s = path_s + TBL; // first tile of product stage s; [n - 1] = all tiles
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
    for (int i = 0; i < DR; ++i) {
      mbar_init(&S.unit_full[i], 1);
      mbar_init(&S.unit_empty[i], 1 + N_DRAIN);  // the issuer and every drain warp
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
  volatile int* fail_v = &S.fail;
  // per-role running counters (every role advances its own copy identically)
  uint32_t seq_base = 0;  // sequence number of chunk 0 of the current tile
  uint32_t grp_base = 0;  // sequence number of the current tile's first accumulation group
  uint32_t ucount = 0;    // tile descriptors passed through the ring
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
  const size_t sbytes = row_state_bytes(cfg.max_ops);
  // Row-tile stride (in K chunks) of every stored product: the widest Z.
  // Row tile r of Z_{s+1} is written while other row tiles of Z_{s-1}, in
  // the same buffer, may still be read; with one stride for all widths the
  // row tiles of different products never share memory.
  const int nkz = 2 * rup(M.max_dim, BK) / BKE;
  const long long gthreads = (long long)gridDim.x * BG_THREADS;
  const long long gtid = (long long)blockIdx.x * BG_THREADS + tid;
  if (alive) {
    int* z = reinterpret_cast<int*>(P.state);
    for (long long i = gtid; i < (long long)(sbytes / 4); i += gthreads) z[i] = 0;
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) alive = false;
  }
  int par = 0;  // state copy of the current string

  for (int it_idx = 0; it_idx < n_items && alive; ++it_idx) {
    const Item it = items[W.order[it_idx]];
    const int c = it.c, q0 = it.q0;
    const size_t slot = size_t(c) * ns + q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const int dp0 = rup(d0, BM);
    const double* E0 = M.E_rel + M.E_off[q0];
    const bool track = cfg.lazy || cfg.bounds != nullptr;
    double* segp = W.seg + slot * size_t(cfg.n_seg_max + 1);

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

    const RowState RS = row_state(P.state + size_t(par) * sbytes, cfg.max_ops);
    unsigned char* next_state = P.state + size_t(par ^ 1) * sbytes;
    par ^= 1;
    const int R = dp0 / BM;

    // ---- tables of the string (every CTA keeps its own copy)
    for (int k = tid; k < n; k += BG_THREADS) {
      op_s[k] = B.op[a0 + k];
      tau_s[k] = B.tau[a0 + k];
    }
    __syncthreads();
    if (tid == 0) {
      const double er0 = M.E_min[q0] - M.E_ref;
      KSum L;
      L.add(-tau_s[0] * er0);
      L.add(-(B.beta - tau_s[n - 1]) * er0);
      double pre = M.log_norm[op_s[0] * ns + q0];
      int q = q0;
      path_s[0] = q0;
      for (int k = 1; k < n; ++k) {
        q = M.s[op_s[k - 1] * ns + q];
        path_s[k] = q;
        const double dt = tau_s[k] - tau_s[k - 1];
        const double er = M.E_min[q] - M.E_ref;
        L.add(-dt * er);
        pre -= dt * er;
        L_s[k] = L.val();
        pre_s[k] = pre;
        pre += M.log_norm[op_s[k] * ns + q];
      }
      path_s[n] = M.s[op_s[n - 1] * ns + q];
      int u = 0;
      for (int s = 1; s <= n - 2; ++s) {
        ustart_s[s] = u;
        u += R * ((2 * rup(M.dims[path_s[s + 1]], BK) + BN - 1) / BN);
      }
      ustart_s[n - 1] = u;
    }
    __syncthreads();

    // Lazy bound after a applied operators (one thread): the stored Z_a row
    // tiles carry the exponents ecum[a - 1][r].
    auto bound = [&](int a) {
      int emx = INT_MIN;
      for (int r = 0; r < R; ++r)
        if (__ldcg(&RS.fr[a * RT_MAX + r]) > 0.0) emx = max(emx, __ldcg(&RS.ecum[(a - 1) * RT_MAX + r]));
      double sfr = 0.0;
      if (emx != INT_MIN)
        for (int r = 0; r < R; ++r) {
          const double f = __ldcg(&RS.fr[a * RT_MAX + r]);
          if (f > 0.0) sfr += ldexp(f, 2 * (__ldcg(&RS.ecum[(a - 1) * RT_MAX + r]) - emx));
        }
      const double ub = (sfr > 0.0) ? 0.5 * it.log_r + 0.5 * log(sfr) + double(emx) * LN2 + L_s[a] +
                                          (it.t_all - pre_s[a])
                                    : -INFINITY;
      segp[a / cfg.S] = ub;
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
        if (flag & FLAG_REJECTED) atomicExch(RS.abort, 1);
        __threadfence();
      }
    };

    // ---- operator 1 (elementwise): Z_1[j][m] = p0[j] F_1[m][j] p1[m]
    {
      const int qb = path_s[1];
      const int d1 = M.dims[qb];
      const int dpk = rup(d1, BK);
      const double dt = tau_s[1] - tau_s[0];
      const double t_first = tau_s[0], t_last = B.beta - tau_s[n - 1];
      const double* Eb = M.E_rel + M.E_off[qb];
      for (int m = tid; m < d1; m += BG_THREADS) p_s[m] = expf(float(-dt * Eb[m]));
      __syncthreads();
      const int64_t off = M.blk_off[op_s[0] * ns + q0];
      int cur_r = -1, ek = 0;
      float f2 = 0.f;
      // the 32 lanes of a warp always share a row (dpk is a multiple of 32),
      // so row-tile partials are flushed warp by warp
      auto flush = [&]() {
        const int ekw = __reduce_max_sync(0xffffffffu, ek);
        const double fw = warp_sum(double(f2));
        if (lane == 0 && cur_r >= 0) {
          atomicMax(&RS.ekey[RT_MAX + cur_r], ekw);
          atomicAdd(&RS.fr[RT_MAX + cur_r], fw);
        }
        ek = 0;
        f2 = 0.f;
      };
      const long long total = (long long)dp0 * dpk;
      for (long long e = gtid; e < total; e += gthreads) {
        const int j = int(e / dpk), m = int(e - (long long)j * dpk);
        const int r = j / BM;
        if (r != cur_r) {
          flush();
          cur_r = r;
        }
        float xr = 0.f, xi = 0.f;
        if (j < d0 && m < d1) {
          const float pj = expf(float(-t_first * E0[j])) * expf(float(-t_last * E0[j])) * p_s[m];
          const int64_t fe = off + int64_t(m) * d0 + j;
          xr = float(cplx ? M.blk[2 * fe] : M.blk[fe]) * pj;
          xi = cplx ? float(M.blk[2 * fe + 1]) * pj : 0.f;
        }
        ek = max(ek, max((__float_as_int(xr) >> 23) & 0xff, (__float_as_int(xi) >> 23) & 0xff));
        f2 += xr * xr + xi * xi;
        const size_t o_r = tiled_off<EB>(j, m, BM, nkz), o_i = tiled_off<EB>(j, dpk + m, BM, nkz);
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
      flush();
      // p_s lives in the stages and Z_1 is read by bulk copies (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
    if (blockIdx.x == 0 && tid == 64 && track && cfg.S == 1) bound(1);

    // ---- products Z_{s+1} = Z_s F_{s+1}^T P_{s+1}, s = 1 .. n - 2
    if (n >= 3) {
      const int total = ustart_s[n - 1];
      const size_t b_tile = B_BYTES / EB, a_tile = A_BYTES / EB;  // elements per staged tile
      if (tid == 32) {
        // producer and scheduler: announces each tile, waits for its input
        // row tile, then streams its chunks through the stages
        int s = 1;
        for (int u = blockIdx.x;; u += gridDim.x) {
          Unit d{-1, 0, 0, 0};
          if (u < total && !*fail_v) {
            while (ustart_s[s + 1] <= u) ++s;
            const int n_nt = (2 * rup(M.dims[path_s[s + 1]], BK) + BN - 1) / BN;
            tile_coords(u - ustart_s[s], R, n_nt, P.order, d.mt, d.nt);
            d.s = s;
            const volatile int* ab = RS.abort;
            d.skip = *ab;
            if (!d.skip && s >= 2) {
              const volatile int* rdy = RS.ready + s * RT_MAX + d.mt;
              bool ok = true;
              if (*rdy == 0) {
                const uint64_t t0 = globaltimer();
                while (*rdy == 0 && *ab == 0) {
                  if (globaltimer() - t0 > P.timeout_ns) {
                    ok = false;
                    break;
                  }
                }
              }
              if (!ok) {
                *fail_v = 1;
                d.s = -1;
              } else if (*ab) {
                d.skip = 1;
              } else {
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");
              }
            }
          }
          const uint32_t us = ucount % DR;
          if (ucount >= DR && !mbar_wait(&S.unit_empty[us], ((ucount / DR) - 1u) & 1u, P.timeout_ns)) {
            *fail_v = 1;
            break;
          }
          S.unit[us] = d;
          mbar_arrive(&S.unit_full[us]);
          ++ucount;
          if (d.s < 0) break;
          if (d.skip) continue;
          const int qa = path_s[d.s], qb = path_s[d.s + 1];
          const int dpk = rup(M.dims[qa], BK), nkc = 2 * dpk / BKE;
          const int dpn = rup(M.dims[qb], BK);
          const T* Bt = reinterpret_cast<const T*>(P.bt) + P.bt_off[op_s[d.s] * ns + qa];
          const size_t b_plane = size_t(rup(2 * dpn, BN) / BN) * nkc * b_tile;
          const T* Ah = Zh[(d.s - 1) & 1];
          const T* Al = Zl[(d.s - 1) & 1];
          bool okp = true;
          for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t q = seq_base + uint32_t(kc);
            const int st = int(q % uint32_t(NST));
            if (*fail_v || (q >= uint32_t(NST) && !mbar_wait(&S.empty[st], ((q / NST) - 1u) & 1u, P.timeout_ns))) {
              okp = false;
              break;
            }
            unsigned char* sb = stage0 + size_t(st) * stage_bytes;
            const size_t ao = (size_t(d.mt) * nkz + kc) * a_tile, bo = (size_t(d.nt) * nkc + kc) * b_tile;
            mbar_arrive_expect_tx(&S.full[st], stage_bytes);
            bulk_g2s(sb, Ah + ao, A_BYTES, &S.full[st]);
            bulk_g2s(sb + A_BYTES, Bt + bo, B_BYTES, &S.full[st]);
            if (SPLIT) {
              bulk_g2s(sb + A_BYTES + B_BYTES, Al + ao, A_BYTES, &S.full[st]);
              bulk_g2s(sb + 2 * A_BYTES + B_BYTES, Bt + b_plane + bo, B_BYTES, &S.full[st]);
            }
            S.issued = q + 1;
          }
          seq_base += uint32_t(nkc);
          if (!okp) {
            *fail_v = 1;
            break;
          }
        }
      } else if (tid == 0) {
        // MMA issuer: only waits for data.  Chunks carry a per-CTA sequence
        // number q (stage q % NST, phase q / NST); groups of GRP chunks carry
        // g and accumulate in tensor-memory bank g % 2, which the drain warps
        // add into FP32 registers while the tensor core fills the other bank.
        for (;;) {
          const uint32_t us = ucount % DR;
          if (*fail_v || !mbar_wait(&S.unit_full[us], (ucount / DR) & 1u, P.timeout_ns)) {
            *fail_v = 1;
            break;
          }
          const Unit d = S.unit[us];
          mbar_arrive(&S.unit_empty[us]);
          ++ucount;
          if (d.s < 0) break;
          if (d.skip) continue;
          const int dpk = rup(M.dims[path_s[d.s]], BK), nkc = 2 * dpk / BKE;
          const int dpn = rup(M.dims[path_s[d.s + 1]], BK);
          const int ncols = min(BN, 2 * dpn - d.nt * BN);
          const int ngrp = (nkc + GRP - 1) / GRP;
          const uint32_t idesc = (PREC == CTQ_BF16X3) ? idesc_bf16(BM, ncols) : idesc_tf32(BM, ncols);
          bool ok = true;
          for (int kc = 0; kc < nkc; ++kc) {
            const uint32_t q = seq_base + uint32_t(kc);
            const uint32_t g = grp_base + uint32_t(kc / GRP);
            const int st = int(q % uint32_t(NST));
            const uint32_t bank = g & 1u;
            if (kc % GRP == 0 && g >= 2u &&
                (*fail_v || !mbar_wait(&S.bank_free[bank], ((g >> 1) - 1u) & 1u, P.timeout_ns))) {
              ok = false;
              break;
            }
            if (*fail_v || !mbar_wait(&S.full[st], (q / NST) & 1u, P.timeout_ns)) {
              ok = false;
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
          seq_base += uint32_t(nkc);
          grp_base += uint32_t(ngrp);
          if (!ok) {
            *fail_v = 1;
            break;
          }
        }
      } else if (warp >= 2) {
        // drain warps: lane quarter warp % 4, column slice (warp - 2) / 4 of
        // COLS columns; they also run the epilogue and publish finished row tiles
        constexpr int COLS = BN / (N_DRAIN / 4);
        const int slice = (warp - 2) >> 2;
        const uint32_t tl = uint32_t(32 * (warp & 3)) << 16;
        for (;;) {
          const uint32_t us = ucount % DR;
          if (!warp_wait(&S.unit_full[us], (ucount / DR) & 1u, P.timeout_ns, fail_v)) {
            *fail_v = 1;
            break;
          }
          const Unit d = S.unit[us];
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.unit_empty[us]);
          ++ucount;
          if (d.s < 0) break;
          if (d.skip) continue;
          const int qb = path_s[d.s + 1];
          const int dpk = rup(M.dims[path_s[d.s]], BK), nkc = 2 * dpk / BKE;
          const int db = M.dims[qb];
          const int dpn = rup(db, BK);
          const int ncols = min(BN, 2 * dpn - d.nt * BN);
          const int ngrp = (nkc + GRP - 1) / GRP;
          // column scale e^{-dt (E - E_min)} 2^{-e_r(s)}: lane l holds columns
          // l, l + 32, ... of this warp's slice
          const int ek_in = __ldcg(&RS.ekey[d.s * RT_MAX + d.mt]);
          const float scale = ek_in ? ldexpf(1.0f, -(ek_in - 127)) : 1.0f;
          float preg[COLS / 32];
          {
            const double dt = tau_s[d.s + 1] - tau_s[d.s];
            const double* Eb = M.E_rel + M.E_off[qb];
#pragma unroll
            for (int i = 0; i < COLS / 32; ++i) {
              const int col = d.nt * BN + slice * COLS + 32 * i + lane;
              const int j = (col < dpn) ? col : col - dpn;
              preg[i] = (j < db) ? expf(float(-dt * Eb[j])) * scale : 0.f;
            }
          }
          float acc[COLS];
#pragma unroll
          for (int cc = 0; cc < COLS; ++cc) acc[cc] = 0.f;
          bool okd = true;
          for (int gi = 0; gi < ngrp; ++gi) {
            const uint32_t g = grp_base + uint32_t(gi);
            const uint32_t bank = g & 1u;
            if (!warp_wait(&S.bank_full[bank], (g >> 1) & 1u, P.timeout_ns, fail_v)) {
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
                for (int cc = 0; cc < 16; ++cc) acc[h * 32 + u * 16 + cc] += __uint_as_float(v[u][cc]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.bank_free[bank]);
          }
          grp_base += uint32_t(ngrp);
          if (!okd) {
            *fail_v = 1;
            break;
          }
          // epilogue from registers: this thread's row, COLS columns of Z_{s+1}
          T* Oh = Zh[d.s & 1];
          T* Ol = Zl[d.s & 1];
          const int row = d.mt * BM + 32 * (warp & 3) + lane;
          int ek = 0;
          float f2 = 0.f;
#pragma unroll
          for (int c0 = 0; c0 < COLS; c0 += 16) {
            const int cb = slice * COLS + c0;  // column within the tile
            if (cb >= ncols) break;
            // 16 consecutive K elements of the next product, written as
            // 16-byte vectors of PER16 elements
            constexpr int PER16 = 16 / EB;
#pragma unroll
            for (int g = 0; g < 16 / PER16; ++g) {
              const size_t o = tiled_off<EB>(row, d.nt * BN + cb + PER16 * g, BM, nkz);
              if constexpr (PREC == CTQ_BF16X3) {  // pairs through one packed conversion
                float xs[PER16];
#pragma unroll
                for (int t2 = 0; t2 < PER16; ++t2) {
                  const int cc = c0 + PER16 * g + t2;
                  const float x = acc[cc] * __shfl_sync(0xffffffffu, preg[cc >> 5], cc & 31);
                  ek = max(ek, (__float_as_int(x) >> 23) & 0xff);
                  f2 += x * x;
                  xs[t2] = x;
                }
                uint32_t hv[4], lv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) split_bf16x2(xs[2 * u], xs[2 * u + 1], hv[u], lv[u]);
                *reinterpret_cast<uint4*>(Oh + o) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<uint4*>(Ol + o) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
              } else {
                T hi[PER16], lo[PER16];
#pragma unroll
                for (int t2 = 0; t2 < PER16; ++t2) {
                  const int cc = c0 + PER16 * g + t2;
                  const float x = acc[cc] * __shfl_sync(0xffffffffu, preg[cc >> 5], cc & 31);
                  ek = max(ek, (__float_as_int(x) >> 23) & 0xff);
                  f2 += x * x;
                  split_store<PREC>(x, hi[t2], lo[t2]);
                }
                *reinterpret_cast<uint4*>(Oh + o) = pack16<PREC>(hi);
                if (SPLIT) *reinterpret_cast<uint4*>(Ol + o) = pack16<PREC>(lo);
              }
            }
          }
          ek = __reduce_max_sync(0xffffffffu, ek);
          const double f2d = warp_sum(double(f2));
          // the stored tile is read by bulk copies (async proxy) of other CTAs next
          asm volatile("fence.proxy.async.global;" ::: "memory");
          __threadfence();
          __syncwarp();
          if (lane == 0) {
            // every drain warp of every column tile reports once; the report
            // that completes a row tile marks it ready, the one that completes
            // the stage takes the checkpoint bound
            atomicMax(&RS.ekey[(d.s + 1) * RT_MAX + d.mt], ek);
            atomicAdd(&RS.fr[(d.s + 1) * RT_MAX + d.mt], f2d);
            __threadfence();
            const int n_nt = (2 * dpn + BN - 1) / BN;
            if (atomicAdd(&RS.cnt[(d.s + 1) * RT_MAX + d.mt], 1) == n_nt * N_DRAIN - 1) {
              __threadfence();
              RS.ecum[d.s * RT_MAX + d.mt] = __ldcg(&RS.ecum[(d.s - 1) * RT_MAX + d.mt]) + (ek_in ? ek_in - 127 : 0);
              __threadfence();
              *((volatile int*)&RS.ready[(d.s + 1) * RT_MAX + d.mt]) = 1;
              if (atomicAdd(&RS.rows[d.s + 1], 1) == R - 1) {
                __threadfence();
                const int a = d.s + 1;
                if (track && a % cfg.S == 0 && a < n) bound(a);
              }
            }
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    if (S.fail) {
      if (tid == 32)  // let issued copies that were never consumed land before leaving
        for (uint32_t q = S.consumed; q < S.issued; ++q)
          mbar_wait(&S.full[q % uint32_t(NST)], (q / NST) & 1u, P.timeout_ns);
      alive = false;
    }
    if (!alive) break;
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }

    // ---- final operator: partial traces sum_{j in r, k} F_n[j][k] Z_{n-1}[j][k]
    const bool aborted = *((volatile int*)RS.abort) != 0;
    if (!aborted) {
      const int ql = path_s[n - 1];
      const int dl = M.dims[ql];
      const int dpk = rup(dl, BK);
      const int64_t off = M.blk_off[op_s[n - 1] * ns + ql];
      const T* Ah = Zh[(n - 2) & 1];
      const T* Al = Zl[(n - 2) & 1];
      int cur_r = -1;
      double vr = 0.0, vi = 0.0;
      auto flush = [&]() {
        const double wr = warp_sum(vr), wi = warp_sum(vi);
        if (lane == 0 && cur_r >= 0) {
          atomicAdd(&RS.part[2 * cur_r], wr);
          atomicAdd(&RS.part[2 * cur_r + 1], wi);
        }
        vr = 0.0;
        vi = 0.0;
      };
      const long long total = (long long)dp0 * dpk;
      for (long long e = gtid; e < total; e += gthreads) {
        const int j = int(e / dpk), k = int(e - (long long)j * dpk);
        const int r = j / BM;
        if (r != cur_r) {
          flush();
          cur_r = r;
        }
        if (j < d0 && k < dl) {
          const size_t o_r = tiled_off<EB>(j, k, BM, nkz), o_i = tiled_off<EB>(j, dpk + k, BM, nkz);
          float zr = elt_val<PREC>(Ah[o_r]), zi = elt_val<PREC>(Ah[o_i]);
          if (SPLIT) {
            zr += elt_val<PREC>(Al[o_r]);
            zi += elt_val<PREC>(Al[o_i]);
          }
          const int64_t fe = off + int64_t(j) * dl + k;
          const float fr_ = float(cplx ? M.blk[2 * fe] : M.blk[fe]);
          const float fi_ = cplx ? float(M.blk[2 * fe + 1]) : 0.f;
          vr += double(fr_ * zr - fi_ * zi);
          vi += double(fr_ * zi + fi_ * zr);
        }
      }
      flush();
    }
    {  // the next string's state (its previous user finished before this string began)
      int* z = reinterpret_cast<int*>(next_state);
      for (long long i = gtid; i < (long long)(sbytes / 4); i += gthreads) z[i] = 0;
    }
    if (!grid_sync(P.bar, P.bar + 1, P.timeout_ns)) { alive = false; break; }
    if (blockIdx.x == 0 && tid == 0) {
      if (aborted) {
        W.res_log[slot] = NAN;
      } else {
        // row tile r of Z_{n-1} carries 2^{-ecum[n-2][r]}
        int emx = INT_MIN;
        for (int r = 0; r < R; ++r)
          if (__ldcg(&RS.part[2 * r]) != 0.0 || __ldcg(&RS.part[2 * r + 1]) != 0.0)
            emx = max(emx, __ldcg(&RS.ecum[(n - 2) * RT_MAX + r]));
        double sr = 0.0, si = 0.0;
        if (emx != INT_MIN)
          for (int r = 0; r < R; ++r) {
            const int sh = __ldcg(&RS.ecum[(n - 2) * RT_MAX + r]) - emx;
            sr += ldexp(__ldcg(&RS.part[2 * r]), sh);
            si += ldexp(__ldcg(&RS.part[2 * r + 1]), sh);
          }
        const bool zero_v = (sr == 0.0 && si == 0.0);
        const double lg = L_s[n - 1] + double(emx) * LN2;
        W.res_val[2 * slot] = sr;
        W.res_val[2 * slot + 1] = si;
        W.res_log[slot] = zero_v ? -INFINITY : lg;
        if (track) segp[it.n_seg] = zero_v ? -INFINITY : log(sqrt(sr * sr + si * si)) + lg;
      }
    }
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
  (void)grid;
  int dmax = h.max_dim;
  const size_t zf = size_t((dmax + BM - 1) / BM * BM) * size_t(2 * ((dmax + BK - 1) / BK * BK));
  return 4 * zf * 4 + 256 + 2 * row_state_bytes(max_ops) + 1024;
}

static int big_stages(int prec) { return prec == CTQ_TF32 ? 4 : 2; }

static size_t big_smem(int prec, int nst, int max_ops) {
  const size_t stages = size_t(nst) * (prec == CTQ_TF32 ? 1 : 2) * (A_BYTES + B_BYTES);
  return std::max(stages, size_t(PVEC) * 4) + big_table_bytes(max_ops);  // the stages also hold p_s
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
  lc->smem = big_smem(prec, big_stages(prec), 256);
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
    if (events) record_timing_event(events[i], st);
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
  s = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(s) + 255) & ~uintptr_t(255));
  P.state = reinterpret_cast<unsigned char*>(s);
  P.nst = cfg.stages > 0 ? cfg.stages : big_stages(P.prec);
  P.order = cfg.tile_order == 0 ? 1 : cfg.tile_order - 1;  // tile_coords codes; row-major by default
  const size_t smem = big_smem(P.prec, P.nst, cfg.max_ops);
  if (P.nst < 2 || P.nst > MAX_NST || smem > size_t(lc.smem_optin)) return CTQ_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(W.counters, 0, COUNTER_BYTES, st) != cudaSuccess) return CTQ_ERR_CUDA;
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
