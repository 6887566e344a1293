// Incremental local trace with a skip list of cached segment products
// (Sec. 3.3.1, skip-list paragraph: products of operator sub-sequences are
// kept, so that a local change of the configuration recomputes O(log k)
// products instead of all k).
//
// One ctq_skiplist holds one configuration (a time-ordered operator
// sequence).  For every starting sector q0 whose string survives, the trace
//     w_q0 = Tr P_{beta - tau_n + tau_1}(q0) F_n P ... P F_2 P_{tau_2 - tau_1} F_1
// is the trace of the wrap-around propagator times the ordered product of
// "leaves" X_i = P_{tau_{i+1} - tau_i}(q_i) F_{alpha_i}(q_{i-1}) (the last leaf
// is F_n alone).  Each operator gets a random height h >= 1 (geometric, 1/2)
// when it is inserted.  Level 0 holds the leaves; the segments of level l
// start at the first operator and at every operator with h > l, and a
// segment's product is the product of the level-(l-1) segments it covers,
// the latest on the left.  The top level is a single segment: the whole
// product.  Every product is cached under a key made from the keys of its
// factors (a leaf's key: operator identity, input sector and time step), so
// after a move only the segments that contain a changed leaf get a new key
// and are recomputed: about one product per level for a local insertion or
// removal, plus the ancestors of the leaves whose sector the move shifted.
//
// Arithmetic: float64 on the SIMT pipe (complex blocks as [Re | Im] rows),
// or, with CTQ_BF16X3, the products on the tensor cores (below; leaves,
// exponents and root traces stay float64).  A stored product is raw: its true value is the stored matrix times
// 2^{E} (E kept on the device beside the matrix's max |entry|), and every
// consumer scales its factors by the exact power of two that brings their
// max |entry| into [1, 2) as it loads them, so the products are the
// renormalised products of the other trace kernels, value for value.  The
// log of the propagators' E_min factors is kept on the host.
//
// Launches: an evaluation first plans every product it needs on the host
// (the cache decides what is new), orders the new products in rounds (a
// product's round is one more than its factors'), and then launches one
// grouped kernel per round over all strings and segments (two on the
// tensor cores: the factors' formatting and the products; CTAs find their
// product by a binary search on tile offsets), after one kernel for the
// new leaves and one clearing the new products' max words; one kernel takes
// every string's root trace.  The task tables go to the device in one copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <unordered_map>
#include <vector>

#include "ctq_internal.h"
#include "tc_ptx.cuh"

namespace ctq {
namespace {

using namespace ptx;

constexpr int SL_MAX_LEVEL = 24;
constexpr int GK = 16;            // K chunk of the product tiles
constexpr int LEAF_CHUNK = 1024;  // elements of a leaf per CTA (256 threads)
constexpr long long EXP_DEAD = LLONG_MIN / 4;

// A leaf X = P_dt(q_out) F (raw, exponent 0).
struct SlLeaf {
  const double* E_out;
  double* out;
  unsigned long long* w;
  int64_t off;
  double dt;
  int d_out, d_in, cplx, tile0;
};
// A product C = (R 2^-r)(L 2^-l), r and l the exponents of max|R|, max|L|.
struct SlProd {
  const double* R;
  const double* L;
  double* C;
  const unsigned long long* wR;
  const unsigned long long* wL;
  unsigned long long* wC;
  int M, K, N, cplx, tile0, tiles_x;
};
// A root: Tr P_t(q0) X, written with X's exponent to out[0..2].
struct SlRoot {
  const double* X;
  const unsigned long long* w;
  const double* E0;
  double* out;
  double t;
  int d, cplx;
};

// Index of the task whose tile range holds CTA b (tile0 ascending, first 0).
template <typename T>
__device__ __forceinline__ int find_task(const T* t, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t[mid].tile0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void atomic_max_abs(unsigned long long* w, double v) {
  // |v| >= 0: the bit patterns of non-negative doubles order like the values
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(w, (unsigned long long)__double_as_longlong(v));
}

// 2^-e for the max word m (0 for an all-zero matrix) and e itself.
__device__ __forceinline__ double norm_of(const unsigned long long* w, int* e) {
  const double m = __longlong_as_double((long long)w[0]);
  if (!(m > 0.0)) {
    *e = 0;
    return 0.0;
  }
  *e = ilogb(m);
  return ldexp(1.0, -*e);
}

__global__ void k_sl_zero(unsigned long long* const* w, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    w[i][0] = 0ull;
    w[i][1] = 0ull;
  }
}

// Leaves: out[m][j] = e^{-dt E_rel(q_out)_m} F[m][j]; complex rows are
// stored [Re(0..d_in) | Im(0..d_in)].
__global__ void k_sl_leaves(const double* blk, const SlLeaf* tasks, int n) {
  __shared__ double p_s[LEAF_CHUNK];  // the propagator of the chunk's rows, one exponential per row
  const SlLeaf T = tasks[find_task(tasks, n, blockIdx.x)];
  const long long total = (long long)T.d_out * T.d_in;
  const long long e0 = (long long)(blockIdx.x - T.tile0) * LEAF_CHUNK;
  const long long e1 = e0 + LEAF_CHUNK < total ? e0 + LEAF_CHUNK : total;
  const int m0 = int(e0 / T.d_in), nrow = int((e1 - 1) / T.d_in) - m0 + 1;  // nrow <= LEAF_CHUNK
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) p_s[i] = T.dt > 0.0 ? exp(-T.dt * T.E_out[m0 + i]) : 1.0;
  __syncthreads();
  double mx = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int m = int(e / T.d_in), j = int(e - (long long)m * T.d_in);
    const double p = p_s[m - m0];
    if (T.cplx) {
      const double re = blk[2 * (T.off + e)] * p, im = blk[2 * (T.off + e) + 1] * p;
      T.out[size_t(m) * 2 * T.d_in + j] = re;
      T.out[size_t(m) * 2 * T.d_in + T.d_in + j] = im;
      mx = fmax(mx, fmax(fabs(re), fabs(im)));
    } else {
      const double v = blk[T.off + e] * p;
      T.out[e] = v;
      mx = fmax(mx, fabs(v));
    }
  }
  atomic_max_abs(T.w, mx);
}

// Products, TILE x TILE outputs per CTA, RR x RR per thread.  Real: R (M x K),
// L (K x N), C (M x N), row-major.  Complex ([Re | Im] rows): the real GEMM
// of [Rr | Ri] (M x 2K) with [[Lr, Li], [-Li, Lr]] (2K x 2N) gives
// [Cr | Ci] (M x 2N).
template <int TILE, int RR>
__global__ void __launch_bounds__((TILE / RR) * (TILE / RR)) k_sl_gemm(const SlProd* tasks, int n) {
  constexpr int NT = (TILE / RR) * (TILE / RR), TPR = TILE / RR;
  __shared__ double As[GK][TILE + 1];
  __shared__ double Bs[GK][TILE + 1];
  const SlProd P = tasks[find_task(tasks, n, blockIdx.x)];
  const int local = blockIdx.x - P.tile0;
  const int row0 = (local / P.tiles_x) * TILE, col0 = (local % P.tiles_x) * TILE;
  int er, el;
  const double sR = norm_of(P.wR, &er), sL = norm_of(P.wL, &el);
  if (local == 0 && threadIdx.x == 0) {
    const long long eR = reinterpret_cast<const long long*>(P.wR)[1], eL = reinterpret_cast<const long long*>(P.wL)[1];
    reinterpret_cast<long long*>(P.wC)[1] = (sR > 0.0 && sL > 0.0) ? eR + er + eL + el : EXP_DEAD;
  }
  const int M = P.M, K = P.K, N = P.N;
  const int Kp = P.cplx ? 2 * K : K, Np = P.cplx ? 2 * N : N;
  const int tx = threadIdx.x % TPR, ty = threadIdx.x / TPR;
  double acc[RR][RR] = {};
  for (int k0 = 0; k0 < Kp; k0 += GK) {
    for (int e = threadIdx.x; e < TILE * GK; e += NT) {
      const int r = e / GK, k = e - r * GK;  // A: row r, column k0 + k
      const int gr = row0 + r, gk = k0 + k;
      As[k][r] = (gr < M && gk < Kp) ? P.R[size_t(gr) * Kp + gk] * sR : 0.0;
      const int kb = e / TILE, c = e - kb * TILE;  // B: row k0 + kb, column c
      const int bk = k0 + kb, bc = col0 + c;
      double v = 0.0;
      if (bk < Kp && bc < Np) {
        if (!P.cplx || bk < K) {
          v = P.L[size_t(bk) * Np + bc];
        } else {
          const int kk = bk - K;
          v = (bc < N) ? -P.L[size_t(kk) * Np + N + bc] : P.L[size_t(kk) * Np + (bc - N)];
        }
      }
      Bs[kb][c] = v * sL;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      double a[RR], b[RR];
#pragma unroll
      for (int i = 0; i < RR; ++i) a[i] = As[k][ty * RR + i];
#pragma unroll
      for (int j = 0; j < RR; ++j) b[j] = Bs[k][tx * RR + j];
#pragma unroll
      for (int i = 0; i < RR; ++i)
#pragma unroll
        for (int j = 0; j < RR; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < RR; ++i) {
    const int r = row0 + ty * RR + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < RR; ++j) {
      const int c = col0 + tx * RR + j;
      if (c < Np) {
        P.C[size_t(r) * Np + c] = acc[i][j];
        mx = fmax(mx, fabs(acc[i][j]));
      }
    }
  }
  atomic_max_abs(P.wC, mx);
}

// Roots, one CTA each: out = (Re, Im) of sum_j e^{-t E_rel(q0)_j} X[j][j]
// and X's exponent bits (EXP_DEAD for a zero product).
__global__ void k_sl_roots(const SlRoot* tasks) {
  const SlRoot T = tasks[blockIdx.x];
  __shared__ double sr[32], si[32];
  double re = 0.0, im = 0.0;
  for (int j = threadIdx.x; j < T.d; j += blockDim.x) {
    const double p = exp(-T.t * T.E0[j]);
    if (T.cplx) {
      re += p * T.X[size_t(j) * 2 * T.d + j];
      im += p * T.X[size_t(j) * 2 * T.d + T.d + j];
    } else {
      re += p * T.X[size_t(j) * T.d + j];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sr[w] = re;
    si[w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      a += sr[i];
      b += si[i];
    }
    const bool dead = !(__longlong_as_double((long long)T.w[0]) > 0.0);
    const long long e = dead ? EXP_DEAD : reinterpret_cast<const long long*>(T.w)[1];
    T.out[0] = dead ? 0.0 : a;
    T.out[1] = dead ? 0.0 : b;
    T.out[2] = __longlong_as_double(e);
  }
}

// ------------------------------------------------ tensor-core products
// CTQ_BF16X3 products: each factor is scaled by its power of two, split
// into bf16 hi / lo planes and laid out as K-major tiles of 8 x 16-byte core
// matrices (k_sl_fmt); then C = A B^T runs on 128 x 256 tiles (k_sl_tc):
// A = the left factor R as stored (M x K', complex rows [Re | Im]), B = the
// rows of the real embedding of the right factor transposed (N' x K'),
// chunks of 32 K elements staged by bulk copies through four 48 KB stages,
// three MMAs per 16 K (hi hi + hi lo + lo hi) into two alternating FP32
// accumulators of 256 tensor-memory columns; every 8 chunks (256 K terms)
// sixteen drain warps fold the full one into FP32 registers while the tensor
// core fills the other (the tensor core's own accumulation never spans more
// than 256 terms), and write the float64 product with its max at the end.
constexpr int TBM = 128, TBN = 256, TKE = 32;                      // tile rows, columns, K per chunk
constexpr uint32_t TA_BYTES = TBM * TKE * 2, TB_BYTES = TBN * TKE * 2;  // one bf16 plane of a staged chunk
constexpr uint32_t TSTAGE = 2 * (TA_BYTES + TB_BYTES);             // hi and lo planes of A and B
constexpr int NSTG = 4;                                            // stages in flight (192 KB)
constexpr int SL_GW = 8;                                           // column tiles per scheduling group
constexpr int SL_DRAIN = 16;                                       // drain warps (four per tensor-memory lane quarter)
constexpr int TC_SL_THREADS = 32 * (1 + SL_DRAIN);                 // warp 0: copies and MMAs
constexpr int SL_GRP = 8;                                          // chunks (256 K terms) per accumulator group
constexpr int FMT_CHUNK = 2048;                                    // operand elements per format CTA
constexpr uint64_t SL_TC_TIMEOUT_NS = 20000000000ull;              // bound of every wait (20 s)

// Element (r, k) of an operand stored as tiles of rpt rows x TKE K elements:
// tile (r / rpt, k / TKE) at ((r / rpt) nkc + k / TKE) rpt TKE, core matrix
// (k % TKE / 8, r % rpt / 8) at (k % TKE / 8 * rpt / 8 + r % rpt / 8) 64,
// element (r % 8) 8 + k % 8.
__device__ __forceinline__ size_t tc_off(int r, int k, int rpt, int nkc) {
  const int rt = r / rpt, rr = r - rt * rpt, kc = k / TKE, kk = k % TKE;
  return (size_t(rt) * nkc + kc) * size_t(rpt) * TKE + size_t((kk >> 3) * (rpt >> 3) + (rr >> 3)) * 64 +
         (rr & 7) * 8 + (kk & 7);
}

// One operand to format.  mode 0: A = the stored rows of R (rows x kp);
// mode 1: B[n][k] = L_emb[k][n], L_emb the real embedding of L (K x N
// complex: [[Lr, Li], [-Li, Lr]], stored rows [Lr | Li]).
struct SlFmt {
  const double* src;
  const unsigned long long* w;
  uint16_t* hi;
  uint16_t* lo;
  int rows, kp, rows_pad, kp_pad, mode, K, N, cplx, rpt, tile0;
};
// One product on the tensor cores: tiled operands, output and records.
struct SlTc {
  const uint16_t* Ah;
  const uint16_t* Al;
  const uint16_t* Bh;
  const uint16_t* Bl;
  double* C;
  const unsigned long long* wR;
  const unsigned long long* wL;
  unsigned long long* wC;
  int M, Np, nkc, tiles_n, tiles_m, tile0;
};

// One thread per 8 consecutive K elements of one operand row (a 16-byte
// core-matrix row of each plane, stored as one vector); consecutive threads
// take consecutive operand rows, so a warp writes 512 contiguous bytes per
// plane (A rows are read as 64-byte segments, L row by row with consecutive
// threads on consecutive columns).
__global__ void k_sl_fmt(const SlFmt* tasks, int n) {
  const SlFmt T = tasks[find_task(tasks, n, blockIdx.x)];
  int e_unused;
  const double sc = norm_of(T.w, &e_unused);
  const int kg_n = T.kp_pad / 8;
  const long long total = (long long)T.rows_pad * kg_n;  // groups of 8 elements
  const long long g0 = (long long)(blockIdx.x - T.tile0) * (FMT_CHUNK / 8);
  const long long g1 = g0 + FMT_CHUNK / 8 < total ? g0 + FMT_CHUNK / 8 : total;
  const int nkc = T.kp_pad / TKE;
  const int Np = T.cplx ? 2 * T.N : T.N;
  for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const int kg = int(g / T.rows_pad);
    const int r = int(g - (long long)kg * T.rows_pad), k0 = 8 * kg;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      float x[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = k0 + t + u;
        double v = 0.0;
        if (r < T.rows && k < T.kp) {
          if (T.mode == 0) {
            v = T.src[size_t(r) * T.kp + k];
          } else if (!T.cplx || k < T.K) {
            v = T.src[size_t(k) * Np + r];
          } else {
            const int kk = k - T.K;
            v = (r < T.N) ? -T.src[size_t(kk) * Np + T.N + r] : T.src[size_t(kk) * Np + (r - T.N)];
          }
        }
        x[u] = float(v * sc);
      }
      const uint32_t h0 = bf16_bits(x[0]), h1 = bf16_bits(x[1]);
      hw[t / 2] = h0 | (h1 << 16);
      lw[t / 2] = bf16_bits(x[0] - bf16_val(h0)) | (bf16_bits(x[1] - bf16_val(h1)) << 16);
    }
    const size_t o = tc_off(r, k0, T.rpt, nkc);  // 8 consecutive elements, 16-byte aligned
    *reinterpret_cast<uint4*>(T.hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(T.lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

__global__ void __launch_bounds__(TC_SL_THREADS, 1)
    k_sl_tc(const SlTc* tasks, int n, uint64_t timeout_ns, int* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[NSTG], empty[NSTG], bank_full[2], bank_free[2];
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  const SlTc T = tasks[find_task(tasks, n, blockIdx.x)];
  const int local = blockIdx.x - T.tile0;
  // tiles in groups of SL_GW column tiles, row tiles fastest within a group:
  // the CTAs resident together share a few block columns and row panels in L2
  const int grp = local / (SL_GW * T.tiles_m), n0 = grp * SL_GW;
  const int gw = min(SL_GW, T.tiles_n - n0), in = local - grp * SL_GW * T.tiles_m;
  const int mt = in / gw, nt = n0 + (in - mt * gw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < NSTG; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bank_full[b], 1);
      mbar_init(&bank_free[b], SL_DRAIN);  // one arrival per drain warp
    }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, 2 * TBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tD = tmem_base;
  volatile int* fail_v = &fail;
  int er, el;
  const double sR = norm_of(T.wR, &er), sL = norm_of(T.wL, &el);
  if (local == 0 && tid == 0) {
    const long long eR = reinterpret_cast<const long long*>(T.wR)[1], eL = reinterpret_cast<const long long*>(T.wL)[1];
    reinterpret_cast<long long*>(T.wC)[1] = (sR > 0.0 && sL > 0.0) ? eR + er + eL + el : EXP_DEAD;
  }
  const int nkc = T.nkc, ngrp = (nkc + SL_GRP - 1) / SL_GRP;
  if (tid == 0) {
    // copies and MMAs: chunks through the stages; group g of SL_GRP chunks
    // accumulates in bank g % 2, which the drain warps fold into registers
    // while the tensor core fills the other bank
    const size_t a_tile = size_t(TBM) * TKE, b_tile = size_t(TBN) * TKE;  // elements of one chunk
    auto issue = [&](int kc) {
      const int st = kc % NSTG;
      unsigned char* base = sm + st * TSTAGE;
      const size_t ao = (size_t(mt) * nkc + kc) * a_tile, bo = (size_t(nt) * nkc + kc) * b_tile;
      mbar_arrive_expect_tx(&full[st], TSTAGE);
      bulk_g2s(base, T.Ah + ao, TA_BYTES, &full[st]);
      bulk_g2s(base + TA_BYTES, T.Bh + bo, TB_BYTES, &full[st]);
      bulk_g2s(base + TA_BYTES + TB_BYTES, T.Al + ao, TA_BYTES, &full[st]);
      bulk_g2s(base + 2 * TA_BYTES + TB_BYTES, T.Bl + bo, TB_BYTES, &full[st]);
    };
    constexpr uint32_t LBO_A = (TBM / 8) * 128, LBO_B = (TBN / 8) * 128;
    const uint32_t idesc = idesc_bf16(TBM, TBN);
    int issued = 0, kc = 0;
    for (; issued < nkc && issued < NSTG; ++issued) issue(issued);
    bool ok = true;
    for (; kc < nkc; ++kc) {
      const int st = kc % NSTG, g = kc / SL_GRP;
      const uint32_t bank = uint32_t(g & 1);
      if (kc % SL_GRP == 0 && g >= 2 && !mbar_wait(&bank_free[bank], uint32_t(((g >> 1) - 1) & 1), timeout_ns)) {
        ok = false;
        break;
      }
      if (!mbar_wait(&full[st], uint32_t((kc / NSTG) & 1), timeout_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(sm + st * TSTAGE), sbh = sa + TA_BYTES, sal = sbh + TB_BYTES, sbl = sal + TA_BYTES;
      const uint32_t tacc = tD + bank * uint32_t(TBN);
      for (int kk = 0; kk < TKE / 16; ++kk) {  // 16 K elements (32 bytes) per MMA
        const uint64_t dah = sdesc(sa + kk * 2 * LBO_A, LBO_A, 128), dbh = sdesc(sbh + kk * 2 * LBO_B, LBO_B, 128);
        mma_bf16_ss(tacc, dah, dbh, idesc, (kc % SL_GRP != 0 || kk > 0) ? 1u : 0u);
        mma_bf16_ss(tacc, dah, sdesc(sbl + kk * 2 * LBO_B, LBO_B, 128), idesc, 1u);
        mma_bf16_ss(tacc, sdesc(sal + kk * 2 * LBO_A, LBO_A, 128), dbh, idesc, 1u);
      }
      mma_commit(&empty[st]);
      if (kc % SL_GRP == SL_GRP - 1 || kc == nkc - 1) mma_commit(&bank_full[bank]);
      if (kc >= 1 && kc + NSTG - 1 < nkc) {  // chunk kc - 1's stage takes chunk kc + NSTG - 1 once its MMAs are done
        if (!mbar_wait(&empty[(kc - 1) % NSTG], uint32_t(((kc - 1) / NSTG) & 1), timeout_ns)) {
          ok = false;
          break;
        }
        issue(kc + NSTG - 1);
        issued = kc + NSTG;
      }
    }
    if (!ok) {
      *fail_v = 1;
      atomicExch(status, CTQ_ERR_TIMEOUT);
      // copies still in flight land in this CTA's shared memory: wait for them (bounded)
      for (int j = kc; j < issued; ++j) mbar_wait(&full[j % NSTG], uint32_t((j / NSTG) & 1), timeout_ns);
    }
  } else if (warp >= 1) {
    // drain warps: lane quarter warp % 4, column slice (warp - 1) / 4 of
    // COLS columns; every group of the accumulator is added into FP32
    // registers (round to nearest)
    constexpr int COLS = TBN / (SL_DRAIN / 4);
    const int half = (warp - 1) >> 2;
    const uint32_t tl = uint32_t(32 * (warp & 3)) << 16;
    float acc[COLS];
#pragma unroll
    for (int c = 0; c < COLS; ++c) acc[c] = 0.f;
    bool okd = true;
    for (int g = 0; g < ngrp; ++g) {
      const uint32_t bank = uint32_t(g & 1);
      const bool ok = !*fail_v && mbar_wait(&bank_full[bank], uint32_t((g >> 1) & 1), timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        okd = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < COLS / 16; ++h) {  // 16 columns per tensor-memory wait
        uint32_t v[16];
        tmem_ld16(tD + bank * uint32_t(TBN) + tl + uint32_t(half * COLS + h * 16), v);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[h * 16 + c] += __uint_as_float(v[c]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bank_free[bank]);
    }
    if (!okd) {
      if (lane == 0) atomicExch(status, CTQ_ERR_TIMEOUT);
      *fail_v = 1;
    } else {
      const int r = mt * TBM + 32 * (warp & 3) + lane;  // this thread's accumulator row
      double mx = 0.0;
      if (r < T.M) {
#pragma unroll
        for (int c = 0; c < COLS; ++c) {
          const int col = nt * TBN + half * COLS + c;
          if (col < T.Np) {
            const double x = double(acc[c]);
            T.C[size_t(r) * T.Np + col] = x;
            mx = fmax(mx, fabs(x));
          }
        }
      }
      atomic_max_abs(T.wC, mx);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tD, 2 * TBN);
  }
}

// ---------------------------------------------------------------- host

uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// 128-bit cache key of a leaf or a segment product (two independent
// 64-bit hashes; a collision needs both to agree).
struct Key {
  uint64_t a, b;
  bool operator==(const Key& o) const { return a == o.a && b == o.b; }
};
struct KeyHash {
  size_t operator()(const Key& k) const { return size_t(k.a ^ (k.b * 0x9e3779b97f4a7c15ull)); }
};

// A cached product: device matrix (rows x cols doubles, complex rows as
// [Re | Im]), its max word and exponent on the device, its log scale on the host.
struct Buf {
  double* p = nullptr;
  size_t elems = 0;
  unsigned long long* maxw = nullptr;  // [0] max|X| bits; [1] exponent (long long)
  int d_out = 0, d_in = 0;
  double L = 0.0;
  uint64_t epoch = 0;  // the evaluation that planned it
  int round = 0;       // its launch round in that evaluation (leaves 0)
  uint64_t used = 0;   // the last evaluation whose configuration needed it
};

class Pool {
 public:
  ~Pool() { release(); }
  double* get(size_t elems) {
    const size_t b = bucket(elems);
    auto it = free_.find(b);
    if (it != free_.end() && !it->second.empty()) {
      double* p = it->second.back();
      it->second.pop_back();
      return p;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, b * sizeof(double)) != cudaSuccess) return nullptr;
    bytes_ += b * sizeof(double);
    return static_cast<double*>(p);
  }
  void put(double* p, size_t elems) { free_[bucket(elems)].push_back(p); }
  unsigned long long* word() {
    if (words_.empty()) {
      void* p = nullptr;
      if (cudaMalloc(&p, 4096 * 16) != cudaSuccess) return nullptr;
      blocks_.push_back(p);
      for (int i = 0; i < 4096; ++i) words_.push_back(static_cast<unsigned long long*>(p) + 2 * i);
    }
    unsigned long long* w = words_.back();
    words_.pop_back();
    return w;
  }
  void put_word(unsigned long long* w) { words_.push_back(w); }
  size_t bytes() const { return bytes_; }
  void release() {
    for (auto& kv : free_)
      for (double* p : kv.second) cudaFree(p);
    free_.clear();
    for (void* p : blocks_) cudaFree(p);
    blocks_.clear();
    words_.clear();
    bytes_ = 0;
  }

 private:
  static size_t bucket(size_t elems) {  // size classes 2^k and 1.5 x 2^k, at least 256
    size_t b = 256;
    while (b < elems) b *= 2;
    const size_t c = b / 4 * 3;
    return (c >= elems && c >= 256) ? c : b;
  }
  std::map<size_t, std::vector<double*>> free_;
  std::vector<unsigned long long*> words_;
  std::vector<void*> blocks_;
  size_t bytes_ = 0;
};

struct Op {
  uint64_t id;
  double t;
  int alpha;
  int h;
};

}  // namespace
}  // namespace ctq

struct ctq_skiplist {
  const ctq_impurity* imp = nullptr;
  const ctq::HostModel* H = nullptr;
  const ctq::DevModel* D = nullptr;
  int device = 0;
  cudaStream_t st = nullptr;
  double beta = 0.0;
  uint64_t rng = 0, next_id = 1;
  std::vector<ctq::Op> ops;
  ctq::Pool pool;
  std::unordered_map<ctq::Key, std::shared_ptr<ctq::Buf>, ctq::KeyHash> cache;
  double* d_res = nullptr;  // [3 n_sec]: trace re, im, exponent bits per q0
  ctq_skiplist_stats stats{};
  uint64_t epoch = 0;
  int num_sms = 1;
  unsigned char* h_tab = nullptr;  // task tables: pinned host staging and device copy
  unsigned char* d_tab = nullptr;
  size_t tab_cap = 0;
  int prec = CTQ_FP64;             // products: CTQ_FP64 (SIMT) or CTQ_BF16X3 (tensor cores)
  unsigned char* d_fmt = nullptr;  // tiled bf16 operands of one round (CTQ_BF16X3)
  size_t fmt_cap = 0;
  int* d_status = nullptr;         // CTQ_ERR_TIMEOUT from a tensor-core product
};

namespace ctq {
namespace {

int sl_height(ctq_skiplist* S) {
  int h = 1;
  S->rng = mix64(S->rng);
  uint64_t r = S->rng;
  while ((r & 1u) && h < SL_MAX_LEVEL - 1) {
    ++h;
    r >>= 1;
  }
  return h;
}

// The work one evaluation launches, planned on the host.
struct Plan {
  std::vector<unsigned long long*> zero;        // max / exponent words of the new leaves and products
  std::vector<SlLeaf> leaves;
  std::vector<std::vector<SlProd>> rounds;      // rounds[r - 1]: products of round r
  std::vector<SlRoot> roots;
  std::vector<std::shared_ptr<Buf>> keep;       // new buffers, alive until their kernels are enqueued
};

std::shared_ptr<Buf> new_buf(ctq_skiplist* S, Plan& P, int d_out, int d_in, int round) {
  auto b = std::shared_ptr<Buf>(new Buf(), [S](Buf* x) {
    if (x->p) S->pool.put(x->p, x->elems);
    if (x->maxw) S->pool.put_word(x->maxw);
    delete x;
  });
  b->d_out = d_out;
  b->d_in = d_in;
  b->elems = size_t(d_out) * d_in * (S->H->is_complex ? 2 : 1);
  b->p = S->pool.get(b->elems);
  b->maxw = S->pool.word();
  if (!b->p || !b->maxw) return nullptr;
  b->epoch = S->epoch;
  b->round = round;
  P.zero.push_back(b->maxw);
  P.keep.push_back(b);
  return b;
}

int round_of(const ctq_skiplist* S, const Buf& b) { return b.epoch == S->epoch ? b.round : 0; }

std::shared_ptr<Buf> make_leaf(ctq_skiplist* S, Plan& P, int alpha, int q_in, int q_out, double dt, int* st) {
  const HostModel& H = *S->H;
  const int ns = H.n_sec, d_in = H.dims[q_in], d_out = H.dims[q_out];
  auto b = new_buf(S, P, d_out, d_in, 0);
  if (!b) { *st = CTQ_ERR_NOMEM; return nullptr; }
  SlLeaf t{};
  t.E_out = S->D->E_rel + H.E_off[q_out];
  t.out = b->p;
  t.w = b->maxw;
  t.off = H.blk_off[size_t(alpha) * ns + q_in];
  t.dt = dt;
  t.d_out = d_out;
  t.d_in = d_in;
  t.cplx = H.is_complex;
  P.leaves.push_back(t);
  b->L = dt > 0.0 ? -dt * (H.E_min[q_out] - H.E_gs) : 0.0;
  S->stats.leaves += 1;
  return b;
}

// C = R L (R applied after L), in the round after its factors'.
std::shared_ptr<Buf> product(ctq_skiplist* S, Plan& P, const std::shared_ptr<Buf>& R, const std::shared_ptr<Buf>& L,
                             int* st) {
  const int round = std::max(round_of(S, *R), round_of(S, *L)) + 1;
  auto b = new_buf(S, P, R->d_out, L->d_in, round);
  if (!b) { *st = CTQ_ERR_NOMEM; return nullptr; }
  const int cplx = S->H->is_complex;
  SlProd t{};
  t.R = R->p;
  t.L = L->p;
  t.C = b->p;
  t.wR = R->maxw;
  t.wL = L->maxw;
  t.wC = b->maxw;
  t.M = R->d_out;
  t.K = R->d_in;
  t.N = L->d_in;
  t.cplx = cplx;
  if (int(P.rounds.size()) < round) P.rounds.resize(round);
  P.rounds[round - 1].push_back(t);
  b->L = R->L + L->L;
  S->stats.products += 1;
  S->stats.flops += 2.0 * R->d_out * double(R->d_in) * L->d_in * (cplx ? 4.0 : 1.0);
  return b;
}

Key leaf_key(const Op& o, int q_in, double dt) {
  uint64_t t;
  std::memcpy(&t, &dt, 8);
  return Key{mix64(o.id * 0x100000001b3ull + uint64_t(q_in)), mix64(t ^ mix64(o.id ^ 0x5bd1e995ull)) | 1ull};
}

// A segment's key depends only on its factors' keys (the same factors give
// the same product at any level); leaf keys have the low bit of b set,
// segment keys clear.
Key seg_key(const Key* kids, int n) {
  uint64_t h1 = 0x243f6a8885a308d3ull, h2 = 0x13198a2e03707344ull ^ uint64_t(n);
  for (int i = 0; i < n; ++i) {
    h1 = mix64(h1 ^ kids[i].a) + kids[i].b;
    h2 = mix64(h2 + kids[i].b) ^ (kids[i].a * 0xff51afd7ed558ccdull);
  }
  return Key{mix64(h1), mix64(h2) & ~1ull};
}

// Plans (or finds in the cache) every segment product of the string that
// starts in sector q0 and its root trace into d_res[3 q0 ..].  Returns the
// root's log scale in *L_root.
int plan_string(ctq_skiplist* S, Plan& P, int q0, const std::vector<int>& path, double* L_root) {
  const int n = int(S->ops.size());
  std::vector<Key> keys(n);
  std::vector<std::shared_ptr<Buf>> bufs(n);
  int st = CTQ_OK;
  for (int i = 0; i < n; ++i) {
    const double dt = (i + 1 < n) ? S->ops[i + 1].t - S->ops[i].t : 0.0;
    keys[i] = leaf_key(S->ops[i], path[i], dt);
    auto it = S->cache.find(keys[i]);
    if (it != S->cache.end()) {
      bufs[i] = it->second;
      S->stats.reused += 1;
    } else {
      bufs[i] = make_leaf(S, P, S->ops[i].alpha, path[i], path[i + 1], dt, &st);
      if (st != CTQ_OK) return st;
      S->cache[keys[i]] = bufs[i];
    }
    bufs[i]->used = S->epoch;
  }
  // levels: segment starts are index 0 and every operator with h > level
  std::vector<int> starts(n);
  for (int i = 0; i < n; ++i) starts[i] = i;
  for (int level = 1; starts.size() > 1; ++level) {
    std::vector<int> ns_;
    for (size_t j = 0; j < starts.size(); ++j)
      if (j == 0 || S->ops[starts[j]].h > level) ns_.push_back(int(j));  // indices into starts
    std::vector<Key> nkeys;
    std::vector<std::shared_ptr<Buf>> nbufs;
    std::vector<int> nstarts;
    for (size_t g = 0; g < ns_.size(); ++g) {
      const int a = ns_[g], b = (g + 1 < ns_.size()) ? ns_[g + 1] : int(starts.size());
      nstarts.push_back(starts[a]);
      if (b - a == 1) {  // one factor: the same product
        nkeys.push_back(keys[a]);
        nbufs.push_back(bufs[a]);
        continue;
      }
      const Key k = seg_key(&keys[a], b - a);
      auto it = S->cache.find(k);
      std::shared_ptr<Buf> buf;
      if (it != S->cache.end()) {
        buf = it->second;
        S->stats.reused += 1;
      } else {
        buf = bufs[a];
        for (int j = a + 1; j < b && st == CTQ_OK; ++j) buf = product(S, P, bufs[j], buf, &st);
        if (st != CTQ_OK) return st;
        S->cache[k] = buf;
      }
      buf->used = S->epoch;
      nkeys.push_back(k);
      nbufs.push_back(buf);
    }
    keys.swap(nkeys);
    bufs.swap(nbufs);
    starts.swap(nstarts);
  }
  const Buf& root = *bufs[0];
  const HostModel& H = *S->H;
  const double t_wrap = S->beta - S->ops[n - 1].t + S->ops[0].t;
  SlRoot r{};
  r.X = root.p;
  r.w = root.maxw;
  r.E0 = S->D->E_rel + H.E_off[q0];
  r.out = S->d_res + 3 * q0;
  r.t = t_wrap;
  r.d = H.dims[q0];
  r.cplx = H.is_complex;
  P.roots.push_back(r);
  *L_root = root.L - t_wrap * (H.E_min[q0] - H.E_gs);
  return CTQ_OK;
}

size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Copies the planned tables to the device (one copy) and enqueues the
// zeroing, leaf, per-round product and root kernels.
int launch_plan(ctq_skiplist* S, Plan& P) {
  // tile offsets: leaves in chunks, products in tiles (the largest of
  // 64 x 64, 32 x 32 and 16 x 16 that gives the round a CTA per SM)
  int leaf_tiles = 0;
  for (SlLeaf& t : P.leaves) {
    t.tile0 = leaf_tiles;
    leaf_tiles += int((int64_t(t.d_out) * t.d_in + LEAF_CHUNK - 1) / LEAF_CHUNK);
  }
  std::vector<int> tile(P.rounds.size()), n_tiles(P.rounds.size());
  const bool tc = S->prec == CTQ_BF16X3;
  // tensor-core rounds: two operands to format and the 128 x 256 tiles of
  // every product, operands in the round's workspace (reused by the next round)
  std::vector<std::vector<SlFmt>> fmts(tc ? P.rounds.size() : 0);
  std::vector<std::vector<SlTc>> tcs(tc ? P.rounds.size() : 0);
  std::vector<int> fmt_tiles(tc ? P.rounds.size() : 0);
  size_t fmt_need = 0;
  for (size_t r = 0; tc && r < P.rounds.size(); ++r) {
    size_t wo = 0;  // bytes into the workspace
    int ft = 0, tt = 0;
    for (const SlProd& t : P.rounds[r]) {
      const int Kp = t.cplx ? 2 * t.K : t.K, Np = t.cplx ? 2 * t.N : t.N;
      const int Kpad = (Kp + TKE - 1) / TKE * TKE, Mpad = (t.M + TBM - 1) / TBM * TBM,
                Npad = (Np + TBN - 1) / TBN * TBN;
      // byte offsets into the workspace, made pointers once it is allocated
      auto at = [](size_t bytes) { return reinterpret_cast<uint16_t*>(static_cast<uintptr_t>(bytes)); };
      const size_t a_el = size_t(Mpad) * Kpad, b_el = size_t(Npad) * Kpad;
      SlFmt fa{t.R, t.wR, at(wo), at(wo + 2 * a_el), t.M, Kp, Mpad, Kpad, 0, t.K, t.N, t.cplx, TBM, ft};
      ft += int((int64_t(a_el) + FMT_CHUNK - 1) / FMT_CHUNK);
      SlFmt fb{t.L, t.wL, at(wo + 4 * a_el), at(wo + 4 * a_el + 2 * b_el), Np, Kp, Npad, Kpad, 1, t.K, t.N, t.cplx,
               TBN, ft};
      ft += int((int64_t(b_el) + FMT_CHUNK - 1) / FMT_CHUNK);
      SlTc g{fa.hi, fa.lo, fb.hi, fb.lo, t.C, t.wR, t.wL, t.wC, t.M, Np, Kpad / TKE, Npad / TBN, Mpad / TBM, tt};
      tt += (Mpad / TBM) * (Npad / TBN);
      wo += 2 * (2 * a_el + 2 * b_el);
      fmts[r].push_back(fa);
      fmts[r].push_back(fb);
      tcs[r].push_back(g);
    }
    fmt_tiles[r] = ft;
    n_tiles[r] = tt;
    fmt_need = std::max(fmt_need, wo);
  }
  for (size_t r = 0; !tc && r < P.rounds.size(); ++r) {
    tile[r] = 16;
    for (int T : {64, 32}) {
      long long nt = 0;
      for (const SlProd& t : P.rounds[r]) {
        const int np = t.cplx ? 2 * t.N : t.N;
        nt += (long long)((t.M + T - 1) / T) * ((np + T - 1) / T);
      }
      if (nt >= S->num_sms) {
        tile[r] = T;
        break;
      }
    }
    int acc = 0;
    for (SlProd& t : P.rounds[r]) {
      const int np = t.cplx ? 2 * t.N : t.N;
      t.tile0 = acc;
      t.tiles_x = (np + tile[r] - 1) / tile[r];
      acc += t.tiles_x * ((t.M + tile[r] - 1) / tile[r]);
    }
    n_tiles[r] = acc;
  }
  // one host staging buffer: zero list, leaves, rounds, roots
  size_t off = 0;
  const size_t o_zero = off;
  off = align16(off + P.zero.size() * sizeof(unsigned long long*));
  const size_t o_leaf = off;
  off = align16(off + P.leaves.size() * sizeof(SlLeaf));
  std::vector<size_t> o_round(P.rounds.size()), o_fmt(P.rounds.size());
  for (size_t r = 0; r < P.rounds.size(); ++r) {
    if (tc) {
      o_fmt[r] = off;
      off = align16(off + fmts[r].size() * sizeof(SlFmt));
      o_round[r] = off;
      off = align16(off + tcs[r].size() * sizeof(SlTc));
    } else {
      o_round[r] = off;
      off = align16(off + P.rounds[r].size() * sizeof(SlProd));
    }
  }
  const size_t o_root = off;
  off = align16(off + P.roots.size() * sizeof(SlRoot));
  if (off == 0) return CTQ_OK;
  if (off > S->tab_cap) {
    // the previous evaluation synchronised the stream: the old tables are idle
    if (S->h_tab) cudaFreeHost(S->h_tab);
    if (S->d_tab) cudaFree(S->d_tab);
    S->h_tab = nullptr;
    S->d_tab = nullptr;
    S->tab_cap = 0;
    const size_t cap = std::max<size_t>(off * 2, 64 * 1024);
    if (cudaMallocHost(&S->h_tab, cap) != cudaSuccess) return CTQ_ERR_NOMEM;
    if (cudaMalloc(&S->d_tab, cap) != cudaSuccess) return CTQ_ERR_NOMEM;
    S->tab_cap = cap;
  }
  if (tc && fmt_need > S->fmt_cap) {  // the stream is idle here (the previous evaluation synchronised)
    if (S->d_fmt) cudaFree(S->d_fmt);
    S->d_fmt = nullptr;
    S->fmt_cap = 0;
    if (cudaMalloc(&S->d_fmt, fmt_need) != cudaSuccess) return CTQ_ERR_NOMEM;
    S->fmt_cap = fmt_need;
  }
  if (tc) {  // the operand offsets become pointers into the workspace
    const uintptr_t shift = reinterpret_cast<uintptr_t>(S->d_fmt);
    auto rebase = [shift](const uint16_t* p) {
      return reinterpret_cast<uint16_t*>(reinterpret_cast<uintptr_t>(p) + shift);
    };
    for (size_t r = 0; r < P.rounds.size(); ++r) {
      for (SlFmt& f : fmts[r]) {
        f.hi = rebase(f.hi);
        f.lo = rebase(f.lo);
      }
      for (SlTc& g : tcs[r]) {
        g.Ah = rebase(g.Ah);
        g.Al = rebase(g.Al);
        g.Bh = rebase(g.Bh);
        g.Bl = rebase(g.Bl);
      }
    }
  }
  std::memcpy(S->h_tab + o_zero, P.zero.data(), P.zero.size() * sizeof(unsigned long long*));
  std::memcpy(S->h_tab + o_leaf, P.leaves.data(), P.leaves.size() * sizeof(SlLeaf));
  for (size_t r = 0; r < P.rounds.size(); ++r) {
    if (tc) {
      std::memcpy(S->h_tab + o_fmt[r], fmts[r].data(), fmts[r].size() * sizeof(SlFmt));
      std::memcpy(S->h_tab + o_round[r], tcs[r].data(), tcs[r].size() * sizeof(SlTc));
    } else {
      std::memcpy(S->h_tab + o_round[r], P.rounds[r].data(), P.rounds[r].size() * sizeof(SlProd));
    }
  }
  std::memcpy(S->h_tab + o_root, P.roots.data(), P.roots.size() * sizeof(SlRoot));
  if (cudaMemcpyAsync(S->d_tab, S->h_tab, off, cudaMemcpyHostToDevice, S->st) != cudaSuccess) return CTQ_ERR_CUDA;
  int launches = 0;
  if (!P.zero.empty()) {
    const int n = int(P.zero.size());
    k_sl_zero<<<std::min((n + 255) / 256, 1024), 256, 0, S->st>>>(
        reinterpret_cast<unsigned long long* const*>(S->d_tab + o_zero), n);
    ++launches;
  }
  if (!P.leaves.empty()) {
    k_sl_leaves<<<leaf_tiles, 256, 0, S->st>>>(S->D->blk, reinterpret_cast<const SlLeaf*>(S->d_tab + o_leaf),
                                                int(P.leaves.size()));
    ++launches;
  }
  for (size_t r = 0; tc && r < P.rounds.size(); ++r) {
    if (P.rounds[r].empty()) continue;
    k_sl_fmt<<<fmt_tiles[r], 256, 0, S->st>>>(reinterpret_cast<const SlFmt*>(S->d_tab + o_fmt[r]),
                                              int(fmts[r].size()));
    k_sl_tc<<<n_tiles[r], TC_SL_THREADS, TSTAGE * NSTG, S->st>>>(
        reinterpret_cast<const SlTc*>(S->d_tab + o_round[r]), int(tcs[r].size()), SL_TC_TIMEOUT_NS, S->d_status);
    launches += 2;
  }
  for (size_t r = 0; !tc && r < P.rounds.size(); ++r) {
    if (P.rounds[r].empty()) continue;
    const SlProd* t = reinterpret_cast<const SlProd*>(S->d_tab + o_round[r]);
    const int n = int(P.rounds[r].size());
    if (tile[r] == 16) k_sl_gemm<16, 2><<<n_tiles[r], 64, 0, S->st>>>(t, n);
    else if (tile[r] == 32) k_sl_gemm<32, 4><<<n_tiles[r], 64, 0, S->st>>>(t, n);
    else k_sl_gemm<64, 4><<<n_tiles[r], 256, 0, S->st>>>(t, n);
    ++launches;
  }
  if (!P.roots.empty()) {
    k_sl_roots<<<int(P.roots.size()), 256, 0, S->st>>>(reinterpret_cast<const SlRoot*>(S->d_tab + o_root));
    ++launches;
  }
  S->stats.launches += launches;
  S->stats.rounds = int(P.rounds.size());
  return cudaPeekAtLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

class DevGuard {
 public:
  explicit DevGuard(int d) {
    cudaGetDevice(&prev_);
    if (prev_ != d) cudaSetDevice(d);
    sw_ = prev_ != d;
  }
  ~DevGuard() {
    if (sw_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0;
  bool sw_ = false;
};

}  // namespace
}  // namespace ctq

using ctq::Op;

extern "C" int ctq_skiplist_create(const ctq_impurity* imp, double beta, uint64_t seed, void* stream,
                                   ctq_skiplist** out) {
  if (!imp || !out || !(beta > 0.0)) return CTQ_ERR_ARG;
  const ctq::HostModel* H = ctq::impurity_host(imp);
  if (H->n_extra != 0) {
    ctq::set_last_error("the skip list takes the operators c and c+ only");
    return CTQ_ERR_UNSUPPORTED;
  }
  auto* S = new ctq_skiplist();
  S->imp = imp;
  S->H = H;
  S->D = ctq::impurity_dev(imp);
  ctq::impurity_device(imp, &S->device);
  S->st = static_cast<cudaStream_t>(stream);
  S->beta = beta;
  S->rng = ctq::mix64(seed ^ 0x5ca1ab1eull);
  ctq::DevGuard g(S->device);
  cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device);
  S->num_sms = std::max(S->num_sms, 1);
  if (cudaMalloc(&S->d_res, sizeof(double) * 3 * std::max(H->n_sec, 1)) != cudaSuccess) {
    delete S;
    return CTQ_ERR_NOMEM;
  }
  *out = S;
  return CTQ_OK;
}

extern "C" int ctq_skiplist_set_precision(ctq_skiplist* S, int precision) {
  if (!S) return CTQ_ERR_ARG;
  if (precision != CTQ_FP64 && precision != CTQ_BF16X3) {
    ctq::set_last_error("the skip list's products run in CTQ_FP64 or CTQ_BF16X3");
    return CTQ_ERR_UNSUPPORTED;
  }
  if (precision == S->prec) return CTQ_OK;
  ctq::DevGuard g(S->device);
  if (precision == CTQ_BF16X3) {
    if (!S->d_status && cudaMalloc(&S->d_status, sizeof(int)) != cudaSuccess) return CTQ_ERR_NOMEM;
    if (cudaFuncSetAttribute(ctq::k_sl_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctq::NSTG * ctq::TSTAGE)) !=
        cudaSuccess)
      return CTQ_ERR_CUDA;
  }
  cudaStreamSynchronize(S->st);
  S->cache.clear();  // products of the other precision are not reused
  S->prec = precision;
  return CTQ_OK;
}

extern "C" void ctq_skiplist_free(ctq_skiplist* S) {
  if (!S) return;
  {
    ctq::DevGuard g(S->device);
    cudaStreamSynchronize(S->st);
    S->cache.clear();
    S->pool.release();
    cudaFree(S->d_res);
    if (S->h_tab) cudaFreeHost(S->h_tab);
    if (S->d_tab) cudaFree(S->d_tab);
    if (S->d_fmt) cudaFree(S->d_fmt);
    if (S->d_status) cudaFree(S->d_status);
  }
  delete S;
}

static int sl_check_ops(const ctq_skiplist* S, int m, const double* tau, const int32_t* op) {
  for (int i = 0; i < m; ++i) {
    if (!(tau[i] >= 0.0 && tau[i] < S->beta)) return CTQ_ERR_ARG;
    if (op && (op[i] < 0 || op[i] >= 2 * S->H->n_flav)) return CTQ_ERR_ARG;
  }
  return CTQ_OK;
}

extern "C" int ctq_skiplist_set(ctq_skiplist* S, int n, const double* tau, const int32_t* op) {
  if (!S || n < 0 || (n > 0 && (!tau || !op))) return CTQ_ERR_ARG;
  if (sl_check_ops(S, n, tau, op) != CTQ_OK) return CTQ_ERR_ARG;
  for (int i = 1; i < n; ++i)
    if (!(tau[i] > tau[i - 1])) return CTQ_ERR_ARG;
  S->ops.clear();
  for (int i = 0; i < n; ++i) S->ops.push_back(Op{S->next_id++, tau[i], op[i], ctq::sl_height(S)});
  return CTQ_OK;
}

extern "C" int ctq_skiplist_insert(ctq_skiplist* S, int m, const double* tau, const int32_t* op) {
  if (!S || m < 0 || (m > 0 && (!tau || !op))) return CTQ_ERR_ARG;
  if (sl_check_ops(S, m, tau, op) != CTQ_OK) return CTQ_ERR_ARG;
  std::vector<Op> add;
  for (int i = 0; i < m; ++i) add.push_back(Op{0, tau[i], op[i], 0});
  for (const Op& a : add)
    for (const Op& o : S->ops)
      if (o.t == a.t) return CTQ_ERR_ARG;
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (tau[i] == tau[j]) return CTQ_ERR_ARG;
  for (Op& a : add) {
    a.id = S->next_id++;
    a.h = ctq::sl_height(S);
    auto it = std::lower_bound(S->ops.begin(), S->ops.end(), a.t, [](const Op& o, double t) { return o.t < t; });
    S->ops.insert(it, a);
  }
  return CTQ_OK;
}

extern "C" int ctq_skiplist_remove(ctq_skiplist* S, int m, const double* tau) {
  if (!S || m < 0 || (m > 0 && !tau)) return CTQ_ERR_ARG;
  std::vector<size_t> idx;
  for (int i = 0; i < m; ++i) {
    auto it = std::lower_bound(S->ops.begin(), S->ops.end(), tau[i], [](const Op& o, double t) { return o.t < t; });
    if (it == S->ops.end() || it->t != tau[i]) return CTQ_ERR_ARG;
    idx.push_back(size_t(it - S->ops.begin()));
  }
  std::sort(idx.begin(), idx.end());
  if (std::adjacent_find(idx.begin(), idx.end()) != idx.end()) return CTQ_ERR_ARG;
  for (size_t k = idx.size(); k-- > 0;) S->ops.erase(S->ops.begin() + idx[k]);
  return CTQ_OK;
}

extern "C" int ctq_skiplist_evaluate(ctq_skiplist* S, double* log_abs, double* phase, ctq_skiplist_stats* stats) {
  if (!S || !log_abs || !phase) return CTQ_ERR_ARG;
  const ctq::HostModel& H = *S->H;
  const int ns = H.n_sec, n = int(S->ops.size());
  ctq::DevGuard g(S->device);
  S->stats = ctq_skiplist_stats{};
  S->epoch += 1;
  ctq::Plan plan;
  std::vector<int> live;
  std::vector<double> Lq(ns, 0.0);
  double lm = -INFINITY;
  double acc_re = 0.0, acc_im = 0.0;
  if (n == 0) {  // w = Z_loc
    for (int q = 0; q < ns; ++q)
      for (int j = 0; j < H.dims[q]; ++j) {
        const double l = -S->beta * (H.E[H.E_off[q] + j] - H.E_gs);
        if (l > lm) { acc_re *= std::exp(lm - l); lm = l; }
        acc_re += std::exp(l - lm);
      }
  } else {
    for (int q0 = 0; q0 < ns; ++q0) {
      std::vector<int> path(n + 1);
      path[0] = q0;
      bool ok = true;
      for (int i = 0; i < n && ok; ++i) {
        const int q = H.s[size_t(S->ops[i].alpha) * ns + path[i]];
        ok = q >= 0;
        path[i + 1] = q;
      }
      if (!ok || path[n] != q0) continue;
      const int st = ctq::plan_string(S, plan, q0, path, &Lq[q0]);
      if (st != CTQ_OK) {  // no cached product may outlive a plan that never ran
        S->cache.clear();
        return st;
      }
      live.push_back(q0);
    }
    const bool tc = S->prec == CTQ_BF16X3;
    if (tc && cudaMemsetAsync(S->d_status, 0, sizeof(int), S->st) != cudaSuccess) return CTQ_ERR_CUDA;
    const int st = ctq::launch_plan(S, plan);
    plan.keep.clear();  // the buffers' kernels are enqueued: later reuse is ordered after them
    if (st != CTQ_OK) {
      cudaStreamSynchronize(S->st);
      S->cache.clear();
      return st;
    }
    std::vector<double> res(3 * std::max(ns, 1));
    int tc_status = 0;
    if (!live.empty() &&
        cudaMemcpyAsync(res.data(), S->d_res, sizeof(double) * 3 * ns, cudaMemcpyDeviceToHost, S->st) != cudaSuccess)
      return CTQ_ERR_CUDA;
    if (tc && cudaMemcpyAsync(&tc_status, S->d_status, sizeof(int), cudaMemcpyDeviceToHost, S->st) != cudaSuccess)
      return CTQ_ERR_CUDA;
    if (cudaStreamSynchronize(S->st) != cudaSuccess) return CTQ_ERR_CUDA;
    if (tc_status != 0) {  // a product gave up waiting: none of this evaluation's products is kept
      S->cache.clear();
      return CTQ_ERR_TIMEOUT;
    }
    for (int q0 : live) {
      long long e;
      std::memcpy(&e, &res[3 * q0 + 2], 8);
      const double re = res[3 * q0], im = res[3 * q0 + 1];
      if (e == ctq::EXP_DEAD || (re == 0.0 && im == 0.0)) continue;
      const double l = Lq[q0] + double(e) * 0.69314718055994530942 + std::log(std::hypot(re, im));
      const double ur = re / std::hypot(re, im), ui = im / std::hypot(re, im);
      if (l > lm) {
        const double f = std::exp(lm - l);
        acc_re *= f;
        acc_im *= f;
        lm = l;
      }
      const double f = std::exp(l - lm);
      acc_re += f * ur;
      acc_im += f * ui;
    }
  }
  // drop every cached product the current configuration no longer uses
  for (auto it = S->cache.begin(); it != S->cache.end();)
    it = it->second->used == S->epoch ? std::next(it) : S->cache.erase(it);
  const double a = std::hypot(acc_re, acc_im);
  if (!(a > 0.0) || lm == -INFINITY) {
    *log_abs = -INFINITY;
    phase[0] = phase[1] = 0.0;
  } else {
    *log_abs = lm + std::log(a) - S->beta * H.E_gs;
    phase[0] = acc_re / a;
    phase[1] = acc_im / a;
  }
  S->stats.n_ops = n;
  S->stats.n_strings = int(live.size());
  S->stats.cached = int64_t(S->cache.size());
  S->stats.device_bytes = int64_t(S->pool.bytes());
  if (stats) *stats = S->stats;
  return cudaGetLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}
