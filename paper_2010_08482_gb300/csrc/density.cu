// Reduced-density-matrix estimator on the GPU (Sec. 2.3, "Estimators",
// Eq. ImpurityDensityMatrix): for every chain C,
//     rho^C_{uv} = beta^{-1} int_0^beta w_loc(C, |v><u|(tau)) / w_loc(C) dtau,
// the projector inserted at every time of the time-ordered product and the
// tau integral taken analytically.  For a surviving sector string q0 -> q1
// -> ... -> q0 and the propagation interval i (length D_i, sector q_i):
//     int w(C, |v><u|(tau)) dtau = (A_i B_i)_{uv} K(E_u, E_v, D_i),
//     A_i = F_i P ... F_1 P_{tau_1}              (the product before the interval),
//     B_i = P_{beta - tau_n} F_n ... F_{i+1}      (the product after it),
//     K(a, b, D) = e^{-D min(a, b)} (1 - e^{-D |a - b|}) / |a - b|   (D e^{-D a} if a = b).
//
//   k_rho   persistent CTAs pull (chain, q0) strings from the work list of
//           k_plan.  A forward pass stores every A_i (normalised, with an
//           exact power-of-two exponent) in the CTA's scratch; a backward
//           pass builds B_i, forms G_i = A_i B_i for every interval and adds
//           G_i o K_i / (beta w_C) into the chain's density matrix (float64
//           atomics; w_C from the trace evaluation that precedes it).
// float64 throughout; blocks of both products live in shared memory (the
// sizes of the shared-memory trace kernel).
//
//   HST     the same two passes give the static improved-estimator ratio
//           (Sec. 2.4, Eq. PImprovedEstimatorStatic) of every annihilator
//           c_f at operator i: with the annihilator replaced by its Bulla
//           operator Q = [c_f, U] (operator code 2 n_f + f),
//             w^U_i = Tr[ Y_i Q P_{Delta_i} A_i ],
//           Y_i the backward product after operator i (its propagator
//           included), A_i the stored forward product before it and
//           P_{Delta_i} the propagator of the interval that ends at
//           operator i (A_0 = 1, P = P_{tau_1}(q0) for the first operator).
//           One extra product per annihilator instead of a full trace of a
//           replaced sequence; h^st_i = sum_{q0} w^U_i / w_C.
#include <algorithm>

#include "device_common.cuh"

namespace ctq {
namespace {

using namespace dev;

template <bool CPLX>
struct Num;
template <>
struct Num<false> {
  using T = double;
};
template <>
struct Num<true> {
  using T = double2;
};

__device__ __forceinline__ int num_key(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ int num_key(double2 v) { return max(num_key(v.x), num_key(v.y)); }
__device__ __forceinline__ double num_zero(double) { return 0.0; }
__device__ __forceinline__ double2 num_zero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double num_one(double) { return 1.0; }
__device__ __forceinline__ double2 num_one(double2) { return make_double2(1.0, 0.0); }
__device__ __forceinline__ double num_scale(double v, double s) { return v * s; }
__device__ __forceinline__ double2 num_scale(double2 v, double s) { return make_double2(v.x * s, v.y * s); }
__device__ __forceinline__ void num_fma(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void num_fma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double num_blk(const double* blk, int64_t i, double) { return __ldg(blk + i); }
__device__ __forceinline__ double2 num_blk(const double* blk, int64_t i, double2) {
  return __ldg(reinterpret_cast<const double2*>(blk) + i);
}

// Largest exponent field of a block held by the CTA, as the scale 2^-e that
// brings max|X| into [1, 2); returns e (0 with *dead set when X == 0).
template <typename T>
__device__ int block_rescale(T* X, int count, int* redi, bool* dead) {
  int k = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) k = max(k, num_key(X[i]));
  k = __reduce_max_sync(0xffffffffu, k);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nw > 1) {
    __syncthreads();
    if ((threadIdx.x & 31) == 0) redi[w] = k;
    __syncthreads();
    k = redi[0];
    for (int i = 1; i < nw; ++i) k = max(k, redi[i]);
  }
  if (k == 0) {
    *dead = true;
    return 0;
  }
  const int e = min(k - 1023, 1022);
  const double s = pow2i(-e);
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) X[i] = num_scale(X[i], s);
  __syncthreads();
  return e;
}

// The interval integral without its e^{-D E_min(q)} factor: energies a, b
// are relative to the sector's lowest level, ea = e^{-D a}, eb = e^{-D b}.
// Well separated levels use the difference quotient of the exponentials
// (relative error below 3 u once D |a - b| > 1/2); close levels the form
// e^{-D min(a, b)} (1 - e^{-D |a - b|}) / |a - b| with expm1.
__device__ __forceinline__ double kernel_rel(double a, double b, double ea, double eb, double D) {
  const double gap = fabs(a - b);
  if (gap == 0.0) return D * ea;
  if (D * gap > 0.5) return (a > b) ? (eb - ea) / gap : (ea - eb) / gap;
  return ((a < b) ? ea : eb) * (-expm1(-D * gap) / gap);
}

template <bool CPLX, bool HST>
__global__ void __launch_bounds__(256) k_rho(DevModel M, BatchView B, EvalCfg cfg, Work W, ctq_result R, RhoParams P) {
  using T = typename Num<CPLX>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int D = M.max_dim;
  const int MO = max(cfg.max_ops, 1);
  T* X = reinterpret_cast<T*>(smem_raw);  // [D * D] running product (backward pass: also G_i = A_i B_i)
  T* Xn = X + size_t(D) * D;              // [D * D]
  short* path = reinterpret_cast<short*>(Xn + size_t(D) * D);  // [MO + 1]
  short* opsm = path + (MO + 1);                               // [MO], then one short of padding
  int* eA = reinterpret_cast<int*>(opsm + MO + 1);             // [MO + 1] exponents of the stored A_i
  double* ex = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(eA + MO + 1) + 7) & ~uintptr_t(7));  // [D]
  // small estimators: the string's contributions are summed in shared memory
  // and added to the chain's estimator once
  double* acc_s = P.local_acc ? ex + D : nullptr;  // [rho_elems]
  __shared__ int redi[32];
  __shared__ int s_item;
  __shared__ double s_L;
  __shared__ double segdummy[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ns = M.n_sec;
  const int n_items = W.counters[0];
  const Item* items = W.items + size_t(B.n_chains) * ns;
  T* Ast = reinterpret_cast<T*>(P.scratch) + size_t(blockIdx.x) * P.scratch_elems;  // stored A_1 .. A_n
  EvalCfg cfg0 = cfg;
  cfg0.lazy = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(&W.counters[3], 1);
    __syncthreads();
    const int it_idx = s_item;
    if (it_idx >= n_items) break;
    const Item it = items[W.order[it_idx]];
    const int c = it.c, q0 = it.q0;
    const int a0 = B.offsets[c];
    const int n = B.offsets[c + 1] - a0;
    const int d0 = M.dims[q0];
    const double lw = R.log_abs[c];
    if (!(lw > -INFINITY) || !(lw < INFINITY)) continue;  // zero or failed chain: no estimator
    // 1 / (beta w_C) with w_C = |w| e^{i phi}; logs relative to e^{-beta E_ref}
    const double logw_rel = lw + B.beta * M.E_ref;
    const double phr = R.phase[2 * c], phi = CPLX ? R.phase[2 * c + 1] : 0.0;
    double* out = P.rho + size_t(c) * P.rho_elems;
    double* dst = acc_s ? acc_s : out;
    if (acc_s) {
      for (size_t i = tid; i < P.rho_elems; i += nt) acc_s[i] = 0.0;
      __syncthreads();
    }

    // ---- the string: operator codes, sectors, total log scale
    for (int i = tid; i < n; i += nt) opsm[i] = short(B.op[a0 + i]);
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
    const double t_first = (n > 0) ? B.tau[a0] : B.beta;
    const double t_last = (n > 0) ? B.beta - B.tau[a0 + n - 1] : 0.0;
    if (n > 0) {
      if (tid < 32) chain_log_scale(M, B, cfg0, a0, n, q0, t_first, t_last, false, path, opsm, segdummy, segdummy, &s_L);
    } else if (tid == 0) {
      s_L = -B.beta * (M.E_min[q0] - M.E_ref);
    }
    __syncthreads();
    const double base = s_L - logw_rel;  // log of (propagator scale) / w_C

    // adds G o K(D) of sector q, scaled by 2^e e^{base} / beta, into rho^C
    auto accumulate = [&](const T* Gm, int q, double Dlen, int e) {
      const int d = M.dims[q];
      const double* Eq = M.E_rel + M.E_off[q];
      const double f = exp(base + double(e) * LN2) / B.beta;
      double* blk = dst + (CPLX ? 2 : 1) * P.rho_off[q];
      __syncthreads();
      for (int u = tid; u < d; u += nt) ex[u] = exp(-Dlen * Eq[u]);
      __syncthreads();
      for (int idx = tid; idx < d * d; idx += nt) {
        const int u = idx / d, v = idx - u * d;
        const double k = kernel_rel(Eq[u], Eq[v], ex[u], ex[v], Dlen) * f;
        if constexpr (CPLX) {
          // (g / w) with w = |w| (phr + i phi): multiply by conj(phase)
          const double gr = Gm[idx].x, gi = Gm[idx].y;
          atomicAdd(blk + 2 * idx, k * (gr * phr + gi * phi));
          atomicAdd(blk + 2 * idx + 1, k * (gi * phr - gr * phi));
        } else {
          atomicAdd(blk + idx, k * Gm[idx] * phr);
        }
      }
    };

    if (HST && n == 0) continue;  // no operator, no ratio
    if (n == 0) {  // one interval (0, beta) with G = identity
      for (int idx = tid; idx < d0 * d0; idx += nt) {
        const int u = idx / d0, v = idx - u * d0;
        X[idx] = (u == v) ? num_one(T()) : num_zero(T());
      }
      __syncthreads();
      accumulate(X, q0, B.beta, 0);
      if (acc_s) {
        __syncthreads();
        for (size_t i = tid; i < P.rho_elems; i += nt)
          if (acc_s[i] != 0.0) atomicAdd(out + i, acc_s[i]);
      }
      continue;
    }

    // ---- forward: A_i (d_{q_i} x d0), i = 1..n, stored normalised with exponents eA[i].
    // A zero product stays in the pass: intervals before it may still carry
    // weight once the projector is inserted.
    bool dead = false;
    {
      const double* E0 = M.E_rel + M.E_off[q0];
      for (int idx = tid; idx < d0 * d0; idx += nt) X[idx] = num_zero(T());
      __syncthreads();
      for (int j = tid; j < d0; j += nt) X[j * d0 + j] = num_scale(num_one(T()), exp(-t_first * E0[j]));
    }
    __syncthreads();
    int eacc = 0;
    size_t aoff = 0;
    int da = d0;
    for (int i = 1; i <= n; ++i) {
      const int qa = path[i - 1], qb = path[i];
      const int db = M.dims[qb];
      const int64_t off = M.blk_off[opsm[i - 1] * ns + qa];
      // Xn = F X  (db x d0)
      for (int idx = tid; idx < db * d0; idx += nt) {
        const int m = idx / d0, j = idx - m * d0;
        T acc = num_zero(T());
        for (int k = 0; k < da; ++k) num_fma(acc, num_blk(M.blk, off + int64_t(m) * da + k, T()), X[k * d0 + j]);
        Xn[idx] = acc;
      }
      __syncthreads();
      bool zero = false;
      eacc += block_rescale(Xn, db * d0, redi, &zero);
      if (tid == 0) eA[i] = eacc;
      for (int idx = tid; idx < db * d0; idx += nt) Ast[aoff + idx] = Xn[idx];
      aoff += size_t(db) * d0;
      // X = P_{Delta_i} Xn for the next operator
      if (i < n) {
        const double dt = B.tau[a0 + i] - B.tau[a0 + i - 1];
        const double* Eb = M.E_rel + M.E_off[qb];
        for (int m = tid; m < db; m += nt) ex[m] = exp(-dt * Eb[m]);
        __syncthreads();
        for (int idx = tid; idx < db * d0; idx += nt) X[idx] = num_scale(Xn[idx], ex[idx / d0]);
      }
      __syncthreads();
      da = db;
    }
    // interval n: (tau_n, beta) in q0, G = A_n, B_n = I
    aoff -= size_t(d0) * d0;  // A_n (d0 x d0) is the last stored product
    if (!HST) accumulate(Ast + aoff, q0, t_last, eA[n]);
    __syncthreads();

    // ---- backward: Y = P_{beta - tau_n}(q0), then B_i = Y F_{i+1}, G_i = A_i B_i
    {
      const double* E0 = M.E_rel + M.E_off[q0];
      for (int idx = tid; idx < d0 * d0; idx += nt) X[idx] = num_zero(T());
      __syncthreads();
      for (int j = tid; j < d0; j += nt) X[j * d0 + j] = num_scale(num_one(T()), exp(-t_last * E0[j]));
    }
    __syncthreads();
    int ebacc = 0;
    int dy = d0;  // columns of Y = dim of path[i + 1]
    for (int i = n - 1; i >= 0 && !dead; --i) {
      const int qa = path[i];  // F_{i+1} maps qa -> path[i + 1]
      const int dq = M.dims[qa];
      const int64_t off = M.blk_off[opsm[i] * ns + qa];
      const T* Ai = nullptr;  // A_i is d_{q_i} x d0 (i >= 1)
      if (i >= 1) {
        aoff -= size_t(dq) * d0;
        Ai = Ast + aoff;
      }
      const double Dlen = (i == 0) ? t_first : (B.tau[a0 + i] - B.tau[a0 + i - 1]);
      // Xn = Y F  (d0 x dq), F is dy x dq
      for (int idx = tid; idx < d0 * dq; idx += nt) {
        const int j = idx / dq, m = idx - j * dq;
        T acc = num_zero(T());
        for (int k = 0; k < dy; ++k) num_fma(acc, X[j * dy + k], num_blk(M.blk, off + int64_t(k) * dq + m, T()));
        Xn[idx] = acc;
      }
      __syncthreads();
      if (HST && opsm[i] < 2 * M.n_flav && (opsm[i] & 1) == 0) {
        // w^U_i / w_C = 2^{e} e^{base} sum_{j, m} (Y Q)_{jm} e^{-Dlen E_m} (A_i)_{mj}, Q dy x dq
        const int64_t qoff = M.blk_off[(2 * M.n_flav + (opsm[i] >> 1)) * ns + qa];
        const double* Eq = M.E_rel + M.E_off[qa];
        for (int m = tid; m < dq; m += nt) ex[m] = exp(-Dlen * Eq[m]);
        __syncthreads();
        T part = num_zero(T());
        if (qoff >= 0) {
          for (int idx = tid; idx < d0 * dq; idx += nt) {
            const int j = idx / dq, m = idx - j * dq;
            if (i == 0 && m != j) continue;  // A_0 = 1
            T yq = num_zero(T());
            for (int k = 0; k < dy; ++k) num_fma(yq, X[j * dy + k], num_blk(M.blk, qoff + int64_t(k) * dq + m, T()));
            const T z = (i == 0) ? num_scale(num_one(T()), ex[m]) : num_scale(Ai[m * d0 + j], ex[m]);
            num_fma(part, yq, z);
          }
        }
        const double f = exp(base + double(ebacc + (i >= 1 ? eA[i] : 0)) * LN2);
        double pr, pi;
        if constexpr (CPLX) {
          pr = part.x;
          pi = part.y;
        } else {
          pr = part;
          pi = 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) {
          pr += __shfl_down_sync(0xffffffffu, pr, o);
          pi += __shfl_down_sync(0xffffffffu, pi, o);
        }
        if ((tid & 31) == 0 && (pr != 0.0 || pi != 0.0) && size_t(a0) + i < P.h_len) {
          // (w^U / |w|) conj(phase)
          double* hdst = P.rho + 2 * (size_t(a0) + i);
          atomicAdd(hdst, f * (pr * phr + pi * phi));
          atomicAdd(hdst + 1, f * (pi * phr - pr * phi));
        }
        __syncthreads();
      }
      ebacc += block_rescale(Xn, d0 * dq, redi, &dead);
      if (dead) break;  // B_i = 0, and so are the products of every earlier interval
      // G_i = A_i B_i (dq x dq) into X (Y is no longer needed); A_0 = I
      T* G = X;
      if (HST) {
        // no interval products: Y = B_i P_{Delta} below
      } else if (i == 0) {
        for (int idx = tid; idx < dq * dq; idx += nt) G[idx] = Xn[idx];
      } else {
        for (int idx = tid; idx < dq * dq; idx += nt) {
          const int u = idx / dq, v = idx - u * dq;
          T acc = num_zero(T());
          for (int k = 0; k < d0; ++k) num_fma(acc, Ai[u * d0 + k], Xn[k * dq + v]);
          G[idx] = acc;
        }
      }
      __syncthreads();
      if (!HST) accumulate(G, qa, Dlen, ebacc + (i >= 1 ? eA[i] : 0));
      __syncthreads();
      // Y = B_i P_{Delta} for the next (earlier) operator
      if (i > 0) {
        const double* Eq = M.E_rel + M.E_off[qa];
        for (int m = tid; m < dq; m += nt) ex[m] = exp(-Dlen * Eq[m]);
        __syncthreads();
        for (int idx = tid; idx < d0 * dq; idx += nt) X[idx] = num_scale(Xn[idx], ex[idx % dq]);
      }
      __syncthreads();
      dy = dq;
    }
    if (acc_s) {  // add this string's contributions to the chain's estimator
      __syncthreads();
      for (size_t i = tid; i < P.rho_elems; i += nt)
        if (acc_s[i] != 0.0) atomicAdd(out + i, acc_s[i]);
    }
  }
}

}  // namespace

constexpr size_t RHO_LOCAL_MAX = 16384;  // bytes of an estimator summed in shared memory

static size_t rho_smem(int max_dim, bool cplx, int max_ops, size_t rho_doubles) {
  const size_t el = cplx ? 16 : 8;
  const size_t mo = size_t(std::max(max_ops, 1));
  // products, path + operator codes + padding, exponents, then (8-byte aligned) e^{-D E}
  size_t b = 2 * size_t(max_dim) * max_dim * el + (2 * mo + 2) * 2 + (mo + 1) * 4 + 8 + size_t(max_dim) * 8 + 16;
  if (rho_doubles * 8 <= RHO_LOCAL_MAX) b += rho_doubles * 8;
  return (b + 15) & ~size_t(15);
}

size_t rho_elems(const HostModel& h) {
  size_t s = 0;
  for (int q = 0; q < h.n_sec; ++q) s += size_t(h.dims[q]) * h.dims[q];
  return s;
}

size_t rho_scratch_bytes(const HostModel& h, int max_ops, int grid) {
  const size_t el = h.is_complex ? 16 : 8;
  return size_t(grid) * size_t(std::max(max_ops, 1) + 1) * h.max_dim * h.max_dim * el + 256;
}

int rho_grid(const DevModel& M, int num_sms, int max_ops, size_t rho_doubles) {
  const size_t smem = rho_smem(M.max_dim, M.is_complex != 0, max_ops, rho_doubles);
  const int per_sm = std::max(1, std::min(16, int((200 * 1024) / (smem + 1024))));
  return num_sms * per_sm;
}

int prepare_rho(int optin) {
  cudaFuncAttributes fa;
  int stat = 0;
  for (const void* fn : {reinterpret_cast<const void*>(k_rho<false, false>), reinterpret_cast<const void*>(k_rho<true, false>),
                         reinterpret_cast<const void*>(k_rho<false, true>), reinterpret_cast<const void*>(k_rho<true, true>)}) {
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return CTQ_ERR_CUDA;
    stat = std::max(stat, int(fa.sharedSizeBytes));
  }
  const int cap = optin - stat;
  if (cudaFuncSetAttribute(k_rho<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
      cudaFuncSetAttribute(k_rho<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
      cudaFuncSetAttribute(k_rho<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
      cudaFuncSetAttribute(k_rho<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess)
    return CTQ_ERR_CUDA;
  return CTQ_OK;
}

int launch_rho(const DevModel& M, int num_sms, int optin, const BatchView& B, const EvalCfg& cfg, const Work& W,
               const ctq_result& R, RhoParams P, size_t rho_total_doubles, void* stream, bool hst) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (hst) P.rho_elems = 0;  // ratios go straight to the output, one pair per operator
  P.local_acc = (!hst && P.rho_elems * 8 <= RHO_LOCAL_MAX) ? 1 : 0;
  const size_t smem = rho_smem(M.max_dim, M.is_complex != 0, cfg.max_ops, P.rho_elems);
  if (smem + 1024 > size_t(optin)) return CTQ_ERR_UNSUPPORTED;
  const int threads = M.max_dim <= 12 ? 32 : (M.max_dim <= 32 ? 128 : 256);
  const int grid = rho_grid(M, num_sms, cfg.max_ops, P.rho_elems);
  if (cudaMemsetAsync(P.rho, 0, rho_total_doubles * sizeof(double), st) != cudaSuccess) return CTQ_ERR_CUDA;
  // the item counter of this pass (the trace pass used counters[1])
  if (cudaMemsetAsync(W.counters + 3, 0, sizeof(int), st) != cudaSuccess) return CTQ_ERR_CUDA;
  if (hst) {
    if (M.is_complex)
      k_rho<true, true><<<grid, threads, smem, st>>>(M, B, cfg, W, R, P);
    else
      k_rho<false, true><<<grid, threads, smem, st>>>(M, B, cfg, W, R, P);
  } else if (M.is_complex) {
    k_rho<true, false><<<grid, threads, smem, st>>>(M, B, cfg, W, R, P);
  } else {
    k_rho<false, false><<<grid, threads, smem, st>>>(M, B, cfg, W, R, P);
  }
  return cudaGetLastError() == cudaSuccess ? CTQ_OK : CTQ_ERR_CUDA;
}

}  // namespace ctq
