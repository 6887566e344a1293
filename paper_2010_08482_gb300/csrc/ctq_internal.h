// Internal declarations shared by the translation units of libctq.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "ctq.h"

namespace ctq {

using cplx = std::complex<double>;

// Sector-decomposed impurity in its eigenbasis, host copy.
//   E is concatenated per sector (E_off[q] .. E_off[q+1]), ascending, mu included.
//   s[alpha * n_sec + q]: target sector of operator alpha on q, or -1.
//   blk_off[alpha * n_sec + q]: element offset of block F_alpha(q)
//     (d_{s(q)} x d_q, row-major) in blk_re / blk_im, or -1.
//   opnorm: spectral norm of each block (0 for absent blocks).
//   Operator codes: 2 f + dag for c_f / c+_f, then n_extra further codes
//   (2 n_flav + f: the Bulla operator [c_f, U] once added).
//   h1: the one-body matrix t - mu (n_flav x n_flav, flavour basis) of a
//     model built from parameters; empty for a loaded model.
struct HostModel {
  int n_flav = 0, n_sec = 0, max_dim = 0, is_complex = 0;
  int n_extra = 0;
  double mu = 0.0, E_gs = 0.0;
  std::vector<int> dims, N, E_off;
  std::vector<double> E, E_min;
  std::vector<int> s;
  std::vector<int64_t> blk_off;
  std::vector<double> blk_re, blk_im;
  std::vector<double> opnorm;
  std::vector<cplx> h1;
  int n_alpha() const { return 2 * n_flav + n_extra; }
};

// Builds the model from physics parameters on the host (Fock space, H_loc,
// sectors, eigensolver, blocks).  Returns a CTQ_* status.
int build_host_model(const ctq_model_params* p, HostModel& m, std::string& err);

// Hermitian eigensolver (cyclic Jacobi): A (n x n, row-major) is destroyed;
// E ascending, V[row * n + col] = component row of eigenvector col.
int jacobi_eigh_real(int n, std::vector<double>& A, std::vector<double>& E, std::vector<double>& V);
int jacobi_eigh_cplx(int n, std::vector<cplx>& A, std::vector<double>& E, std::vector<cplx>& V);

// Set-up linear algebra for sectors too large for the host Jacobi solver
// (eigen_device.cu): cuSOLVER eigensolver and cuBLAS block transforms on the
// impurity's device, libraries loaded on first use.
class DeviceSectorLA {
 public:
  DeviceSectorLA();
  ~DeviceSectorLA();
  int init(int device, bool cplx, int n_sec, std::string& err);
  int eigh(int q, int n, const std::vector<cplx>& H, std::vector<double>& E, std::vector<cplx>* Vc,
           std::vector<double>* Vr, std::string& err);
  bool has(int q) const;
  int block(int q, int qp, const std::vector<int>& src, const std::vector<int>& dst, const std::vector<double>& sg,
            double* re, double* im, std::string& err);

 private:
  struct Impl;
  Impl* impl_;
};

// Sectors above this dimension are diagonalised on the device.
constexpr int kJacobiMaxDim = 160;

// Device-side view of a model (all pointers on the model's device).
struct DevModel {
  int n_flav, n_alpha, n_sec, max_dim, is_complex;
  double E_ref;         // reference energy (E_gs); logs are kept relative to -beta E_ref
  const int* dims;      // [n_sec]
  const double* log_dim;  // [n_sec]  log(dims[q]) (rank factor of the bounds, no device logarithm)
  const int* E_off;     // [n_sec + 1]
  const double* E_rel;  // [sum dims]  E_q,j - E_min(q)  (>= 0)
  const float* E_relf;  // [sum dims]  the same in float32 (mixed-precision propagators)
  const double* E_min;  // [n_sec]
  const int* s;         // [n_alpha * n_sec]
  const int64_t* blk_off;  // [n_alpha * n_sec]  element offsets, -1 absent
  const double* blk;    // real: re; complex: interleaved (re, im)
  const float* blk_x2;  // two-float copy of blk (hi, lo per real number; CTQ_F32X2), nullptr if absent
  const double* log_norm;  // [n_alpha * n_sec]  log ||F||_2 (-inf absent)
  // distinct values of E_rel per sector (bitwise equal states share one
  // propagator entry): level values, per-sector offsets, state -> level
  const double* lev_E;     // [sum n_lev]
  const int* lev_off;      // [n_sec + 1]
  const int* lev_idx;      // [sum dims]  level of each state within its sector
  int max_lev;             // largest number of levels of one sector
};

struct BatchView {
  int n_chains;
  double beta;
  const int32_t* offsets;
  const double* tau;
  const int32_t* op;
  const double* log_threshold;
};

struct EvalCfg {
  int lazy;         // early reject enabled (and thresholds present)
  int has_thr;      // thresholds present
  int S;            // segment length
  int n_seg_max;    // ceil(max_ops / S)
  int max_ops;      // longest chain allowed (longer chains are flagged invalid)
  double margin;    // safety margin (log units) applied to bounds before rejecting
  double* bounds;   // result bounds [C x (n_seg_max + 1)] or nullptr
  int debug;        // ctq_eval_opts.debug_flags
  int threads;      // launch tuning (ctq_eval_opts), 0 = default
  int ctas_per_sm;
  int stages;
  int tile_order;
};

// A work item: one surviving (chain, q0) string.
struct Item {
  int c;
  int q0;
  int r;         // min over the string of the sector dimension (rank bound)
  int n_seg;     // ceil(n / S)
  double t_all;  // sum of log ||F_i||_2 and -dtau (E_min - E_ref) over the string (plan kernel)
  double log_r;  // log r, from the host table of log(dims)
  float cost;    // work estimate: d0 sum_i d_i d_{i+1} + PLAN_OP_COST n (orders the work list)
};

// Work-list ordering: strings are pulled in decreasing order of their cost
// estimate, in ORDER_CLASSES classes of 1/8 octave (counting sort).
constexpr int ORDER_CLASSES = 512;
constexpr size_t COUNTER_BYTES = 256;  // counters region, cleared before every evaluation

// Views of the caller's workspace.
struct Work {
  int* counters;   // [0] n_items, [1] next item, [2] device error bits, [3] estimator next item,
                   // [4] plan CTAs done
  Item* items;     // [2 C n_sec] staging slots per (c, q0), then the compacted list
  int* order;      // [C * n_sec] list position -> compacted item, most expensive first
  double* res_val; // [C * n_sec * 2]  scaled trace value (re, im)
  // All logs below are relative: the true value carries an extra e^{-beta E_ref}.
  double* res_log; // [C * n_sec]      log scale of res_val (-inf: zero)
  double* live;    // [C * n_sec]      live log upper bound per (c, q0)
  double* lvl0;    // [C * n_sec]      level-0 log bound per (c, q0)
  double* seg;     // [C * n_sec * (n_seg_max + 1)] per-segment log bounds
  int* chain_flag; // [C]  bit 0 invalid, bit 1 rejected early
};

enum : int { FLAG_INVALID = 1, FLAG_REJECTED = 2 };

size_t workspace_layout(int n_chains, int n_sec, int n_seg_max, void* base, Work* w);

// Helpers for entry points defined outside api.cpp.
void set_last_error(const std::string& msg);
// Records a caller's timing event on `stream`; while the stream is being
// captured into a CUDA graph the record becomes an event-record node of the
// graph (so that every replay records it), otherwise a plain record.
void record_timing_event(void* event, void* stream);
int impurity_device(const ctq_impurity* imp, int* device);
// The impurity's host model and its device view (nullptr for a null handle).
const HostModel* impurity_host(const ctq_impurity* imp);
const DevModel* impurity_dev(const ctq_impurity* imp);

// Launch shape of the trace kernel, fixed per impurity when it is uploaded
// (so that evaluation makes no attribute or occupancy query, e.g. while a
// CUDA graph is being captured).
struct LaunchCfg {
  int threads = 0;
  size_t smem = 0;
  int per_sm = 0;   // resident CTAs per SM (0: shape not supported)
  int num_sms = 0;
  int regs = 0;     // registers per thread of the kernel
  int regs_small = 0;  // registers per thread of the 32-thread variant (small blocks), if any
  int smem_optin = 0;  // opt-in shared memory per block of the device
};

// Kernel parameters specific to the tensor-core path (trace_tc.cu).
struct TcParams {
  const void* blk = nullptr;     // pre-formatted blocks (hi, lo) in core-matrix order
  const int64_t* off = nullptr;  // [n_alpha * n_sec] byte offsets into blk, -1 absent
  int prec = CTQ_TF32;           // CTQ_TF32, CTQ_TF32X3 or CTQ_BF16X3
  int stage_bytes = 0;           // bytes per shared-memory stage
  int tmem_cols = 256;           // TMEM columns allocated per CTA
  uint64_t timeout_ns = 0;
};

// Per-impurity parameters and scratch of the large-block path (trace_big.cu).
struct BigParams {
  const void* bt = nullptr;       // embedded blocks: tiles (hi, then lo), per (alpha, q)
  const int64_t* bt_off = nullptr;  // [n_alpha * n_sec] element offsets, -1 absent
  int prec = CTQ_TF32X3;          // CTQ_TF32, CTQ_TF32X3 or CTQ_BF16X3
  int nst = 3;                    // pipeline stages
  int order = 0;                  // tile order (ctq_eval_opts.tile_order)
  uint64_t timeout_ns = 0;
  float* zbuf = nullptr;          // scratch: 2 x (hi, lo) Z buffers
  size_t zfloats = 0;             // floats of one Z plane
  unsigned* bar = nullptr;        // grid barrier: count, generation
  unsigned char* state = nullptr; // two copies of the per-string row-tile state of the product schedule
};

// Per-impurity parameters and scratch of the float64 large-block path (trace_big64.cu).
struct Big64Params {
  const double* bt = nullptr;       // embedded float64 blocks, row-major, per (alpha, q)
  const float* bt_x2 = nullptr;     // the same as two-float pairs (CTQ_F32X2), same element offsets
  const int64_t* bt_off = nullptr;  // [n_alpha * n_sec] element offsets, -1 absent
  uint64_t timeout_ns = 0;
  double* zbuf = nullptr;           // scratch: two Z buffers
  size_t zelems = 0;                // elements of one Z buffer
  unsigned* bar = nullptr;          // grid barrier: count, generation
  int* ekey = nullptr;              // [max_ops + 2] max exponent field per operator
  double* fr = nullptr;             // [max_ops + 2] ||Z||^2 per operator
  double* part = nullptr;           // [2 * grid] final-trace partial sums
  int* abort_flag = nullptr;
  int order = 0;                    // tile order (ctq_eval_opts.tile_order)
};

// Density-matrix estimator (density.cu).
struct RhoParams {
  double* rho = nullptr;            // [C x rho_elems] per-chain estimator, sector blocks
  size_t rho_elems = 0;             // doubles per chain (complex: two per element)
  const int64_t* rho_off = nullptr; // [n_sec] element offset of each sector block (sum of d^2 before it)
  void* scratch = nullptr;          // per-CTA storage of the forward products
  size_t scratch_elems = 0;         // elements (real or complex) per CTA
  int local_acc = 0;                // estimator summed in shared memory per string
  size_t h_len = 0;                 // static ratios: operator slots of the output (pairs)
};
size_t rho_elems(const HostModel& h);
size_t rho_scratch_bytes(const HostModel& h, int max_ops, int grid);
int rho_grid(const DevModel& M, int num_sms, int max_ops, size_t rho_doubles);
int prepare_rho(int optin);
int launch_rho(const DevModel& M, int num_sms, int optin, const BatchView& B, const EvalCfg& cfg, const Work& W,
               const ctq_result& R, RhoParams P, size_t rho_total_doubles, void* stream, bool hst = false);

// Static improved-estimator ratios h^st = w^U / w (improved.cu).
int launch_static_ratios(int m, const int* chain, int n_chains, const double* log_abs, const double* phase,
                         const double* log_abs_u, const double* phase_u, double* h, void* stream);

size_t big64_block_elems(int dn, int dk);
int format_big64_blocks(const HostModel& h, const double* d_blk, void* out, const std::vector<int64_t>& off, bool x2);
size_t big64_scratch_bytes(const HostModel& h, int max_ops, int grid);
int prepare_eval_big64(int num_sms, LaunchCfg* lc);
int launch_eval_big64(const DevModel& M, const LaunchCfg& lc, Big64Params P, const BatchView& B, const EvalCfg& cfg,
                      const Work& W, const ctq_result* R, void* scratch, void* stream, void* const* events,
                      bool x2 = false);
bool fp64_shared_kernel_fits(const DevModel& M, int optin);

size_t big_block_elems(int dn, int dk);
int format_big_blocks(const HostModel& h, const double* d_blk, void* out, const std::vector<int64_t>& off, int prec);
size_t big_scratch_bytes(const HostModel& h, int max_ops, int grid);
int prepare_eval_big(int prec, int num_sms, LaunchCfg* lc);
int launch_eval_big(const DevModel& M, const LaunchCfg& lc, BigParams P, const BatchView& B, const EvalCfg& cfg,
                    const Work& W, const ctq_result* R, void* scratch, void* stream, void* const* events);

// Launchers (trace_fp64.cu, trace_tc.cu).  Return a CTQ_* status.
int build_tc_blocks(const HostModel& h, int prec, std::vector<unsigned char>& out, std::vector<int64_t>& off,
                    int* stage_bytes);
int prepare_eval_tc(const DevModel& M, int prec, int stage_bytes, int num_sms, LaunchCfg* lc);
int launch_eval_tc(const DevModel& M, const LaunchCfg& lc, const TcParams& P, const BatchView& B,
                   const EvalCfg& cfg, const Work& W, const ctq_result* R, void* stream, void* const* events);
int prepare_eval_fp64(const DevModel& M, int num_sms, LaunchCfg* lc);
int launch_eval_fp64(const DevModel& M, const LaunchCfg& lc, const BatchView& B, const EvalCfg& cfg,
                     const Work& W, const ctq_result* R, void* stream, void* const* events, bool x2 = false);

}  // namespace ctq
