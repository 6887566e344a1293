/*
 * ctq.h -- C ABI of the GB300 local-trace library (libctq.so).
 *
 * The library evaluates the CT-HYB local trace of arXiv 2010.08482,
 * Eq. pweight1 in the sector form of Sec. 3.3.1 ("Computing the local
 * impurity trace"):
 *
 *   w(C) = sum_{q0} Tr P_{beta - tau_n}(q_n) F_{alpha_n}(q_{n-1}) ...
 *                      F_{alpha_1}(q0) P_{tau_1}(q0),
 *
 * for batches of already time-ordered operator sequences, on one GPU, with
 * the lazy-trace norm bounds (Sec. 3.3.1, lazy-trace paragraph) for early
 * rejection.  The time-ordering permutation sign is the caller's
 * (Sec. 3.3.1 states the product after T_tau has been applied).
 *
 * Conventions for every entry point:
 *   - return 0 (CTQ_OK) on success, a negative CTQ_ERR_* code otherwise;
 *     no C++ exception crosses the ABI; ctq_strerror() names the code.
 *   - the library never frees caller buffers; objects it creates are freed
 *     by the matching ctq_free_* call.
 *   - "device" pointers are CUDA global-memory pointers on the impurity's
 *     device; "host" pointers are ordinary CPU memory.
 *   - operator code alpha = 2*f + dag (dag = 1: c^dagger), flavour f in the
 *     paper's order: all spin-down orbitals, then all spin-up (App. A,
 *     Eqs. enumProduct / enumCoupled).  After ctq_add_bulla_operators the
 *     codes 2*n_flav + f name the Bulla operators [c_f, U].
 */
#ifndef CTQ_H
#define CTQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes returned by the entry points ---------------------------- */
#define CTQ_OK 0
#define CTQ_ERR_ARG (-1)         /* invalid argument (null, size, value)        */
#define CTQ_ERR_NOMEM (-2)       /* host or device allocation failed            */
#define CTQ_ERR_CUDA (-3)        /* a CUDA runtime call failed                  */
#define CTQ_ERR_TIMEOUT (-4)     /* a bounded device wait expired               */
#define CTQ_ERR_UNSUPPORTED (-5) /* combination not built (e.g. precision)      */
#define CTQ_ERR_NUMERIC (-6)     /* eigensolver did not converge                */
#define CTQ_ERR_WORKSPACE (-7)   /* workspace smaller than ctq_workspace_size() */

/* ---- per-chain status written by ctq_eval_traces -------------------------- */
#define CTQ_CHAIN_OK 0             /* trace computed; no decision requested    */
#define CTQ_CHAIN_ZERO 1           /* no surviving q0, or the trace is exactly 0 */
#define CTQ_CHAIN_REJECTED_EARLY 2 /* bound below threshold: trace not finished */
#define CTQ_CHAIN_ACCEPTED 3       /* full trace, log|w| >= threshold           */
#define CTQ_CHAIN_REJECTED 4       /* full trace, log|w| <  threshold           */
#define CTQ_CHAIN_ERR_ARG (-1)     /* malformed sequence (see ctq_batch)        */
#define CTQ_CHAIN_ERR_TIMEOUT (-4) /* a bounded device wait expired: no result  */

/* ---- ctq_eval_opts.debug_flags ------------------------------------------- */
#define CTQ_DEBUG_STALL_WAIT 1 /* tensor-core kernels first wait on an event that
                                  never happens (bounded by timeout_ns), to test
                                  the timeout path; every chain then reports
                                  CTQ_CHAIN_ERR_TIMEOUT */

/* ---- enums ------------------------------------------------------------------ */
#define CTQ_KANAMORI 0 /* U, U' = U - 2J, J (rotationally invariant Kanamori)    */
#define CTQ_SLATER 1   /* Slater-Condon, F0 = U, J fixes F2, F4 (, F6)            */

#define CTQ_MU_GIVEN 0        /* mu as given                                      */
#define CTQ_MU_PH_SYMMETRIC 1 /* mu such that E_gs(n0 - 1) = E_gs(n0 + 1)         */

#define CTQ_SECTORS_N_SZ 0 /* sectors labelled by (N_down, N_up)                 */
#define CTQ_SECTORS_N 1    /* sectors labelled by N                               */

#define CTQ_FP64 0   /* all products in float64                                  */
#define CTQ_TF32 1   /* tensor-core TF32 products, FP32 accumulation             */
#define CTQ_BF16X3 2 /* three-term bf16 split products, FP32 accumulation        */
#define CTQ_TF32X3 3 /* three-term tf32 split products, FP32 accumulation        */
#define CTQ_F32X2 4  /* two-float (hi + lo float32, ~48-bit) products on the FP32
                        pipe; propagators, log scale and final sum in float64   */

/*
 * Local-Hamiltonian parameters (Eq. ImpurityHamiltonian, Sec. 2.1):
 *   H = sum_ij c+_i (t_ij - mu delta_ij) c_j + 1/2 sum_ijkl U_ijkl c+_i c+_j c_k c_l.
 * n_orb orbitals, n_f = 2 n_orb flavours.  interaction = CTQ_KANAMORI uses a
 * generic orbital basis; CTQ_SLATER uses the real-harmonic product basis of
 * App. A with l = 2 (d) or 3 (f).  soc_xi adds xi l.s (Slater shells).  cf_re /
 * cf_im (host, n_f x n_f row-major, nullable) add an Hermitian one-body term
 * t_ij in the flavour basis.  n_min / n_max (-1: none) truncate the Hilbert
 * space to N in [n_min, n_max]; an operator leaving the window maps to the
 * zero sector.  device: CUDA ordinal that receives the blocks (-1: host only,
 * ctq_eval_traces then fails with CTQ_ERR_ARG).
 */
typedef struct {
  int n_orb;
  int l;
  int interaction;
  double U, J;
  int mu_mode;
  double mu;
  int n0;
  double soc_xi;
  const double* cf_re;
  const double* cf_im;
  int sector_mode;
  int n_min, n_max;
  int device;
} ctq_model_params;

typedef struct ctq_impurity ctq_impurity;

typedef struct {
  int n_flav;      /* flavours (spin-orbitals)                              */
  int n_sec;       /* sectors                                               */
  int max_dim;     /* largest sector dimension                              */
  int is_complex;  /* 1 if the blocks are complex                           */
  double mu;       /* chemical potential used                               */
  double E_gs;     /* ground-state energy (mu included)                     */
  int64_t n_block_elems; /* total elements over all nonzero blocks          */
  int n_alpha;     /* operator codes: 2 n_flav, or 3 n_flav with the Bulla
                      operators (ctq_add_bulla_operators)                    */
} ctq_info;

/*
 * Build the sector-decomposed impurity (Sec. 3.2 "Structure", phase (1):
 * decompose the Hilbert space into invariant spaces, diagonalise each, build
 * the operator matrices in the eigenbasis; Sec. 3.3.1 sector map s_alpha(q)).
 * Host work, then an upload of the blocks to p->device.  *out is owned by the
 * library (free with ctq_free_impurity).  Errors: CTQ_ERR_ARG (bad params),
 * CTQ_ERR_NUMERIC, CTQ_ERR_NOMEM, CTQ_ERR_CUDA.
 */
int ctq_build_impurity(const ctq_model_params* p, ctq_impurity** out);

/*
 * Load an impurity given directly in its eigenbasis (all host arrays, copied):
 *   dims[n_sec], N[n_sec] (particle number per sector),
 *   energies: sum(dims) float64, sector by sector, ascending within a sector,
 *   s_table[(2 n_flav) x n_sec] int32: target sector of alpha on q, or -1,
 *   blocks_re / blocks_im: every nonzero block F_alpha(q) (d_{s(q)} x d_q,
 *     row-major, <m(q')|c_alpha|n(q)>) concatenated in (alpha, q) order;
 *     blocks_im may be NULL for a real impurity,
 *   opnorm (nullable): ||F_alpha(q)||_2 per (alpha, q) in the same order;
 *     NULL: estimated by power iteration and inflated by 1e-9 relative.
 * Same ownership and errors as ctq_build_impurity.
 */
int ctq_load_impurity(int n_flav, int n_sec, const int* dims, const int* N, const double* energies,
                      const int* s_table, const double* blocks_re, const double* blocks_im,
                      const double* opnorm, double mu, int device, ctq_impurity** out);

/*
 * Add the Bulla operators B_f = [c_f, U] of the improved estimator for the
 * self-energy (Sec. 2.4, Eq. ImprCorrFunc and Eq. PImprovedEstimatorStatic:
 * the static ratio h^st replaces one annihilator c_f(tau) of a configuration
 * by [c_f, U](tau), U the interaction part of H_loc) as operator codes
 * 2 n_flav + f, f = 0 .. n_flav - 1.  Their blocks are formed on the host in
 * the impurity's eigenbasis from the identity
 *   <m|[c_f, U]|n> = <m|c_f|n> (E_n - E_m) - sum_j h_fj <m|c_j|n>,
 * with h = t - mu the one-body part of H_loc (Eq. ImpurityHamiltonian):
 * h_re / h_im (host, n_flav x n_flav row-major, flavour basis; h_im nullable)
 * or, when both are NULL, the matrix ctq_build_impurity used (an impurity
 * from ctq_load_impurity then fails with CTQ_ERR_ARG).  B_f maps each sector
 * where c_f does, so its sector map equals that of c_f; a one-body term that
 * links sectors differently is CTQ_ERR_UNSUPPORTED.  Block norms for the
 * lazy bounds: power iteration up to 400 x 400, the Frobenius norm above.
 * Every device copy of the impurity is then rebuilt (blocks and
 * precision-specific operand formats; ~1.5x the block memory), so no
 * evaluation on this impurity may be in flight.  Once per impurity (a second
 * call is CTQ_ERR_ARG).  Errors: CTQ_ERR_ARG, CTQ_ERR_UNSUPPORTED,
 * CTQ_ERR_NOMEM, CTQ_ERR_CUDA; after a device error the impurity has no
 * device copy and must be freed.
 */
int ctq_add_bulla_operators(ctq_impurity* imp, const double* h_re, const double* h_im);

int ctq_impurity_info(const ctq_impurity* imp, ctq_info* out);

/*
 * Copy sector data to host arrays (each nullable): dims[n_sec], N[n_sec],
 * E_min[n_sec], s_table[(2 n_flav) x n_sec] (the c / c+ codes; a Bulla
 * operator 2 n_flav + f maps sectors as c_f, code 2 f, does).
 */
int ctq_get_sectors(const ctq_impurity* imp, int* dims, int* N, double* E_min, int* s_table);

/* Energies of sector q (host, dims[q] float64, ascending, mu included). */
int ctq_get_energies(const ctq_impurity* imp, int q, double* E);

/*
 * Copy block F_alpha(q) to host arrays re / im (d_{s(q)} x d_q row-major; im
 * nullable, zero-filled for real impurities when given).  CTQ_ERR_ARG if the
 * block is zero (s_alpha(q) = -1).
 */
int ctq_get_block(const ctq_impurity* imp, int alpha, int q, double* re, double* im);

/*
 * A batch of time-ordered operator sequences (device pointers, caller-owned):
 *   offsets[n_chains + 1] int32, nondecreasing; chain c owns entries
 *     offsets[c] .. offsets[c+1]-1 of tau and op,
 *   tau   float64, strictly increasing within a chain, in [0, beta),
 *   op    int32 alpha codes in [0, n_alpha) (ctq_info.n_alpha),
 *   log_threshold[n_chains] float64 (nullable): Metropolis threshold
 *     T = log r + log|w_old| - log(other ratios), the random number r drawn
 *     first (App. B, Eq. decide); accept iff log|w| >= T.
 * A chain that breaks these rules gets status CTQ_CHAIN_ERR_ARG.
 */
typedef struct {
  int n_chains;
  double beta;
  const int32_t* offsets;
  const double* tau;
  const int32_t* op;
  const double* log_threshold;
} ctq_batch;

/*
 * precision: CTQ_FP64 (any impurity).  CTQ_TF32 and CTQ_TF32X3 run on the
 *   tensor cores: real impurities with sector blocks <= 112 states use the
 *   small-block kernel, any other impurity with blocks <= 3072 states the
 *   large-block kernel (complex blocks in their real embedding).  CTQ_BF16X3
 *   (bf16 hi / lo operands, hi*hi + hi*lo + lo*hi) runs on both kernels.
 *   CTQ_F32X2 runs the float64 kernel of the impurity (shared-memory or
 *   large-block) with two-float block products.
 *   Other combinations: CTQ_ERR_UNSUPPORTED.
 * lazy: 1 = stop a chain as soon as its upper bound falls below its threshold
 *   (needs log_threshold).  segment: operators per bound refinement (>= 1).
 * max_ops: largest 2k in the batch (sizes the bounds output).
 * timeout_ns: limit for bounded device waits (0: library default).
 * timing_events (nullable): ctq_launches_per_eval() + 1 cudaEvent_t handles,
 *   recorded on `stream` before the first kernel and after each kernel, so a
 *   caller can time every kernel of the evaluation on its launching stream.
 *   While `stream` is being captured into a CUDA graph they are captured as
 *   event-record nodes (cudaEventRecordExternal), recorded on every replay.
 * debug_flags: 0, or CTQ_DEBUG_STALL_WAIT (test of the timeout path).
 * Launch tuning (0 everywhere = library defaults; the package's autotuner
 * picks them per impurity, precision and batch shape):
 *   threads_per_cta: FP64 and two-float kernel, 32 to 512 in steps of 32;
 *   ctas_per_sm: upper bound on the resident CTAs per SM of the FP64 and
 *     small-block trace kernels;
 *   stages: large-block kernel pipeline stages, >= 2 and as many as fit in
 *     shared memory (CTQ_ERR_UNSUPPORTED otherwise);
 *   tile_order: large-block kernel tile order, 0 the library default
 *     (row-major for the tensor-core kernel, whose products overlap row tile
 *     by row tile; column-major for the float64 one), 1 column-major (a B
 *     tile is shared by consecutive CTAs), 2 row-major, 3 groups of 8 column
 *     tiles row by row.
 * Out-of-range values: CTQ_ERR_ARG.
 * When a bounded wait expires, every chain of the call gets
 * CTQ_CHAIN_ERR_TIMEOUT (log_abs NaN); the context stays usable.
 */
typedef struct {
  int precision;
  int lazy;
  int segment;
  int max_ops;
  int64_t timeout_ns;
  void* const* timing_events;
  int32_t debug_flags;
  int32_t threads_per_cta;
  int32_t ctas_per_sm;
  int32_t stages;
  int32_t tile_order;
} ctq_eval_opts;

/*
 * Results (device pointers, caller-owned):
 *   log_abs[n_chains]  log|w| with every energy shift undone (-inf if w = 0,
 *                      NaN if not evaluated),
 *   phase[2 n_chains]  (re, im) of w/|w| (real impurities: (+-1, 0)),
 *   status[n_chains]   CTQ_CHAIN_*,
 *   bounds (nullable)  [n_chains x (n_seg + 1)], n_seg = ceil(max_ops/segment):
 *                      column 0 the level-0 bound log B, column s >= 1 the
 *                      refined bound after min(s*segment, 2k) operators (the
 *                      last is log sum_q0 |w_q0|); NaN where not evaluated.
 */
typedef struct {
  double* log_abs;
  double* phase;
  int32_t* status;
  double* bounds;
} ctq_result;

/* Bytes of device workspace ctq_eval_traces needs for this batch shape. */
size_t ctq_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts);

/*
 * Evaluate the local traces of a batch.  Asynchronous on `stream` (a
 * cudaStream_t; NULL = legacy default stream): only kernel launches and
 * memsets are enqueued, nothing is allocated and nothing synchronises, so the
 * call may be captured in a CUDA graph.  workspace: device memory of at least
 * ctq_workspace_size() bytes, 256-byte aligned, used only for the duration of
 * the enqueued work (calls that overlap on the GPU must not share it).
 * Errors: CTQ_ERR_ARG, CTQ_ERR_WORKSPACE, CTQ_ERR_UNSUPPORTED, CTQ_ERR_CUDA.
 */
int ctq_eval_traces(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                    const ctq_result* result, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Allocation-free variant of ctq_eval_traces, for callers that cannot provide
 * a workspace: a C or Fortran Monte Carlo driver that owns no device
 * allocator, code whose device memory belongs to another runtime's pool, or
 * code that must not call cudaMalloc on a latency-critical path (it can
 * synchronise the device).  No counterpart in the paper.
 *
 * The scratch is a file-scope device array of CTQ_STATIC_SCRATCH_BYTES inside
 * the library; every GPU that loads the library holds it until the process
 * exits.  The call allocates nothing and makes no allocating library call.
 * Batches whose ctq_workspace_size() exceeds CTQ_STATIC_SCRATCH_BYTES are
 * rejected with CTQ_ERR_WORKSPACE (ctq_last_error_message() gives the sizes).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the rest of the process;
 * make that first call before any stream capture.  A device reset
 * (cudaDeviceReset, by the caller or by another runtime in the process)
 * destroys the array together with the context, and the kept address then
 * points nowhere: do not call this entry point on a device that has been
 * reset since its first call there.  All calls share the one array: calls
 * whose work overlaps on the GPU (other streams, other threads) race on it
 * and must be serialised by the caller.  Every call re-initialises the parts of the scratch it reads.
 * Arguments, results and the other errors are those of ctq_eval_traces.
 */
#define CTQ_STATIC_SCRATCH_BYTES (32u << 20)
int ctq_eval_traces_static(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                           const ctq_result* result, void* stream);

/*
 * Incremental local trace of one configuration with a skip list of cached
 * segment products (Sec. 3.3.1, skip-list paragraph): after a local change
 * (a pair inserted or removed) only the products of the segments that
 * contain a changed operator are recomputed, about one per level of the
 * skip list (O(log k)), plus the ancestors of operators whose sector the
 * change shifted.  Products in float64 on the SIMT pipe (or on the tensor
 * cores, ctq_skiplist_set_precision), renormalised by exact powers of two;
 * operators c and c+ only (codes 2 f + dag).  An evaluation launches one
 * kernel per dependency round of its new products (two on the tensor cores:
 * the factors' formatting and the products; all strings and segments
 * together), plus one for the new leaves, one clearing their bookkeeping
 * words and one for the root traces, after a single host-to-device copy of
 * its task tables.
 *
 * ctq_skiplist_create: the handle works on imp's device, enqueues its
 *   kernels on `stream` (cudaStream_t, NULL = legacy default) and allocates
 *   its own device memory (released by ctq_skiplist_free); beta > 0; seed
 *   draws the operators' skip-list heights.  Errors: CTQ_ERR_ARG,
 *   CTQ_ERR_UNSUPPORTED (an impurity with Bulla operators), CTQ_ERR_NOMEM.
 * ctq_skiplist_set: replaces the configuration by n operators (host arrays,
 *   tau strictly increasing in [0, beta), op = 2 f + dag); no product is
 *   kept from the previous configuration.
 * ctq_skiplist_insert: adds m operators (host arrays, any order; times in
 *   [0, beta), distinct from each other and from the configuration's).
 * ctq_skiplist_remove: removes the m operators at exactly these times.
 * ctq_skiplist_evaluate: computes what the current configuration needs
 *   (cached products are reused), synchronises `stream` and returns, on the
 *   host, log|w| (-inf if w = 0) and the phase (re, im) of the raw trace of
 *   the time-ordered product, as ctq_eval_traces does, and, if stats is not
 *   NULL, the work done by this call.  Products no longer used are released.
 *   CTQ_ERR_TIMEOUT: a tensor-core product gave up one of its bounded waits
 *   (20 s); no product of that call is kept.
 * ctq_skiplist_set_precision: CTQ_FP64 (default: float64 SIMT products) or
 *   CTQ_BF16X3 (products on the tensor cores: each factor scaled to max
 *   |entry| in [1, 2), split into bf16 hi / lo, hi hi + hi lo + lo hi with
 *   FP32 accumulation folded into registers every 256 K terms, stored in
 *   float64; leaves, exponents and the root traces stay float64; products
 *   are computed on 128 x 256 tiles, so small blocks are mostly padding and
 *   the float64 products are the faster choice for them).  Changing it
 *   releases every cached product.
 *   Errors: CTQ_ERR_ARG, CTQ_ERR_UNSUPPORTED (another precision), CTQ_ERR_NOMEM.
 * Errors of set / insert / remove: CTQ_ERR_ARG (nothing changed).
 */
typedef struct ctq_skiplist ctq_skiplist;
typedef struct {
  int64_t products;      /* segment products computed by this evaluation */
  int64_t leaves;        /* leaves (propagator x block) formed */
  int64_t reused;        /* cached leaves and products found */
  int64_t cached;        /* products held after the evaluation */
  double flops;          /* real flops of the products (complex counts 4 x) */
  int n_ops;             /* operators of the configuration */
  int n_strings;         /* surviving starting sectors */
  int64_t device_bytes;  /* device memory held by the handle */
  int64_t launches;      /* kernels this evaluation launched */
  int rounds;            /* dependency rounds of its products */
} ctq_skiplist_stats;
int ctq_skiplist_create(const ctq_impurity* imp, double beta, uint64_t seed, void* stream, ctq_skiplist** out);
int ctq_skiplist_set(ctq_skiplist* sl, int n, const double* tau, const int32_t* op);
int ctq_skiplist_insert(ctq_skiplist* sl, int m, const double* tau, const int32_t* op);
int ctq_skiplist_remove(ctq_skiplist* sl, int m, const double* tau);
int ctq_skiplist_evaluate(ctq_skiplist* sl, double* log_abs, double* phase, ctq_skiplist_stats* stats);
int ctq_skiplist_set_precision(ctq_skiplist* sl, int precision);
void ctq_skiplist_free(ctq_skiplist* sl);

/*
 * Static part of the improved estimator for the self-energy (Sec. 2.4,
 * Eq. PImprovedEstimatorStatic): h^st_i = w^U_i / w_loc(C_{chain[i]}) from
 * the results of two ctq_eval_traces calls, one on the configurations
 * (n_chains entries of log_abs / phase) and one on m sequences, each a
 * configuration with one annihilator c_f replaced by its Bulla operator
 * (code 2 n_flav + f; log_abs_u / phase_u).  All device pointers, on the
 * current device: chain[m] int32, the configuration of each sequence;
 * h[2 m] float64 out, (re, im) pairs.  An entry is NaN when its
 * configuration has w = 0, was rejected or failed (log_abs -inf or NaN), its
 * sequence failed, or chain[i] is outside [0, n_chains); w^U = 0 gives 0.
 * One kernel, asynchronous on `stream` (cudaStream_t), graph-capturable.
 * Errors: CTQ_ERR_ARG (m < 0, n_chains < 0, a NULL pointer with m > 0),
 * CTQ_ERR_CUDA.
 */
int ctq_static_ratios(int m, const int32_t* chain, int n_chains, const double* log_abs, const double* phase,
                      const double* log_abs_u, const double* phase_u, double* h, void* stream);

/*
 * The same ratios for every annihilator of every configuration in one pass
 * (Sec. 2.4, Eq. PImprovedEstimatorStatic), without replaced sequences: after
 * the float64 trace evaluation of the batch (ctq_eval_traces, results in
 * `result`), the forward products A_i and backward products Y_i of each
 * surviving string (those of the density-matrix estimator) give
 *   w^U_i = Tr[ Y_i Q_i P_{Delta_i} A_i ]
 * for the annihilator at operator i replaced by Q_i = [c_f, U], one product
 * per annihilator instead of a trace of a replaced sequence.  The impurity
 * must hold the Bulla operators (ctq_add_bulla_operators).
 * h: device float64 [2 n_ops], n_ops = offsets[n_chains] (the batch's total
 * operator count): entry 2 k, 2 k + 1 is h^st (re, im) of the operator with
 * global index k when it is an annihilator (code 2 f), 0 otherwise; every
 * entry of a chain whose status is not CTQ_CHAIN_OK is 0.  Writes beyond
 * n_ops are skipped.  CTQ_FP64 without lazy rejects, blocks that fit the
 * shared-memory kernel (CTQ_ERR_UNSUPPORTED otherwise).  Workspace:
 * ctq_static_ratio_workspace_size() bytes, 256-byte aligned.  Asynchronous on
 * `stream`; enqueues the trace evaluation, one memset and the ratio kernel.
 * Errors: CTQ_ERR_ARG, CTQ_ERR_WORKSPACE, CTQ_ERR_UNSUPPORTED, CTQ_ERR_CUDA.
 */
size_t ctq_static_ratio_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts);
int ctq_eval_static_ratios(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                           const ctq_result* result, double* h, int n_ops, void* workspace, size_t workspace_bytes,
                           void* stream);

/*
 * Number of kernels one ctq_eval_traces call enqueues (for launch accounting).
 */
int ctq_launches_per_eval(const ctq_impurity* imp, const ctq_eval_opts* opts);

/*
 * Which trace kernel ctq_eval_traces runs for this impurity and precision:
 * CTQ_KERNEL_FP64_SHARED (float64, blocks in shared memory),
 * CTQ_KERNEL_FP64_LARGE (float64, persistent large-block kernel),
 * CTQ_KERNEL_TC_SMALL (tensor cores, running product in tensor memory),
 * CTQ_KERNEL_TC_LARGE (tensor cores, persistent large-block kernel), or a
 * negative CTQ_ERR_* code when the combination is not built.  Host only.
 */
#define CTQ_KERNEL_FP64_SHARED 0
#define CTQ_KERNEL_FP64_LARGE 1
#define CTQ_KERNEL_TC_SMALL 2
#define CTQ_KERNEL_TC_LARGE 3
int ctq_trace_kernel(const ctq_impurity* imp, int precision);

/*
 * Reduced-density-matrix estimator (Sec. 2.3, Eq. ImpurityDensityMatrix):
 * for every chain C,
 *   rho^C_{uv} = beta^{-1} int_0^beta w_loc(C, |v><u|(tau)) / w_loc(C) dtau
 * with u, v eigenstates of the same sector, the tau integral taken in closed
 * form over every propagation interval.  float64, impurities whose blocks
 * fit the shared-memory FP64 kernel (CTQ_ERR_UNSUPPORTED otherwise).
 *
 * ctq_density_size: doubles of one chain's estimator: the sector blocks
 *   d_q x d_q, row-major (u row, v column), in sector order; complex
 *   impurities store (re, im) pairs.
 * ctq_density_workspace_size: workspace bytes for n_chains chains (the trace
 *   evaluation's workspace plus per-CTA storage of the forward products).
 * ctq_eval_density_matrices: evaluates the traces exactly as ctq_eval_traces
 *   with CTQ_FP64 (result: log|w|, phase, status; bounds nullable) and then
 *   writes rho (device, caller-owned, n_chains x ctq_density_size doubles).
 *   Chains with w = 0, rejected or invalid chains get an all-zero estimator.
 *   opts->precision must be CTQ_FP64 and opts->lazy 0.  Asynchronous on
 *   `stream`.  Errors: as ctq_eval_traces.
 */
size_t ctq_density_size(const ctq_impurity* imp);
size_t ctq_density_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts);
int ctq_eval_density_matrices(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                              const ctq_result* result, double* rho, void* workspace, size_t workspace_bytes,
                              void* stream);

void ctq_free_impurity(ctq_impurity* imp);

/*
 * Measures the sustained fused-multiply-add rate of one arithmetic pipe on
 * `device` (kind 0: float64 FMA, 1: float32 FMA, 8 independent chains per
 * thread; kind 2: the float64 warp-level MMA mma.sync.m8n8k4.f64, 8
 * independent accumulators per warp, 256 multiply-adds per instruction),
 * 8 CTAs of 256 threads per SM.  *flops_per_s receives 2 x multiply-adds /
 * second.  Allocates and frees a small device buffer; synchronises the
 * device.  No counterpart in the paper: it states the arithmetic roofline of
 * the small-block trace.  Errors: CTQ_ERR_ARG, CTQ_ERR_NOMEM, CTQ_ERR_CUDA.
 */
int ctq_probe_fma_rate(int device, int kind, int iters, double* flops_per_s);

/*
 * Accuracy hook of the propagators' exponential: for the n host values x[i]
 * (the propagator arguments -dtau (E - E_min) <= 0), computes on `device`
 * y_table[i] = the table-driven e^x the float64 trace kernel uses (Tang's
 * method, 64 entries) and y_lib[i] = the CUDA library's exp(x[i]), both
 * written to host arrays of n doubles owned by the caller.  Allocates and
 * frees device buffers and synchronises.  No counterpart in the paper.
 * Errors: CTQ_ERR_ARG, CTQ_ERR_NOMEM, CTQ_ERR_CUDA.
 */
int ctq_probe_exp(int device, int n, const double* x, double* y_table, double* y_lib);

/*
 * Diagnostic of the small-block kernel's tensor-core operand conventions
 * (every precision): computes D = A B^T on `device` with one tcgen05 MMA sequence
 * (A: host 128 x K row-major floats, placed in tensor memory; B: host N x K
 * row-major floats, staged in shared memory as K-major core matrices; D: host
 * 128 x N row-major floats), split = CTQ_TF32, CTQ_TF32X3 or CTQ_BF16X3
 * (the split modes: hi*hi + hi*lo + lo*hi).
 * N in [16, 112] and K in [16, 112], both multiples of 16.  Allocates and frees
 * device buffers and synchronises.  No counterpart in the paper.
 * Errors: CTQ_ERR_ARG, CTQ_ERR_NOMEM, CTQ_ERR_CUDA, CTQ_ERR_TIMEOUT.
 */
int ctq_tc_gemm_check(int device, const float* A, const float* B, float* D, int N, int K, int split);

/*
 * Diagnostic of the large-block kernel's operand conventions: D = A B^T with
 * A (host 128 x K row-major floats) and B (host N x K row-major floats) split
 * and tiled on the device like the running product and the embedded blocks,
 * staged chunk by chunk with bulk copies, and multiplied with the same
 * descriptors and MMA kinds (precision CTQ_TF32, CTQ_TF32X3 or CTQ_BF16X3);
 * D: host 128 x N row-major floats.  N in [16, 128], multiple of 16; K in
 * [64, 4096], multiple of 64.  Allocates and frees device buffers and
 * synchronises.  No counterpart in the paper.
 * Errors: CTQ_ERR_ARG, CTQ_ERR_NOMEM, CTQ_ERR_CUDA, CTQ_ERR_TIMEOUT.
 */
int ctq_big_gemm_check(int device, const float* A, const float* B, float* D, int N, int K, int precision);

const char* ctq_strerror(int code);

/* Message of the last failing call on this host thread ("" if none). */
const char* ctq_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* CTQ_H */
