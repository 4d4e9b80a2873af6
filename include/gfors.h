/*
 * gfors.h -- C ABI of the B300 (sm_103a) GFORS hot path.
 *
 * GFORS (arXiv 2510.27117) attacks the binary integer program of Eq. (1)
 *
 *     min  <x, Qx> + <c, x>   s.t.  A x >= b,  B x = d,  x in {0,1}^n
 *
 * by running the PDHG update of Alg. 2 on the penalised saddle form Eq. (2)
 * (K = -[A;B], r = (b;d), y = (u,v), u >= 0, penalty rho <x, 1-x>) and, every
 * k_int iterations, drawing k_r rounds of k_b binary candidates from the
 * current iterate (Alg. 3 and the customised samplers of Section 2.4.2),
 * scoring them on the original data and keeping the best feasible one
 * (EvalBest of Alg. 1).
 *
 * Conventions shared by every call:
 *  - Matrices cross the boundary as HOST CSR (int64 row pointers, int32
 *    column indices, double values), borrowed for the duration of the call
 *    and copied.  Duplicate entries are summed.
 *  - A handle owns all device memory of one batch of instances.  Instances
 *    are independent; they share one device launch per kernel (the batch is
 *    laid out block-diagonally in HBM).
 *  - Work is enqueued asynchronously on the handle's CUDA stream.  Calls that
 *    return host data (gfors_incumbent, gfors_lp_stats, gfors_get_*,
 *    gfors_eval_candidates, gfors_state_export, gfors_run) synchronise it.
 *  - Errors are status codes; nothing throws across the ABI.  A CUDA error or
 *    a device wait that ran out of time marks the handle failed: later calls
 *    return GFORS_E_STATE until gfors_destroy.  gfors_last_error() explains.
 *  - One handle per host thread at a time; handles are not thread-safe.
 *  - The library never falls back to the CPU.  It needs an sm_103a device.
 */
#ifndef GFORS_H
#define GFORS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GFORS_API __attribute__((visibility("default")))
#else
#define GFORS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfors_ctx* gfors_handle;

typedef enum {
  GFORS_OK = 0,
  GFORS_E_ARG = 1,         /* bad argument or malformed / infeasible input   */
  GFORS_E_CUDA = 2,        /* a CUDA runtime call failed                     */
  GFORS_E_OOM = 3,         /* device allocation failed                       */
  GFORS_E_TIMEOUT = 4,     /* a bounded device-side wait gave up             */
  GFORS_E_STATE = 5,       /* handle failed earlier, or call out of order    */
  GFORS_E_UNSUPPORTED = 6  /* valid input this build does not handle         */
} gfors_status;

/* Sparse matrix in CSR form, host memory, borrowed. */
typedef struct {
  int64_t rows, cols, nnz;
  const int64_t* row_ptr; /* rows + 1 entries, row_ptr[0] = 0             */
  const int32_t* col_idx; /* nnz entries in [0, cols)                      */
  const double* val;      /* nnz entries                                   */
} gfors_csr;

/* Q of Eq. (1): kind 0 = none (Q = 0), 1 = dense row-major n x n host
 * array, 2 = CSR.  Q need not be symmetric: the gradient uses (Q + Q^T)/2
 * (Eq. 1 assumes symmetry without loss of generality); scoring uses x^T Q x. */
typedef struct {
  int32_t kind;
  const double* dense_rowmajor;
  gfors_csr sparse;
} gfors_qmat;

/* Parameters (Alg. 1, Section 3).  gfors_default_params() fills the
 * defaults named in the comments. */
typedef struct {
  double sigma;        /* tau1 tau2 <= sigma after Preprocess (Sec. 3); 0.99 */
  double rho_min;      /* UpdatePenalty (Sec. 3); 1e-3                      */
  double rho_max;      /* 1.0                                               */
  double T;            /* 20                                                */
  double p;            /* 2                                                 */
  double delta;        /* minimum increment; 0                              */
  int32_t k_int;       /* sampling interval (Alg. 1); 50                    */
  int32_t k_r;         /* sampling rounds per trigger; 1                    */
  int32_t k_b;         /* candidates per round; 1024 (multiple of 32)       */
  int32_t tau_cap_by_L;/* -1 auto (on iff Q != 0), 0 off, 1 on: tau1 <=
                          1/(2L), L = 2(||Q||+rho) (Eq. 2, Prop. 2)          */
  uint64_t seed;       /* Philox key                                        */
  double x0;           /* start point: value in [0,1] = constant vector;
                          negative = Philox uniform draws                   */
  double halt_tol;     /* CheckHalt tolerance; 1e-4                         */
  int32_t stall_window;/* CheckHalt stall window in triggers; 20            */
  int32_t inst_base;   /* Philox instance id of the batch's first instance  */
  int32_t sample_chunk;/* candidates evaluated per device pass (memory cap,
                          the role Sec. 2.1 gives k_b); 0 = k_b              */
  int32_t eval_mode;   /* 0 auto, 1 materialised bits, 2 fused sample+eval
                          (single-row instances), 3 dense tensor-core
                          scoring (dense small-integer Q), 4 dense scoring
                          on CUDA cores (checking), 5 the same as 3,
                          6 tensor-core scoring with bf16 operands (auto
                          uses FP8 E4M3 operands when every entry of
                          offdiag(Q+Q^T) is exact in E4M3)                  */
  double power_tol;    /* power-iteration stop tolerance; 1e-12            */
  int32_t power_maxit; /* power-iteration cap; 5000                         */
  double wait_timeout_s;/* limit of every device-side wait; 2.0             */
  int32_t pdhg_mode;   /* 0 auto: one persistent cooperative launch per call
                          for a single dense instance that fits shared
                          memory; one block per instance for instances whose
                          matrix fits a block's shared memory (one
                          thread-block cluster of 16 or 8 CTAs per instance
                          when every instance's cluster fits one wave); the
                          fused one-row kernels for batches of one-row
                          instances; otherwise CUDA graphs of per-iteration
                          launches.  1 per-iteration launches only.  2 as 0,
                          plus one cooperative launch per call for sparse
                          problems that fit the L2 cache.  3 as 0 without
                          the clusters (one block per instance)            */
} gfors_params;

GFORS_API void gfors_default_params(gfors_params* prm);
GFORS_API const char* gfors_version(void);

/* Device allocation hook (optional).  When set, every device buffer of a
 * later gfors_load* comes from alloc(size, ctx) and returns via free(ptr,
 * ctx); alloc returning NULL yields GFORS_E_OOM.  NULL functions restore
 * cudaMalloc / cudaFree. */
typedef void* (*gfors_alloc_fn)(size_t size, void* ctx);
typedef void (*gfors_free_fn)(void* ptr, void* ctx);
GFORS_API gfors_status gfors_set_allocator(gfors_alloc_fn alloc, gfors_free_fn free_fn,
                                 void* ctx);

/* Load one instance (Eq. 1) and run Preprocess (Section 3): K = -[A;B] rows
 * divided by their 2-norms, Q and c divided by ||Q||_2 + ||c||_2, K and r
 * divided by ||K||_2; the two spectral norms come from FP64 power
 * iterations on the device.  A and/or B may be NULL (m1 = 0 / m2 = 0), Q may
 * be NULL (Q = 0).  b has A->rows entries, d has B->rows, c has n.
 * cuda_stream: the cudaStream_t all of the handle's work is enqueued on
 * (NULL: the handle creates and owns a non-blocking stream).
 * Infeasible empty rows and malformed CSR give GFORS_E_ARG. */
GFORS_API gfors_status gfors_load(const gfors_csr* A, const double* b, const gfors_csr* B,
                        const double* d, const gfors_qmat* Q, const double* c,
                        int64_t n, const gfors_params* prm, void* cuda_stream,
                        gfors_handle* out);

/* Batch of ninst independent instances in one handle (arrays of per-instance
 * pointers; A[i]/B[i]/Q[i] entries may be NULL).  Instance i uses Philox
 * instance id prm->inst_base + i, so a batch reproduces single-instance runs
 * bit for bit. */
GFORS_API gfors_status gfors_load_batch(int32_t ninst, const gfors_csr* const* A,
                              const double* const* b, const gfors_csr* const* B,
                              const double* const* d, const gfors_qmat* const* Q,
                              const double* const* c, const int64_t* n,
                              const gfors_params* prm, void* cuda_stream,
                              gfors_handle* out);

/* Customised sampling (Section 2.4.2) for instance inst.
 * mode 0: plain Bernoulli (Alg. 3) for every variable.
 * mode 1: one-hot groups -- ngroups disjoint groups (grp_ptr[ngroups+1]
 *         offsets into grp_idx, variable indices) each receive exactly one 1
 *         per candidate, drawn from p restricted to the group; the other
 *         variables stay Bernoulli.
 * mode 2: axial 3D assignment over n = I^3 variables x_ijk at (i I + j) I + k;
 *         every candidate is a feasible assignment by construction.
 * Groups are copied. */
GFORS_API gfors_status gfors_set_groups(gfors_handle h, int32_t inst, int32_t mode,
                              int64_t ngroups, const int64_t* grp_ptr,
                              const int64_t* grp_idx, int32_t axial_I);

/* Algorithm 4 (customized sampling for the 3D assignment, Section 2.4.2)
 * for instance inst, n = I^3 variables x_ijk at (i I + j) I + k, 1 <= I <= 64:
 * the gamma*I largest entries of p (p descending, then index ascending) give
 * a greedy conflict-free partial assignment; every candidate completes it with
 * Fisher-Yates permutations of the free j's and k's (Philox stream 6) and
 * applies up to L best strictly improving pairwise interchanges (exchange of
 * j or of k between two triples; exact integer costs; ties to the smallest
 * (a, b, type)).  Every candidate is a feasible assignment.  Needs integral
 * costs, 0 <= gamma <= I, I * gamma * I <= 16384, L >= 0. */
GFORS_API gfors_status gfors_set_assign3d_custom(gfors_handle h, int32_t inst, int32_t I,
                                                 int32_t gamma, int32_t L);

/* Monotone relaxation (Section 2.4.3), group repair for instance inst: the
 * caller has relaxed equality groups sum_{k in G} x_k = 1 to sum >= 1 (rows
 * of A; valid when costs are non-negative); after sampling, every candidate
 * keeps, in each group, its selected member of least cost c_k (ties to the
 * member listed first) and clears the others, before the closure below.
 * Dropping a member must not be able to violate any other row (the caller's
 * claim).  grp_ptr (ngroups + 1, grp_ptr[0] = 0) / grp_idx: disjoint groups
 * of local variable indices.  Needs integral costs; GFORS_E_UNSUPPORTED on
 * a dense-Q or fused single-row batch. */
/* Monotone relaxation (Section 2.4.3), general repair for instance inst:
 * the caller has relaxed equality rows with 0/1 coefficients to covering
 * rows sum_{k in R} x_k >= 1 (rows of A; valid when costs are
 * non-negative, so dropping a selected variable never raises the
 * objective).  After sampling (and any group repair, before the closure),
 * every candidate visits its selected variables of these rows in decreasing
 * cost c_k, ties to the larger index first, and drops each one whose rows
 * all keep another selected member ("reverse delete").  The result is a
 * minimal cover of the rows the candidate covered, never more expensive;
 * on disjoint rows it keeps the cheapest selected member (ties to the lower
 * index), as gfors_set_repair_groups does.  row_ptr (nrows + 1, row_ptr[0]
 * = 0) / row_idx: local variable indices; rows may overlap.  Once per
 * instance (GFORS_E_STATE after), needs integral costs; GFORS_E_UNSUPPORTED
 * on a dense-Q or fused single-row batch.  The repair is the paper's
 * "customized repair step", read here as reverse delete. */
GFORS_API gfors_status gfors_set_repair_rows(gfors_handle h, int32_t inst, int64_t nrows,
                                             const int64_t* row_ptr, const int64_t* row_idx);

GFORS_API gfors_status gfors_set_repair_groups(gfors_handle h, int32_t inst, int64_t ngroups,
                                               const int64_t* grp_ptr, const int64_t* grp_idx);

/* Monotone relaxation with repair (Section 2.4.3) for instance inst: after
 * sampling, rep_var[q] <- rep_var[q] OR (OR of rep_idx[rep_ptr[q] ..
 * rep_ptr[q+1])).  Valid when the repaired variables have non-negative
 * cost (facility opening). */
GFORS_API gfors_status gfors_set_closure(gfors_handle h, int32_t inst, int64_t nrep,
                               const int64_t* rep_var, const int64_t* rep_ptr,
                               const int64_t* rep_idx);

/* nsteps iterations of Alg. 1's loop body without sampling: k <- k+1;
 * rho <- UpdatePenalty (the counter advances once per k_int iterations);
 * FirstOrderStep (Alg. 2).  Asynchronous. */
GFORS_API gfors_status gfors_pdhg_steps(gfors_handle h, int64_t nsteps);

/* nrounds rounds of RandSampleStep + EvalBest (Alg. 1) on every instance,
 * proposal p = x_k (proposal 0), the attached learned network (1), half of
 * each (2: the first half of every round from the network), or both (3:
 * every round draws k_b candidates from x_k -- exactly those of proposal 0
 * -- and then k_b from the network under round id | 2^31).  Round r uses
 * Philox round id first_round_id + r.  Each round scores its candidates on
 * the ORIGINAL data (violation count, objective) and updates the device
 * incumbent.  Asynchronous. */
GFORS_API gfors_status gfors_sample_eval(gfors_handle h, int32_t nrounds,
                               uint32_t first_round_id, int32_t proposal);

/* EvalBest(round(x_k)) of Alg. 1 (x_i = 1 iff x_i > 0.5), round id
 * 0xFFFFFFFF.  Asynchronous. */
GFORS_API gfors_status gfors_final_round(gfors_handle h);

/* Alg. 1 end to end: iterate until CheckHalt (Section 3) holds for every
 * instance, max_iters iterations, or time_budget_s seconds (<= 0: none);
 * then the final rounding.  Sampling triggers every k_int iterations
 * (k_r rounds each, proposal as in gfors_sample_eval).  *iters_out (may be
 * NULL) receives the iteration count.  Synchronises. */
GFORS_API gfors_status gfors_run(gfors_handle h, int64_t max_iters, double time_budget_s,
                       int32_t proposal, int64_t* iters_out);

/* Alg. 1 as ONE CUDA-graph launch, with CheckHalt (Section 3) decided on
 * the device: no host synchronisation between sampling triggers.  The body
 * of a conditional while node is one trigger: k_int PDHG iterations, k_r
 * rounds (proposal as in gfors_sample_eval), the FP64 CheckHalt sums, and a
 * one-block kernel that evaluates CheckHalt (the indicators and stall rule
 * of gfors_run), the iteration budget and, when target_obj (HOST,
 * ninst int64, may be NULL) is given, whether every instance b holds a
 * feasible incumbent with objective <= target_obj[b]; that kernel sets the
 * loop condition.  After the graph come the iterations after the last
 * trigger when the budget (not CheckHalt or the targets) ended the loop,
 * then the final rounding.  With target_obj NULL the results equal
 * gfors_run's with time_budget_s <= 0: the same iterates, candidates,
 * incumbents and halting decisions.  *iters_out and *triggers_out (may be
 * NULL) receive the iteration count and the triggers the graph ran.  Needs
 * an even k_int, the iteration count at a trigger boundary, and a PDHG path
 * without cooperative launches (not "persistent" or "cooperative" in
 * gfors_pdhg_path); otherwise GFORS_E_UNSUPPORTED.  The instantiated graph
 * is kept on the handle, one per proposal, and reused until the groups,
 * closure, repair groups or lane counts change; the budget, the first
 * trigger and the targets are read from device memory.  Synchronises. */
GFORS_API gfors_status gfors_run_graph(gfors_handle h, int64_t max_iters, int32_t proposal,
                                       const int64_t* target_obj, int64_t* iters_out,
                                       int64_t* triggers_out);
/* Build and keep that graph without running it (set-up work, e.g. before a
 * timed run); the same conditions and errors as gfors_run_graph. */
GFORS_API gfors_status gfors_run_graph_prepare(gfors_handle h, int32_t proposal);

/* Incumbent of instance inst: *found = 0/1, objective on the original data
 * (*obj_i exact for integer data, *obj_f always), the round id and sample
 * index that produced it, and x_best as n bytes (0/1) into x_out (may be
 * NULL).  Synchronises. */
GFORS_API gfors_status gfors_incumbent(gfors_handle h, int32_t inst, int32_t* found,
                             int64_t* obj_i, double* obj_f, uint32_t* round_id,
                             int32_t* sample, uint8_t* x_out);

/* Relaxation statistics of instance inst at the current iterate, FP64
 * reductions on the preprocessed problem (CheckHalt indicators, Section 3):
 * out[0] primal residual, out[1] gap (Q = 0: relative duality gap against
 * the Lagrangian dual bound; else ||s^x|| of Thm. 2), out[2] binary gap,
 * out[3] c^T x + x^T Q x (scaled), out[4] dual bound (NaN if Q != 0),
 * out[5] ||s^x_k||, out[6] rho, out[7] k.  Synchronises. */
GFORS_API gfors_status gfors_lp_stats(gfors_handle h, int32_t inst, double out[8]);

/* Scales found by Preprocess for instance inst: out[0] ||Q_sym||_2,
 * out[1] s_obj = ||Q||_2 + ||c||_2, out[2] ||K_rownormalised||_2, out[3]
 * ||Q_hat||_2, out[4] power iterations for Q, out[5] for K, out[6] tau1,
 * out[7] tau2 (current rho).  Synchronises. */
GFORS_API gfors_status gfors_get_scales(gfors_handle h, int32_t inst, double out[8]);

/* Iterate of instance inst as FP32 host arrays: x = x_k, xbar = xbar_k,
 * x_prev = x_{k-1} (n entries each), y (m1+m2 entries).  Any pointer may be
 * NULL.  Synchronises. */
GFORS_API gfors_status gfors_get_iterate(gfors_handle h, int32_t inst, float* x,
                               float* xbar, float* x_prev, float* y);

/* Overwrite the iterate of instance inst (x_k, xbar_k, y_k; x_{k-1} set to
 * x).  Any pointer may be NULL (left unchanged).  Asynchronous. */
GFORS_API gfors_status gfors_set_iterate(gfors_handle h, int32_t inst, const float* x,
                               const float* xbar, const float* y);

/* Set the iteration counter k (all instances) and the penalty rho (rho < 0:
 * keep the schedule's value); the penalty counter becomes floor(k/k_int).
 * Asynchronous. */
GFORS_API gfors_status gfors_set_counters(gfors_handle h, int64_t k, double rho);

/* Score k explicit candidates X (k x n bytes, sample-major, 0/1) of
 * instance inst on the original data with the same device evaluator that
 * sampling uses: viol[k] violation counts, obj_i[k] exact objectives
 * (integer data), obj_f[k] FP64 objectives.  The incumbent is untouched.
 * Synchronises. */
GFORS_API gfors_status gfors_eval_candidates(gfors_handle h, int32_t inst, int32_t k,
                                   const uint8_t* X, int32_t* viol,
                                   int64_t* obj_i, double* obj_f);

/* Candidates and scores of the LAST sampled chunk of instance inst:
 * X_out (chunk x n bytes, may be NULL), viol, obj_i (chunk entries, may be
 * NULL); *count receives the chunk length.  Synchronises. */
GFORS_API gfors_status gfors_get_samples(gfors_handle h, int32_t inst, uint8_t* X_out,
                               int32_t* viol, int64_t* obj_i, int32_t* count);

/* Learned proposal (an added pattern, no counterpart in the paper).
 * Weights of the per-variable MLP  h1 = relu(W1 f + b1), h2 = relu(W2 h1 +
 * b2), p = clip(sigmoid(w3 . h2 + b3), 2^-24, 1 - 2^-24) (the sampler's
 * resolution: every variable keeps a draw weight floor(p 2^24) >= 1), F = 8 features,
 * H = 128 hidden units, packed as W1[H*F] b1[H] W2[H*H] b2[H] w3[H] b3[1]
 * (FP32 masters; the kernels round weights to bf16).  nW must equal
 * gfors_mlp_nparams(F, H). */
GFORS_API int64_t gfors_mlp_nparams(int32_t F, int32_t H);
GFORS_API gfors_status gfors_set_proposal(gfors_handle h, const float* W, int64_t nW);

/* Features of the learned proposal at the current iterate, FP32 [n x 8]
 * row-major into feat (host), for instance inst: 1 standardised cost over
 * the instance, 2 column degree / max degree, 3 x_k, 4 x_k - x at the
 * previous call, 5 feature 1 minus its minimum over the variable's group
 * (one-hot group or axial slab; the instance when ungrouped), 6 x_k / max of
 * x_k over the group (x_k when ungrouped), 7 tau1 delta of the last primal
 * step, 8 rho / rho_max.  Each call (and each learned sampling round)
 * advances the previous-trigger snapshot of feature 4.  Synchronises. */
GFORS_API gfors_status gfors_get_features(gfors_handle h, int32_t inst, float* feat);

/* MLP kernels on caller DEVICE buffers (cuda_stream as in gfors_load):
 * forward: feat [nv x F] -> z [nv] logits, p [nv] probabilities (p may be
 * NULL); loss_grad: mean BCE on logits against label [nv] (0/1), gradient
 * into grad [nparams] (overwritten), loss into *loss_dev (device double);
 * adam: one Adam step (t >= 1) on W [nparams] with moments m, v [nparams]
 * (FP32).  W is packed as in gfors_set_proposal. */
GFORS_API gfors_status gfors_mlp_forward(int32_t F, int32_t H, const float* W_dev,
                               int64_t nv, const float* feat_dev, float* z_dev,
                               float* p_dev, void* cuda_stream);
GFORS_API gfors_status gfors_mlp_loss_grad(int32_t F, int32_t H, const float* W_dev,
                                 int64_t nv, const float* feat_dev,
                                 const float* label_dev, float* grad_dev,
                                 double* loss_dev, void* cuda_stream);
GFORS_API gfors_status gfors_mlp_adam(int64_t nparams, float* W_dev, const float* grad_dev,
                            float* m_dev, float* v_dev, int64_t t, double lr,
                            double beta1, double beta2, double eps,
                            void* cuda_stream);

/* Checkpoint / resume of the whole solver state (iterates, counters,
 * penalty, incumbents, halting trackers).  export: with buf == NULL only
 * *len is set; otherwise *len must hold the buffer size.  A resumed handle
 * (same instance data and parameters) continues bit-identically.
 * Synchronises. */
GFORS_API gfors_status gfors_state_export(gfors_handle h, void* buf, size_t* len);
GFORS_API gfors_status gfors_state_import(gfors_handle h, const void* buf, size_t len);

/* Phase timing with CUDA events recorded on the handle's stream (no
 * counterpart in the paper; measurement support).  enable = 1 clears and
 * starts recording, 0 stops.  gfors_profile_read synchronises and writes,
 * for each of nphases phases, the summed milliseconds and the number of
 * timed launches: 0 PDHG iterations (per captured pair or single step;
 * counts iterations), 1 bit sampling, 2 sparse evaluation, 3 dense scoring,
 * 4 incumbent update, 5 fused sample+evaluate, 6 CheckHalt statistics,
 * 7 dense sampling, 8 the sparse-Q objective kernel (also inside 2). */
GFORS_API gfors_status gfors_profile(gfors_handle h, int32_t enable);
GFORS_API gfors_status gfors_profile_read(gfors_handle h, int32_t nphases, double* ms,
                                          int64_t* counts);

/* Failure injection for tests of the bounded device-side waits (failure
 * detection of this library; the paper has no counterpart).  kind 1: in
 * the next launch of the persistent dense PDHG kernel (pdhg_mode 0, one
 * dense instance) or of the cooperative sparse kernel (pdhg_mode 2), block
 * `block` waits at its first grid barrier without arriving there.  The
 * other blocks' waits, bounded by wait_timeout_s, run out; every block
 * then leaves the kernel, the next synchronising call returns
 * GFORS_E_TIMEOUT and the handle is failed (later calls GFORS_E_STATE until
 * gfors_destroy).  Nothing faults and the CUDA context stays usable.  A
 * block index beyond the grid injects nothing.  kind 0 clears a pending
 * injection.  One launch consumes it.  GFORS_E_ARG for another kind or a
 * negative block. */
GFORS_API gfors_status gfors_debug_inject(gfors_handle h, int32_t kind, int32_t block);

/* Allocation-free fused sampling + evaluation of one single-row instance
 * (the knapsack form a.x >= rhs).  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they
 * need the pass -- code running while a CUDA graph is captured on its
 * thread, serving loops that never touch an allocator after start-up, hosts
 * whose device memory all belongs to their own pool.  It draws the same
 * candidates as gfors_sample_eval on a single-row handle and returns the
 * same scores, without any allocation.
 *   p_dev [n]   FP32 probabilities (device); a_dev [n] int32 row
 *               coefficients; c_dev [n] int64 costs; rhs the row's bound
 *   seed, inst_id, round_id, first_sample: the Philox key, instance id,
 *               round id and first candidate index (as in gfors_sample_eval)
 *   nsamples    candidates first_sample .. first_sample + nsamples - 1;
 *               at most GFORS_NOALLOC_MAX_SAMPLES, and first_sample +
 *               nsamples at most INT32_MAX, else GFORS_E_ARG
 *   viol_dev [nsamples] int32 out: 1 if a.x < rhs; obj_dev [nsamples]
 *               int64 out: c.x  (device buffers owned by the caller)
 * Enqueued on cuda_stream, asynchronous.  Its only scratch is a file-scope
 * device array of GFORS_NOALLOC_MAX_SAMPLES int64 that every device using
 * the library keeps until the process exits.  The first call on a device
 * looks up that array's address and should come before any stream capture;
 * the address is cached for the process, so do not call this after a
 * cudaDeviceReset.  Calls share the array (each clears what it uses first): calls that overlap
 * on the GPU race. */
#define GFORS_NOALLOC_MAX_SAMPLES 16384
GFORS_API gfors_status gfors_fused_eval_noalloc(const float* p_dev, const int32_t* a_dev,
                                                const int64_t* c_dev, int64_t n, int64_t rhs,
                                                uint64_t seed, uint32_t inst_id,
                                                uint32_t round_id, int32_t first_sample,
                                                int32_t nsamples, int32_t* viol_dev,
                                                int64_t* obj_dev, void* cuda_stream);

/* ---- Autotuner of the batched PDHG path (the batching pattern of the
 * method's implementation; the paper itself prescribes no tuning).
 * Rows (dual step, Alg. 2 line for y) and columns (primal step) are processed
 * in five length buckets -- lengths <= 2, <= 8, <= 32, <= 128, <= 2048;
 * longer ones are split into fixed chunks -- with `lanes` threads per row /
 * column.  lanes[10] = rows' five buckets then columns' five, each 1, 2, 4,
 * 8, 16 or 32.  A lane count changes only the FP32 summation order inside a
 * row / column (results stay within the per-step tolerance of the FP64
 * reference; a fixed choice is deterministic).
 *
 * gfors_autotune times every candidate lane count of every non-empty bucket
 * on the device (scratch outputs: the solver state is untouched) and keeps
 * the fastest.  cache_path (may be NULL) names a JSON file keyed by
 * gfors_tune_key: on a hit the stored choice is applied without timing
 * (*hit = 1), else the timed choice is stored (file created if absent).
 * out_lanes (may be NULL) receives the choice.  Synchronises; drops captured
 * CUDA graphs of the iteration.  Errors: GFORS_E_ARG (cache not writable),
 * GFORS_E_CUDA. */
GFORS_API gfors_status gfors_autotune(gfors_handle h, const char* cache_path,
                                      int32_t out_lanes[10], int32_t* hit);
/* Apply an explicit choice (GFORS_E_ARG if a value is not a lane count) /
 * read the current one. */
GFORS_API gfors_status gfors_set_lanes(gfors_handle h, const int32_t lanes[10]);
GFORS_API gfors_status gfors_get_lanes(gfors_handle h, int32_t lanes[10]);
/* Cache key of this handle: device name, then log2 classes of the total
 * variables, rows and nonzeros and of every bucket's row / column count.
 * GFORS_E_ARG if len is too small. */
GFORS_API gfors_status gfors_tune_key(gfors_handle h, char* buf, size_t len);
/* Host-only cache access (no device needed): look up key in the JSON file at
 * path (*found = 0 when the file or key is absent), or insert / replace an
 * entry (GFORS_E_ARG for invalid lanes, a key containing quotes, backslashes
 * or control characters, or an unwritable path). */
GFORS_API gfors_status gfors_tune_cache_lookup(const char* path, const char* key,
                                               int32_t lanes[10], int32_t* found);
GFORS_API gfors_status gfors_tune_cache_store(const char* path, const char* key,
                                              const int32_t lanes[10]);

/* Dense-Q scoring of instance inst: out[0] = 1 if Q is held as a dense
 * small-integer matrix, out[1] = 1 if the tensor-core scorer is exact for it
 * (n max|W2| < 2^24 and int32 tile partials), out[2] = 1 if it scores with
 * FP8 E4M3 operands (else bf16), out[3] = max|W2|, W2 = offdiag(Q + Q^T).
 * Host only. */
GFORS_API gfors_status gfors_dense_info(gfors_handle h, int32_t inst, int64_t out[4]);

/* ---- TU reformulation (Thm. 5, Section 2.4.1), host only, no GPU needed.
 * Removes the equality rows J of B by x_I = s + S x_Ibar (s = B_JI^-1 d_J,
 * S = -B_JI^-1 B_JIbar).  A signed-permutation B_JI (every row J[k] has
 * exactly one entry +-1 in the columns I, every column of I has its entry in
 * exactly one of those rows) is used directly; any other B_JI is inverted by
 * Gauss-Jordan elimination in exact integer arithmetic, S stored explicitly.
 * The new problem is over x_Ibar, Ibar = the other columns in ascending
 * order:
 *   A' = [A_.I S + A_.Ibar; S; -S],  b' = [b - A_.I s; -s; s - 1] (a
 *   bounds row that every x in [0, 1] satisfies is left out),
 *   B' = B_JbarI S + B_JbarIbar (rows of B outside J, ascending),
 *   d' = d_Jbar - B_JbarI s,  Q' = S^T Q_II S + S^T Q_IIbar + Q_IbarI S +
 *   Q_IbarIbar,  c' = S^T (Q_II + Q_II^T) s + Q_IIbar^T s + Q_IbarI s +
 *   S^T c_I + c_Ibar,  objective constant c0' = s^T Q_II s + c_I^T s.
 * Q is used as given (not symmetrised).  Exactness needs B_J totally
 * unimodular; that is the caller's claim, not checked.
 * gfors_tu_reformulate: n, A, b, B, d, Q, c as in gfors_load (A, Q may be
 *   NULL); J, I: nJ row / column indices.  *out receives an object owned by
 *   the caller (gfors_tu_free).  GFORS_E_ARG for malformed input or
 *   repeated / out-of-range indices, a singular B_JI or non-integral B_J,
 *   d_J; GFORS_E_UNSUPPORTED when the elimination meets a pivot other than
 *   +-1 or an entry outside {-1, 0, 1} (B_J not TU) or S would exceed 2^28
 *   entries (the paper keeps an LU factor instead; not built).
 * gfors_tu_sizes: out[0] = n', out[1] = rows of A', out[2] = nnz(A'),
 *   out[3] = rows of B', out[4] = nnz(B'), out[5] = 1 if Q' exists,
 *   out[6] = nnz(Q'), out[7] = |I|.
 * gfors_tu_copy: copies the CSR arrays (row_ptr, col_idx, val; sized from
 *   gfors_tu_sizes), b', d', c' (n'), c0' and Ibar (n') into caller buffers;
 *   any pointer may be NULL to skip that array.
 * gfors_tu_recover: k candidates over x_Ibar (k x n' bytes, row-major) to
 *   candidates of the original problem (k x n bytes); GFORS_E_ARG if some
 *   x_I falls outside {0, 1} (that candidate violates the bounds rows). */
typedef struct gfors_tu_s* gfors_tu;
GFORS_API gfors_status gfors_tu_reformulate(int64_t n, const gfors_csr* A, const double* b,
                                            const gfors_csr* B, const double* d,
                                            const gfors_qmat* Q, const double* c,
                                            int64_t nJ, const int64_t* J, const int64_t* I,
                                            gfors_tu* out);
GFORS_API gfors_status gfors_tu_sizes(gfors_tu t, int64_t out[8]);
GFORS_API gfors_status gfors_tu_copy(gfors_tu t, int64_t* Ap, int32_t* Ac, double* Av,
                                     double* b, int64_t* Bp, int32_t* Bc, double* Bv,
                                     double* d, int64_t* Qp, int32_t* Qc, double* Qv,
                                     double* c, double* c0, int64_t* Ibar);
GFORS_API gfors_status gfors_tu_recover(gfors_tu t, int64_t k, const uint8_t* Xbar,
                                        uint8_t* X);
GFORS_API void gfors_tu_free(gfors_tu t);

/* Which kernels run the PDHG iterations (Alg. 2) of this handle, fixed at
 * load: bucketed row / column kernels with CUDA-graph replay, the one-row
 * streaming kernels (every instance one row, no Q), one block per instance
 * (instances that fit shared memory), one cooperative launch per call
 * (pdhg_mode 2), the persistent dense-Q launch, or one thread-block cluster
 * per instance (few instances that fit shared memory; xbar and y exchanged in
 * distributed shared memory).  Host only. */
enum {
  GFORS_PATH_BUCKETS = 0,
  GFORS_PATH_ONE_ROW = 1,
  GFORS_PATH_SMALL = 2,
  GFORS_PATH_COOPERATIVE = 3,
  GFORS_PATH_PERSISTENT = 4,
  GFORS_PATH_CLUSTER = 5
};
GFORS_API gfors_status gfors_pdhg_path(gfors_handle h, int32_t* path);

/* ---- Several devices (Section 3's sampling rounds split by candidate).
 * gfors_sample_eval_range: as gfors_sample_eval, but only candidates
 * [s_begin, s_end) of every round (multiples of 32, within k_b).  Candidate
 * indices stay global within the round (Philox counters as in Algorithm 3),
 * so devices that each take a disjoint range of the same rounds from the same
 * iterate draw together exactly the candidates of the whole round, and the
 * lexicographic minimum of their incumbent keys is the one-device incumbent.
 * Asynchronous. */
GFORS_API gfors_status gfors_sample_eval_range(gfors_handle h, int32_t nrounds,
                                               uint32_t first_round_id, int32_t proposal,
                                               int32_t s_begin, int32_t s_end);
/* ---- Asynchronous host I/O (serving loops: one synchronisation per batch
 * of steps instead of one per call).
 * gfors_set_iterate_async: as gfors_set_iterate, but only enqueued on the
 *   handle's stream; the host arrays must stay valid and unchanged until the
 *   stream has passed the copies (pinned memory makes them asynchronous).
 * gfors_incumbent_async: enqueues the copy of instance inst's incumbent key
 *   (objective, round id, candidate index; all INT64_MAX when none) into
 *   key_host[3] (host memory, pinned for asynchrony); valid after
 *   gfors_synchronize or any synchronisation of the stream.
 * gfors_synchronize: waits for everything enqueued on the handle's stream. */
GFORS_API gfors_status gfors_set_iterate_async(gfors_handle h, int32_t inst, const float* x,
                                               const float* xbar, const float* y);
GFORS_API gfors_status gfors_incumbent_async(gfors_handle h, int32_t inst, int64_t* key_host);
GFORS_API gfors_status gfors_synchronize(gfors_handle h);

/* Incumbent key of instance inst -- (objective, round id, candidate index);
 * all three INT64_MAX when none was found -- written to key_dev[3] (DEVICE
 * memory, caller-owned), enqueued on the handle's stream (asynchronous), for
 * a min-reduction across devices without a host round trip. */
GFORS_API gfors_status gfors_incumbent_key_async(gfors_handle h, int32_t inst,
                                                 int64_t* key_dev);

/* Kernel-launch counter of this handle (device kernels enqueued so far). */
GFORS_API int64_t gfors_launch_count(gfors_handle h);

/* Text of the last error on h (h == NULL: the calling thread's last load
 * error).  Valid until the next call on the same handle / thread. */
GFORS_API const char* gfors_last_error(gfors_handle h);

GFORS_API void gfors_destroy(gfors_handle h);

#ifdef __cplusplus
}
#endif
#endif /* GFORS_H */
