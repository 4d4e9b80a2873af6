// internal.cuh -- host-side context of a GFORS handle and kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "gfors.h"

// ---------------------------------------------------------------------------
// Work lists of the PDHG kernels.  Rows (dual step) and columns (primal
// step) are bucketed by length; each bucket is processed by groups of
// `lanes` threads; lengths above kLongLen are split into chunks whose
// partial sums are combined in a fixed order by a finalising kernel.
// ---------------------------------------------------------------------------
constexpr int kLongLen = 2048;     // rows/cols longer than this are chunked
constexpr int kChunkLen = 2048;    // nnz per partial-sum chunk
constexpr int kGLong = 256;       // general rows above this length: a block each in evaluation

struct GfChunk {                    // one partial-sum chunk of a long row/col
  int32_t id;                       // row (dual) or column (primal)
  int32_t part;                     // 0: K entries, 1: Q entries (primal)
  int64_t t0, t1;                   // nnz range
};

// Consecutive rows (columns) of one instance inside one length bucket.
struct GfRun {
  int64_t first;                    // first row / column id
  int64_t nnz0;                     // offset of its first nonzero (uniform runs)
  int32_t count;                    // rows / columns in the run
  int32_t len;                      // common length, -1 if lengths differ
  int32_t inst;
  int32_t pad;
};

struct GfBucket {
  int lanes = 1;
  int32_t* ids = nullptr;           // device row / column ids (when runs == nullptr)
  int32_t count = 0;
  GfRun* runs = nullptr;            // device runs covering the bucket, in order
  int64_t* run_ptr = nullptr;       // device prefix of run counts (nruns + 1)
  int32_t nruns = 0;
  bool short_ok = false;            // every member has <= 2 nonzeros
};

struct GfLongSet {
  GfChunk* chunks = nullptr;        // device
  int32_t nchunks = 0;
  int32_t* ids = nullptr;           // device: long row / column ids
  int32_t* chunk_ptr = nullptr;     // device: nlong + 1 offsets into chunks
  int32_t nlong = 0;
  float2* partial = nullptr;        // device: (s, c) per chunk
};

// Long K^T columns of one length in slices of 32 (sliced ELL): entry e of
// the slice's column l sits at off + 32 e + l, so that a warp reads 32
// columns' entries (and, for columns whose rows are consecutive, the dual
// values) contiguously.  Each block (slice, chunk c) writes the chunk
// partials of the clong layout (kChunkLen entries per column chunk).
struct GfColSlices {
  int32_t nslices = 0, nblocks = 0;
  int4* blk = nullptr;              // per block: (slice, chunk, columns, 0)
  int64_t* off = nullptr;           // per slice: first entry
  int32_t* len = nullptr;           // per slice: entries per column
  int32_t* pbase = nullptr;         // [slice][32]: partial index of chunk 0 (-1: empty lane)
  int32_t* sidx = nullptr;          // interleaved row indices (-1: empty lane)
  float* sval = nullptr;            // interleaved scaled values
};
// ---------------------------------------------------------------------------
// Evaluation structures (original, unscaled, integer data).
// ---------------------------------------------------------------------------
struct GfURow {                     // all coefficients equal: count in [L, U]
  int32_t inst;
  int32_t len;
  int64_t t0;                       // into ucols
  int32_t L, U;                     // U < 0: no upper bound
};
struct GfPRow {                     // at most two nonzeros: truth table
  int32_t inst;
  int32_t v1, v2;                   // global variables (v2 = -1 if absent)
  uint32_t table;                   // bit (x1 + 2 x2) set = violated
};
struct GfGRow {                     // general integer row
  int32_t inst;
  int32_t len;
  int64_t t0;                       // into gcols / gvals
  long long rhs;
  int32_t eq;
  int32_t pad;
};
struct GfPChunk {                   // run of P rows (v1 + e stride, v2), e < len, one table
  int32_t inst;
  int32_t v1, v2;
  uint32_t table;
  int32_t len;                      // <= kPChunk
  int32_t stride;                   // > 0
  int32_t pad[2];
};
struct GfPSlice {                   // up to 32 P-row chunks side by side: lane l has
  int32_t inst;                     // hub v2 + l and rows (v1 + l + e stride, v2 + l)
  int32_t v1, v2;
  uint32_t table;
  int32_t len;
  int32_t stride;
  int32_t lanes;
  int32_t pad;
};
constexpr int kPChunk = 256;        // rows per P-row run chunk (one warp)
constexpr int kPSliceRows = 64;     // rows per warp of a slice of runs
constexpr int kMinPRun = 64;        // runs at least this long are evaluated as chunks
struct GfObjChunk {                 // linear-objective chunk: vars [v0, v1)
  int32_t inst;
  int32_t v0, v1;
  int32_t pad;
};
struct GfQChunk {                   // sparse-Q chunk: pair blocks [r0, r1)
  int32_t inst;
  int32_t r0, r1;
  int32_t pad;
};

struct GfDenseQ {                   // dense +-small-integer Q (tensor-core path)
  int inst = -1;
  int64_t n = 0, ld = 0;            // ld: row stride in elements (mult. of 64)
  __nv_bfloat16* W2 = nullptr;      // off-diagonal of Q + Q^T, n x ld
  uint8_t* W2i8 = nullptr;          // W2 + 128 as bytes when max|W2| <= 127 (PDHG GEMV)
  float* qdiag = nullptr;           // diag(Q_sym) / s_obj
  float qscale = 0.f;               // 0.5 / s_obj
  long long* lin = nullptr;         // c_i + Q_ii (original, integer)
  uint8_t* W2f8 = nullptr;          // same as FP8 E4M3 when max|W2| <= 16 (scoring)
  __nv_bfloat16* Xs = nullptr;      // candidates, sample-major, chunk x ld (bf16, or
                                    // FP8 E4M3 bytes in the same buffer when f8)
  uint32_t* Xb = nullptr;           // same as bit words, chunk x ld/32
  uint32_t* thr = nullptr;          // Bernoulli thresholds of the current chunk (ld)
  int chunk = 0;
  bool tc_ok = false;               // tensor-core scoring exact (n max|W2| < 2^24)
  bool f8 = false;                  // score with FP8 operands (exact, twice the rate)
  long long w2max = 0;
};

struct GfInstHost {
  int64_t n = 0, npad = 0, m1 = 0, m2 = 0;
  int64_t var_off = 0, row_off = 0;
  int qkind = 0;                    // 0 none, 1 dense tensor-core path, 2 sparse
  bool integral = true;
  double normQ_raw = 0, s_obj = 1, normK = 0, s_K = 1, normQhat = 0;
  int itQ = 0, itK = 0;
  int cap = 0;
  int group_mode = 0;               // 0 Bernoulli, 1 one-hot groups, 2 axial,
                                    // 3 Algorithm 4 (customized 3D assignment)
  int axial_I = 0;
  int a4_gamma = 1, a4_L = 0;       // Algorithm 4: entries gamma*I, steps L
  bool a4_gain32 = false;           // Algorithm 4 gains fit in int32 (4 max|c| < 2^31)
  int64_t ngroups = 0;
  int64_t grp_off = 0;              // offset into the group tables
  int64_t nrep = 0, rep_off = 0;
  bool single_row = false;          // eligible for fused sample+eval
  int dense_idx = -1;
  bool rr_set = false;              // general repair rows attached
};

struct gfors_ctx {
  gfors_params prm;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int dev = 0;
  int num_sms = 148;
  bool failed = false;
  std::string err;
  long long launches = 0;
  // test injection (gfors_debug_inject): this block of the next persistent
  // or cooperative PDHG launch skips its first grid-barrier arrival; -1 none
  int inject_skip_block = -1;

  int ninst = 0;
  std::vector<GfInstHost> ih;
  int64_t N = 0, M = 0, nnzK = 0, nnzQ = 0;

  // allocation bookkeeping
  std::vector<void*> allocs;

  // instance tables (device)
  int64_t* var_off_d = nullptr;     // ninst + 1
  int32_t* var_inst = nullptr;      // N
  int32_t* row_inst = nullptr;      // M
  uint8_t* row_eq = nullptr;        // M

  // scaled problem (FP32)
  int64_t* Kp = nullptr; int32_t* Kc = nullptr; float* Kv = nullptr;
  int64_t* Tp = nullptr; int32_t* Tr = nullptr; float* Tv = nullptr;
  int64_t* Qp = nullptr; int32_t* Qc = nullptr; float* Qv = nullptr;
  float* rhat = nullptr;
  float* chat = nullptr;
  uint8_t* var_live = nullptr;      // 1 for real variables, 0 for padding

  // iterate
  float* x[2] = {nullptr, nullptr}; // x_k lives in x[k & 1]
  float* xbar = nullptr;
  float* y = nullptr;
  float* qbuf = nullptr;            // dense-Q products when K is present

  // device state
  GfDState* dstate = nullptr;
  GfIParam* iprm = nullptr;         // [2][ninst]
  GfSched sched;
  GfSched* sched_d = nullptr;
  double* normQhat_d = nullptr;     // ninst
  int32_t* cap_d = nullptr;         // ninst
  long long k_host = 0;             // mirrors dstate->k
  int n_rho_host = 0;
  double rho_host = 0;

  // PDHG work lists
  std::vector<GfBucket> rb, cb;     // row / column buckets
  GfLongSet rlong, clong;
  GfColSlices csl;                  // long K^T columns in slices of 32
  std::vector<GfDenseQ> dense;

  // sampling
  uint8_t* var_grouped = nullptr;   // N: 1 if drawn by a group sampler
  // 4-variable groups with a variable the Bernoulli sampler draws (any
  // variable not drawn by a group sampler, padding included), built on the
  // device when stale (n_bit_g4 < 0)
  // monotone-relaxation repair groups (Section 2.4.3), global variable ids
  std::vector<int64_t> h_rg_ptr, h_rg_idx;
  int64_t* rg_ptr = nullptr;
  int64_t* rg_idx = nullptr;
  int64_t nrg = 0;
  // general monotone-relaxation repair (reverse delete over relaxed covering
  // rows): rows (global ids, CSR), per instance segment the row variables
  // in decreasing cost, each with its rows; per (row, candidate) counts
  int64_t nrr = 0, nrr_seg = 0;
  int64_t *rr_ptr = nullptr, *rr_idx = nullptr;   // rows
  int64_t *rr_optr = nullptr, *rr_order = nullptr;  // segments of the order
  int64_t *rr_vptr = nullptr, *rr_vrow = nullptr;   // rows of each order position
  int32_t* rr_cnt = nullptr;                         // nrr x chunk
  std::vector<int64_t> h_rr_ptr, h_rr_idx, h_rr_optr, h_rr_order, h_rr_vptr, h_rr_vrow;
  long long* key_stage = nullptr;    // 3 per instance: gfors_incumbent_async
  int32_t* bit_g4 = nullptr;
  int32_t* bit_count = nullptr;
  int64_t n_bit_g4 = -1;
  int64_t ngroups_tot = 0;
  int64_t* grp_ptr = nullptr;       // global groups (ngroups_tot + 1)
  int64_t* grp_idx = nullptr;       // global variable ids
  int32_t* grp_inst = nullptr;      // instance of each group
  int32_t* grp_local = nullptr;     // group index within its instance
  unsigned long long* grp_cw = nullptr;  // cumulative weights (per member)
  int64_t* grp_step = nullptr;      // per group: members grp_idx[ptr] + t step
                                    // (arithmetic lists), 0 = read the list
  unsigned long long* grp_cw2 = nullptr; // a second set (two proposals in one call)
  const float* cw_src[2] = {nullptr, nullptr};  // p whose weights each set holds
  bool cw_cache = false;            // within one sampling call: p does not change
  // objective of one-hot picks: valid when no later repair changes a grouped
  // variable; objective chunks over 32-variable slabs with an ungrouped
  // variable and, per slab, the mask of its grouped lanes
  bool pick_obj_valid = false;
  long long repair_version = 0;     // bumped when repair groups / rows / closure change
  long long pick_obj_rv = -1, pick_obj_gv = -1;
  long long* objp = nullptr;        // [ninst][chunk] costs of the picks
  GfObjChunk* ochunks_ng = nullptr; int64_t nochunks_ng = 0;
  uint32_t* slab_gmask = nullptr;   // N / 32
  std::vector<int64_t> h_grp_ptr, h_grp_idx;
  std::vector<int32_t> h_grp_inst, h_grp_local;
  bool groups_dirty = false;
  int64_t nrep_tot = 0;
  int64_t* rep_var = nullptr; int64_t* rep_ptr = nullptr; int64_t* rep_idx = nullptr;
  int64_t* rep_step = nullptr;      // per repaired variable: list = rep_idx[ptr] + t step
                                    // (arithmetic lists), 0 = read the list
  std::vector<int64_t> h_rep_var, h_rep_ptr, h_rep_idx;
  bool closure_dirty = false;
  int chunk = 0;                    // candidates per pass (multiple of 32)
  int kw = 0;                       // chunk / 32 words per variable
  uint32_t* X = nullptr;            // variable-major bits, N x kw
  int32_t* viol = nullptr;          // ninst x chunk
  long long* obj = nullptr;         // ninst x chunk
  int last_chunk_len = 0;
  int last_mode = 0;                // how the last chunk was sampled
  int last_s0 = 0;

  // evaluation (integer data)
  bool all_integral = true;
  GfURow* urows = nullptr; int64_t nurows = 0; int32_t* ucols = nullptr;
  int64_t nurows_cls[3] = {0, 0, 0};  // urows of each class, stored in class order
  GfPRow* prows = nullptr; int64_t nprows = 0;
  GfPChunk* pchunks = nullptr; int64_t npchunks = 0;   // long runs of P rows
  GfPSlice* pslices = nullptr; int64_t npslices = 0;   // runs side by side
  GfGRow* grows = nullptr; int64_t ngrows = 0; int32_t* gcols = nullptr; int32_t* gvals = nullptr;
  int64_t ngrows_short = 0;         // rows [0, ngrows_short) have <= kGLong entries
  long long* cint = nullptr;        // N, original integer costs
  GfObjChunk* ochunks = nullptr; int64_t nochunks = 0;
  // sparse Q for evaluation: pairs (QIi < QIc) with w = q_ij + q_ji in
  // blocks of 32 (each instance padded with weight-0 pairs), per block the
  // bias -min w and the bit width of the weight span; clin = c + diag(Q)
  // (null when no instance has a sparse Q)
  int32_t* QIi = nullptr; int32_t* QIc = nullptr; long long* QIv = nullptr;
  long long* QIb = nullptr; uint8_t* QIw = nullptr; long long* clin = nullptr;
  // per 32-variable group of the linear costs used in evaluation: bias
  // -min c and bit width of the cost span
  long long* cgbias = nullptr; uint8_t* cgP = nullptr;
  GfQChunk* qchunks = nullptr; int64_t nqchunks = 0;
  // fused single-row path
  bool fused_ok = false;
  int32_t* frow_w = nullptr;        // N: coefficient of the single row (0 for padding)
  int32_t* f_c32 = nullptr;         // N: costs as int32 when every row / cost sum fits
  uint32_t* fthr = nullptr;         // N: Bernoulli thresholds of the current chunk
  long long* frhs = nullptr;        // ninst
  long long* fsum = nullptr;        // ninst x chunk row sums
  int32_t* fblk = nullptr;          // fused work blocks: (inst, v0, v1) triples
  int64_t nfblk = 0;

  // incumbents
  GfInc* inc = nullptr;             // ninst
  uint8_t* xbest = nullptr;         // N (0/1 bytes)

  // statistics
  double* stats_part = nullptr;     // per stats chunk partials
  double* stats = nullptr;          // ninst x 8 (row sums)
  double* stats2 = nullptr;         // ninst x 8 (variable sums)
  int32_t* vchunk = nullptr; int64_t nvchunk = 0;   // var chunks (inst, v0, v1)
  int32_t* rchunk = nullptr; int64_t nrchunk = 0;   // row chunks (inst, r0, r1)
  int32_t* vchunk_iptr = nullptr;   // ninst + 1
  int32_t* rchunk_iptr = nullptr;   // ninst + 1
  uint8_t* inst_dense = nullptr;    // ninst: 1 if dense tensor-core Q
  float* qbuf2 = nullptr;           // N scratch (Q dx)
  float* dxbuf = nullptr;           // N scratch (x - x_prev)
  const float* last_p = nullptr;    // proposal of the last sampled chunk

  // halting trackers (host)
  std::vector<double> h_best;       // ninst x 3
  std::vector<long long> h_last;    // ninst x 3
  long long h_trig = 0;

  // learned proposal
  float* mlp_W = nullptr;
  int64_t mlp_np = 0;
  float* feat = nullptr;            // N x 8
  float* x_trig_prev = nullptr;     // x at the previous trigger
  float* crel = nullptr;            // N: cstd - min of cstd over the variable's group
  long long feat_grp_version = -1;  // group tables the static features were built for
  float* p_learn = nullptr;         // N
  float* dlast = nullptr;           // tau1 * delta of the last step (N)
  float* degnorm = nullptr;         // column degree / max (N)
  float* cstd = nullptr;            // standardised c (N)
  float* grpmax = nullptr;          // N: max_{group} x (scratch)
  float* p_learn_z = nullptr;       // N: logits of the learned proposal
  uint8_t* var_grouped_feat = nullptr;  // N: 1 if in a one-hot group / axial slab
  long long grp_version = 0;        // bumped whenever groups change
  // device-side Alg. 1 loop (gfors_run_graph): per-instance constants and
  // CheckHalt state of the halt kernel, the trigger graph while it is built
  bool capturing = false;
  int32_t* halt_n = nullptr;        // ninst: n of each instance
  int32_t* halt_q = nullptr;        // ninst: qkind of each instance
  double* halt_best = nullptr;      // 3 ninst
  long long* halt_last = nullptr;   // 3 ninst
  long long* halt_tgt = nullptr;    // ninst: target objectives
  long long* halt_ctl = nullptr;    // [0] triggers run, [1] CheckHalt trigger count,
                                    // [2] halt reason (0 budget, 1 CheckHalt, 2 targets),
                                    // [3] trigger budget, [4] first trigger's index,
                                    // [5] targets on
  long long struct_version = 0;     // bumped when the launches of a trigger change
  struct RunGraph {                 // instantiated whole-run graph, per proposal
    cudaGraphExec_t exec = nullptr;
    long long sv = -1, gv = -1;     // struct_version / grp_version it was built for
    long long per_trig = 0;         // kernel launches in one trigger
  } run_graph[4];

  // CUDA graphs of one PDHG iteration pair, by parity of its first iteration
  cudaGraphExec_t g_pair = nullptr;
  cudaGraphExec_t g_iter2[2] = {nullptr, nullptr};
  // pairs of "light" iterations: they do not store tau1 delta (a feature of
  // the learned proposal) and, in one-row batches, not xbar either (only the
  // K xbar partials the next dual step reads); every call's last two
  // iterations run in full, so both are current between calls
  cudaGraphExec_t g_light2[2] = {nullptr, nullptr};
  bool light_iter = false;
  long long pair_launches = 0;
  bool use_graphs = true;
  // single-row batches (one constraint row per instance, no Q): fused
  // primal step + K xbar partials, then a per-instance dual step
  bool single_ok = false;
  bool sr_valid = false;            // partials of K xbar match the state
  int32_t* sr_chunk = nullptr;      // (inst, v0, v1) per chunk of <= 2048 variables
  int64_t sr_nchunk = 0;
  int32_t* sr_ciptr = nullptr;      // ninst + 1 offsets into the chunks
  int64_t* sr_row = nullptr;        // global row of each instance
  float* sr_kv = nullptr;           // K entry of every variable (0 if none)
  float2* sr_part = nullptr;        // [2][sr_nchunk] compensated partial sums
  // Algorithm 4 scratch: slab top lists, partial assignment
  unsigned long long* a4_cand = nullptr;   // up to 16384 keys
  int32_t* a4_J0 = nullptr;                // 64
  int32_t* a4_K0 = nullptr;                // 64
  // L2-resident sparse problems: one cooperative launch per call
  bool coop_ok = false;
  int32_t *coop_rblk = nullptr, *coop_rwarp = nullptr, *coop_cblk = nullptr,
          *coop_cwarp = nullptr, *coop_cthr = nullptr;
  int32_t coop_n[5] = {0, 0, 0, 0, 0};
  unsigned* coop_bar = nullptr;
  // small instances: one block per instance, matrix in shared memory
  bool small_ok = false;
  struct GfSmallInst* small_tab = nullptr;
  uint16_t* small_perm = nullptr;   // N: each instance's columns by decreasing length
  long long* small_k0 = nullptr;    // st->k snapshotted before each small launch
  int cluster_C = 0;                // > 0: one cluster of this many CTAs per instance
  size_t cluster_smem = 0;
  size_t small_smem = 0;
  // persistent cooperative PDHG launch (dense instance, matrix in smem)
  bool persist_ok = false;
  size_t persist_smem = 0;
  int64_t persist_per = 0;          // rows per block
  int persist_grid = 0;             // blocks (each owns >= 1 row)
  unsigned* persist_bar = nullptr;  // grid-barrier counter
  unsigned host_round = 0;          // round id of the next round (host mirror)
  // phase profiling (CUDA events on the handle's stream)
  bool prof = false;
  struct ProfRec { int phase; int count; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  unsigned last_round = 0;          // round id of the last sampled chunk
};

typedef gfors_ctx GfCtx;

// ---- error handling -------------------------------------------------------
gfors_status gf_fail(GfCtx* h, gfors_status st, const std::string& msg);
gfors_status gf_cuda(GfCtx* h, cudaError_t e, const char* what);
#define GF_CK(h, call)                                        \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return gf_cuda((h), _e, #call);    \
  } while (0)

void* gf_alloc(GfCtx* h, size_t bytes);   // NULL on failure (status set)
template <class T>
T* gf_alloc_t(GfCtx* h, size_t count) {
  return static_cast<T*>(gf_alloc(h, sizeof(T) * (count > 0 ? count : 1)));
}
void gf_free_all(GfCtx* h);
void gf_free_one(GfCtx* h, void* p);

// ---- launchers (each returns cudaGetLastError of its launch) --------------
cudaError_t gf_launch_pdhg_iter(GfCtx* h, int parity);
cudaError_t gf_launch_dense_gemv_q(GfCtx* h, const GfDenseQ& dq, const float* x,
                                   float* out);   // out = Q_hat x (FP32)
cudaError_t gf_launch_power(GfCtx* h, int which, const int64_t* Kp, const int32_t* Kc,
                            const double* Kv, const int64_t* Tp, const int32_t* Tr,
                            const double* Tv, int64_t mrows, double* norms, int* iters);
// pick_obj (may be NULL): set when the one-hot picks also left their costs
// in objp (gf_launch_eval then evaluates the other variables only)
cudaError_t gf_launch_sample(GfCtx* h, const float* p, int s0, int len, bool for_dense,
                             bool* pick_obj = nullptr);
cudaError_t gf_ensure_bit_list(GfCtx* h);
cudaError_t gf_prepare_features(GfCtx* h);
cudaError_t gf_launch_eval(GfCtx* h, int s0, int len, bool pick_obj = false);
// Whether (and the tables with which) the objective of the one-hot groups'
// variables can come from the picks: rebuilt when groups or repairs change.
cudaError_t gf_ensure_pick_obj(GfCtx* h);
// Interleaved scaled values of the long-column slices (at load).
cudaError_t gf_fill_slices(GfCtx* h, const int64_t* src_d);
cudaError_t gf_launch_fused(GfCtx* h, const float* p, int s0, int len);
cudaError_t gf_launch_dense_score(GfCtx* h, const GfDenseQ& dq, int s0, int len);
cudaError_t gf_launch_incumbent(GfCtx* h, int s0, int len, int mode, bool last_chunk);
cudaError_t gf_launch_stats(GfCtx* h);
cudaError_t gf_launch_features(GfCtx* h);
cudaError_t gf_launch_mlp_proposal(GfCtx* h);
cudaError_t gf_launch_final_round(GfCtx* h);

// phase profiling: returns an index to pass to gf_prof_end (or -1)
int gf_prof_begin(GfCtx* h, int phase);
void gf_prof_end(GfCtx* h, int idx, int count);

// bit words of bf16 candidate rows (k_sample.cu)
__global__ void k_dense_bits(const void* __restrict__ Xs, int len, int64_t ld,
                             uint32_t* __restrict__ Xb, int f8);

// helpers used by several files
int64_t gf_round_up(int64_t v, int64_t m);
