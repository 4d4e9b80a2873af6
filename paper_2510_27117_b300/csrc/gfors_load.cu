// gfors_load.cu -- loading a batch of instances and Preprocess (Section 3).
//
// Host (FP64): K = -[A;B] and r = (b;d) per instance (Eq. 2), duplicate
// entries summed, every row divided by its 2-norm; Q symmetrised as
// (Q + Q^T)/2 (Eq. 1); integer rows classified for exact evaluation;
// the batch concatenated block-diagonally; K^T built as CSC.
// Device (FP64): ||Q_sym||_2 and ||K_rownormalised||_2 by power iteration;
// then s_obj = ||Q||_2 + ||c||_2, s_K = ||K||_2 and the FP32 scaled copies
// Q/s_obj, c/s_obj, K/s_K, r/s_K used by the PDHG kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <tuple>

#include <cuda_fp8.h>

#include "internal.cuh"

static thread_local std::string g_thread_err;
static gfors_alloc_fn g_alloc = nullptr;
static gfors_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::mutex g_alloc_mu;

extern cudaError_t gf_power_run(GfCtx* h, int which, const int64_t* Mp, const int32_t* Mc,
                                const double* Mv, const int64_t* Tp, const int32_t* Tr,
                                const double* Tv, int64_t mrows, const int32_t* rch,
                                int64_t nrch, const int32_t* rptr,
                                const double* const* dense_diag, double* norms, int* iters);
extern cudaError_t gf_scale_to_f32(GfCtx* h, const double* Kd, const double* Td,
                                   const double* rd, const double* cd, const double* Qd,
                                   const double* sK, const double* sobj);
void gf_set_slot(GfCtx* h, int parity, double rho);

int64_t gf_round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

gfors_status gf_fail(GfCtx* h, gfors_status st, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (st == GFORS_E_CUDA || st == GFORS_E_TIMEOUT) h->failed = true;
  } else {
    g_thread_err = msg;
  }
  return st;
}

gfors_status gf_cuda(GfCtx* h, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return gf_fail(h, GFORS_E_OOM, std::string("out of device memory in ") + what);
  }
  return gf_fail(h, GFORS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* gf_alloc(GfCtx* h, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc) {
      p = g_alloc(bytes, g_alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) h->allocs.push_back(p);
  return p;
}

void gf_free_one(GfCtx* h, void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  for (size_t q = 0; q < h->allocs.size(); ++q)
    if (h->allocs[q] == p) {
      h->allocs.erase(h->allocs.begin() + q);
      if (g_free) g_free(p, g_alloc_ctx);
      else cudaFree(p);
      return;
    }
}

void gf_free_all(GfCtx* h) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  for (void* p : h->allocs) {
    if (g_free) g_free(p, g_alloc_ctx);
    else cudaFree(p);
  }
  h->allocs.clear();
}

extern "C" void gfors_default_params(gfors_params* p) {
  memset(p, 0, sizeof(*p));
  p->sigma = 0.99;
  p->rho_min = 1e-3;
  p->rho_max = 1.0;
  p->T = 20.0;
  p->p = 2.0;
  p->delta = 0.0;
  p->k_int = 50;
  p->k_r = 1;
  p->k_b = 1024;
  p->tau_cap_by_L = -1;
  p->seed = 0x5EED0000ull;
  p->x0 = 0.5;
  p->halt_tol = 1e-4;
  p->stall_window = 20;
  p->inst_base = 0;
  p->sample_chunk = 0;
  p->eval_mode = 0;
  p->power_tol = 1e-12;
  p->power_maxit = 5000;
  p->wait_timeout_s = 2.0;
  p->pdhg_mode = 0;
}

extern "C" const char* gfors_version(void) { return "gfors-b300 0.1 (sm_103a)"; }

extern "C" gfors_status gfors_set_allocator(gfors_alloc_fn a, gfors_free_fn f, void* ctx) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if ((a == nullptr) != (f == nullptr)) {
    g_thread_err = "gfors_set_allocator: give both functions or neither";
    return GFORS_E_ARG;
  }
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
  return GFORS_OK;
}

extern "C" const char* gfors_last_error(gfors_handle h) {
  return h ? h->err.c_str() : g_thread_err.c_str();
}

extern "C" int64_t gfors_launch_count(gfors_handle h) { return h ? h->launches : 0; }

// ---------------------------------------------------------------------------
namespace {

// Rows in flat CSR form: local columns ascending, no duplicates, no zeros.
struct RowSet {
  std::vector<int64_t> ptr{0};
  std::vector<int32_t> col;
  std::vector<double> val;
  size_t size() const { return ptr.size() - 1; }
  int64_t len(size_t j) const { return ptr[j + 1] - ptr[j]; }
  const int32_t* c(size_t j) const { return col.data() + ptr[j]; }
  const double* v(size_t j) const { return val.data() + ptr[j]; }
  void add(int32_t cc, double vv) { col.push_back(cc); val.push_back(vv); }
  void close() { ptr.push_back((int64_t)col.size()); }
};

bool check_csr(const gfors_csr* M, int64_t ncols, std::string& why) {
  if (!M) return true;
  if (M->rows < 0 || M->nnz < 0 || M->cols != ncols) {
    why = "CSR shape mismatch (cols must equal n)";
    return false;
  }
  if (M->rows > 0 && !M->row_ptr) { why = "CSR row_ptr is NULL"; return false; }
  if (M->rows > 0 && M->row_ptr[0] != 0) { why = "CSR row_ptr[0] != 0"; return false; }
  for (int64_t r = 0; r < M->rows; ++r)
    if (M->row_ptr[r + 1] < M->row_ptr[r]) { why = "CSR row_ptr not monotone"; return false; }
  if (M->rows > 0 && M->row_ptr[M->rows] != M->nnz) { why = "CSR nnz mismatch"; return false; }
  if (M->nnz > 0 && (!M->col_idx || !M->val)) { why = "CSR arrays NULL"; return false; }
  for (int64_t t = 0; t < M->nnz; ++t) {
    if (M->col_idx[t] < 0 || M->col_idx[t] >= ncols) { why = "CSR column out of range"; return false; }
    if (!std::isfinite(M->val[t])) { why = "CSR value not finite"; return false; }
  }
  return true;
}

// Row r of M appended to R with duplicate columns summed (in input order),
// columns ascending and zero sums dropped.
void append_merged(RowSet& R, const gfors_csr* M, int64_t r,
                   std::vector<std::pair<int32_t, double>>& e) {
  const int64_t t0 = M->row_ptr[r], t1 = M->row_ptr[r + 1];
  bool sorted = true;
  for (int64_t t = t0 + 1; t < t1 && sorted; ++t) sorted = M->col_idx[t] > M->col_idx[t - 1];
  if (sorted) {
    for (int64_t t = t0; t < t1; ++t)
      if (M->val[t] != 0.0) R.add(M->col_idx[t], M->val[t]);
  } else {
    e.clear();
    for (int64_t t = t0; t < t1; ++t) e.emplace_back(M->col_idx[t], M->val[t]);
    std::stable_sort(e.begin(), e.end(),
                     [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                       return x.first < y.first;
                     });
    for (size_t q = 0; q < e.size();) {
      size_t u = q;
      double sum = 0.0;
      while (u < e.size() && e[u].first == e[q].first) sum += e[u++].second;
      if (sum != 0.0) R.add(e[q].first, sum);
      q = u;
    }
  }
  R.close();
}

bool is_int31(double v) { return std::floor(v) == v && std::fabs(v) < 2147483648.0; }

long long floor_div(long long a, long long b) {   // b != 0
  long long q = a / b, r = a % b;
  if (r != 0 && ((r < 0) != (b < 0))) --q;
  return q;
}
long long ceil_div(long long a, long long b) { return -floor_div(-a, b); }

// Host-side staging of one instance before concatenation.
struct Stage {
  RowSet orig;                    // A rows then B rows, original values (merged)
  std::vector<double> r;          // (b; d), divided by the row norms
  std::vector<uint8_t> eq;
  std::vector<double> rownorm;    // rows of K = -orig / rownorm
  std::vector<long long> rhs;     // integer right-hand sides (evaluation)
  RowSet Qsym;                    // (Q + Q^T)/2 per variable (sparse Q)
  RowSet Qorig;                   // original Q rows (sparse Q)
  bool dense = false;             // dense small-integer Q (tensor-core path)
  GfDenseQ dq;
  std::vector<double> dense_diag;
  std::vector<__nv_bfloat16> dense_w2;
  // evaluation rows of this instance (local offsets into ucols / gcols)
  std::vector<GfURow> ur;
  std::vector<int32_t> ucols;
  std::vector<GfPRow> pr;
  std::vector<GfPChunk> pch;
  std::vector<GfPSlice> psl;
  std::vector<GfGRow> gr;
  std::vector<int32_t> gcols, gvals;
  gfors_status status = GFORS_OK;
  std::string err;
};

// Run f(q) for q in [0, count) on up to hardware_concurrency threads; an
// exception in f(q) is returned as text (first failing q).
template <class F>
std::string parallel_for(int count, F&& f) {
  const int nt = std::min<int>(count, std::max(1u, std::thread::hardware_concurrency()));
  std::vector<std::string> errs(count);
  auto run = [&](int q) {
    try {
      f(q);
    } catch (const std::exception& ex) {
      errs[q] = ex.what();
    } catch (...) {
      errs[q] = "unknown exception";
    }
  };
  if (nt <= 1) {
    for (int q = 0; q < count; ++q) run(q);
  } else {
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&]() {
        for (int q; (q = next.fetch_add(1)) < count;) run(q);
      });
    for (auto& x : th) x.join();
  }
  for (int q = 0; q < count; ++q)
    if (!errs[q].empty()) return "instance " + std::to_string(q) + ": " + errs[q];
  return std::string();
}

// Preprocess step 1 and the Q classification of one instance (host, FP64).
void stage_instance(int q, GfInstHost& I, Stage& S, const gfors_params& P,
                    const gfors_csr* Aq, const double* bq, const gfors_csr* Bq,
                    const double* dq_rhs, const gfors_qmat* Qq, const double* cq) {
  auto fail = [&](const std::string& why) {
    S.status = GFORS_E_ARG;
    S.err = "instance " + std::to_string(q) + ": " + why;
  };
  std::string why;
  if (!check_csr(Aq, I.n, why) || !check_csr(Bq, I.n, why)) return fail(why);
  bool integral = true;
  for (int64_t i = 0; i < I.n; ++i) {
    if (!std::isfinite(cq[i])) return fail("c not finite");
    integral &= is_int31(cq[i]);
  }
  // rows of K = -[A;B] (Eq. 2) and the original rows for evaluation
  std::vector<std::pair<int32_t, double>> scratch;
  const int64_t nnz0 = (Aq ? Aq->nnz : 0) + (Bq ? Bq->nnz : 0);
  S.orig.ptr.reserve(I.m1 + I.m2 + 1);
  S.orig.col.reserve(nnz0);
  S.orig.val.reserve(nnz0);
  for (int part = 0; part < 2; ++part) {
    const gfors_csr* M = part ? Bq : Aq;
    const double* rhs = part ? dq_rhs : bq;
    if (!M) continue;
    for (int64_t r = 0; r < M->rows; ++r) {
      if (!std::isfinite(rhs[r])) return fail("rhs not finite");
      append_merged(S.orig, M, r, scratch);
      const size_t j = S.orig.size() - 1;
      for (int64_t u = 0; u < S.orig.len(j); ++u) integral &= is_int31(S.orig.v(j)[u]);
      integral &= is_int31(rhs[r]);
      S.r.push_back(rhs[r]);
      S.eq.push_back((uint8_t)part);
      S.rhs.push_back(is_int31(rhs[r]) ? (long long)rhs[r] : 0);
    }
  }
  // Preprocess step 1: row 2-norms
  S.rownorm.resize(S.orig.size());
  for (size_t j = 0; j < S.orig.size(); ++j) {
    double sq = 0.0;
    for (int64_t u = 0; u < S.orig.len(j); ++u) sq += S.orig.v(j)[u] * S.orig.v(j)[u];
    sq = sqrt(sq);
    S.rownorm[j] = sq;
    if (sq > 0.0) {
      S.r[j] /= sq;
    } else if ((!S.eq[j] && S.r[j] > 0.0) || (S.eq[j] && S.r[j] != 0.0)) {
      return fail("empty row " + std::to_string(j) + " cannot be satisfied");
    }
  }
  // Q
  I.qkind = 0;
  if (Qq && Qq->kind == 1) {
    if (!Qq->dense_rowmajor) return fail("dense Q pointer is NULL");
    const double* Qd = Qq->dense_rowmajor;
    bool qint = true;
    long long w2max = 0;
    for (int64_t i = 0; i < I.n && qint; ++i)
      for (int64_t j = 0; j < I.n; ++j) {
        const double v = Qd[i * I.n + j];
        if (!std::isfinite(v)) return fail("Q not finite");
        if (!is_int31(v)) { qint = false; break; }
        if (i != j) {
          double w = v + Qd[j * I.n + i];
          if (std::fabs(w) > (double)w2max) w2max = (long long)std::fabs(w);
        }
      }
    const bool tc = qint && integral && I.m1 + I.m2 == 0 && w2max <= 256 &&
                    (double)I.n * (double)w2max < 16777216.0 && P.eval_mode != 1 &&
                    P.eval_mode != 2;
    if (tc) {
      I.qkind = 1;
      GfDenseQ& dq = S.dq;
      dq.inst = q;
      dq.n = I.n;
      dq.ld = gf_round_up(I.n, 64);
      dq.w2max = w2max;
      {
        // tensor-core scoring keeps every per-tile partial in int32:
        // 128 rows x (n max|W2| + 2 max|c_i + Q_ii|) < 2^31
        double maxlin = 0.0;
        for (int64_t i = 0; i < I.n; ++i)
          maxlin = std::max(maxlin, std::fabs(cq[i] + Qd[i * I.n + i]));
        dq.tc_ok = 128.0 * ((double)I.n * (double)w2max + 2.0 * maxlin) < 2147483648.0;
      }
      S.dense_w2.assign((size_t)I.n * dq.ld, __float2bfloat16(0.0f));
      S.dense_diag.resize(I.n);
      for (int64_t i = 0; i < I.n; ++i) {
        for (int64_t j = 0; j < I.n; ++j)
          if (i != j)
            S.dense_w2[(size_t)i * dq.ld + j] =
                __float2bfloat16((float)(Qd[i * I.n + j] + Qd[j * I.n + i]));
        S.dense_diag[i] = Qd[i * I.n + i];
      }
      S.dense = true;
    } else {
      I.qkind = 2;
      for (int64_t i = 0; i < I.n; ++i) {
        for (int64_t j = 0; j < I.n; ++j) {
          const double v = Qd[i * I.n + j];
          if (v != 0.0) S.Qorig.add((int32_t)j, v);
          const double sv = 0.5 * (v + Qd[j * I.n + i]);
          if (sv != 0.0) S.Qsym.add((int32_t)j, sv);
          integral &= is_int31(v);
        }
        S.Qorig.close();
        S.Qsym.close();
      }
    }
  } else if (Qq && Qq->kind == 2) {
    if (!check_csr(&Qq->sparse, I.n, why) || Qq->sparse.rows != I.n) return fail("Q: " + why);
    I.qkind = 2;
    std::vector<std::vector<std::pair<int32_t, double>>> sym(I.n);
    for (int64_t i = 0; i < I.n; ++i) {
      append_merged(S.Qorig, &Qq->sparse, i, scratch);
      for (int64_t t = 0; t < S.Qorig.len(i); ++t) {
        const int32_t j = S.Qorig.c(i)[t];
        const double v = S.Qorig.v(i)[t];
        integral &= is_int31(v);
        sym[i].emplace_back(j, 0.5 * v);
        sym[j].emplace_back((int32_t)i, 0.5 * v);
      }
    }
    bool any = false;
    for (int64_t i = 0; i < I.n; ++i) {
      auto& e = sym[i];
      std::stable_sort(e.begin(), e.end(),
                       [](const std::pair<int32_t, double>& x,
                          const std::pair<int32_t, double>& y) { return x.first < y.first; });
      for (size_t u = 0; u < e.size();) {
        size_t w = u;
        double sum = 0.0;
        while (w < e.size() && e[w].first == e[u].first) sum += e[w++].second;
        if (sum != 0.0) { S.Qsym.add(e[u].first, sum); any = true; }
        u = w;
      }
      S.Qsym.close();
    }
    if (!any) I.qkind = 0;
  } else if (Qq && Qq->kind != 0) {
    return fail("Q.kind must be 0, 1 or 2");
  }
  I.integral = integral;
  I.cap = (P.tau_cap_by_L < 0) ? (I.qkind != 0) : (P.tau_cap_by_L != 0);
  I.single_row = (I.m1 == 1 && I.m2 == 0 && I.qkind == 0);
}

// P rows in runs (v1 in constant steps, one v2, one table; e.g. linking
// rows x_ij <= y_i over j) become chunks of up to kPChunk rows that carry no
// per-row data; the rest stay single rows.  Row order changes no count.
void extract_p_runs(std::vector<GfPRow>& pr, std::vector<GfPChunk>& pch) {
  // orient each two-variable row so that its more frequent variable (a hub
  // such as y_i) is v2: swapping x1 and x2 swaps bits 1 and 2 of the table
  {
    if (pr.empty()) return;
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    for (const GfPRow& R : pr) {
      lo = std::min(lo, R.v1);
      hi = std::max(hi, R.v1);
      if (R.v2 >= 0) {
        lo = std::min(lo, R.v2);
        hi = std::max(hi, R.v2);
      }
    }
    std::vector<int32_t> cnt_v((size_t)((int64_t)hi - lo + 1), 0);
    auto cnt = [&](int32_t v) -> int32_t& { return cnt_v[(size_t)(v - lo)]; };
    for (const GfPRow& R : pr) {
      ++cnt(R.v1);
      if (R.v2 >= 0) ++cnt(R.v2);
    }
    for (GfPRow& R : pr) {
      if (R.v2 < 0) continue;
      const int32_t a = cnt(R.v1), b = cnt(R.v2);
      if (a > b || (a == b && R.v1 > R.v2)) {
        std::swap(R.v1, R.v2);
        const uint32_t t = R.table;
        R.table = (t & 9u) | ((t & 2u) << 1) | ((t & 4u) >> 1);
      }
    }
  }
  std::sort(pr.begin(), pr.end(), [](const GfPRow& a, const GfPRow& b) {
    if (a.table != b.table) return a.table < b.table;
    if (a.v2 != b.v2) return a.v2 < b.v2;
    return a.v1 < b.v1;
  });
  std::vector<GfPRow> rest;
  size_t i = 0;
  while (i < pr.size()) {
    const auto same = [&](size_t k) {
      return pr[k].table == pr[i].table && pr[k].v2 == pr[i].v2;
    };
    size_t j = i + 1;
    int64_t d = 0;
    if (j < pr.size() && same(j) && pr[j].v1 > pr[i].v1) {
      d = (int64_t)pr[j].v1 - pr[i].v1;
      while (j < pr.size() && same(j) && (int64_t)pr[j].v1 - pr[j - 1].v1 == d) ++j;
    }
    if (j - i >= (size_t)kMinPRun && pr[i].v2 >= 0 && d <= INT32_MAX) {
      for (size_t a = i; a < j; a += kPChunk) {
        GfPChunk C{};
        C.inst = pr[i].inst;
        C.v1 = pr[a].v1;
        C.v2 = pr[i].v2;
        C.table = pr[i].table;
        C.len = (int32_t)std::min<size_t>(kPChunk, j - a);
        C.stride = (int32_t)d;
        pch.push_back(C);
      }
    } else {
      rest.insert(rest.end(), pr.begin() + i, pr.begin() + j);
    }
    i = j;
  }
  pr.swap(rest);
}

// Chunks of equal table, stride and length whose hubs are consecutive and
// whose first rows are consecutive (v1 - v2 equal; e.g. the same customer
// range of consecutive facilities' linking rows) are put side by side in
// slices of up to 32: lane l of a warp then reads variable v1 + l + e stride,
// adjacent to its neighbours'.  Chunks in no slice of 8 or more stay.
void slice_p_chunks(std::vector<GfPChunk>& pch, std::vector<GfPSlice>& psl) {
  std::vector<size_t> ord(pch.size());
  std::iota(ord.begin(), ord.end(), 0);
  auto key = [&](size_t i) {
    const GfPChunk& C = pch[i];
    return std::make_tuple(C.table, C.stride, C.len, (int64_t)C.v1 - C.v2, C.v2);
  };
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return key(a) < key(b); });
  std::vector<GfPChunk> rest;
  size_t i = 0;
  while (i < ord.size()) {
    const GfPChunk& A = pch[ord[i]];
    size_t j = i + 1;
    while (j < ord.size()) {
      const GfPChunk& B = pch[ord[j]];
      const GfPChunk& P = pch[ord[j - 1]];
      if (B.table != A.table || B.stride != A.stride || B.len != A.len ||
          (int64_t)B.v1 - B.v2 != (int64_t)A.v1 - A.v2 || B.v2 != P.v2 + 1)
        break;
      ++j;
    }
    if (j - i >= 8) {
      for (size_t a = i; a < j; a += 32) {
        const GfPChunk& C = pch[ord[a]];
        // kPSliceRows rows per warp (more, shorter warps)
        for (int32_t e0 = 0; e0 < C.len; e0 += kPSliceRows) {
          GfPSlice S{};
          S.inst = C.inst;
          S.v1 = (int32_t)(C.v1 + (int64_t)e0 * C.stride);
          S.v2 = C.v2;
          S.table = C.table;
          S.len = std::min<int32_t>(kPSliceRows, C.len - e0);
          S.stride = C.stride;
          S.lanes = (int32_t)std::min<size_t>(32, j - a);
          psl.push_back(S);
        }
      }
    } else {
      for (size_t a = i; a < j; ++a) rest.push_back(pch[ord[a]]);
    }
    i = j;
  }
  pch.swap(rest);
}

// Integer evaluation rows of one instance (original data): P rows (<= 2
// nonzeros, truth table), U rows (equal coefficients: a count bound), G rows.
void stage_eval_rows(int q, const GfInstHost& I, Stage& S) {
  for (size_t j = 0; j < S.orig.size(); ++j) {
    const int32_t* oc = S.orig.c(j);
    const double* ov = S.orig.v(j);
    const long long rhs = S.rhs[j];
    const bool eq = S.eq[j] != 0;
    const int len = (int)S.orig.len(j);
    if (len <= 2) {
      GfPRow R;
      R.inst = q;
      R.v1 = len >= 1 ? (int32_t)(I.var_off + oc[0]) : 0;
      R.v2 = len >= 2 ? (int32_t)(I.var_off + oc[1]) : -1;
      R.table = 0;
      for (int m = 0; m < 4; ++m) {
        const int x1 = m & 1, x2 = (m >> 1) & 1;
        if (len < 1 && x1) continue;
        if (len < 2 && x2) continue;
        long long sum = (len >= 1 ? (long long)ov[0] * x1 : 0) +
                        (len >= 2 ? (long long)ov[1] * x2 : 0);
        const bool bad = eq ? (sum != rhs) : (sum < rhs);
        if (bad) R.table |= 1u << m;
      }
      if (len == 0) R.v1 = (int32_t)I.var_off;      // read any word; table uses x1=0
      if (len == 0 && R.table) R.table = 0xFu;      // constant violated row
      if (R.table) S.pr.push_back(R);
      continue;
    }
    bool uni = len < 65536;
    for (int t = 1; t < len && uni; ++t) uni = (ov[t] == ov[0]);
    bool placed = false;
    if (uni) {
      const long long a = (long long)ov[0];
      long long L = 0, U = -1;
      bool ok = true;
      if (!eq) {
        if (a > 0) { L = std::max(0ll, ceil_div(rhs, a)); U = -1; }
        else { U = floor_div(rhs, a); L = 0; if (U < 0) ok = false; }
        if (L > len) ok = false;
      } else {
        if (rhs % a != 0) ok = false;
        else { L = U = rhs / a; if (L < 0 || L > len) ok = false; }
      }
      if (ok && U >= len) U = -1;
      if (ok) {
        if (L <= 0 && U < 0) { placed = true; }      // never violated
        else if (L < 65536 && U < 65536) {
          GfURow R;
          R.inst = q;
          R.len = len;
          R.t0 = (int64_t)S.ucols.size();             // local; shifted on concatenation
          R.L = (int32_t)L;
          R.U = (int32_t)U;
          for (int t = 0; t < len; ++t) S.ucols.push_back((int32_t)(I.var_off + oc[t]));
          S.ur.push_back(R);
          placed = true;
        }
      }
    }
    if (!placed) {
      GfGRow R;
      R.inst = q;
      R.len = len;
      R.t0 = (int64_t)S.gcols.size();                 // local; shifted on concatenation
      R.rhs = rhs;
      R.eq = eq;
      R.pad = 0;
      for (int t = 0; t < len; ++t) {
        S.gcols.push_back((int32_t)(I.var_off + oc[t]));
        S.gvals.push_back((int32_t)ov[t]);
      }
      S.gr.push_back(R);
    }
  }
  extract_p_runs(S.pr, S.pch);
  slice_p_chunks(S.pch, S.psl);
}

}  // namespace

void gf_set_slot(GfCtx* h, int parity, double rho) {
  std::vector<GfIParam> v(h->ninst);
  for (int b = 0; b < h->ninst; ++b) {
    double t1 = sqrt(h->prm.sigma);
    if (h->ih[b].cap) {
      double L = 2.0 * (h->ih[b].normQhat + rho);
      if (L > 0.0 && 1.0 / (2.0 * L) < t1) t1 = 1.0 / (2.0 * L);
    }
    double t2 = h->prm.sigma / t1;
    GfIParam q;
    q.tau1 = (float)t1; q.tau2 = (float)t2; q.rho = (float)rho; q.pad = 0.f;
    q.tau1d = t1; q.tau2d = t2; q.rhod = rho; q.normQ = h->ih[b].normQhat;
    v[b] = q;
  }
  cudaMemcpyAsync(h->iprm + (size_t)parity * h->ninst, v.data(), sizeof(GfIParam) * h->ninst,
                  cudaMemcpyHostToDevice, h->stream);
}

// Runs of a bucket's (ascending) ids: maximal stretches of consecutive ids of
// one instance; uniform when all have the same length (ptr differences).
// Used instead of the id list when there are at most kMaxRuns of them, or
// when they hold at least kMinRunLen ids on average (a kernel finds a run by
// binary search over the run offsets, once per row group or block, which
// long runs amortise).
constexpr int kMaxRuns = 4096;
constexpr int64_t kMinRunLen = 32;
// Blocks of 32 sparse-Q pairs per evaluation chunk (one CUDA block of 8 warps).
constexpr int kQChunkBlocks = 64;
static bool make_runs(const std::vector<int32_t>& ids, const std::vector<int64_t>& ptr,
                      const std::vector<int32_t>& inst_of, std::vector<GfRun>& runs,
                      std::vector<int64_t>& run_ptr) {
  runs.clear();
  run_ptr.assign(1, 0);
  for (size_t u = 0; u < ids.size(); ++u) {
    const int32_t id = ids[u];
    const int32_t len = (int32_t)(ptr[id + 1] - ptr[id]);
    GfRun* R = runs.empty() ? nullptr : &runs.back();
    if (R && id == R->first + R->count && inst_of[id] == R->inst) {
      if (R->len != len) R->len = -1;
      R->count++;
    } else {
      // many short runs: the id list serves better
      if ((int64_t)runs.size() >= kMaxRuns &&
          (int64_t)runs.size() * kMinRunLen > (int64_t)ids.size())
        return false;
      if (runs.size() >= (size_t)INT32_MAX) return false;
      runs.push_back(GfRun{id, ptr[id], 1, len, inst_of[id], 0});
    }
  }
  int64_t acc = 0;
  for (const GfRun& R : runs) run_ptr.push_back(acc += R.count);
  return true;
}

static gfors_status load_impl(GfCtx* h, int32_t ninst, const gfors_csr* const* A,
                              const double* const* b, const gfors_csr* const* B,
                              const double* const* d, const gfors_qmat* const* Q,
                              const double* const* c, const int64_t* n) {
  const gfors_params& P = h->prm;
  if (ninst <= 0) return gf_fail(h, GFORS_E_ARG, "ninst must be positive");
  if (P.k_int < 1 || P.k_r < 0 || P.k_b < 32 || P.k_b % 32 != 0)
    return gf_fail(h, GFORS_E_ARG, "need k_int >= 1, k_r >= 0, k_b a positive multiple of 32");
  if (!(P.sigma > 0.0) || !(P.sigma <= 1.0))
    return gf_fail(h, GFORS_E_ARG, "sigma must lie in (0, 1]");
  if (P.sample_chunk < 0 || P.sample_chunk % 32 != 0)
    return gf_fail(h, GFORS_E_ARG, "sample_chunk must be a multiple of 32");
  h->ninst = ninst;
  h->ih.assign(ninst, GfInstHost());
  std::vector<Stage> st(ninst);
  int64_t voff = 0, roff = 0;
  for (int q = 0; q < ninst; ++q) {          // sizes and offsets (serial)
    GfInstHost& I = h->ih[q];
    if (!n || n[q] <= 0) return gf_fail(h, GFORS_E_ARG, "n must be positive");
    if (n[q] >= (1ll << 30)) return gf_fail(h, GFORS_E_UNSUPPORTED, "n >= 2^30");
    if (!c || !c[q]) return gf_fail(h, GFORS_E_ARG, "c is NULL");
    const gfors_csr* Aq = A ? A[q] : nullptr;
    const gfors_csr* Bq = B ? B[q] : nullptr;
    I.n = n[q];
    I.npad = gf_round_up(I.n, 64);
    I.m1 = Aq ? std::max<int64_t>(0, Aq->rows) : 0;
    I.m2 = Bq ? std::max<int64_t>(0, Bq->rows) : 0;
    if (I.m1 && (!b || !b[q])) return gf_fail(h, GFORS_E_ARG, "b is NULL");
    if (I.m2 && (!d || !d[q])) return gf_fail(h, GFORS_E_ARG, "d is NULL");
    I.var_off = voff;
    I.row_off = roff;
    voff += I.npad;
    roff += I.m1 + I.m2;
  }
  {
    const std::string ex = parallel_for(ninst, [&](int q) {
      stage_instance(q, h->ih[q], st[q], P, A ? A[q] : nullptr, b ? b[q] : nullptr,
                     B ? B[q] : nullptr, d ? d[q] : nullptr, Q ? Q[q] : nullptr, c[q]);
    });
    if (!ex.empty()) return gf_fail(h, GFORS_E_OOM, "staging: " + ex);
  }
  for (int q = 0; q < ninst; ++q) {
    if (st[q].status != GFORS_OK) return gf_fail(h, st[q].status, st[q].err);
    GfInstHost& I = h->ih[q];
    if (st[q].dense) {
      I.dense_idx = (int)h->dense.size();
      h->dense.push_back(st[q].dq);
    }
    h->all_integral &= I.integral;
  }
  h->N = voff;
  h->M = roff;
  const int64_t N = h->N, M = h->M;
  if (N >= (1ll << 31) - 64) return gf_fail(h, GFORS_E_UNSUPPORTED, "total variables >= 2^31");

  // ---------------- concatenate K (FP64, global indices) and build CSC
  std::vector<int64_t> Kp(M + 1, 0);
  std::vector<int32_t> row_inst(M), Kc;
  std::vector<double> Kd, rd(M);
  std::vector<uint8_t> row_eq(M);
  for (int q = 0; q < ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    for (size_t j = 0; j < st[q].orig.size(); ++j) {
      const int64_t gj = I.row_off + (int64_t)j;
      Kp[gj + 1] = st[q].orig.len(j);
      row_inst[gj] = q;
      rd[gj] = st[q].r[j];
      row_eq[gj] = st[q].eq[j];
    }
  }
  for (int64_t j = 0; j < M; ++j) Kp[j + 1] += Kp[j];
  h->nnzK = Kp[M];
  if (h->nnzK >= (1ll << 31)) return gf_fail(h, GFORS_E_UNSUPPORTED, "nnz(K) >= 2^31");
  Kc.resize(h->nnzK);
  Kd.resize(h->nnzK);
  std::vector<int64_t> Tp(N + 1, 0);
  std::vector<int32_t> Tr(h->nnzK);
  std::vector<double> Td(h->nnzK);
  {
    // per instance (disjoint row, column and nnz ranges): K rows with global
    // columns and values -a / ||a||, column counts, then the transpose
    std::string ex = parallel_for(ninst, [&](int q) {
      const GfInstHost& I = h->ih[q];
      const Stage& S = st[q];
      for (size_t j = 0; j < S.orig.size(); ++j) {
        int64_t t = Kp[I.row_off + (int64_t)j];
        const double nr = S.rownorm[j];
        for (int64_t u = 0; u < S.orig.len(j); ++u, ++t) {
          Kc[t] = (int32_t)(I.var_off + S.orig.c(j)[u]);
          const double k = -S.orig.v(j)[u];
          Kd[t] = nr > 0.0 ? k / nr : k;
          Tp[Kc[t] + 1]++;
        }
      }
    });
    if (!ex.empty()) return gf_fail(h, GFORS_E_OOM, "K: " + ex);
    for (int64_t i = 0; i < N; ++i) Tp[i + 1] += Tp[i];
    ex = parallel_for(ninst, [&](int q) {
      const GfInstHost& I = h->ih[q];
      std::vector<int64_t> fill(Tp.begin() + I.var_off, Tp.begin() + I.var_off + I.npad);
      for (int64_t j = I.row_off; j < I.row_off + I.m1 + I.m2; ++j)
        for (int64_t t = Kp[j]; t < Kp[j + 1]; ++t) {
          const int64_t pos = fill[Kc[t] - I.var_off]++;
          Tr[pos] = (int32_t)j;
          Td[pos] = Kd[t];
        }
    });
    if (!ex.empty()) return gf_fail(h, GFORS_E_OOM, "K^T: " + ex);
  }
  // Q_sym (sparse instances), global indices
  std::vector<int64_t> Qp(N + 1, 0);
  std::vector<int32_t> Qc;
  std::vector<double> Qd;
  for (int q = 0; q < ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    if (I.qkind != 2) continue;
    for (int64_t i = 0; i < I.n; ++i) Qp[I.var_off + i + 1] = st[q].Qsym.len(i);
  }
  for (int64_t i = 0; i < N; ++i) Qp[i + 1] += Qp[i];
  h->nnzQ = Qp[N];
  Qc.resize(h->nnzQ);
  Qd.resize(h->nnzQ);
  for (int q = 0; q < ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    if (I.qkind != 2) continue;
    for (int64_t i = 0; i < I.n; ++i) {
      int64_t t = Qp[I.var_off + i];
      for (int64_t u = 0; u < st[q].Qsym.len(i); ++u, ++t) {
        Qc[t] = (int32_t)(I.var_off + st[q].Qsym.c(i)[u]);
        Qd[t] = st[q].Qsym.v(i)[u];
      }
    }
  }
  std::vector<int32_t> var_inst(N);
  std::vector<uint8_t> live(N, 0);
  std::vector<int64_t> var_off(ninst + 1);
  std::vector<double> cd(N, 0.0);
  std::vector<long long> cint(N, 0);
  for (int q = 0; q < ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    var_off[q] = I.var_off;
    for (int64_t i = 0; i < I.npad; ++i) var_inst[I.var_off + i] = q;
    for (int64_t i = 0; i < I.n; ++i) {
      live[I.var_off + i] = 1;
      cd[I.var_off + i] = c[q][i];
      cint[I.var_off + i] = I.integral ? (long long)c[q][i] : 0;
    }
  }
  var_off[ninst] = N;

  // ---------------- device allocations
  cudaStream_t s = h->stream;
#define ALLOC(ptr, T, cnt)                                          \
  do {                                                              \
    ptr = gf_alloc_t<T>(h, (size_t)(cnt));                          \
    if (!ptr) return gf_fail(h, GFORS_E_OOM, "allocating " #ptr);   \
  } while (0)
#define UP(dst, src, T, cnt) \
  GF_CK(h, cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)(cnt), cudaMemcpyHostToDevice, s))

  ALLOC(h->var_off_d, int64_t, ninst + 1);
  ALLOC(h->var_inst, int32_t, N);
  ALLOC(h->var_live, uint8_t, N);
  ALLOC(h->row_inst, int32_t, M);
  ALLOC(h->row_eq, uint8_t, M);
  ALLOC(h->Kp, int64_t, M + 1);
  ALLOC(h->Kc, int32_t, h->nnzK);
  ALLOC(h->Kv, float, h->nnzK);
  ALLOC(h->Tp, int64_t, N + 1);
  ALLOC(h->Tr, int32_t, h->nnzK);
  ALLOC(h->Tv, float, h->nnzK);
  ALLOC(h->Qp, int64_t, N + 1);
  ALLOC(h->Qc, int32_t, h->nnzQ);
  ALLOC(h->Qv, float, h->nnzQ);
  ALLOC(h->rhat, float, M);
  ALLOC(h->chat, float, N);
  UP(h->var_off_d, var_off.data(), int64_t, ninst + 1);
  UP(h->var_inst, var_inst.data(), int32_t, N);
  UP(h->var_live, live.data(), uint8_t, N);
  UP(h->row_inst, row_inst.data(), int32_t, M);
  UP(h->row_eq, row_eq.data(), uint8_t, M);
  UP(h->Kp, Kp.data(), int64_t, M + 1);
  UP(h->Kc, Kc.data(), int32_t, h->nnzK);
  UP(h->Tp, Tp.data(), int64_t, N + 1);
  UP(h->Tr, Tr.data(), int32_t, h->nnzK);
  UP(h->Qp, Qp.data(), int64_t, N + 1);
  UP(h->Qc, Qc.data(), int32_t, h->nnzQ);

  // chunk tables for deterministic per-instance reductions
  {
    std::vector<int32_t> vch, vptr(ninst + 1), rch, rptr(ninst + 1);
    for (int q = 0; q < ninst; ++q) {
      const GfInstHost& I = h->ih[q];
      vptr[q] = (int32_t)(vch.size() / 3);
      for (int64_t a = 0; a < I.npad; a += 2048) {
        vch.push_back(q);
        vch.push_back((int32_t)(I.var_off + a));
        vch.push_back((int32_t)(I.var_off + std::min<int64_t>(I.npad, a + 2048)));
      }
      rptr[q] = (int32_t)(rch.size() / 3);
      for (int64_t a = 0; a < I.m1 + I.m2; a += 2048) {
        rch.push_back(q);
        rch.push_back((int32_t)(I.row_off + a));
        rch.push_back((int32_t)(I.row_off + std::min<int64_t>(I.m1 + I.m2, a + 2048)));
      }
    }
    vptr[ninst] = (int32_t)(vch.size() / 3);
    rptr[ninst] = (int32_t)(rch.size() / 3);
    h->nvchunk = (int64_t)vch.size() / 3;
    h->nrchunk = (int64_t)rch.size() / 3;
    ALLOC(h->vchunk, int32_t, vch.size());
    ALLOC(h->rchunk, int32_t, rch.size() + 3);
    ALLOC(h->vchunk_iptr, int32_t, ninst + 1);
    ALLOC(h->rchunk_iptr, int32_t, ninst + 1);
    UP(h->vchunk, vch.data(), int32_t, vch.size());
    if (!rch.empty()) UP(h->rchunk, rch.data(), int32_t, rch.size());
    UP(h->vchunk_iptr, vptr.data(), int32_t, ninst + 1);
    UP(h->rchunk_iptr, rptr.data(), int32_t, ninst + 1);
  }

  // dense operands
  std::vector<double*> ddiag(h->dense.size(), nullptr);
  for (size_t u = 0; u < h->dense.size(); ++u) {
    GfDenseQ& dq = h->dense[u];
    ALLOC(dq.W2, __nv_bfloat16, dq.n * dq.ld);
    if (dq.w2max <= 127) {             // biased byte copy for the PDHG GEMV (exact)
      ALLOC(dq.W2i8, uint8_t, dq.n * dq.ld);
      std::vector<uint8_t> w8((size_t)dq.n * dq.ld);
      const std::vector<__nv_bfloat16>& wb = st[dq.inst].dense_w2;
      for (size_t t = 0; t < w8.size(); ++t)
        w8[t] = (uint8_t)((int)__bfloat162float(wb[t]) + 128);
      UP(dq.W2i8, w8.data(), uint8_t, w8.size());
    }
    // FP8 E4M3 copy for the tensor-core scorer when every entry of W2 is
    // exactly representable in E4M3 (3 mantissa bits: all integers up to 16,
    // even ones up to 32, ...); the 0/1 candidates always are
    if (dq.tc_ok && P.eval_mode != 4 && P.eval_mode != 6) {
      std::vector<uint8_t> w8((size_t)dq.n * dq.ld);
      const std::vector<__nv_bfloat16>& wb = st[dq.inst].dense_w2;
      bool exact = true;
      for (size_t t = 0; t < w8.size() && exact; ++t) {
        const float v = __bfloat162float(wb[t]);
        const __nv_fp8_e4m3 q(v);
        exact = (float)q == v;
        w8[t] = q.__x;
      }
      if (exact) {
        ALLOC(dq.W2f8, uint8_t, dq.n * dq.ld);
        UP(dq.W2f8, w8.data(), uint8_t, w8.size());
        dq.f8 = true;
      }
    }
    ALLOC(dq.qdiag, float, dq.ld);
    ALLOC(dq.lin, long long, dq.ld);
    ALLOC(ddiag[u], double, dq.n);
    UP(dq.W2, st[dq.inst].dense_w2.data(), __nv_bfloat16, dq.n * dq.ld);
    UP(ddiag[u], st[dq.inst].dense_diag.data(), double, dq.n);
    std::vector<long long> lin(dq.ld, 0);
    for (int64_t i = 0; i < dq.n; ++i)
      lin[i] = (long long)c[dq.inst][i] + (long long)st[dq.inst].dense_diag[i];
    UP(dq.lin, lin.data(), long long, dq.ld);
  }

  // ---------------- Preprocess on the device: spectral norms (FP64)
  double *Kd_d = nullptr, *Td_d = nullptr, *Qd_d = nullptr, *rd_d = nullptr, *cd_d = nullptr;
  ALLOC(Kd_d, double, h->nnzK);
  ALLOC(Td_d, double, h->nnzK);
  ALLOC(Qd_d, double, h->nnzQ);
  ALLOC(rd_d, double, M);
  ALLOC(cd_d, double, N);
  UP(Kd_d, Kd.data(), double, h->nnzK);
  UP(Td_d, Td.data(), double, h->nnzK);
  UP(Qd_d, Qd.data(), double, h->nnzQ);
  UP(rd_d, rd.data(), double, M);
  UP(cd_d, cd.data(), double, N);
  GF_CK(h, cudaStreamSynchronize(s));
  std::vector<double> nQ(ninst, 0.0), nK(ninst, 0.0);
  std::vector<int> itQ(ninst, 0), itK(ninst, 0);
  GF_CK(h, gf_power_run(h, 1, h->nnzQ ? h->Qp : nullptr, Qc.empty() ? nullptr : h->Qc, Qd_d,
                        nullptr, nullptr, nullptr, N, nullptr, 0, nullptr, ddiag.data(),
                        nQ.data(), itQ.data()));
  if (M > 0)
    GF_CK(h, gf_power_run(h, 0, h->Kp, h->Kc, Kd_d, h->Tp, h->Tr, Td_d, M, h->rchunk,
                          h->nrchunk, h->rchunk_iptr, nullptr, nK.data(), itK.data()));
  std::vector<double> sK(ninst), sobj(ninst), nQhat(ninst);
  std::vector<int32_t> capv(ninst);
  for (int q = 0; q < ninst; ++q) {
    GfInstHost& I = h->ih[q];
    double cn = 0.0;
    for (int64_t i = 0; i < I.n; ++i) cn += c[q][i] * c[q][i];
    I.normQ_raw = nQ[q];
    I.s_obj = nQ[q] + sqrt(cn);
    if (I.s_obj == 0.0) I.s_obj = 1.0;
    I.normK = nK[q];
    I.s_K = nK[q] > 0.0 ? nK[q] : 1.0;
    I.normQhat = nQ[q] / I.s_obj;
    I.itQ = itQ[q];
    I.itK = itK[q];
    sK[q] = I.s_K;
    sobj[q] = I.s_obj;
    nQhat[q] = I.normQhat;
    capv[q] = I.cap;
  }
  double *sK_d = nullptr, *sobj_d = nullptr;
  ALLOC(sK_d, double, ninst);
  ALLOC(sobj_d, double, ninst);
  ALLOC(h->normQhat_d, double, ninst);
  ALLOC(h->cap_d, int32_t, ninst);
  UP(sK_d, sK.data(), double, ninst);
  UP(sobj_d, sobj.data(), double, ninst);
  UP(h->normQhat_d, nQhat.data(), double, ninst);
  UP(h->cap_d, capv.data(), int32_t, ninst);
  GF_CK(h, gf_scale_to_f32(h, Kd_d, Td_d, rd_d, cd_d, Qd_d, sK_d, sobj_d));
  for (GfDenseQ& dq : h->dense) {
    const GfInstHost& I = h->ih[dq.inst];
    std::vector<float> qd(dq.ld, 0.0f);
    for (int64_t i = 0; i < dq.n; ++i) qd[i] = (float)(st[dq.inst].dense_diag[i] / I.s_obj);
    UP(dq.qdiag, qd.data(), float, dq.ld);
    dq.qscale = (float)(0.5 / I.s_obj);
  }

  // ---------------- PDHG work lists (length buckets, long chunks)
  auto bucket_of = [](int64_t len) {
    if (len <= 2) return 0;
    if (len <= 8) return 1;
    if (len <= 32) return 2;
    if (len <= 128) return 3;
    if (len <= kLongLen) return 4;
    return 5;
  };
  static const int lanes_of[5] = {1, 4, 8, 16, 32};
  {
    std::vector<std::vector<int32_t>> rl(5);
    std::vector<GfChunk> ch;
    std::vector<int32_t> lid, lptr;
    for (int64_t j = 0; j < M; ++j) {
      const int64_t len = Kp[j + 1] - Kp[j];
      const int bk = bucket_of(len);
      if (bk < 5) {
        rl[bk].push_back((int32_t)j);
      } else {
        lid.push_back((int32_t)j);
        lptr.push_back((int32_t)ch.size());
        for (int64_t t = Kp[j]; t < Kp[j + 1]; t += kChunkLen)
          ch.push_back(GfChunk{(int32_t)j, 0, t, std::min(Kp[j + 1], t + kChunkLen)});
      }
    }
    lptr.push_back((int32_t)ch.size());
    for (int bk = 0; bk < 5; ++bk) {
      GfBucket B;
      B.lanes = lanes_of[bk];
      B.short_ok = bk == 0;
      B.count = (int32_t)rl[bk].size();
      if (B.count) {
        std::vector<GfRun> runs;
        std::vector<int64_t> rptr;
        if (make_runs(rl[bk], Kp, row_inst, runs, rptr)) {
          B.nruns = (int32_t)runs.size();
          ALLOC(B.runs, GfRun, runs.size());
          ALLOC(B.run_ptr, int64_t, rptr.size());
          UP(B.runs, runs.data(), GfRun, runs.size());
          UP(B.run_ptr, rptr.data(), int64_t, rptr.size());
        } else {
          ALLOC(B.ids, int32_t, B.count);
          UP(B.ids, rl[bk].data(), int32_t, B.count);
        }
      }
      h->rb.push_back(B);
    }
    h->rlong.nlong = (int32_t)lid.size();
    h->rlong.nchunks = (int32_t)ch.size();
    if (!lid.empty()) {
      ALLOC(h->rlong.ids, int32_t, lid.size());
      ALLOC(h->rlong.chunk_ptr, int32_t, lptr.size());
      ALLOC(h->rlong.chunks, GfChunk, ch.size());
      ALLOC(h->rlong.partial, float2, ch.size());
      UP(h->rlong.ids, lid.data(), int32_t, lid.size());
      UP(h->rlong.chunk_ptr, lptr.data(), int32_t, lptr.size());
      UP(h->rlong.chunks, ch.data(), GfChunk, ch.size());
    }
  }
  {
    std::vector<std::vector<int32_t>> cl(5);
    std::vector<GfChunk> ch;
    std::vector<int32_t> lid, lptr;
    for (int q = 0; q < ninst; ++q) {
      const GfInstHost& I = h->ih[q];
      if (I.qkind == 1) continue;            // dense kernel handles these
      for (int64_t i = I.var_off; i < I.var_off + I.n; ++i) {
        const int64_t lt = Tp[i + 1] - Tp[i], lq = Qp[i + 1] - Qp[i];
        const int bk = bucket_of(lt + lq);
        if (bk < 5) {
          cl[bk].push_back((int32_t)i);
        } else {
          lid.push_back((int32_t)i);
          lptr.push_back((int32_t)ch.size());
          for (int64_t t = Tp[i]; t < Tp[i + 1]; t += kChunkLen)
            ch.push_back(GfChunk{(int32_t)i, 0, t, std::min(Tp[i + 1], t + kChunkLen)});
          for (int64_t t = Qp[i]; t < Qp[i + 1]; t += kChunkLen)
            ch.push_back(GfChunk{(int32_t)i, 1, t, std::min(Qp[i + 1], t + kChunkLen)});
        }
      }
    }
    lptr.push_back((int32_t)ch.size());
    for (int bk = 0; bk < 5; ++bk) {
      GfBucket B;
      B.lanes = lanes_of[bk];
      B.short_ok = bk == 0;
      B.count = (int32_t)cl[bk].size();
      if (B.count) {
        std::vector<GfRun> runs;
        std::vector<int64_t> rptr;
        if (make_runs(cl[bk], Tp, var_inst, runs, rptr)) {
          B.nruns = (int32_t)runs.size();
          ALLOC(B.runs, GfRun, runs.size());
          ALLOC(B.run_ptr, int64_t, rptr.size());
          UP(B.runs, runs.data(), GfRun, runs.size());
          UP(B.run_ptr, rptr.data(), int64_t, rptr.size());
        } else {
          ALLOC(B.ids, int32_t, B.count);
          UP(B.ids, cl[bk].data(), int32_t, B.count);
        }
      }
      h->cb.push_back(B);
    }
    // runs of at least 8 consecutive long columns of one length (one
    // instance, no Q part) in slices of 32 with interleaved entries; their
    // chunks are marked part 2 (done by the slice kernel)
    std::vector<int4> sblk;
    std::vector<int64_t> soff, ssrc;
    std::vector<int32_t> slen, spb, sidx;
    for (size_t q = 0; q < lid.size();) {
      const int64_t i0 = lid[q];
      const int64_t L = Tp[i0 + 1] - Tp[i0];
      auto fits = [&](size_t k) {
        const int64_t i = lid[k];
        return Qp[i + 1] == Qp[i] && Tp[i + 1] - Tp[i] == L && var_inst[i] == var_inst[i0];
      };
      if (!fits(q)) {
        ++q;
        continue;
      }
      size_t r = q + 1;
      while (r < lid.size() && fits(r)) ++r;
      if (r - q >= 8 && L <= (int64_t)INT32_MAX / 32) {
        for (size_t a = q; a < r; a += 32) {
          const int nc = (int)std::min<size_t>(32, r - a);
          const int sl = (int)slen.size();
          soff.push_back((int64_t)sidx.size());
          slen.push_back((int32_t)L);
          for (int l = 0; l < 32; ++l) {
            if (l < nc) {
              spb.push_back(lptr[a + l]);
              ssrc.push_back(Tp[lid[a + l]]);
              for (int c = lptr[a + l]; c < lptr[a + l + 1]; ++c) ch[c].part = 2;
            } else {
              spb.push_back(-1);
              ssrc.push_back(-1);
            }
          }
          sidx.resize(sidx.size() + (size_t)L * 32);
          for (int64_t e = 0; e < L; ++e)
            for (int l = 0; l < 32; ++l)
              sidx[(size_t)(soff[sl] + 32 * e + l)] = (l < nc) ? Tr[Tp[lid[a + l]] + e] : -1;
          for (int64_t c = 0; c * kChunkLen < L; ++c) sblk.push_back(make_int4(sl, (int)c, nc, 0));
        }
      }
      q = r;
    }
    h->csl.nslices = (int32_t)slen.size();
    h->csl.nblocks = (int32_t)sblk.size();
    if (!slen.empty()) {
      ALLOC(h->csl.blk, int4, sblk.size());
      ALLOC(h->csl.off, int64_t, soff.size());
      ALLOC(h->csl.len, int32_t, slen.size());
      ALLOC(h->csl.pbase, int32_t, spb.size());
      ALLOC(h->csl.sidx, int32_t, sidx.size());
      ALLOC(h->csl.sval, float, sidx.size());
      int64_t* ssrc_d = gf_alloc_t<int64_t>(h, ssrc.size());
      if (!ssrc_d) return gf_fail(h, GFORS_E_OOM, "column slices");
      UP(h->csl.blk, sblk.data(), int4, sblk.size());
      UP(h->csl.off, soff.data(), int64_t, soff.size());
      UP(h->csl.len, slen.data(), int32_t, slen.size());
      UP(h->csl.pbase, spb.data(), int32_t, spb.size());
      UP(h->csl.sidx, sidx.data(), int32_t, sidx.size());
      UP(ssrc_d, ssrc.data(), int64_t, ssrc.size());
      GF_CK(h, gf_fill_slices(h, ssrc_d));
      GF_CK(h, cudaStreamSynchronize(s));
    }
    h->clong.nlong = (int32_t)lid.size();
    h->clong.nchunks = (int32_t)ch.size();
    if (!lid.empty()) {
      ALLOC(h->clong.ids, int32_t, lid.size());
      ALLOC(h->clong.chunk_ptr, int32_t, lptr.size());
      ALLOC(h->clong.chunks, GfChunk, ch.size());
      ALLOC(h->clong.partial, float2, ch.size());
      UP(h->clong.ids, lid.data(), int32_t, lid.size());
      UP(h->clong.chunk_ptr, lptr.data(), int32_t, lptr.size());
      UP(h->clong.chunks, ch.data(), GfChunk, ch.size());
    }
  }

  // ---------------- evaluation structures (integer data)
  {
    {
      const std::string ex = parallel_for(ninst, [&](int q) {
        if (h->ih[q].integral) stage_eval_rows(q, h->ih[q], st[q]);
      });
      if (!ex.empty()) return gf_fail(h, GFORS_E_OOM, "evaluation rows: " + ex);
    }
    std::vector<GfURow> ur;
    std::vector<int32_t> ucols;
    std::vector<GfPRow> pr;
    std::vector<GfPChunk> pch;
    std::vector<GfPSlice> psl;
    std::vector<GfGRow> gr;
    std::vector<int32_t> gcols, gvals;
    std::vector<GfObjChunk> oc;
    std::vector<GfQChunk> qc;
    std::vector<int32_t> QIi, QIc;
    for (int q = 0; q < ninst; ++q) {
      const GfInstHost& I = h->ih[q];
      if (!I.integral) continue;
      Stage& S = st[q];
      for (GfURow R : S.ur) {
        R.t0 += (int64_t)ucols.size();
        ur.push_back(R);
      }
      ucols.insert(ucols.end(), S.ucols.begin(), S.ucols.end());
      pr.insert(pr.end(), S.pr.begin(), S.pr.end());
      pch.insert(pch.end(), S.pch.begin(), S.pch.end());
      psl.insert(psl.end(), S.psl.begin(), S.psl.end());
      for (GfGRow R : S.gr) {
        R.t0 += (int64_t)gcols.size();
        gr.push_back(R);
      }
      gcols.insert(gcols.end(), S.gcols.begin(), S.gcols.end());
      gvals.insert(gvals.end(), S.gvals.begin(), S.gvals.end());
      std::vector<int32_t>().swap(S.ucols);
      std::vector<int32_t>().swap(S.gcols);
      std::vector<int32_t>().swap(S.gvals);
      // dense tensor-core instances: the scorer adds c + diag(Q) itself
      if (I.qkind != 1)
        for (int64_t a = 0; a < I.n; a += 1024)
          oc.push_back(GfObjChunk{q, (int32_t)(I.var_off + a),
                                  (int32_t)(I.var_off + std::min<int64_t>(I.n, a + 1024)), 0});
    }
    // Sparse Q for evaluation: x^T Q x = sum_i q_ii x_i + sum_{i<j} w_ij x_i x_j
    // with w_ij = q_ij + q_ji; the diagonal joins the linear costs (x_i^2 =
    // x_i), every pair (i < j) is stored once, in blocks of 32 with the
    // block's bias -min w and the bit width of max w - min w (bit-plane
    // evaluation).
    std::vector<long long> clin;
    std::vector<long long> QIv;
    std::vector<long long> QIb;
    std::vector<uint8_t> QIw;
    bool anyq = false;
    for (int q = 0; q < ninst; ++q) anyq |= h->ih[q].integral && h->ih[q].qkind == 2;
    if (anyq) {
      clin = cint;
      std::vector<std::vector<std::pair<int32_t, long long>>> pr2(ninst);
      std::vector<std::vector<int64_t>> cnt(ninst);
      const std::string ex = parallel_for(ninst, [&](int q) {
        const GfInstHost& I = h->ih[q];
        if (!I.integral || I.qkind != 2) return;
        const RowSet& Qo = st[q].Qorig;
        std::vector<int64_t>& pp = cnt[q];
        pp.assign(I.n + 1, 0);
        for (int64_t i = 0; i < I.n; ++i)
          for (int64_t u = 0; u < Qo.len(i); ++u) {
            const int64_t j = Qo.c(i)[u];
            if (j != i) pp[std::min(i, j) + 1]++;
          }
        for (int64_t i = 0; i < I.n; ++i) pp[i + 1] += pp[i];
        std::vector<std::pair<int32_t, long long>>& e = pr2[q];
        e.resize(pp[I.n]);
        std::vector<int64_t> fill(pp.begin(), pp.end() - 1);
        for (int64_t i = 0; i < I.n; ++i)
          for (int64_t u = 0; u < Qo.len(i); ++u) {
            const int64_t j = Qo.c(i)[u];
            const long long v = (long long)Qo.v(i)[u];
            if (j == i) clin[I.var_off + i] += v;
            else e[fill[std::min(i, j)]++] = {(int32_t)std::max(i, j), v};
          }
        // per row: sort by column, merge, drop zero sums; compact in place
        int64_t outp = 0;
        for (int64_t i = 0; i < I.n; ++i) {
          const int64_t a = pp[i], b = pp[i + 1];
          std::sort(e.begin() + a, e.begin() + b);
          const int64_t start = outp;
          for (int64_t u = a; u < b;) {
            int64_t w = u;
            long long sum = 0;
            while (w < b && e[w].first == e[u].first) sum += e[w++].second;
            if (sum != 0) e[outp++] = {e[u].first, sum};
            u = w;
          }
          pp[i] = start;
        }
        pp[I.n] = outp;
        e.resize(outp);
      });
      if (!ex.empty()) return gf_fail(h, GFORS_E_OOM, "sparse Q pairs: " + ex);
      // flat pair list, each instance padded to whole blocks of 32 with
      // weight-0 pairs; per block the bias -min w and the span's bit width
      for (int q = 0; q < ninst; ++q) {
        const GfInstHost& I = h->ih[q];
        if (cnt[q].empty()) continue;
        const int64_t np = (int64_t)pr2[q].size();
        const int64_t nb = (np + 31) / 32;
        const int64_t pb0 = (int64_t)QIi.size() / 32;
        for (int64_t i = 0; i < I.n; ++i)
          for (int64_t u = cnt[q][i]; u < cnt[q][i + 1]; ++u) {
            QIi.push_back((int32_t)(I.var_off + i));
            QIc.push_back((int32_t)(I.var_off + pr2[q][u].first));
            QIv.push_back(pr2[q][u].second);
          }
        while ((int64_t)QIi.size() % 32) {
          QIi.push_back((int32_t)I.var_off);
          QIc.push_back((int32_t)I.var_off);
          QIv.push_back(0);
        }
        for (int64_t bk = 0; bk < nb; ++bk) {
          long long lo = QIv[(pb0 + bk) * 32], hi = lo;
          for (int l = 1; l < 32; ++l) {
            lo = std::min(lo, QIv[(pb0 + bk) * 32 + l]);
            hi = std::max(hi, QIv[(pb0 + bk) * 32 + l]);
          }
          const unsigned long long span = (unsigned long long)(hi - lo);
          int bits = 0;
          while (bits < 64 && (span >> bits) != 0ull) ++bits;
          QIb.push_back(-lo);
          QIw.push_back((uint8_t)bits);
        }
        for (int64_t bk = 0; bk < nb; bk += kQChunkBlocks)
          qc.push_back(GfQChunk{q, (int32_t)(pb0 + bk),
                                (int32_t)(pb0 + std::min<int64_t>(nb, bk + kQChunkBlocks)), 0});
        std::vector<std::pair<int32_t, long long>>().swap(pr2[q]);
      }
    }
    // uniform rows grouped by evaluation class (any-of, at-most-one with at
    // least one, general count), one kernel instance per class
    {
      auto cls = [](const GfURow& R) {
        const bool no_upper = R.U < 0 || R.U >= R.len;
        return (R.L <= 1 && no_upper) ? 0 : (R.U == 1 && R.L <= 1) ? 1 : 2;
      };
      std::stable_sort(ur.begin(), ur.end(),
                       [&](const GfURow& a, const GfURow& b) { return cls(a) < cls(b); });
      for (int c = 0; c < 3; ++c) h->nurows_cls[c] = 0;
      for (const GfURow& R : ur) ++h->nurows_cls[cls(R)];
    }
    h->nurows = (int64_t)ur.size();
    h->nprows = (int64_t)pr.size();
    h->npchunks = (int64_t)pch.size();
    h->npslices = (int64_t)psl.size();
    // general rows longer than kGLong entries after the others: those get a
    // block per (row, candidate word) in evaluation (row order does not
    // change any count)
    std::stable_partition(gr.begin(), gr.end(), [](const GfGRow& R) { return R.len <= kGLong; });
    h->ngrows_short = 0;
    for (const GfGRow& R : gr) h->ngrows_short += (R.len <= kGLong) ? 1 : 0;
    h->ngrows = (int64_t)gr.size();
    h->nochunks = (int64_t)oc.size();
    h->nqchunks = (int64_t)qc.size();
    ALLOC(h->urows, GfURow, ur.size());
    ALLOC(h->ucols, int32_t, ucols.size());
    ALLOC(h->prows, GfPRow, pr.size());
    ALLOC(h->pchunks, GfPChunk, pch.size());
    ALLOC(h->pslices, GfPSlice, psl.size());
    ALLOC(h->grows, GfGRow, gr.size());
    ALLOC(h->gcols, int32_t, gcols.size());
    ALLOC(h->gvals, int32_t, gvals.size());
    ALLOC(h->ochunks, GfObjChunk, oc.size());
    // cost bit planes per 32-variable group (linear-objective evaluation)
    std::vector<long long> cgb(N / 32);
    std::vector<uint8_t> cgp(N / 32);
    {
      const std::vector<long long>& cl = anyq ? clin : cint;
      for (int64_t g = 0; g < N / 32; ++g) {
        long long lo = cl[32 * g], hi = lo;
        for (int l = 1; l < 32; ++l) {
          lo = std::min(lo, cl[32 * g + l]);
          hi = std::max(hi, cl[32 * g + l]);
        }
        const unsigned long long span = (unsigned long long)(hi - lo);
        int bits = 0;
        while (bits < 64 && (span >> bits) != 0ull) ++bits;
        cgb[g] = -lo;
        cgp[g] = (uint8_t)bits;
      }
    }
    ALLOC(h->cgbias, long long, N / 32);
    ALLOC(h->cgP, uint8_t, N / 32);
    UP(h->cgbias, cgb.data(), long long, N / 32);
    UP(h->cgP, cgp.data(), uint8_t, N / 32);
    ALLOC(h->qchunks, GfQChunk, qc.size());
    ALLOC(h->QIi, int32_t, QIi.size());
    ALLOC(h->QIc, int32_t, QIc.size());
    ALLOC(h->QIv, long long, QIv.size());
    ALLOC(h->QIb, long long, QIb.size());
    ALLOC(h->QIw, uint8_t, QIw.size());
    if (anyq) ALLOC(h->clin, long long, N);
    ALLOC(h->cint, long long, N);
    if (!ur.empty()) UP(h->urows, ur.data(), GfURow, ur.size());
    if (!ucols.empty()) UP(h->ucols, ucols.data(), int32_t, ucols.size());
    if (!pr.empty()) UP(h->prows, pr.data(), GfPRow, pr.size());
    if (!pch.empty()) UP(h->pchunks, pch.data(), GfPChunk, pch.size());
    if (!psl.empty()) UP(h->pslices, psl.data(), GfPSlice, psl.size());
    if (!gr.empty()) UP(h->grows, gr.data(), GfGRow, gr.size());
    if (!gcols.empty()) UP(h->gcols, gcols.data(), int32_t, gcols.size());
    if (!gvals.empty()) UP(h->gvals, gvals.data(), int32_t, gvals.size());
    if (!oc.empty()) UP(h->ochunks, oc.data(), GfObjChunk, oc.size());
    if (!qc.empty()) UP(h->qchunks, qc.data(), GfQChunk, qc.size());
    if (!QIi.empty()) UP(h->QIi, QIi.data(), int32_t, QIi.size());
    if (!QIc.empty()) UP(h->QIc, QIc.data(), int32_t, QIc.size());
    if (!QIv.empty()) UP(h->QIv, QIv.data(), long long, QIv.size());
    if (!QIb.empty()) UP(h->QIb, QIb.data(), long long, QIb.size());
    if (!QIw.empty()) UP(h->QIw, QIw.data(), uint8_t, QIw.size());
    if (anyq) UP(h->clin, clin.data(), long long, N);
    UP(h->cint, cint.data(), long long, N);
  }

  // ---------------- fused single-row path (every instance one >= row, no Q)
  {
    bool ok = h->all_integral && P.eval_mode != 1 && P.eval_mode != 3;
    for (int q = 0; q < ninst && ok; ++q) ok = h->ih[q].single_row;
    long long worst = 0;
    if (ok) {
      for (int q = 0; q < ninst && ok; ++q) {
        long long s = 0;
        for (int64_t u = 0; u < st[q].orig.len(0); ++u) s += (long long)std::fabs(st[q].orig.v(0)[u]);
        worst = std::max(worst, s);
      }
    }
    h->fused_ok = ok;
    if (ok) {
      std::vector<int32_t> w(N, 0), blk;
      std::vector<long long> rhs(ninst);
      for (int q = 0; q < ninst; ++q) {
        const GfInstHost& I = h->ih[q];
        const RowSet& o = st[q].orig;
        for (int64_t t = 0; t < o.len(0); ++t) w[I.var_off + o.c(0)[t]] = (int32_t)o.v(0)[t];
        rhs[q] = st[q].rhs[0];
        for (int64_t a = 0; a < I.npad; a += 8192) {
          blk.push_back(q);
          blk.push_back((int32_t)(I.var_off + a));
          blk.push_back((int32_t)(I.var_off + std::min<int64_t>(I.npad, a + 8192)));
        }
      }
      // longest slices first (better tail)
      h->nfblk = (int64_t)blk.size() / 3;
      ALLOC(h->frow_w, int32_t, N);
      ALLOC(h->frhs, long long, ninst);
      ALLOC(h->fblk, int32_t, blk.size());
      UP(h->frow_w, w.data(), int32_t, N);
      UP(h->frhs, rhs.data(), long long, ninst);
      UP(h->fblk, blk.data(), int32_t, blk.size());
      ALLOC(h->fthr, uint32_t, N);
      // a block sums at most 8192 products of one instance: int32 partial
      // sums are exact when every |coefficient| and |cost| is below 2^31/8192
      long long maxw = 0, maxc = 0;
      for (int64_t i = 0; i < N; ++i) {
        maxw = std::max(maxw, std::llabs((long long)w[i]));
        maxc = std::max(maxc, std::llabs(cint[i]));
      }
      if (maxw < (1ll << 31) / 8192 && maxc < (1ll << 31) / 8192) {
        std::vector<int32_t> c32(N);
        for (int64_t i = 0; i < N; ++i) c32[i] = (int32_t)cint[i];
        ALLOC(h->f_c32, int32_t, N);
        UP(h->f_c32, c32.data(), int32_t, N);
      }
    }
  }

  // ---------------- iterate, state, sampling buffers
  h->chunk = P.sample_chunk > 0 ? std::min(P.sample_chunk, P.k_b) : P.k_b;
  h->kw = h->chunk / 32;
  ALLOC(h->x[0], float, N);
  ALLOC(h->x[1], float, N);
  ALLOC(h->xbar, float, N);
  ALLOC(h->y, float, M);
  ALLOC(h->dlast, float, N);
  ALLOC(h->qbuf, float, N);
  ALLOC(h->qbuf2, float, N);
  ALLOC(h->dxbuf, float, N);
  ALLOC(h->dstate, GfDState, 1);
  ALLOC(h->iprm, GfIParam, 2 * ninst);
  ALLOC(h->sched_d, GfSched, 1);
  ALLOC(h->X, uint32_t, (size_t)N * h->kw);
  ALLOC(h->viol, int32_t, (size_t)ninst * h->chunk);
  ALLOC(h->obj, long long, (size_t)ninst * h->chunk);
  ALLOC(h->objp, long long, (size_t)ninst * h->chunk);
  if (h->fused_ok) ALLOC(h->fsum, long long, (size_t)ninst * h->chunk);
  ALLOC(h->inc, GfInc, ninst);
  ALLOC(h->xbest, uint8_t, N);
  ALLOC(h->var_grouped, uint8_t, N);
  ALLOC(h->bit_g4, int32_t, N / 4 + 1);
  ALLOC(h->bit_count, int32_t, 1);
  h->n_bit_g4 = -1;
  ALLOC(h->var_grouped_feat, uint8_t, N);
  GF_CK(h, cudaMemsetAsync(h->var_grouped_feat, 0, N, s));
  ALLOC(h->stats_part, double, 8 * (h->nrchunk + h->nvchunk + 1));
  ALLOC(h->stats, double, 8 * ninst);
  ALLOC(h->stats2, double, 8 * ninst);
  ALLOC(h->inst_dense, uint8_t, ninst);
  for (GfDenseQ& dq : h->dense) {
    dq.chunk = h->chunk;
    ALLOC(dq.Xs, __nv_bfloat16, (size_t)h->chunk * dq.ld);
    ALLOC(dq.Xb, uint32_t, (size_t)h->chunk * (dq.ld / 32));
    ALLOC(dq.thr, uint32_t, (size_t)dq.ld);
  }
  {
    std::vector<uint8_t> grouped(N, 0), idense(ninst, 0);
    for (const GfDenseQ& dq : h->dense) {
      idense[dq.inst] = 1;
      const GfInstHost& I = h->ih[dq.inst];
      for (int64_t i = 0; i < I.npad; ++i) grouped[I.var_off + i] = 1;  // no bit sampling
    }
    UP(h->var_grouped, grouped.data(), uint8_t, N);
    UP(h->inst_dense, idense.data(), uint8_t, ninst);
  }
  GF_CK(h, cudaMemsetAsync(h->inc, 0, sizeof(GfInc) * ninst, s));
  GF_CK(h, cudaMemsetAsync(h->xbest, 0, N, s));
  GF_CK(h, cudaMemsetAsync(h->y, 0, sizeof(float) * std::max<int64_t>(M, 1), s));
  GF_CK(h, cudaMemsetAsync(h->dlast, 0, sizeof(float) * N, s));
  GF_CK(h, cudaMemsetAsync(h->qbuf, 0, sizeof(float) * N, s));
  GF_CK(h, cudaMemsetAsync(h->qbuf2, 0, sizeof(float) * N, s));
  // start point x_0 (Alg. 1): constant, or Philox uniforms (stream 5)
  {
    std::vector<float> x0(N, 0.0f);
    for (int q = 0; q < ninst; ++q) {
      const GfInstHost& I = h->ih[q];
      if (P.x0 >= 0.0) {
        const float v = (float)std::min(1.0, P.x0);
        for (int64_t i = 0; i < I.n; ++i) x0[I.var_off + i] = v;
      }
    }
    UP(h->x[0], x0.data(), float, N);
    if (P.x0 < 0.0) {
      extern cudaError_t gf_launch_x0_random(GfCtx * h);
      GF_CK(h, gf_launch_x0_random(h));
    }
    GF_CK(h, cudaMemcpyAsync(h->x[1], h->x[0], sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
    GF_CK(h, cudaMemcpyAsync(h->xbar, h->x[0], sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
  }
  h->sched = GfSched{P.sigma, P.rho_min, P.rho_max, P.T, P.p, P.delta, P.k_int, ninst};
  UP(h->sched_d, &h->sched, GfSched, 1);
  h->k_host = 0;
  h->n_rho_host = 0;
  h->rho_host = std::min(P.rho_min, P.rho_max);
  GfDState ds;
  memset(&ds, 0, sizeof(ds));
  ds.k = 0;
  ds.n_rho = 0;
  ds.rho = h->rho_host;
  ds.round_id = 0;
  UP(h->dstate, &ds, GfDState, 1);
  gf_set_slot(h, 1, h->rho_host);     // iteration 1 reads slot 1
  {
    extern bool gf_persistent_setup(GfCtx * h);
    extern bool gf_single_setup(GfCtx * h);
    h->persist_ok = (P.pdhg_mode != 1) && gf_persistent_setup(h);
    h->single_ok = gf_single_setup(h);
    // rows with one common coefficient (the small path keeps one value per row)
    extern bool gf_small_setup(GfCtx * h, const std::vector<uint8_t>& uniform,
                               const std::vector<int64_t>& kp, const std::vector<int64_t>& tp);
    std::vector<uint8_t> uniform(ninst, 1);
    for (int q = 0; q < ninst; ++q) {
      const RowSet& o = st[q].orig;
      for (size_t j = 0; j < o.size() && uniform[q]; ++j)
        for (int64_t u = 1; u < o.len(j); ++u)
          if (o.v(j)[u] != o.v(j)[0]) { uniform[q] = 0; break; }
    }
    GF_CK(h, cudaStreamSynchronize(s));
    h->small_ok = gf_small_setup(h, uniform, Kp, Tp);
    extern bool gf_coop_setup(GfCtx * h, const std::vector<int64_t>& kp,
                              const std::vector<int64_t>& tp);
    h->coop_ok = gf_coop_setup(h, Kp, Tp);
  }
  GF_CK(h, cudaStreamSynchronize(s));
  h->h_best.assign(3 * ninst, INFINITY);
  h->h_last.assign(3 * ninst, 0);
  h->h_trig = 0;
  return GFORS_OK;
#undef ALLOC
#undef UP
}

static gfors_status make_ctx(const gfors_params* prm, void* stream, GfCtx** out) {
  if (!out) { g_thread_err = "out handle is NULL"; return GFORS_E_ARG; }
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    g_thread_err = std::string("no CUDA device: ") + cudaGetErrorString(e);
    return GFORS_E_CUDA;
  }
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    g_thread_err = "cudaGetDeviceProperties failed";
    return GFORS_E_CUDA;
  }
  if (!(pr.major == 10 && pr.minor == 3)) {
    g_thread_err = "this build targets sm_103a (B300); device is sm_" + std::to_string(pr.major) +
                   std::to_string(pr.minor);
    return GFORS_E_UNSUPPORTED;
  }
  GfCtx* h = new GfCtx();
  if (prm) h->prm = *prm; else gfors_default_params(&h->prm);
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {          // own a stream: graph capture needs a non-legacy stream
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      g_thread_err = "cudaStreamCreate failed";
      return GFORS_E_CUDA;
    }
    h->own_stream = true;
  }
  h->dev = dev;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->num_sms <= 0) h->num_sms = 148;
  *out = h;
  return GFORS_OK;
}

extern "C" gfors_status gfors_load_batch(int32_t ninst, const gfors_csr* const* A,
                                         const double* const* b, const gfors_csr* const* B,
                                         const double* const* d, const gfors_qmat* const* Q,
                                         const double* const* c, const int64_t* n,
                                         const gfors_params* prm, void* cuda_stream,
                                         gfors_handle* out) {
  GfCtx* h = nullptr;
  gfors_status st = make_ctx(prm, cuda_stream, &h);
  if (st != GFORS_OK) return st;
  st = load_impl(h, ninst, A, b, B, d, Q, c, n);
  if (st != GFORS_OK) {
    g_thread_err = h->err;
    cudaStreamSynchronize(h->stream);
    gf_free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return st;
  }
  *out = h;
  return GFORS_OK;
}

extern "C" gfors_status gfors_load(const gfors_csr* A, const double* b, const gfors_csr* B,
                                   const double* d, const gfors_qmat* Q, const double* c,
                                   int64_t n, const gfors_params* prm, void* cuda_stream,
                                   gfors_handle* out) {
  const gfors_csr* Aa[1] = {A};
  const double* ba[1] = {b};
  const gfors_csr* Ba[1] = {B};
  const double* da[1] = {d};
  const gfors_qmat* Qa[1] = {Q};
  const double* ca[1] = {c};
  int64_t na[1] = {n};
  return gfors_load_batch(1, Aa, ba, Ba, da, Qa, ca, na, prm, cuda_stream, out);
}

extern "C" void gfors_destroy(gfors_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->g_pair) cudaGraphExecDestroy(h->g_pair);
  for (int q = 0; q < 2; ++q) {
    if (h->g_iter2[q]) cudaGraphExecDestroy(h->g_iter2[q]);
    if (h->g_light2[q]) cudaGraphExecDestroy(h->g_light2[q]);
  }
  for (auto& rg : h->run_graph)
    if (rg.exec) cudaGraphExecDestroy(rg.exec);
  gf_free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}
