// gfors_tu.cu -- TU reformulation (Thm. 5, Section 2.4.1) on the host.
// When B_JI is a signed permutation (every row j of J has exactly one entry,
// +1 or -1, in the columns I, and every column of I has its entry in exactly
// one row of J), B_JI^-1 is the transposed permutation and for the row j
// whose pivot is I_k (sign sigma)
//
//   x_{I_k} = s_k + S_k x_Ibar,   s_k = sigma d_j,   S_k = -sigma B_{j,Ibar},
//
// so S is as sparse as B_JIbar.  Any other invertible B_JI goes through
// Gauss-Jordan elimination of the rows J on the columns I in exact integer
// arithmetic (every pivot is +-1 and every entry stays in {-1, 0, 1} when
// B_J is totally unimodular), and S is stored explicitly (the paper's remark
// keeps an LU factor instead, to save memory when S fills in; here a fill
// above 2^28 entries is reported as unsupported).  The new problem over
// x_Ibar (Ibar ascending) is
//
//   Q'  = S^T Q_II S + S^T Q_IIbar + Q_IbarI S + Q_IbarIbar
//   c'  = S^T (Q_II + Q_II^T) s + Q_IIbar^T s + Q_IbarI s + S^T c_I + c_Ibar
//   c0' = s^T Q_II s + c_I^T s
//   A'  = [A_.I S + A_.Ibar ;  S ; -S],   b' = [b - A_.I s ; -s ; s - 1]
//         (a bounds row that every x in [0, 1] satisfies is left out)
//   B'  = B_JbarI S + B_JbarIbar,         d' = d_Jbar - B_JbarI s
//
// Q is used as given (not symmetrised), so integral data stay integral.  The
// theorem needs B_J to be totally unimodular; that is the caller's claim.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

struct SpRows {                       // rows as (column, value) lists
  std::vector<int64_t> ptr{0};
  std::vector<int32_t> col;
  std::vector<double> val;
  // append a row from unsorted (column, value) pairs: sum duplicates, drop 0
  void add_row(std::vector<std::pair<int32_t, double>>& e) {
    std::sort(e.begin(), e.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                return a.first < b.first;
              });
    for (size_t u = 0; u < e.size();) {
      size_t w = u;
      double s = 0.0;
      while (w < e.size() && e[w].first == e[u].first) s += e[w++].second;
      if (s != 0.0) {
        col.push_back(e[u].first);
        val.push_back(s);
      }
      u = w;
    }
    ptr.push_back((int64_t)col.size());
  }
  int64_t rows() const { return (int64_t)ptr.size() - 1; }
};

}  // namespace

struct gfors_tu_s {
  int64_t n = 0, nbar = 0;
  std::vector<int64_t> I, Ibar;       // pivot columns (given order), the rest
  std::vector<int64_t> pos;           // n: index in Ibar, or -1 - k for pivot k
  std::vector<double> s;              // |I|
  SpRows S;                           // |I| rows over Ibar indices
  SpRows A, B, Q;                     // reformulated data
  std::vector<double> b, d, c;
  double c0 = 0.0;
  bool hasQ = false;
};

static bool csr_ok(const gfors_csr* M, int64_t n) {
  if (!M) return true;
  if (M->rows < 0 || M->cols != n || M->nnz < 0) return false;
  if (M->rows > 0 && (!M->row_ptr || M->row_ptr[0] != 0 || M->row_ptr[M->rows] != M->nnz))
    return false;
  if (M->nnz > 0 && (!M->col_idx || !M->val)) return false;
  for (int64_t r = 0; r < M->rows; ++r)
    if (M->row_ptr[r + 1] < M->row_ptr[r]) return false;
  for (int64_t t = 0; t < M->nnz; ++t)
    if (M->col_idx[t] < 0 || M->col_idx[t] >= n) return false;
  return true;
}

extern "C" gfors_status gfors_tu_reformulate(int64_t n, const gfors_csr* A, const double* b,
                                             const gfors_csr* B, const double* d,
                                             const gfors_qmat* Q, const double* c, int64_t nJ,
                                             const int64_t* J, const int64_t* I,
                                             gfors_tu* out) {
  if (!out) return GFORS_E_ARG;
  *out = nullptr;
  if (n <= 0 || n >= (1ll << 30) || !c || !B || !d || nJ <= 0 || !J || !I) return GFORS_E_ARG;
  if (!csr_ok(A, n) || !csr_ok(B, n) || (A && A->rows > 0 && !b)) return GFORS_E_ARG;
  if (nJ > B->rows || nJ >= n) return GFORS_E_ARG;
  if (Q && Q->kind == 1 && !Q->dense_rowmajor) return GFORS_E_ARG;
  if (Q && Q->kind == 2 && (!csr_ok(&Q->sparse, n) || Q->sparse.rows != n)) return GFORS_E_ARG;
  gfors_tu_s* t = new gfors_tu_s();
  t->n = n;
  t->pos.assign(n, 0);
  std::vector<int64_t> rowJ(B->rows, -1);          // row of B -> k (pivot index)
  for (int64_t k = 0; k < nJ; ++k) {
    if (J[k] < 0 || J[k] >= B->rows || rowJ[J[k]] >= 0 || I[k] < 0 || I[k] >= n ||
        t->pos[I[k]] != 0) {
      delete t;
      return GFORS_E_ARG;
    }
    rowJ[J[k]] = k;
    t->pos[I[k]] = -1 - k;
  }
  t->I.assign(I, I + nJ);
  for (int64_t i = 0; i < n; ++i)
    if (t->pos[i] == 0) {
      t->pos[i] = (int64_t)t->Ibar.size();
      t->Ibar.push_back(i);
    }
  t->nbar = (int64_t)t->Ibar.size();
  // Fast path: B_JI a signed permutation (row J[k] has one entry +-1 in
  // the columns I, every column of I in exactly one of those rows).
  std::vector<int64_t> row_of_pivot(nJ, -1);
  std::vector<double> sigma(nJ, 0.0);
  bool perm = true;
  for (int64_t k = 0; k < nJ && perm; ++k) {
    const int64_t j = J[k];
    int hits = 0;
    for (int64_t u = B->row_ptr[j]; u < B->row_ptr[j + 1]; ++u) {
      const int64_t p = t->pos[B->col_idx[u]];
      if (p >= 0 || B->val[u] == 0.0) continue;
      const int64_t kk = -1 - p;
      ++hits;
      if ((B->val[u] != 1.0 && B->val[u] != -1.0) || row_of_pivot[kk] >= 0) hits = 99;
      row_of_pivot[kk] = j;
      sigma[kk] = B->val[u];
    }
    perm = hits == 1;
  }
  t->s.assign(nJ, 0.0);
  if (perm) {
    // s and S (row k of S belongs to pivot column I[k])
    for (int64_t k = 0; k < nJ; ++k) {
      const int64_t j = row_of_pivot[k];
      t->s[k] = sigma[k] * d[j];
      std::vector<std::pair<int32_t, double>> e;
      for (int64_t u = B->row_ptr[j]; u < B->row_ptr[j + 1]; ++u) {
        const int64_t p = t->pos[B->col_idx[u]];
        if (p >= 0) e.emplace_back((int32_t)p, -sigma[k] * B->val[u]);
      }
      t->S.add_row(e);
    }
  } else {
    // General B_JI: Gauss-Jordan elimination of the rows J on the pivot
    // columns I in exact integer arithmetic.  For a totally unimodular B_J
    // every pivot is +-1 and every entry stays in {-1, 0, 1}; a pivot of
    // another size means B_J is not TU (unsupported), a missing one that
    // B_JI is singular (bad argument).  Columns are kept in one index space:
    // pivot k as -1 - k, Ibar columns as their position.
    typedef std::vector<std::pair<int64_t, long long>> Row;   // sorted by key
    std::vector<Row> R(nJ);
    std::vector<long long> rhs(nJ);
    std::vector<std::vector<int64_t>> rows_with(nJ);     // pivot k -> rows holding it
    for (int64_t r = 0; r < nJ; ++r) {
      const int64_t j = J[r];
      for (int64_t u = B->row_ptr[j]; u < B->row_ptr[j + 1]; ++u) {
        const double v = B->val[u];
        if (v == 0.0) continue;
        if (v != std::floor(v) || std::fabs(v) > 1e15 || d[j] != std::floor(d[j])) {
          delete t;
          return GFORS_E_ARG;                       // B_J, d_J must be integral
        }
        R[r].emplace_back(t->pos[B->col_idx[u]], (long long)v);
      }
      std::sort(R[r].begin(), R[r].end());
      // merge duplicates
      Row m;
      for (const auto& e2 : R[r]) {
        if (!m.empty() && m.back().first == e2.first) m.back().second += e2.second;
        else m.push_back(e2);
      }
      m.erase(std::remove_if(m.begin(), m.end(), [](const std::pair<int64_t, long long>& e2) {
                return e2.second == 0;
              }), m.end());
      R[r].swap(m);
      rhs[r] = (long long)d[j];
      for (const auto& e2 : R[r])
        if (e2.first < 0) rows_with[-1 - e2.first].push_back(r);
    }
    auto coef = [](const Row& row, int64_t kk) -> long long {
      auto it = std::lower_bound(row.begin(), row.end(), std::make_pair(kk, LLONG_MIN));
      return (it != row.end() && it->first == kk) ? it->second : 0;
    };
    std::vector<int64_t> piv_row(nJ, -1);
    std::vector<uint8_t> used(nJ, 0);
    int64_t fill = 0;
    for (int64_t r = 0; r < nJ; ++r) fill += (int64_t)R[r].size();
    for (int64_t k = 0; k < nJ; ++k) {
      const int64_t kk = -1 - k;
      int64_t pr = -1;
      for (int64_t r : rows_with[k])
        if (!used[r] && coef(R[r], kk) != 0) { pr = r; break; }
      if (pr < 0) {
        delete t;
        return GFORS_E_ARG;                         // B_JI singular
      }
      const long long pv = coef(R[pr], kk);
      if (pv != 1 && pv != -1) {
        delete t;
        return GFORS_E_UNSUPPORTED;                 // B_J not totally unimodular
      }
      used[pr] = 1;
      piv_row[k] = pr;
      if (pv == -1) {
        for (auto& e2 : R[pr]) e2.second = -e2.second;
        rhs[pr] = -rhs[pr];
      }
      // eliminate pivot k from every other row that holds it
      const std::vector<int64_t> holders = rows_with[k];
      for (int64_t r : holders) {
        if (r == pr) continue;
        const long long f = coef(R[r], kk);
        if (f == 0) continue;
        Row out;
        out.reserve(R[r].size() + R[pr].size());
        size_t a1 = 0, b1 = 0;
        while (a1 < R[r].size() || b1 < R[pr].size()) {
          if (b1 == R[pr].size() || (a1 < R[r].size() && R[r][a1].first < R[pr][b1].first)) {
            out.push_back(R[r][a1++]);
          } else if (a1 == R[r].size() || R[pr][b1].first < R[r][a1].first) {
            const long long v = -f * R[pr][b1].second;
            const int64_t c2 = R[pr][b1++].first;
            out.emplace_back(c2, v);
            if (c2 < 0) rows_with[-1 - c2].push_back(r);
          } else {
            const long long v = R[r][a1].second - f * R[pr][b1].second;
            if (v != 0) out.emplace_back(R[r][a1].first, v);
            ++a1;
            ++b1;
          }
        }
        for (const auto& e2 : out)
          if (e2.second > 1 || e2.second < -1) {
            delete t;
            return GFORS_E_UNSUPPORTED;             // B_J not totally unimodular
          }
        fill += (int64_t)out.size() - (int64_t)R[r].size();
        R[r].swap(out);
        rhs[r] -= f * rhs[pr];
      }
      if (fill > (1ll << 28)) {
        delete t;
        return GFORS_E_UNSUPPORTED;                 // S too dense to hold
      }
    }
    // row piv_row[k] now reads x_{I_k} + sum_Ibar a x = rhs
    for (int64_t k = 0; k < nJ; ++k) {
      const int64_t r = piv_row[k];
      t->s[k] = (double)rhs[r];
      std::vector<std::pair<int32_t, double>> e;
      for (const auto& e2 : R[r])
        if (e2.first >= 0) e.emplace_back((int32_t)e2.first, -(double)e2.second);
      t->S.add_row(e);
    }
  }
  auto add_srow = [&](std::vector<std::pair<int32_t, double>>& e, int64_t k, double a) {
    for (int64_t u = t->S.ptr[k]; u < t->S.ptr[k + 1]; ++u)
      e.emplace_back(t->S.col[u], a * t->S.val[u]);
  };
  // A' = [A_.I S + A_.Ibar ; S ; -S]
  std::vector<std::pair<int32_t, double>> e;
  const int64_t m1 = A ? A->rows : 0;
  for (int64_t r = 0; r < m1; ++r) {
    e.clear();
    double rhs = b[r];
    for (int64_t u = A->row_ptr[r]; u < A->row_ptr[r + 1]; ++u) {
      const int64_t p = t->pos[A->col_idx[u]];
      if (p >= 0) e.emplace_back((int32_t)p, A->val[u]);
      else { add_srow(e, -1 - p, A->val[u]); rhs -= A->val[u] * t->s[-1 - p]; }
    }
    t->A.add_row(e);
    t->b.push_back(rhs);
  }
  // bounds rows of x_I, except those every x in [0, 1] satisfies (sum of
  // the negative coefficients at least the right-hand side)
  for (int sign = 1; sign >= -1; sign -= 2)
    for (int64_t k = 0; k < nJ; ++k) {
      const double rhs = sign > 0 ? -t->s[k] : t->s[k] - 1.0;
      double lo = 0.0;
      for (int64_t u = t->S.ptr[k]; u < t->S.ptr[k + 1]; ++u)
        lo += std::min(0.0, sign * t->S.val[u]);
      if (lo >= rhs) continue;
      e.clear();
      add_srow(e, k, (double)sign);
      t->A.add_row(e);
      t->b.push_back(rhs);
    }
  // B' = B_JbarI S + B_JbarIbar over the rows of B outside J
  for (int64_t r = 0; r < B->rows; ++r) {
    if (rowJ[r] >= 0) continue;
    e.clear();
    double rhs = d[r];
    for (int64_t u = B->row_ptr[r]; u < B->row_ptr[r + 1]; ++u) {
      const int64_t p = t->pos[B->col_idx[u]];
      if (p >= 0) e.emplace_back((int32_t)p, B->val[u]);
      else { add_srow(e, -1 - p, B->val[u]); rhs -= B->val[u] * t->s[-1 - p]; }
    }
    t->B.add_row(e);
    t->d.push_back(rhs);
  }
  // linear part: c' = S^T c_I + c_Ibar, c0' = c_I^T s
  t->c.assign(t->nbar, 0.0);
  for (int64_t q = 0; q < t->nbar; ++q) t->c[q] = c[t->Ibar[q]];
  for (int64_t k = 0; k < nJ; ++k) {
    const double ck = c[t->I[k]];
    t->c0 += ck * t->s[k];
    for (int64_t u = t->S.ptr[k]; u < t->S.ptr[k + 1]; ++u) t->c[t->S.col[u]] += ck * t->S.val[u];
  }
  // quadratic part, entry by entry of Q (x_a q x_b with x_I = s + S x_Ibar)
  if (Q && Q->kind != 0) {
    t->hasQ = true;
    std::vector<std::vector<std::pair<int32_t, double>>> qr(t->nbar);
    auto entry = [&](int64_t a, int64_t bb, double q) {
      if (q == 0.0) return;
      const int64_t pa = t->pos[a], pb = t->pos[bb];
      if (pa >= 0 && pb >= 0) {
        qr[pa].emplace_back((int32_t)pb, q);
      } else if (pa < 0 && pb >= 0) {          // (s_k + S_k x) q x_b
        const int64_t k = -1 - pa;
        t->c[pb] += t->s[k] * q;
        for (int64_t u = t->S.ptr[k]; u < t->S.ptr[k + 1]; ++u)
          qr[t->S.col[u]].emplace_back((int32_t)pb, t->S.val[u] * q);
      } else if (pa >= 0 && pb < 0) {          // x_a q (s_k + S_k x)
        const int64_t k = -1 - pb;
        t->c[pa] += q * t->s[k];
        for (int64_t u = t->S.ptr[k]; u < t->S.ptr[k + 1]; ++u)
          qr[pa].emplace_back(t->S.col[u], q * t->S.val[u]);
      } else {                                 // (s_k1 + S_k1 x) q (s_k2 + S_k2 x)
        const int64_t k1 = -1 - pa, k2 = -1 - pb;
        t->c0 += t->s[k1] * q * t->s[k2];
        for (int64_t u = t->S.ptr[k1]; u < t->S.ptr[k1 + 1]; ++u)
          t->c[t->S.col[u]] += t->S.val[u] * q * t->s[k2];
        for (int64_t u = t->S.ptr[k2]; u < t->S.ptr[k2 + 1]; ++u)
          t->c[t->S.col[u]] += t->s[k1] * q * t->S.val[u];
        for (int64_t u = t->S.ptr[k1]; u < t->S.ptr[k1 + 1]; ++u)
          for (int64_t w = t->S.ptr[k2]; w < t->S.ptr[k2 + 1]; ++w)
            qr[t->S.col[u]].emplace_back(t->S.col[w], t->S.val[u] * q * t->S.val[w]);
      }
    };
    if (Q->kind == 1) {
      for (int64_t a = 0; a < n; ++a)
        for (int64_t bb = 0; bb < n; ++bb) entry(a, bb, Q->dense_rowmajor[a * n + bb]);
    } else {
      for (int64_t a = 0; a < n; ++a)
        for (int64_t u = Q->sparse.row_ptr[a]; u < Q->sparse.row_ptr[a + 1]; ++u)
          entry(a, Q->sparse.col_idx[u], Q->sparse.val[u]);
    }
    for (int64_t q = 0; q < t->nbar; ++q) t->Q.add_row(qr[q]);
  }
  *out = t;
  return GFORS_OK;
}

extern "C" gfors_status gfors_tu_sizes(gfors_tu t, int64_t out[8]) {
  if (!t || !out) return GFORS_E_ARG;
  out[0] = t->nbar;
  out[1] = t->A.rows();
  out[2] = (int64_t)t->A.col.size();
  out[3] = t->B.rows();
  out[4] = (int64_t)t->B.col.size();
  out[5] = t->hasQ ? 1 : 0;
  out[6] = t->hasQ ? (int64_t)t->Q.col.size() : 0;
  out[7] = (int64_t)t->I.size();
  return GFORS_OK;
}

extern "C" gfors_status gfors_tu_copy(gfors_tu t, int64_t* Ap, int32_t* Ac, double* Av,
                                      double* b, int64_t* Bp, int32_t* Bc, double* Bv,
                                      double* d, int64_t* Qp, int32_t* Qc, double* Qv,
                                      double* c, double* c0, int64_t* Ibar) {
  if (!t) return GFORS_E_ARG;
  auto cp = [](const SpRows& M, int64_t* p, int32_t* cc, double* v) {
    if (p) std::copy(M.ptr.begin(), M.ptr.end(), p);
    if (cc) std::copy(M.col.begin(), M.col.end(), cc);
    if (v) std::copy(M.val.begin(), M.val.end(), v);
  };
  cp(t->A, Ap, Ac, Av);
  cp(t->B, Bp, Bc, Bv);
  if (t->hasQ) cp(t->Q, Qp, Qc, Qv);
  if (b) std::copy(t->b.begin(), t->b.end(), b);
  if (d) std::copy(t->d.begin(), t->d.end(), d);
  if (c) std::copy(t->c.begin(), t->c.end(), c);
  if (c0) *c0 = t->c0;
  if (Ibar) std::copy(t->Ibar.begin(), t->Ibar.end(), Ibar);
  return GFORS_OK;
}

extern "C" gfors_status gfors_tu_recover(gfors_tu t, int64_t k, const uint8_t* Xbar,
                                         uint8_t* X) {
  if (!t || k < 0 || (k > 0 && (!Xbar || !X))) return GFORS_E_ARG;
  bool in_range = true;
  for (int64_t r = 0; r < k; ++r) {
    const uint8_t* xb = Xbar + r * t->nbar;
    uint8_t* x = X + r * t->n;
    for (int64_t q = 0; q < t->nbar; ++q) x[t->Ibar[q]] = xb[q] ? 1 : 0;
    for (size_t kk = 0; kk < t->I.size(); ++kk) {
      double v = t->s[kk];
      for (int64_t u = t->S.ptr[kk]; u < t->S.ptr[kk + 1]; ++u)
        if (xb[t->S.col[u]]) v += t->S.val[u];
      in_range &= (v == 0.0 || v == 1.0);
      x[t->I[kk]] = v == 1.0 ? 1 : 0;
    }
  }
  return in_range ? GFORS_OK : GFORS_E_ARG;
}

extern "C" void gfors_tu_free(gfors_tu t) { delete t; }
