/*
 * gfors_oracle.c -- plain, slow, single-threaded FP64 reference of the GFORS
 * hot path (arXiv 2510.27117).  TEST INFRASTRUCTURE ONLY: the CUDA library
 * never links, loads or calls this file; only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg do.  It shares no code, header, table
 * or constant with the CUDA sources.
 *
 * Every routine follows one passage of the paper, cited in its comment:
 *   Eq. (1)      problem  min <x,Qx>+<c,x>, Ax>=b, Bx=d, x in {0,1}^n
 *   Eq. (2)      saddle form, K=-[A;B], r=(b;d), y=(u,v), u>=0
 *   Alg. 1       GFORS loop (penalty update, first-order step, sampling
 *                trigger every k_int iterations, EvalBest, CheckHalt,
 *                final EvalBest(round(x_k)))
 *   Alg. 2       PDHG update (FirstOrderStep)
 *   Alg. 3       generic Bernoulli sampling (RandSampleStep)
 *   Section 2.4.2 customized sampling (one-hot groups, axial 3D picks)
 *   Section 2.4.3 monotone relaxation with repair (facility-location closure)
 *   Section 3    Preprocess, UpdatePenalty, CheckHalt, EvalBest
 * Where the paper leaves a detail open, the reading used is stated in place.
 *
 * Parity status: every function here is pinned by tests/test_oracle_pins.py
 * against closed forms, library routines, brute force or invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Multi-core build (test infrastructure: the CPU baseline's multi-core leg).
 * Compiled with -fopenmp, the loops marked ORC_PAR_FOR run their iterations
 * on all host threads.  Each marked loop writes disjoint outputs per
 * iteration (one row, one sample) with unchanged per-element arithmetic,
 * so both builds give identical results. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PAR_FOR
#endif

int32_t orc_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================
 * Philox4x32-10 counter-based generator, written from its published
 * definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with the
 * round key bumped by the Weyl increments between rounds.
 * ====================================================================== */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += ORC_PHILOX_W0;
    k1 += ORC_PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of every random draw of the method (a reading: the paper
 * only asks for Bernoulli(p_i) draws, Alg. 3).  One Philox call covers four
 * consecutive indices:  counter = (idx>>2, s, round_id, inst | stream<<28),
 * key = (seed low word, seed high word), lane = idx & 3.
 * stream 0: Bernoulli per variable; 1: one-hot group draw; 2: axial 3D step;
 * 3: power-iteration start vector; 5: random start x0. */
uint32_t orc_philox_lane(uint64_t seed, uint32_t stream, uint32_t inst,
                         uint32_t round_id, uint32_t s, uint64_t idx) {
  uint32_t ctr[4] = {(uint32_t)(idx >> 2), s, round_id,
                     (inst & 0x0FFFFFFFu) | (stream << 28)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[idx & 3u];
}

void orc_philox_lanes(uint64_t seed, uint32_t stream, uint32_t inst,
                      uint32_t round_id, uint32_t s, int64_t count,
                      uint32_t* out) {
  for (int64_t i = 0; i < count; ++i)
    out[i] = orc_philox_lane(seed, stream, inst, round_id, s, (uint64_t)i);
}

/* ======================================================================
 * Sparse helpers (CSR: int64 row pointers, int32 columns, double values).
 * ====================================================================== */
static void csr_mv(int64_t m, const int64_t* rp, const int32_t* ci,
                   const double* v, const double* x, double* out) {
  ORC_PAR_FOR
  for (int64_t j = 0; j < m; ++j) {
    double s = 0.0;
    for (int64_t t = rp[j]; t < rp[j + 1]; ++t) s += v[t] * x[ci[t]];
    out[j] = s;
  }
}

static void csr_mtv(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                    const double* v, const double* y, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
  for (int64_t j = 0; j < m; ++j)
    for (int64_t t = rp[j]; t < rp[j + 1]; ++t) out[ci[t]] += v[t] * y[j];
}

/* Q x for qkind 1 (dense row-major n x n) or 2 (CSR); 0 means Q = 0. */
static void q_mv(int qkind, int64_t n, const double* Qd, const int64_t* Qp,
                 const int32_t* Qc, const double* Qv, const double* x,
                 double* out) {
  if (qkind == 1) {
    ORC_PAR_FOR
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += Qd[i * n + j] * x[j];
      out[i] = s;
    }
  } else if (qkind == 2) {
    csr_mv(n, Qp, Qc, Qv, x, out);
  } else {
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
  }
}

static double norm2(int64_t n, const double* v) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

/* ======================================================================
 * Preprocess, first bullet (Section 3): divide each row of K (and the
 * matching entry of r) by the row's 2-norm.  Empty rows are left as they
 * are; an empty >= row with r_j > 0 (i.e. 0 >= b_j > 0) or an empty equality
 * row with r_j != 0 is infeasible and reported (returns -1 - j).
 * ====================================================================== */
int64_t orc_row_normalize(int64_t m, int64_t m1, const int64_t* rp,
                          double* val, double* r, double* rownorm) {
  for (int64_t j = 0; j < m; ++j) {
    double s = 0.0;
    for (int64_t t = rp[j]; t < rp[j + 1]; ++t) s += val[t] * val[t];
    s = sqrt(s);
    rownorm[j] = s;
    if (s > 0.0) {
      for (int64_t t = rp[j]; t < rp[j + 1]; ++t) val[t] /= s;
      r[j] /= s;
    } else if ((j < m1 && r[j] > 0.0) || (j >= m1 && r[j] != 0.0)) {
      return -1 - j;
    }
  }
  return 0;
}

/* ======================================================================
 * Spectral norms for Preprocess (Section 3, second and third bullets).  The
 * paper does not say how they are obtained; the reading used is the power
 * iteration on M^T M:
 *   v_0 = normalised Philox start vector, entries ((u+0.5) 2^-31 - 1),
 *         u = Philox lane (stream 3, s = which, round 0, index j);
 *   for t = 0,1,...: w = M v_t; lambda_t = ||w||^2; z = M^T w;
 *         v_{t+1} = z/||z||; stop once t >= 1 and
 *         |lambda_t - lambda_{t-1}| <= tol * lambda_t, or t = maxit-1;
 *   ||M||_2 = sqrt(lambda_t).
 * which = 0 for K (m x n CSR), 1 for Q (qkind dense/CSR, n x n, symmetric).
 * ====================================================================== */
static void power_start(int64_t n, uint64_t seed, uint32_t inst, uint32_t which,
                        double* v) {
  for (int64_t j = 0; j < n; ++j) {
    uint32_t u = orc_philox_lane(seed, 3u, inst, 0u, which, (uint64_t)j);
    v[j] = ((double)u + 0.5) * (1.0 / 2147483648.0) - 1.0;
  }
  double s = norm2(n, v);
  for (int64_t j = 0; j < n; ++j) v[j] /= s;
}

double orc_power_norm_K(int64_t m, int64_t n, const int64_t* rp,
                        const int32_t* ci, const double* val, uint64_t seed,
                        uint32_t inst, double tol, int32_t maxit,
                        int32_t* iters) {
  if (m == 0 || n == 0) { *iters = 0; return 0.0; }
  double* v = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  double* w = malloc(sizeof(double) * m);
  power_start(n, seed, inst, 0u, v);
  double lam = 0.0, lam_prev = 0.0;
  int32_t t;
  for (t = 0; t < maxit; ++t) {
    csr_mv(m, rp, ci, val, v, w);
    lam = 0.0;
    for (int64_t j = 0; j < m; ++j) lam += w[j] * w[j];
    csr_mtv(m, n, rp, ci, val, w, z);
    double zn = norm2(n, z);
    if (zn == 0.0) break;
    for (int64_t i = 0; i < n; ++i) v[i] = z[i] / zn;
    if (t >= 1 && fabs(lam - lam_prev) <= tol * lam) break;
    lam_prev = lam;
  }
  *iters = (t < maxit) ? t + 1 : maxit;
  free(v); free(z); free(w);
  return sqrt(lam);
}

double orc_power_norm_Q(int32_t qkind, int64_t n, const double* Qd,
                        const int64_t* Qp, const int32_t* Qc, const double* Qv,
                        uint64_t seed, uint32_t inst, double tol, int32_t maxit,
                        int32_t* iters) {
  if (qkind == 0 || n == 0) { *iters = 0; return 0.0; }
  double* v = malloc(sizeof(double) * n);
  double* z = malloc(sizeof(double) * n);
  double* w = malloc(sizeof(double) * n);
  power_start(n, seed, inst, 1u, v);
  double lam = 0.0, lam_prev = 0.0;
  int32_t t;
  for (t = 0; t < maxit; ++t) {
    q_mv(qkind, n, Qd, Qp, Qc, Qv, v, w);
    lam = 0.0;
    for (int64_t j = 0; j < n; ++j) lam += w[j] * w[j];
    q_mv(qkind, n, Qd, Qp, Qc, Qv, w, z); /* Q symmetric: Q^T w = Q w */
    double zn = norm2(n, z);
    if (zn == 0.0) break;
    for (int64_t i = 0; i < n; ++i) v[i] = z[i] / zn;
    if (t >= 1 && fabs(lam - lam_prev) <= tol * lam) break;
    lam_prev = lam;
  }
  *iters = (t < maxit) ? t + 1 : maxit;
  free(v); free(z); free(w);
  return sqrt(lam);
}

/* ======================================================================
 * Step sizes.  Preprocess makes ||K||_2 = 1 so that the PDHG condition
 * reads tau1*tau2 <= sigma (Section 3).  Reading of the split: tau1 =
 * sqrt(sigma), capped at 1/(2L) with L = 2(||Q||+rho) (Eq. 2's smoothness
 * constant, the cap of Prop. 2) when cap != 0; tau2 = sigma / tau1.
 * ====================================================================== */
void orc_step_sizes(double sigma, double normQ, double rho, int32_t cap,
                    double* tau1, double* tau2) {
  double t1 = sqrt(sigma);
  if (cap) {
    double L = 2.0 * (normQ + rho);
    if (L > 0.0 && 1.0 / (2.0 * L) < t1) t1 = 1.0 / (2.0 * L);
  }
  *tau1 = t1;
  *tau2 = sigma / t1;
}

/* ======================================================================
 * UpdatePenalty (Section 3):  rho~_n = rho_min (1 + n/T)^p,
 * rho_n = clip(rho~_n, rho_{n-1} + delta, rho_max).  Reading: clip(v, lo,
 * hi) = min(max(v, lo), hi) (so rho_max wins when lo > hi); rho_0 =
 * min(rho_min, rho_max); n counts completed sampling triggers.
 * ====================================================================== */
double orc_rho_update(int64_t n, double rho_prev, double rho_min,
                      double rho_max, double T, double p, double delta) {
  if (n == 0) return rho_min < rho_max ? rho_min : rho_max;
  double rt = rho_min * pow(1.0 + (double)n / T, p);
  double lo = rho_prev + delta;
  double v = rt < lo ? lo : rt;
  return v > rho_max ? rho_max : v;
}

/* ======================================================================
 * FirstOrderStep = PDHG update, Alg. 2, in the order printed there:
 *   y_k    = Proj_{R+^{m1} x R^{m2}}( y_{k-1} + tau2 (K xbar_{k-1} + r) )
 *   delta  = c + rho + K^T y_k + 2 Q x_{k-1} - 2 rho x_{k-1}
 *   x_k    = Proj_{[0,1]^n}( x_{k-1} - tau1 delta )
 *   xbar_k = 2 x_k - x_{k-1}
 * (K, r, Q, c already preprocessed; Q symmetric).  y is updated in place.
 * ====================================================================== */
void orc_pdhg_step(int64_t n, int64_t m, int64_t m1, const int64_t* Kp,
                   const int32_t* Kc, const double* Kv, const double* r,
                   int32_t qkind, const double* Qd, const int64_t* Qp,
                   const int32_t* Qc, const double* Qv, const double* c,
                   double tau1, double tau2, double rho, const double* x_prev,
                   const double* xbar_prev, double* y, double* x_out,
                   double* xbar_out, double* delta_out) {
  double* Kx = malloc(sizeof(double) * (m > 0 ? m : 1));
  double* KTy = malloc(sizeof(double) * (n > 0 ? n : 1));
  double* Qx = malloc(sizeof(double) * (n > 0 ? n : 1));
  csr_mv(m, Kp, Kc, Kv, xbar_prev, Kx);
  ORC_PAR_FOR
  for (int64_t j = 0; j < m; ++j) {
    double yj = y[j] + tau2 * (Kx[j] + r[j]);
    if (j < m1 && yj < 0.0) yj = 0.0;
    y[j] = yj;
  }
  csr_mtv(m, n, Kp, Kc, Kv, y, KTy);
  q_mv(qkind, n, Qd, Qp, Qc, Qv, x_prev, Qx);
  ORC_PAR_FOR
  for (int64_t i = 0; i < n; ++i) {
    double delta = c[i] + rho + KTy[i] + 2.0 * Qx[i] - 2.0 * rho * x_prev[i];
    double xi = x_prev[i] - tau1 * delta;
    if (xi < 0.0) xi = 0.0;
    if (xi > 1.0) xi = 1.0;
    x_out[i] = xi;
    xbar_out[i] = 2.0 * xi - x_prev[i];
    if (delta_out) delta_out[i] = delta;
  }
  free(Kx); free(KTy); free(Qx);
}

/* ======================================================================
 * RandSampleStep, generic Bernoulli (Alg. 3): X[l,i] ~ Bernoulli(p_i).
 * Reading of the draw: threshold t_i = floor(p_i 2^24) taken from the FP32
 * probability (exact: scaling by 2^24 is exact), X = 1 iff (u >> 8) < t_i,
 * u = Philox lane (stream 0, instance, round, sample l, variable i).
 * X is sample-major bytes (k x n).  mask (optional) skips variables with
 * mask[i] != 0 (they belong to one-hot groups and are drawn there).
 * ====================================================================== */
static uint32_t prob_threshold(float p) {
  if (!(p > 0.0f)) return 0u;      /* also maps NaN to 0 */
  if (p >= 1.0f) return 16777216u;
  return (uint32_t)floor((double)p * 16777216.0);
}

/* Candidates first .. first+k-1 of a round (row s - first of X). */
void orc_bernoulli_from(int64_t n, int32_t first, int32_t k, const float* p, uint64_t seed,
                        uint32_t inst, uint32_t round_id, const uint8_t* mask,
                        uint8_t* X) {
  ORC_PAR_FOR
  for (int32_t r = 0; r < k; ++r)
    for (int64_t i = 0; i < n; ++i) {
      if (mask && mask[i]) continue;
      uint32_t u = orc_philox_lane(seed, 0u, inst, round_id, (uint32_t)(first + r),
                                   (uint64_t)i);
      X[(int64_t)r * n + i] = ((u >> 8) < prob_threshold(p[i])) ? 1 : 0;
    }
}

void orc_bernoulli(int64_t n, int32_t k, const float* p, uint64_t seed,
                   uint32_t inst, uint32_t round_id, const uint8_t* mask,
                   uint8_t* X) {
  orc_bernoulli_from(n, 0, k, p, seed, inst, round_id, mask, X);
}

/* Categorical pick over a list of candidate variables (customized sampling,
 * Section 2.4.2, read as one draw per group): weights w = floor(p 2^24) in
 * list order, W = sum w; if W > 0 pick the first position whose inclusive
 * prefix exceeds floor(u W / 2^32) (exact 128-bit product); if W = 0 pick
 * position floor(u len / 2^32). */
static int64_t categorical_pick(int64_t len, const int64_t* idx, const float* p,
                                uint32_t u) {
  uint64_t W = 0;
  for (int64_t t = 0; t < len; ++t) W += prob_threshold(p[idx[t]]);
  if (W == 0) return (int64_t)(((uint64_t)u * (uint64_t)len) >> 32);
  unsigned __int128 prod = (unsigned __int128)u * (unsigned __int128)W;
  uint64_t r = (uint64_t)(prod >> 32);
  uint64_t acc = 0;
  for (int64_t t = 0; t < len; ++t) {
    acc += prob_threshold(p[idx[t]]);
    if (acc > r) return t;
  }
  return len - 1; /* unreachable: r < W */
}

/* One-hot groups: each disjoint group G (an assignment-type equality row
 * sum_{i in G} x_i = 1) receives exactly one 1; u = Philox lane (stream 1,
 * index = group number). */
void orc_onehot(int64_t n, int64_t ngroups, const int64_t* gp,
                const int64_t* gi, int32_t k, const float* p, uint64_t seed,
                uint32_t inst, uint32_t round_id, uint8_t* X) {
  ORC_PAR_FOR
  for (int32_t s = 0; s < k; ++s)
    for (int64_t g = 0; g < ngroups; ++g) {
      int64_t len = gp[g + 1] - gp[g];
      if (len <= 0) continue;
      uint32_t u = orc_philox_lane(seed, 1u, inst, round_id, (uint32_t)s,
                                   (uint64_t)g);
      int64_t pick = categorical_pick(len, gi + gp[g], p, u);
      for (int64_t t = 0; t < len; ++t) X[(int64_t)s * n + gi[gp[g] + t]] = 0;
      X[(int64_t)s * n + gi[gp[g] + pick]] = 1;
    }
}

/* Axial 3D assignment (Eq. assign3d) sampled feasibly by construction, a
 * customized RandSampleStep in the sense of Section 2.4.2: for i = 0..I-1
 * draw one (j,k) among the pairs whose j and k are both still unused, by the
 * categorical rule above over x_ijk (index (i I + j) I + k) in (j,k)
 * row-major order; u = Philox lane (stream 2, index i). */
void orc_axial3d(int32_t I, int32_t k, const float* p, uint64_t seed,
                 uint32_t inst, uint32_t round_id, uint8_t* X) {
  int64_t n = (int64_t)I * I * I;
  int64_t* cand = malloc(sizeof(int64_t) * (size_t)I * I);
  uint8_t* usedJ = malloc((size_t)I);
  uint8_t* usedK = malloc((size_t)I);
  for (int32_t s = 0; s < k; ++s) {
    memset(X + (int64_t)s * n, 0, (size_t)n);
    memset(usedJ, 0, (size_t)I);
    memset(usedK, 0, (size_t)I);
    for (int32_t i = 0; i < I; ++i) {
      int64_t len = 0;
      for (int32_t j = 0; j < I; ++j) {
        if (usedJ[j]) continue;
        for (int32_t kk = 0; kk < I; ++kk)
          if (!usedK[kk]) cand[len++] = ((int64_t)i * I + j) * I + kk;
      }
      uint32_t u = orc_philox_lane(seed, 2u, inst, round_id, (uint32_t)s,
                                   (uint64_t)i);
      int64_t v = cand[categorical_pick(len, cand, p, u)];
      X[(int64_t)s * n + v] = 1;
      usedJ[(v / I) % I] = 1;
      usedK[v % I] = 1;
    }
  }
  free(cand); free(usedJ); free(usedK);
}

/* Algorithm 4 (customized sampling for the 3D assignment, Section 2.4.2):
 * the largest gamma*I entries of p give a greedy partial assignment, every
 * candidate completes it at random and improves it by L pairwise
 * interchanges.  The paper fixes the outline only; readings used here:
 *  (a) the gamma*I largest entries of p, ordered by p descending, then by
 *      variable index ascending;
 *  (b) greedy: an entry (i,j,k) is accepted when i, j and k are all unused;
 *  (c) completion: the free j's and the free k's (each ascending) are
 *      shuffled by Fisher-Yates (q = F-1 down to 1, r = floor(u (q+1) / 2^32)
 *      with u the Philox lane of stream 6, index t for the t-th draw: the j's
 *      first, then the k's) and handed in turn to the free i's (ascending);
 *  (d) improvement: up to L steps, each applying the single best strictly
 *      improving interchange between the triples of i = a and i = b (a < b):
 *      type 0 exchanges their j, type 1 their k; exact integer costs; ties
 *      to the smallest (a, b, type); a step without improvement ends it. */
static int cmp_desc_pv(const void* x, const void* y) {
  const double* a = (const double*)x;
  const double* b = (const double*)y;
  if (a[0] != b[0]) return a[0] > b[0] ? -1 : 1;      /* p descending */
  return a[1] < b[1] ? -1 : (a[1] > b[1] ? 1 : 0);     /* index ascending */
}

void orc_assign3d_custom(int32_t I, int32_t gamma, int32_t L, int32_t k, const float* p,
                         const int64_t* cost, uint64_t seed, uint32_t inst,
                         uint32_t round_id, uint8_t* X) {
  const int64_t n = (int64_t)I * I * I;
  const int64_t K = (int64_t)gamma * I;
  double* pv = malloc(sizeof(double) * 2 * (size_t)n);
  for (int64_t v = 0; v < n; ++v) { pv[2 * v] = (double)p[v]; pv[2 * v + 1] = (double)v; }
  qsort(pv, (size_t)n, 2 * sizeof(double), cmp_desc_pv);
  int32_t* J0 = malloc(sizeof(int32_t) * (size_t)I);
  int32_t* K0 = malloc(sizeof(int32_t) * (size_t)I);
  uint8_t* uj = calloc((size_t)I, 1);
  uint8_t* uk = calloc((size_t)I, 1);
  for (int32_t i = 0; i < I; ++i) J0[i] = K0[i] = -1;
  for (int64_t e = 0; e < K && e < n; ++e) {
    const int64_t v = (int64_t)pv[2 * e + 1];
    const int32_t i = (int32_t)(v / ((int64_t)I * I)), j = (int32_t)((v / I) % I),
                  kk = (int32_t)(v % I);
    if (J0[i] < 0 && !uj[j] && !uk[kk]) { J0[i] = j; K0[i] = kk; uj[j] = 1; uk[kk] = 1; }
  }
  int32_t* J = malloc(sizeof(int32_t) * (size_t)I);
  int32_t* Kk = malloc(sizeof(int32_t) * (size_t)I);
  int32_t* fi = malloc(sizeof(int32_t) * (size_t)I);
  int32_t* fj = malloc(sizeof(int32_t) * (size_t)I);
  int32_t* fk = malloc(sizeof(int32_t) * (size_t)I);
#define C3(i, j, kk) cost[((int64_t)(i) * I + (j)) * I + (kk)]
  for (int32_t s = 0; s < k; ++s) {
    int32_t F = 0, Fj = 0, Fk = 0;
    for (int32_t i = 0; i < I; ++i) {
      J[i] = J0[i]; Kk[i] = K0[i];
      if (J0[i] < 0) fi[F++] = i;
      if (!uj[i]) fj[Fj++] = i;
      if (!uk[i]) fk[Fk++] = i;
    }
    uint64_t t = 0;
    for (int32_t q = F - 1; q >= 1; --q) {
      const uint32_t u = orc_philox_lane(seed, 6u, inst, round_id, (uint32_t)s, t++);
      const int32_t r = (int32_t)(((uint64_t)u * (uint64_t)(q + 1)) >> 32);
      const int32_t tmp = fj[q]; fj[q] = fj[r]; fj[r] = tmp;
    }
    for (int32_t q = F - 1; q >= 1; --q) {
      const uint32_t u = orc_philox_lane(seed, 6u, inst, round_id, (uint32_t)s, t++);
      const int32_t r = (int32_t)(((uint64_t)u * (uint64_t)(q + 1)) >> 32);
      const int32_t tmp = fk[q]; fk[q] = fk[r]; fk[r] = tmp;
    }
    for (int32_t e = 0; e < F; ++e) { J[fi[e]] = fj[e]; Kk[fi[e]] = fk[e]; }
    for (int32_t step = 0; step < L; ++step) {
      int64_t best = 0;
      int32_t ba = -1, bb = -1, bt = -1;
      for (int32_t a = 0; a < I; ++a)
        for (int32_t b = a + 1; b < I; ++b) {
          const int64_t old = C3(a, J[a], Kk[a]) + C3(b, J[b], Kk[b]);
          const int64_t d0 = C3(a, J[b], Kk[a]) + C3(b, J[a], Kk[b]) - old;
          const int64_t d1 = C3(a, J[a], Kk[b]) + C3(b, J[b], Kk[a]) - old;
          if (d0 < best) { best = d0; ba = a; bb = b; bt = 0; }
          if (d1 < best) { best = d1; ba = a; bb = b; bt = 1; }
        }
      if (ba < 0) break;
      if (bt == 0) { const int32_t tmp = J[ba]; J[ba] = J[bb]; J[bb] = tmp; }
      else { const int32_t tmp = Kk[ba]; Kk[ba] = Kk[bb]; Kk[bb] = tmp; }
    }
    memset(X + (int64_t)s * n, 0, (size_t)n);
    for (int32_t i = 0; i < I; ++i) X[(int64_t)s * n + ((int64_t)i * I + J[i]) * I + Kk[i]] = 1;
  }
#undef C3
  free(pv); free(J0); free(K0); free(uj); free(uk); free(J); free(Kk); free(fi); free(fj);
  free(fk);
}

/* Monotone relaxation with repair (Section 2.4.3), facility-location form:
 * y <- y OR (OR of x_k over the repair list), valid because the opening
 * costs are non-negative. */
void orc_closure(int64_t n, int64_t nrep, const int64_t* rv, const int64_t* rp,
                 const int64_t* ri, int32_t k, uint8_t* X) {
  ORC_PAR_FOR
  for (int32_t s = 0; s < k; ++s)
    for (int64_t q = 0; q < nrep; ++q) {
      uint8_t v = X[(int64_t)s * n + rv[q]];
      for (int64_t t = rp[q]; t < rp[q + 1]; ++t) v |= X[(int64_t)s * n + ri[t]];
      X[(int64_t)s * n + rv[q]] = v;
    }
}

/* Repair after a monotone relaxation (Section 2.4.3): an equality group
 * sum_{k in G} x_k = 1 relaxed to sum >= 1 lets a candidate select several
 * members; the repair keeps the selected member of least cost c_k (ties to
 * the member listed first) and clears the others, so the candidate meets
 * the equality again whenever it selected any member.  Valid when dropping
 * a member can violate no other constraint (the caller's claim). */
void orc_repair_min(int64_t n, int64_t ng, const int64_t* gp, const int64_t* gi,
                    const int64_t* cost, int32_t k, uint8_t* X) {
  ORC_PAR_FOR
  for (int32_t s = 0; s < k; ++s) {
    uint8_t* x = X + (int64_t)s * n;
    for (int64_t g = 0; g < ng; ++g) {
      int64_t keep = -1;
      for (int64_t t = gp[g]; t < gp[g + 1]; ++t)
        if (x[gi[t]] && (keep < 0 || cost[gi[t]] < cost[keep])) keep = gi[t];
      for (int64_t t = gp[g]; t < gp[g + 1]; ++t)
        if (gi[t] != keep) x[gi[t]] = 0;
    }
  }
}

/* General repair after a monotone relaxation (Section 2.4.3): equality rows
 * with 0/1 coefficients relaxed to covering rows sum_{k in R} x_k >= 1, and
 * c >= 0, so dropping a selected variable never raises the objective.  The
 * repair (a reading: the paper leaves it problem-specific) visits each
 * candidate's selected variables of these rows in decreasing cost, ties to
 * the larger index first, and drops a variable when every relaxed row that
 * contains it keeps another selected member ("reverse delete").  The
 * result is a minimal cover of the rows the candidate covered.  Rows are
 * CSR (rp, ri: variable lists); they may overlap. */
static const int64_t* g_rr_cost;
static int cmp_rr_order(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  if (g_rr_cost[x] != g_rr_cost[y]) return g_rr_cost[x] > g_rr_cost[y] ? -1 : 1;
  return x > y ? -1 : (x < y ? 1 : 0);
}

void orc_repair_rows(int64_t n, int64_t nr, const int64_t* rp, const int64_t* ri,
                     const int64_t* cost, int32_t k, uint8_t* X) {
  /* rows of each variable (CSC of the relaxed rows) */
  int64_t* deg = calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t t = 0; t < rp[nr]; ++t) deg[ri[t] + 1]++;
  for (int64_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
  int64_t* vr = malloc(sizeof(int64_t) * (size_t)(rp[nr] > 0 ? rp[nr] : 1));
  int64_t* fill = calloc((size_t)n, sizeof(int64_t));
  for (int64_t r = 0; r < nr; ++r)
    for (int64_t t = rp[r]; t < rp[r + 1]; ++t) vr[deg[ri[t]] + fill[ri[t]]++] = r;
  /* the variables of relaxed rows in decreasing cost (larger index first) */
  int64_t nv = 0;
  int64_t* order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t v = 0; v < n; ++v)
    if (deg[v + 1] > deg[v]) order[nv++] = v;
  g_rr_cost = cost;
  qsort(order, (size_t)nv, sizeof(int64_t), cmp_rr_order);
  int64_t* cnt = malloc(sizeof(int64_t) * (size_t)(nr > 0 ? nr : 1));
  for (int32_t s = 0; s < k; ++s) {
    uint8_t* x = X + (int64_t)s * n;
    for (int64_t r = 0; r < nr; ++r) {
      cnt[r] = 0;
      for (int64_t t = rp[r]; t < rp[r + 1]; ++t) cnt[r] += x[ri[t]];
    }
    for (int64_t q = 0; q < nv; ++q) {
      const int64_t v = order[q];
      if (!x[v]) continue;
      int removable = 1;
      for (int64_t t = deg[v]; t < deg[v + 1]; ++t)
        if (cnt[vr[t]] < 2) { removable = 0; break; }
      if (!removable) continue;
      x[v] = 0;
      for (int64_t t = deg[v]; t < deg[v + 1]; ++t) cnt[vr[t]]--;
    }
  }
  free(deg); free(vr); free(fill); free(order); free(cnt);
}

/* ======================================================================
 * EvalBest, evaluation half (Section 3 and Eq. 1), on the ORIGINAL data:
 *   viol_s = #{j : A_j X_s < b_j} + #{j : B_j X_s != d_j}
 *   obj_s  = X_s^T Q X_s + c^T X_s
 * Integer version: exact int64 arithmetic (all data integral).
 * qkind: 0 none, 1 dense (n x n int64), 2 CSR (int64 values).
 * ====================================================================== */
void orc_eval_int(int64_t n, int64_t m1, const int64_t* Ap, const int32_t* Ac,
                  const int64_t* Av, const int64_t* b, int64_t m2,
                  const int64_t* Bp, const int32_t* Bc, const int64_t* Bv,
                  const int64_t* d, int32_t qkind, const int64_t* Qd,
                  const int64_t* Qp, const int32_t* Qc, const int64_t* Qv,
                  const int64_t* c, int32_t k, const uint8_t* X, int32_t* viol,
                  int64_t* obj) {
  ORC_PAR_FOR
  for (int32_t s = 0; s < k; ++s) {
    const uint8_t* x = X + (int64_t)s * n;
    int32_t v = 0;
    for (int64_t j = 0; j < m1; ++j) {
      int64_t acc = 0;
      for (int64_t t = Ap[j]; t < Ap[j + 1]; ++t) acc += Av[t] * (int64_t)x[Ac[t]];
      if (acc < b[j]) ++v;
    }
    for (int64_t j = 0; j < m2; ++j) {
      int64_t acc = 0;
      for (int64_t t = Bp[j]; t < Bp[j + 1]; ++t) acc += Bv[t] * (int64_t)x[Bc[t]];
      if (acc != d[j]) ++v;
    }
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) o += c[i] * (int64_t)x[i];
    if (qkind == 1) {
      for (int64_t i = 0; i < n; ++i) {
        if (!x[i]) continue;
        for (int64_t j = 0; j < n; ++j) o += Qd[i * n + j] * (int64_t)x[j];
      }
    } else if (qkind == 2) {
      for (int64_t i = 0; i < n; ++i) {
        if (!x[i]) continue;
        for (int64_t t = Qp[i]; t < Qp[i + 1]; ++t) o += Qv[t] * (int64_t)x[Qc[t]];
      }
    }
    viol[s] = v;
    obj[s] = o;
  }
}

/* Same in FP64 for non-integral data; a row counts as violated when it
 * misses its right-hand side by more than 1e-9 (1 + |rhs|) (a reading). */
void orc_eval_f64(int64_t n, int64_t m1, const int64_t* Ap, const int32_t* Ac,
                  const double* Av, const double* b, int64_t m2,
                  const int64_t* Bp, const int32_t* Bc, const double* Bv,
                  const double* d, int32_t qkind, const double* Qd,
                  const int64_t* Qp, const int32_t* Qc, const double* Qv,
                  const double* c, int32_t k, const uint8_t* X, int32_t* viol,
                  double* obj) {
  ORC_PAR_FOR
  for (int32_t s = 0; s < k; ++s) {
    const uint8_t* x = X + (int64_t)s * n;
    int32_t v = 0;
    for (int64_t j = 0; j < m1; ++j) {
      double acc = 0.0;
      for (int64_t t = Ap[j]; t < Ap[j + 1]; ++t) acc += Av[t] * x[Ac[t]];
      if (acc < b[j] - 1e-9 * (1.0 + fabs(b[j]))) ++v;
    }
    for (int64_t j = 0; j < m2; ++j) {
      double acc = 0.0;
      for (int64_t t = Bp[j]; t < Bp[j + 1]; ++t) acc += Bv[t] * x[Bc[t]];
      if (fabs(acc - d[j]) > 1e-9 * (1.0 + fabs(d[j]))) ++v;
    }
    double o = 0.0;
    for (int64_t i = 0; i < n; ++i) o += c[i] * x[i];
    if (qkind == 1) {
      for (int64_t i = 0; i < n; ++i)
        if (x[i])
          for (int64_t j = 0; j < n; ++j) o += Qd[i * n + j] * x[j];
    } else if (qkind == 2) {
      for (int64_t i = 0; i < n; ++i)
        if (x[i])
          for (int64_t t = Qp[i]; t < Qp[i + 1]; ++t) o += Qv[t] * x[Qc[t]];
    }
    viol[s] = v;
    obj[s] = o;
  }
}

/* ======================================================================
 * EvalBest, incumbent half (Alg. 1): among the feasible samples of a round
 * (viol = 0) take the least objective, earliest sample first; it replaces
 * (z_best, x_best) only when strictly better, so earlier rounds win ties.
 * Returns the index of the replacing sample or -1.
 * ====================================================================== */
int32_t orc_incumbent_update(int32_t k, const int32_t* viol, const int64_t* obj,
                             uint32_t round_id, int32_t* found,
                             int64_t* best_obj, uint32_t* best_round,
                             int32_t* best_s) {
  int32_t pick = -1;
  for (int32_t s = 0; s < k; ++s) {
    if (viol[s] != 0) continue;
    if (pick < 0 || obj[s] < obj[pick]) pick = s;
  }
  if (pick < 0) return -1;
  if (*found && !(obj[pick] < *best_obj)) return -1;
  *found = 1;
  *best_obj = obj[pick];
  *best_round = round_id;
  *best_s = pick;
  return pick;
}

/* Final candidate round(x_k) of Alg. 1: x_i = 1 iff x_i > 0.5 (a reading:
 * the tie 0.5 goes to 0). */
void orc_round(int64_t n, const double* x, uint8_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (x[i] > 0.5) ? 1 : 0;
}

/* ======================================================================
 * CheckHalt indicators (Section 3 names three; definitions are a reading),
 * all on the preprocessed problem, x = x_k, xp = x_{k-1}:
 *   out[0] P_res = ||(max(0, K_I x + r_I), K_E x + r_E)||_2 / (1 + ||r||_2)
 *   out[1] Gap   : Q = 0: |c^T x - D(y)| / (1 + |c^T x| + |D(y)|) with the
 *                  Lagrangian dual bound D(y) = r^T y + sum_i min(0,(c+K^T y)_i);
 *                  Q != 0: ||s^x_k||_2, the primal residual of Thm. 2,
 *                  s^x = (xp - x)/tau1 + 2(Q - rho I)(x - xp)
 *   out[2] B_gap = (1/n) sum_i min(x_i, 1 - x_i)
 *   out[3] c^T x + x^T Q x (scaled relaxation objective)
 *   out[4] D(y) (Q = 0) or NaN
 *   out[5] ||s^x_k||_2
 * ====================================================================== */
void orc_halt_stats(int64_t n, int64_t m, int64_t m1, const int64_t* Kp,
                    const int32_t* Kc, const double* Kv, const double* r,
                    int32_t qkind, const double* Qd, const int64_t* Qp,
                    const int32_t* Qc, const double* Qv, const double* c,
                    double tau1, double rho, const double* x, const double* xp,
                    const double* y, double* out) {
  double* Kx = malloc(sizeof(double) * (m > 0 ? m : 1));
  double* KTy = malloc(sizeof(double) * (n > 0 ? n : 1));
  double* Qx = malloc(sizeof(double) * (n > 0 ? n : 1));
  double* dx = malloc(sizeof(double) * (n > 0 ? n : 1));
  double* Qdx = malloc(sizeof(double) * (n > 0 ? n : 1));
  csr_mv(m, Kp, Kc, Kv, x, Kx);
  double pr = 0.0, rn = 0.0;
  for (int64_t j = 0; j < m; ++j) {
    double v = Kx[j] + r[j];
    if (j < m1 && v < 0.0) v = 0.0;
    pr += v * v;
    rn += r[j] * r[j];
  }
  out[0] = sqrt(pr) / (1.0 + sqrt(rn));
  q_mv(qkind, n, Qd, Qp, Qc, Qv, x, Qx);
  double pobj = 0.0, bg = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    pobj += c[i] * x[i] + x[i] * Qx[i];
    bg += (x[i] < 1.0 - x[i]) ? x[i] : 1.0 - x[i];
  }
  out[2] = n > 0 ? bg / (double)n : 0.0;
  out[3] = pobj;
  for (int64_t i = 0; i < n; ++i) dx[i] = x[i] - xp[i];
  q_mv(qkind, n, Qd, Qp, Qc, Qv, dx, Qdx);
  double sx = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double v = -dx[i] / tau1 + 2.0 * Qdx[i] - 2.0 * rho * dx[i];
    sx += v * v;
  }
  out[5] = sqrt(sx);
  if (qkind == 0) {
    csr_mtv(m, n, Kp, Kc, Kv, y, KTy);
    double D = 0.0;
    for (int64_t j = 0; j < m; ++j) D += r[j] * y[j];
    for (int64_t i = 0; i < n; ++i) {
      double g = c[i] + KTy[i];
      if (g < 0.0) D += g;
    }
    out[4] = D;
    out[1] = fabs(pobj - D) / (1.0 + fabs(pobj) + fabs(D));
  } else {
    out[4] = NAN;
    out[1] = out[5];
  }
  free(Kx); free(KTy); free(Qx); free(dx); free(Qdx);
}

/* ======================================================================
 * Brute force over {0,1}^n (n <= 24) for Eq. (1) with integer data: the
 * least objective over feasible points, ties to the smallest binary code
 * (bit i of the code = x_i).  Returns 1 if a feasible point exists.
 * ====================================================================== */
int32_t orc_brute_force(int64_t n, int64_t m1, const int64_t* Ap,
                        const int32_t* Ac, const int64_t* Av, const int64_t* b,
                        int64_t m2, const int64_t* Bp, const int32_t* Bc,
                        const int64_t* Bv, const int64_t* d, int32_t qkind,
                        const int64_t* Qd, const int64_t* Qp, const int32_t* Qc,
                        const int64_t* Qv, const int64_t* c, int64_t* best_obj,
                        uint8_t* best_x, int64_t* nfeasible) {
  if (n > 24) return -1;
  uint8_t* x = malloc((size_t)n);
  int32_t found = 0;
  int64_t nf = 0;
  for (uint64_t code = 0; code < (1ull << n); ++code) {
    for (int64_t i = 0; i < n; ++i) x[i] = (uint8_t)((code >> i) & 1u);
    int32_t v;
    int64_t o;
    orc_eval_int(n, m1, Ap, Ac, Av, b, m2, Bp, Bc, Bv, d, qkind, Qd, Qp, Qc,
                 Qv, c, 1, x, &v, &o);
    if (v != 0) continue;
    ++nf;
    if (!found || o < *best_obj) {
      found = 1;
      *best_obj = o;
      memcpy(best_x, x, (size_t)n);
    }
  }
  free(x);
  *nfeasible = nf;
  return found;
}

/* ======================================================================
 * Fractional knapsack (Dantzig's greedy): max p^T x s.t. w^T x <= cap,
 * 0 <= x <= 1, w > 0.  Items by decreasing p_i / w_i (ties by index), filled
 * whole while they fit, the first that does not fit taken fractionally.
 * This is the LP relaxation the PDHG limit (rho = 0) must reach.
 * ====================================================================== */
static const double* g_ratio;
static int cmp_ratio(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  if (g_ratio[i] > g_ratio[j]) return -1;
  if (g_ratio[i] < g_ratio[j]) return 1;
  return (i < j) ? -1 : (i > j);
}

double orc_knapsack_lp(int64_t n, const double* w, const double* p, double cap,
                       double* x) {
  double* ratio = malloc(sizeof(double) * n);
  int64_t* ord = malloc(sizeof(int64_t) * n);
  for (int64_t i = 0; i < n; ++i) { ratio[i] = p[i] / w[i]; ord[i] = i; x[i] = 0.0; }
  g_ratio = ratio;
  qsort(ord, (size_t)n, sizeof(int64_t), cmp_ratio);
  double left = cap, val = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    int64_t i = ord[t];
    if (w[i] <= left) { x[i] = 1.0; left -= w[i]; val += p[i]; }
    else { x[i] = left / w[i]; val += p[i] * x[i]; break; }
  }
  free(ratio); free(ord);
  return val;
}

/* ======================================================================
 * Learned proposal (an added pattern; the paper has none): per-variable MLP
 *   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3,
 *   p  = clip(sigmoid(z), 2^-24, 1 - 2^-24)
 * (the clip bounds are the Bernoulli / categorical threshold's resolution:
 * every probability keeps a weight floor(p 2^24) of at least 1)
 * with F inputs, H hidden units; weights (not biases, not activations)
 * rounded to bf16 by round-to-nearest-even when round_bf16 != 0, computed
 * in FP64.  Weight layout: W1 [H x F] row-major, W2 [H x H] row-major.
 * ====================================================================== */
float orc_bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) { /* inf / nan: keep, quiet nan */
    if (u & 0x007FFFFFu) u |= 0x00400000u;
    u &= 0xFFFF0000u;
  } else {
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
  }
  float r;
  memcpy(&r, &u, 4);
  return r;
}

static double wq(const float* w, int64_t i, int32_t rb) {
  return rb ? (double)orc_bf16_round(w[i]) : (double)w[i];
}

/* forward: z_out[v] (logit) and p_out[v]; h1/h2 (nv x H) optional. */
void orc_mlp_forward(int64_t nv, int32_t F, int32_t H, const float* feat,
                     const float* W1, const float* b1, const float* W2,
                     const float* b2, const float* w3, const float* b3,
                     int32_t rb, double* z_out, double* p_out, double* h1_out,
                     double* h2_out) {
  double* h1 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  for (int64_t v = 0; v < nv; ++v) {
    const float* f = feat + v * F;
    for (int32_t a = 0; a < H; ++a) {
      double s = b1[a];
      for (int32_t q = 0; q < F; ++q) s += wq(W1, (int64_t)a * F + q, rb) * (double)f[q];
      h1[a] = s > 0.0 ? s : 0.0;
    }
    for (int32_t a = 0; a < H; ++a) {
      double s = b2[a];
      for (int32_t q = 0; q < H; ++q) s += wq(W2, (int64_t)a * H + q, rb) * h1[q];
      h2[a] = s > 0.0 ? s : 0.0;
    }
    double z = b3[0];
    for (int32_t a = 0; a < H; ++a) z += wq(w3, a, rb) * h2[a];
    double p = 1.0 / (1.0 + exp(-z));
    if (p < 0x1p-24) p = 0x1p-24;
    if (p > 1.0 - 0x1p-24) p = 1.0 - 0x1p-24;
    z_out[v] = z;
    p_out[v] = p;
    if (h1_out) memcpy(h1_out + v * H, h1, sizeof(double) * H);
    if (h2_out) memcpy(h2_out + v * H, h2, sizeof(double) * H);
  }
  free(h1); free(h2);
}

/* Mean binary cross-entropy on the logit, loss = (1/nv) sum softplus(z) - y z
 * (the unclipped sigmoid; the clip only guards sampling), and its gradient
 * with respect to the fp32 master weights, the bf16 rounding passed straight
 * through; relu'(0) = 0.  Gradients are written (not accumulated). */
double orc_mlp_loss_grad(int64_t nv, int32_t F, int32_t H, const float* feat,
                         const float* label, const float* W1, const float* b1,
                         const float* W2, const float* b2, const float* w3,
                         const float* b3, int32_t rb, double* gW1, double* gb1,
                         double* gW2, double* gb2, double* gw3, double* gb3) {
  double* pre1 = malloc(sizeof(double) * H);
  double* h1 = malloc(sizeof(double) * H);
  double* pre2 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  double* d2 = malloc(sizeof(double) * H);
  double* d1 = malloc(sizeof(double) * H);
  memset(gW1, 0, sizeof(double) * (size_t)H * F);
  memset(gb1, 0, sizeof(double) * H);
  memset(gW2, 0, sizeof(double) * (size_t)H * H);
  memset(gb2, 0, sizeof(double) * H);
  memset(gw3, 0, sizeof(double) * H);
  gb3[0] = 0.0;
  double loss = 0.0;
  for (int64_t v = 0; v < nv; ++v) {
    const float* f = feat + v * F;
    for (int32_t a = 0; a < H; ++a) {
      double s = b1[a];
      for (int32_t q = 0; q < F; ++q) s += wq(W1, (int64_t)a * F + q, rb) * (double)f[q];
      pre1[a] = s;
      h1[a] = s > 0.0 ? s : 0.0;
    }
    for (int32_t a = 0; a < H; ++a) {
      double s = b2[a];
      for (int32_t q = 0; q < H; ++q) s += wq(W2, (int64_t)a * H + q, rb) * h1[q];
      pre2[a] = s;
      h2[a] = s > 0.0 ? s : 0.0;
    }
    double z = b3[0];
    for (int32_t a = 0; a < H; ++a) z += wq(w3, a, rb) * h2[a];
    double y = (double)label[v];
    double sp = z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
    loss += sp - y * z;
    double dz = (1.0 / (1.0 + exp(-z)) - y) / (double)nv;
    gb3[0] += dz;
    for (int32_t a = 0; a < H; ++a) {
      gw3[a] += dz * h2[a];
      d2[a] = (pre2[a] > 0.0) ? dz * wq(w3, a, rb) : 0.0;
    }
    for (int32_t a = 0; a < H; ++a) {
      gb2[a] += d2[a];
      for (int32_t q = 0; q < H; ++q) gW2[(int64_t)a * H + q] += d2[a] * h1[q];
    }
    for (int32_t q = 0; q < H; ++q) {
      double s = 0.0;
      for (int32_t a = 0; a < H; ++a) s += wq(W2, (int64_t)a * H + q, rb) * d2[a];
      d1[q] = (pre1[q] > 0.0) ? s : 0.0;
    }
    for (int32_t a = 0; a < H; ++a) {
      gb1[a] += d1[a];
      for (int32_t q = 0; q < F; ++q) gW1[(int64_t)a * F + q] += d1[a] * (double)f[q];
    }
  }
  free(pre1); free(h1); free(pre2); free(h2); free(d2); free(d1);
  return loss / (double)nv;
}

/* Adam (Kingma & Ba 2014), step t >= 1, in place on fp32 masters with
 * double moments: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void orc_adam(int64_t np, float* w, const double* g, double* m, double* v,
              int64_t t, double lr, double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    w[i] = (float)((double)w[i] - lr * mh / (sqrt(vh) + eps));
  }
}
