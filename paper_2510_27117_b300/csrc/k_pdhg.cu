// k_pdhg.cu -- FirstOrderStep (PDHG update, Alg. 2) on the preprocessed
// problem of Eq. (2), FP32 storage with compensated FP32 accumulation:
//   y_k    = Proj_{R+^{m1} x R^{m2}}( y_{k-1} + tau2 (K xbar_{k-1} + r) )
//   delta  = c + rho + K^T y_k + 2 Q x_{k-1} - 2 rho x_{k-1}
//   x_k    = Proj_{[0,1]^n}( x_{k-1} - tau1 delta ),   xbar_k = 2 x_k - x_{k-1}
// The batch is block-diagonal: every row / column carries its instance id,
// whose step sizes come from the iteration's parameter slot.  UpdatePenalty
// (Section 3) for the NEXT iteration is folded into block 0 of the first
// primal kernel of each iteration (it writes the other parity slot).
#include <functional>

#include "internal.cuh"
#include "penalty.cuh"

namespace {

using gf::CSum;

// ---------------------------------------------------------------------------
// Dual step over a bucket of rows, `LANES` threads per row.
// ---------------------------------------------------------------------------
template <int LANES>
__global__ void __launch_bounds__(256)
k_dual_rows(const int32_t* __restrict__ rows, int32_t nrows,
            const int64_t* __restrict__ Kp, const int32_t* __restrict__ Kc,
            const float* __restrict__ Kv, const float* __restrict__ xbar,
            const float* __restrict__ r, const uint8_t* __restrict__ row_eq,
            const int32_t* __restrict__ row_inst,
            const GfIParam* __restrict__ ip, float* __restrict__ y) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t grp = gid / LANES;
  const int lane = (int)(gid % LANES);
  if (grp >= nrows) return;                 // whole groups exit together
  const int j = rows[grp];
  const int64_t t0 = Kp[j], t1 = Kp[j + 1];
  // the update's own operands, loaded before the row's gathers
  float yo = 0.f, rj = 0.f, tau2 = 0.f;
  uint8_t eq = 1;
  if (lane == 0) {
    yo = y[j];
    rj = r[j];
    eq = row_eq[j];
    tau2 = ip[row_inst[j]].tau2;
  }
  CSum acc;
  gf::gather_dot<4>(acc, Kc, Kv, xbar, t0 + lane, t1, LANES);
  gf::csum_group_reduce<LANES>(acc);
  if (lane == 0) {
    float v = yo + tau2 * (acc.value() + rj);
    if (!eq && v < 0.f) v = 0.f;
    y[j] = v;
  }
}

// Run index of group g: the largest r with run_ptr[r] <= g (binary search
// over at most a few thousand run offsets, cached).
GF_DEV int run_of(const int64_t* __restrict__ run_ptr, int nruns, int64_t g) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(run_ptr + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Dual step over a bucket given as runs of consecutive rows: the row id and
// instance come from the run, and for equal-length runs the nonzero range
// too (no id list, no row-pointer loads).  Same arithmetic as k_dual_rows.
template <int LANES>
__global__ void __launch_bounds__(256)
k_dual_runs(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr, int nruns,
            int64_t nrows, const int64_t* __restrict__ Kp, const int32_t* __restrict__ Kc,
            const float* __restrict__ Kv, const float* __restrict__ xbar,
            const float* __restrict__ r, const uint8_t* __restrict__ row_eq,
            const GfIParam* __restrict__ ip, float* __restrict__ y) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t grp = gid / LANES;
  const int lane = (int)(gid % LANES);
  if (grp >= nrows) return;                 // whole groups exit together
  const int q = nruns == 1 ? 0 : run_of(run_ptr, nruns, grp);
  const GfRun R = runs[q];
  const int64_t off = grp - __ldg(run_ptr + q);
  const int64_t j = R.first + off;
  const int64_t t0 = R.len >= 0 ? R.nnz0 + off * R.len : Kp[j];
  const int64_t t1 = R.len >= 0 ? t0 + R.len : Kp[j + 1];
  float yo = 0.f, rj = 0.f;                 // loaded before the row's gathers
  uint8_t eq = 1;
  if (lane == 0) {
    yo = y[j];
    rj = r[j];
    eq = row_eq[j];
  }
  CSum acc;
  gf::gather_dot<4>(acc, Kc, Kv, xbar, t0 + lane, t1, LANES);
  gf::csum_group_reduce<LANES>(acc);
  if (lane == 0) {
    const float tau2 = ip[R.inst].tau2;
    float v = yo + tau2 * (acc.value() + rj);
    if (!eq && v < 0.f) v = 0.f;
    y[j] = v;
  }
}

// ---------------------------------------------------------------------------
// Rows / columns with at most two nonzeros (the length bucket <= 2), given as
// runs: kShortRpt of them per thread, kShortRpt * 256 consecutive ones per
// block, so that a thread issues the loads of all its rows before it uses
// any (several independent gathers in flight instead of one dependent
// chain).  Sums as in the one-lane run kernels: the same two compensated
// adds in the same order, so the results are identical.
// ---------------------------------------------------------------------------
constexpr int kShortRpt = 4;

struct ShortRow {
  int64_t id, t0;
  int n, inst;                    // n = -1: no row
};

GF_DEV void short_rows(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr,
                       int nruns, int64_t count, const int64_t* __restrict__ ptr,
                       ShortRow (&w)[kShortRpt]) {
  const int64_t base = (int64_t)blockIdx.x * (256 * kShortRpt) + threadIdx.x;
  int64_t lo = 0, hi = -1;
  GfRun R{};
#pragma unroll
  for (int u = 0; u < kShortRpt; ++u) {
    const int64_t g = base + (int64_t)u * 256;
    w[u].n = -1;
    if (g >= count) continue;
    if (g >= hi) {
      const int q = nruns == 1 ? 0 : run_of(run_ptr, nruns, g);
      R = runs[q];
      lo = __ldg(run_ptr + q);
      hi = __ldg(run_ptr + q + 1);
    }
    const int64_t off = g - lo;
    w[u].id = R.first + off;
    w[u].inst = R.inst;
    if (R.len >= 0) {
      w[u].t0 = R.nnz0 + off * R.len;
      w[u].n = R.len;
    } else {
      w[u].t0 = ptr[w[u].id];
      w[u].n = (int)(ptr[w[u].id + 1] - w[u].t0);
    }
  }
}

// The block's rows, when they all lie in one run of two-entry rows whose
// nonzeros start at an even offset (nearly every block of a large bucket):
// row ids and nonzero offsets are then affine in the thread index, and each
// (index, value) pair is one 8-byte load.  Otherwise (run boundaries, the
// last block, other lengths) the general per-row bookkeeping of short_rows.
struct ShortBlock {
  GfRun R;
  int64_t off0;      // offset in the run of this thread's first row
  bool fast;
};
GF_DEV ShortBlock short_block(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr,
                              int nruns) {
  const int64_t b0 = (int64_t)blockIdx.x * (256 * kShortRpt);
  const int q = nruns == 1 ? 0 : run_of(run_ptr, nruns, b0);
  ShortBlock B;
  B.R = runs[q];
  const int64_t lo = __ldg(run_ptr + q), hi = __ldg(run_ptr + q + 1);
  B.off0 = b0 - lo + threadIdx.x;
  B.fast = B.R.len == 2 && !(B.R.nnz0 & 1) && b0 + 256 * kShortRpt <= hi;
  return B;
}

__global__ void __launch_bounds__(256, 4)
k_dual_short(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr, int nruns,
             int64_t nrows, const int64_t* __restrict__ Kp, const int32_t* __restrict__ Kc,
             const float* __restrict__ Kv, const float* __restrict__ xbar,
             const float* __restrict__ r, const uint8_t* __restrict__ row_eq,
             const GfIParam* __restrict__ ip, float* __restrict__ y) {
  const ShortBlock B = short_block(runs, run_ptr, nruns);
  if (B.fast) {
    const float tau2 = ip[B.R.inst].tau2;
    int2 c[kShortRpt];
    float2 v[kShortRpt];
    float yo[kShortRpt], rr[kShortRpt], xa[kShortRpt], xb[kShortRpt];
    uint8_t eq[kShortRpt];
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      const int64_t off = B.off0 + u * 256, j = B.R.first + off, t = B.R.nnz0 + 2 * off;
      c[u] = *reinterpret_cast<const int2*>(Kc + t);
      v[u] = *reinterpret_cast<const float2*>(Kv + t);
      yo[u] = y[j];
      rr[u] = r[j];
      eq[u] = row_eq[j];
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      xa[u] = xbar[c[u].x];
      xb[u] = xbar[c[u].y];
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      CSum acc;
      acc.add(__fmul_rn(v[u].x, xa[u]));
      acc.add(__fmul_rn(v[u].y, xb[u]));
      float val = yo[u] + tau2 * (acc.value() + rr[u]);
      if (!eq[u] && val < 0.f) val = 0.f;
      y[B.R.first + B.off0 + u * 256] = val;
    }
    return;
  }
  ShortRow w[kShortRpt];
  short_rows(runs, run_ptr, nruns, nrows, Kp, w);
  int c0[kShortRpt], c1[kShortRpt];
  float v0[kShortRpt], v1[kShortRpt], yo[kShortRpt], rr[kShortRpt];
  float xa[kShortRpt], xb[kShortRpt];
  uint8_t eq[kShortRpt];
#pragma unroll
  for (int u = 0; u < kShortRpt; ++u) {
    c0[u] = w[u].n >= 1 ? Kc[w[u].t0] : 0;
    v0[u] = w[u].n >= 1 ? Kv[w[u].t0] : 0.f;
    c1[u] = w[u].n >= 2 ? Kc[w[u].t0 + 1] : 0;
    v1[u] = w[u].n >= 2 ? Kv[w[u].t0 + 1] : 0.f;
    yo[u] = w[u].n >= 0 ? y[w[u].id] : 0.f;
    rr[u] = w[u].n >= 0 ? r[w[u].id] : 0.f;
    eq[u] = w[u].n >= 0 ? row_eq[w[u].id] : 1;
  }
#pragma unroll
  for (int u = 0; u < kShortRpt; ++u) {
    xa[u] = w[u].n >= 1 ? xbar[c0[u]] : 0.f;
    xb[u] = w[u].n >= 2 ? xbar[c1[u]] : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kShortRpt; ++u) {
    if (w[u].n < 0) continue;
    CSum acc;
    if (w[u].n >= 1) acc.add(__fmul_rn(v0[u], xa[u]));
    if (w[u].n >= 2) acc.add(__fmul_rn(v1[u], xb[u]));
    const float tau2 = ip[w[u].inst].tau2;
    float v = yo[u] + tau2 * (acc.value() + rr[u]);
    if (!eq[u] && v < 0.f) v = 0.f;
    y[w[u].id] = v;
  }
}

// Columns with at most two K^T entries and no Q entries.
__global__ void __launch_bounds__(256, 4)
k_primal_short(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr, int nruns,
               int64_t ncols, const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
               const float* __restrict__ Tv, const float* __restrict__ y,
               const float* __restrict__ x_old, const float* __restrict__ chat,
               const GfIParam* __restrict__ ip, float* __restrict__ x_new,
               float* __restrict__ xbar, float* __restrict__ dlast, int advance,
               GfDState* st, const GfSched* sc, const double* normQ, const int32_t* cap,
               GfIParam* ip_next) {
  const ShortBlock B = short_block(runs, run_ptr, nruns);
  if (B.fast) {
    const GfIParam p = ip[B.R.inst];
    int2 c[kShortRpt];
    float2 v[kShortRpt];
    float xo[kShortRpt], ch[kShortRpt], ya[kShortRpt], yb[kShortRpt];
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      const int64_t off = B.off0 + u * 256, i = B.R.first + off, t = B.R.nnz0 + 2 * off;
      c[u] = *reinterpret_cast<const int2*>(Tr + t);
      v[u] = *reinterpret_cast<const float2*>(Tv + t);
      xo[u] = x_old[i];
      ch[u] = chat[i];
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      ya[u] = y[c[u].x];
      yb[u] = y[c[u].y];
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      CSum acc;
      acc.add(__fmul_rn(v[u].x, ya[u]));
      acc.add(__fmul_rn(v[u].y, yb[u]));
      const float delta = ch[u] + p.rho + acc.value() - 2.0f * p.rho * xo[u];
      float xn = xo[u] - p.tau1 * delta;
      xn = fminf(1.0f, fmaxf(0.0f, xn));
      const int64_t i = B.R.first + B.off0 + u * 256;
      x_new[i] = xn;
      xbar[i] = 2.0f * xn - xo[u];
      if (dlast) dlast[i] = p.tau1 * delta;
    }
  } else {
    ShortRow w[kShortRpt];
    short_rows(runs, run_ptr, nruns, ncols, Tp, w);
    int c0[kShortRpt], c1[kShortRpt];
    float v0[kShortRpt], v1[kShortRpt], xo[kShortRpt], ch[kShortRpt];
    float ya[kShortRpt], yb[kShortRpt];
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      c0[u] = w[u].n >= 1 ? Tr[w[u].t0] : 0;
      v0[u] = w[u].n >= 1 ? Tv[w[u].t0] : 0.f;
      c1[u] = w[u].n >= 2 ? Tr[w[u].t0 + 1] : 0;
      v1[u] = w[u].n >= 2 ? Tv[w[u].t0 + 1] : 0.f;
      xo[u] = w[u].n >= 0 ? x_old[w[u].id] : 0.f;
      ch[u] = w[u].n >= 0 ? chat[w[u].id] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      ya[u] = w[u].n >= 1 ? y[c0[u]] : 0.f;
      yb[u] = w[u].n >= 2 ? y[c1[u]] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kShortRpt; ++u) {
      if (w[u].n < 0) continue;
      CSum acc;
      if (w[u].n >= 1) acc.add(__fmul_rn(v0[u], ya[u]));
      if (w[u].n >= 2) acc.add(__fmul_rn(v1[u], yb[u]));
      const GfIParam p = ip[w[u].inst];
      const float delta = ch[u] + p.rho + acc.value() - 2.0f * p.rho * xo[u];
      float xn = xo[u] - p.tau1 * delta;
      xn = fminf(1.0f, fmaxf(0.0f, xn));
      x_new[w[u].id] = xn;
      xbar[w[u].id] = 2.0f * xn - xo[u];
      if (dlast) dlast[w[u].id] = p.tau1 * delta;
    }
  }
  if (advance && blockIdx.x == 0) advance_penalty(st, sc, normQ, cap, ip, ip_next);
}

// ---------------------------------------------------------------------------
// Primal step over a bucket of columns (K^T in CSC and, optionally, sparse
// symmetric Q rows), `LANES` threads per column, fused projection and
// extrapolation.  Block 0 of the kernel flagged `advance` also runs
// UpdatePenalty for the next iteration.
// ---------------------------------------------------------------------------
template <int LANES>
__global__ void __launch_bounds__(256)
k_primal_cols(const int32_t* __restrict__ cols, int32_t ncols,
              const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
              const float* __restrict__ Tv, const int64_t* __restrict__ Qp,
              const int32_t* __restrict__ Qc, const float* __restrict__ Qv,
              const float* __restrict__ y, const float* __restrict__ x_old,
              const float* __restrict__ chat, const int32_t* __restrict__ var_inst,
              const GfIParam* __restrict__ ip, float* __restrict__ x_new,
              float* __restrict__ xbar, float* __restrict__ dlast, int advance,
              GfDState* st, const GfSched* sc, const double* normQ,
              const int32_t* cap, GfIParam* ip_next) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t grp = gid / LANES;
  const int lane = (int)(gid % LANES);
  if (grp < ncols) {
    const int i = cols[grp];
    float xo = 0.f, ch = 0.f;               // loaded before the column's gathers
    if (lane == 0) {
      xo = x_old[i];
      ch = chat[i];
    }
    CSum acc;
    gf::gather_dot<4>(acc, Tr, Tv, y, Tp[i] + lane, Tp[i + 1], LANES);
    if (Qp) {
      for (int64_t t = Qp[i] + lane; t < Qp[i + 1]; t += LANES)
        acc.add(2.0f * __fmul_rn(Qv[t], x_old[Qc[t]]));
    }
    gf::csum_group_reduce<LANES>(acc);
    if (lane == 0) {
      const GfIParam q = ip[var_inst[i]];
      const float delta = ch + q.rho + acc.value() - 2.0f * q.rho * xo;
      float xn = xo - q.tau1 * delta;
      xn = fminf(1.0f, fmaxf(0.0f, xn));
      x_new[i] = xn;
      xbar[i] = 2.0f * xn - xo;
      if (dlast) dlast[i] = q.tau1 * delta;
    }
  }
  if (advance && blockIdx.x == 0) advance_penalty(st, sc, normQ, cap, ip, ip_next);
}

// Primal step over a bucket given as runs of consecutive columns (instance
// from the run; CSC range implicit for equal-length runs).  Same arithmetic
// as k_primal_cols.
template <int LANES>
__global__ void __launch_bounds__(256)
k_primal_runs(const GfRun* __restrict__ runs, const int64_t* __restrict__ run_ptr, int nruns,
              int64_t ncols, const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
              const float* __restrict__ Tv, const int64_t* __restrict__ Qp,
              const int32_t* __restrict__ Qc, const float* __restrict__ Qv,
              const float* __restrict__ y, const float* __restrict__ x_old,
              const float* __restrict__ chat, const GfIParam* __restrict__ ip,
              float* __restrict__ x_new, float* __restrict__ xbar, float* __restrict__ dlast,
              int advance, GfDState* st, const GfSched* sc, const double* normQ,
              const int32_t* cap, GfIParam* ip_next) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t grp = gid / LANES;
  const int lane = (int)(gid % LANES);
  if (grp < ncols) {
    const int q = nruns == 1 ? 0 : run_of(run_ptr, nruns, grp);
    const GfRun R = runs[q];
    const int64_t off = grp - __ldg(run_ptr + q);
    const int64_t i = R.first + off;
    const int64_t t0 = R.len >= 0 ? R.nnz0 + off * R.len : Tp[i];
    const int64_t t1 = R.len >= 0 ? t0 + R.len : Tp[i + 1];
    float xo = 0.f, ch = 0.f;               // loaded before the column's gathers
    if (lane == 0) {
      xo = x_old[i];
      ch = chat[i];
    }
    CSum acc;
    if (LANES == 1 && (R.len == 3 || R.len == 4)) {
      // one lane, three or four entries: every index and value load first,
      // then the gathers, then the adds in entry order (the loop's sum)
      int c[4];
      float v[4], g[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        c[e] = e < R.len ? Tr[t0 + e] : 0;
        v[e] = e < R.len ? Tv[t0 + e] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) g[e] = e < R.len ? y[c[e]] : 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < R.len) acc.add(__fmul_rn(v[e], g[e]));
    } else {
      gf::gather_dot<4>(acc, Tr, Tv, y, t0 + lane, t1, LANES);
    }
    if (Qp) {
      for (int64_t t = Qp[i] + lane; t < Qp[i + 1]; t += LANES)
        acc.add(2.0f * __fmul_rn(Qv[t], x_old[Qc[t]]));
    }
    gf::csum_group_reduce<LANES>(acc);
    if (lane == 0) {
      const GfIParam p = ip[R.inst];
      const float delta = ch + p.rho + acc.value() - 2.0f * p.rho * xo;
      float xn = xo - p.tau1 * delta;
      xn = fminf(1.0f, fmaxf(0.0f, xn));
      x_new[i] = xn;
      xbar[i] = 2.0f * xn - xo;
      if (dlast) dlast[i] = p.tau1 * delta;
    }
  }
  if (advance && blockIdx.x == 0) advance_penalty(st, sc, normQ, cap, ip, ip_next);
}

// ---------------------------------------------------------------------------
// Long rows / columns: partial compensated sums of fixed chunks, combined in
// chunk order by the finalising kernels (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_long_partial(const GfChunk* __restrict__ ch, int32_t nch,
               const int32_t* __restrict__ idx, const float* __restrict__ val,
               const float* __restrict__ vec, const int32_t* __restrict__ Qc,
               const float* __restrict__ Qv, const float* __restrict__ xq,
               float2* __restrict__ partial) {
  const int c = blockIdx.x;
  if (c >= nch) return;
  const GfChunk k = ch[c];
  if (k.part == 2) return;                     // a column slice computes this chunk
  CSum acc;
  if (k.part == 0) {
    // chunks of kChunkLen = 8 x 256 entries: all eight gathers in flight
    gf::gather_dot<8>(acc, idx, val, vec, k.t0 + threadIdx.x, k.t1, (int)blockDim.x);
  } else {
    for (int64_t t = k.t0 + threadIdx.x; t < k.t1; t += blockDim.x)
      acc.add(2.0f * __fmul_rn(Qv[t], xq[Qc[t]]));
  }
  gf::csum_group_reduce<32>(acc);
  __shared__ float ss[8], sc_[8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = acc.s; sc_[w] = acc.c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum tot;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot.merge(ss[q], sc_[q]);
    partial[c] = make_float2(tot.s, tot.c);
  }
}

// Long K^T columns in slices of 32 (sliced ELL): block (slice, chunk c),
// warp w takes entries e = e0 + w, e0 + w + 8, ... (four loads in flight),
// lane l column l; the warps' compensated sums are merged in warp order and
// written as the partial of chunk c of each column.
__global__ void __launch_bounds__(256)
k_long_slices(const int4* __restrict__ blk, const int64_t* __restrict__ off,
              const int32_t* __restrict__ len, const int32_t* __restrict__ pbase,
              const int32_t* __restrict__ sidx, const float* __restrict__ sval,
              const float* __restrict__ vec, float2* __restrict__ partial) {
  const int4 B = blk[blockIdx.x];
  const int sl = B.x, c = B.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t L = len[sl], base = off[sl];
  const int64_t e0 = (int64_t)c * kChunkLen, e1 = min(L, e0 + (int64_t)kChunkLen);
  CSum acc;
  for (int64_t e = e0 + warp; e < e1; e += 32) {
    int32_t r[4];
    float v[4], g[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t ee = e + 8 * u;
      r[u] = -1;
      v[u] = 0.0f;
      if (ee < e1) {
        r[u] = sidx[base + 32 * ee + lane];
        v[u] = sval[base + 32 * ee + lane];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) g[u] = r[u] >= 0 ? vec[r[u]] : 0.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (r[u] >= 0) acc.add(__fmul_rn(v[u], g[u]));
  }
  __shared__ float ss[8][32], sc_[8][32];
  ss[warp][lane] = acc.s;
  sc_[warp][lane] = acc.c;
  __syncthreads();
  if (warp == 0) {
    CSum tot;
    for (int q = 0; q < 8; ++q) tot.merge(ss[q][lane], sc_[q][lane]);
    const int pb = pbase[sl * 32 + lane];
    if (pb >= 0) partial[pb + c] = make_float2(tot.s, tot.c);
  }
}

__global__ void k_fill_slices(const int64_t* __restrict__ src, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ len, int32_t nslices,
                              const float* __restrict__ Tv, float* __restrict__ sval) {
  const int sl = blockIdx.y;
  if (sl >= nslices) return;
  const int64_t L = len[sl];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 32 * L;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(t & 31);
    const int64_t e = t >> 5;
    const int64_t s0 = src[sl * 32 + l];
    sval[off[sl] + t] = s0 >= 0 ? Tv[s0 + e] : 0.0f;
  }
}

__global__ void k_dual_long_final(const int32_t* __restrict__ ids,
                                  const int32_t* __restrict__ cptr, int32_t nlong,
                                  const float2* __restrict__ partial,
                                  const float* __restrict__ r,
                                  const uint8_t* __restrict__ row_eq,
                                  const int32_t* __restrict__ row_inst,
                                  const GfIParam* __restrict__ ip,
                                  float* __restrict__ y) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nlong) return;
  const int j = ids[q];
  CSum acc;
  for (int c = cptr[q]; c < cptr[q + 1]; ++c) acc.merge(partial[c].x, partial[c].y);
  const float tau2 = ip[row_inst[j]].tau2;
  float v = y[j] + tau2 * (acc.value() + r[j]);
  if (!row_eq[j] && v < 0.f) v = 0.f;
  y[j] = v;
}

__global__ void __launch_bounds__(256)
k_primal_long_final(const int32_t* __restrict__ ids, const int32_t* __restrict__ cptr,
                    int32_t nlong, const float2* __restrict__ partial,
                    const float* __restrict__ x_old, const float* __restrict__ chat,
                    const int32_t* __restrict__ var_inst,
                    const GfIParam* __restrict__ ip, float* __restrict__ x_new,
                    float* __restrict__ xbar, float* __restrict__ dlast, int advance,
                    GfDState* st, const GfSched* sc, const double* normQ,
                    const int32_t* cap, GfIParam* ip_next) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nlong) {
    const int i = ids[q];
    CSum acc;
    for (int c = cptr[q]; c < cptr[q + 1]; ++c) acc.merge(partial[c].x, partial[c].y);
    const GfIParam p = ip[var_inst[i]];
    const float xo = x_old[i];
    const float delta = chat[i] + p.rho + acc.value() - 2.0f * p.rho * xo;
    float xn = fminf(1.0f, fmaxf(0.0f, xo - p.tau1 * delta));
    x_new[i] = xn;
    xbar[i] = 2.0f * xn - xo;
    if (dlast) dlast[i] = p.tau1 * delta;
  }
  if (advance && blockIdx.x == 0) advance_penalty(st, sc, normQ, cap, ip, ip_next);
}

// ---------------------------------------------------------------------------
// Dense symmetric Q stored as W2 = offdiag(Q + Q^T) in bf16 (exact small
// integers) plus diag(Q_sym): (Q_hat x)_i = qscale (W2 x)_i + qdiag_i x_i.
// One warp per variable, x staged in shared memory, 16-byte bf16 loads,
// 8-term plain FP32 chunks folded into a compensated accumulator.  Also sums
// the column of K^T for the same variable, then applies the primal update.
// mode 0: primal update; mode 1: out[i] = (Q_hat x)_i only.
// ---------------------------------------------------------------------------
constexpr int kDenseWarps = 16;

__global__ void __launch_bounds__(kDenseWarps * 32)
k_dense_primal(const __nv_bfloat16* __restrict__ W2, int64_t ld, int64_t n,
               int64_t v0, const float* __restrict__ qdiag, float qscale,
               const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
               const float* __restrict__ Tv, const float* __restrict__ y,
               const float* __restrict__ x_old, const float* __restrict__ chat,
               const GfIParam* __restrict__ ip, int inst, float* __restrict__ x_new,
               float* __restrict__ xbar, float* __restrict__ dlast, int mode,
               float* __restrict__ out, int advance, GfDState* st,
               const GfSched* sc, const double* normQ, const int32_t* cap,
               GfIParam* ip_next) {
  extern __shared__ float4 xs4[];
  float* xs = reinterpret_cast<float*>(xs4);
  for (int64_t j = threadIdx.x; j < ld; j += blockDim.x)
    xs[j] = (j < n) ? x_old[v0 + j] : 0.0f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GfIParam q = ip[inst];
  for (int64_t i = (int64_t)blockIdx.x * kDenseWarps + warp; i < n;
       i += (int64_t)gridDim.x * kDenseWarps) {
    const uint4* row = reinterpret_cast<const uint4*>(W2 + i * ld);
    const int64_t n8 = ld / 8;                 // 16-byte words in the row
    CSum acc;
    // 8 independent 16-byte loads in flight per lane (memory-level
    // parallelism), then 8-term plain FP32 chunks into the compensated sum
    for (int64_t b8 = 0; b8 < n8; b8 += 8 * 32) {
      uint4 w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j8 = b8 + lane + 32 * u;
        w[u] = (j8 < n8) ? __ldg(row + j8) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j8 = b8 + lane + 32 * u;
        if (j8 >= n8) break;
        const float4 xa = xs4[2 * j8], xb = xs4[2 * j8 + 1];
        const __nv_bfloat162* wp = reinterpret_cast<const __nv_bfloat162*>(&w[u]);
        const float2 w0 = __bfloat1622float2(wp[0]), w1 = __bfloat1622float2(wp[1]);
        const float2 w2 = __bfloat1622float2(wp[2]), w3 = __bfloat1622float2(wp[3]);
        float part = w0.x * xa.x;
        part = fmaf(w0.y, xa.y, part);
        part = fmaf(w1.x, xa.z, part);
        part = fmaf(w1.y, xa.w, part);
        part = fmaf(w2.x, xb.x, part);
        part = fmaf(w2.y, xb.y, part);
        part = fmaf(w3.x, xb.z, part);
        part = fmaf(w3.y, xb.w, part);
        acc.add(part);
      }
    }
    // K^T column of this variable, folded in at the 1/(2 qscale) scale so a
    // single compensated sum carries 2 (Q_hat x)_i + (K^T y)_i below.
    gf::csum_group_reduce<32>(acc);
    CSum g;
    if (Tp) {
      for (int64_t t = Tp[v0 + i] + lane; t < Tp[v0 + i + 1]; t += 32)
        g.add(__fmul_rn(Tv[t], y[Tr[t]]));
      gf::csum_group_reduce<32>(g);
    }
    if (lane == 0) {
      const float xo = xs[i];
      CSum s;                              // 2 (Q_hat x)_i + (K^T y)_i
      s.merge(__fmul_rn(2.0f * qscale, acc.s), __fmul_rn(2.0f * qscale, acc.c));
      s.add(__fmul_rn(2.0f * qdiag[i], xo));
      s.merge(g.s, g.c);
      if (mode == 1) {
        out[i] = 0.5f * s.value();
      } else {
        const float delta = chat[v0 + i] + q.rho + s.value() - 2.0f * q.rho * xo;
        float xn = fminf(1.0f, fmaxf(0.0f, xo - q.tau1 * delta));
        x_new[v0 + i] = xn;
        xbar[v0 + i] = 2.0f * xn - xo;
        if (dlast) dlast[v0 + i] = q.tau1 * delta;
      }
    }
  }
  if (advance && blockIdx.x == 0) {
    __syncthreads();
    advance_penalty(st, sc, normQ, cap, ip, ip_next);
  }
}

// Same step with W2 stored as int8 (exact when max|W2| <= 127): 16 entries
// per 16-byte load, one 1024-thread block per SM, each block a contiguous
// range of rows, eight loads in flight per lane, 8-term plain chunks folded
// into the compensated sum.
constexpr int kI8Warps = 32;

__global__ void __launch_bounds__(kI8Warps * 32, 1)
k_dense_primal_i8(const uint8_t* __restrict__ W2, int64_t ld, int64_t n, int64_t v0,
                  const float* __restrict__ qdiag, float qscale,
                  const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
                  const float* __restrict__ Tv, const float* __restrict__ y,
                  const float* __restrict__ x_old, const float* __restrict__ chat,
                  const GfIParam* __restrict__ ip, int inst, float* __restrict__ x_new,
                  float* __restrict__ xbar, float* __restrict__ dlast, int mode,
                  float* __restrict__ out, int advance, GfDState* st, const GfSched* sc,
                  const double* normQ, const int32_t* cap, GfIParam* ip_next) {
  extern __shared__ float4 xs4[];
  float* xs = reinterpret_cast<float*>(xs4);
  for (int64_t j = threadIdx.x; j < ld; j += blockDim.x) xs[j] = (j < n) ? x_old[v0 + j] : 0.0f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const GfIParam q = ip[inst];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  const int64_t nq = ld / 4;                  // 4-entry words per row
  for (int64_t i = r0 + warp; i < r1; i += kI8Warps) {
    CSum acc = gf::i8_row_dot(reinterpret_cast<const uint32_t*>(W2 + i * ld), xs4, nq, lane);
    gf::csum_group_reduce<32>(acc);
    CSum g;
    if (Tp) {
      for (int64_t t = Tp[v0 + i] + lane; t < Tp[v0 + i + 1]; t += 32)
        g.add(__fmul_rn(Tv[t], y[Tr[t]]));
      gf::csum_group_reduce<32>(g);
    }
    if (lane == 0) {
      const float xo = xs[i];
      CSum s;                              // 2 (Q_hat x)_i + (K^T y)_i
      s.merge(__fmul_rn(2.0f * qscale, acc.s), __fmul_rn(2.0f * qscale, acc.c));
      s.add(__fmul_rn(2.0f * qdiag[i], xo));
      s.merge(g.s, g.c);
      if (mode == 1) {
        out[i] = 0.5f * s.value();
      } else {
        const float delta = chat[v0 + i] + q.rho + s.value() - 2.0f * q.rho * xo;
        float xn = fminf(1.0f, fmaxf(0.0f, xo - q.tau1 * delta));
        x_new[v0 + i] = xn;
        xbar[v0 + i] = 2.0f * xn - xo;
        if (dlast) dlast[v0 + i] = q.tau1 * delta;
      }
    }
  }
  if (advance && blockIdx.x == 0) {
    __syncthreads();
    advance_penalty(st, sc, normQ, cap, ip, ip_next);
  }
}

template <int L>
cudaError_t launch_dual(GfCtx* h, const GfBucket& b, const GfIParam* ip, float* y) {
  int64_t threads = (int64_t)b.count * L;
  int blocks = (int)((threads + 255) / 256);
  if (L == 1 && b.runs && b.short_ok) {
    k_dual_short<<<(unsigned)((b.count + 256 * kShortRpt - 1) / (256 * kShortRpt)), 256, 0,
                   h->stream>>>(b.runs, b.run_ptr, b.nruns, b.count, h->Kp, h->Kc, h->Kv,
                                h->xbar, h->rhat, h->row_eq, ip, y);
  } else if (b.runs)
    k_dual_runs<L><<<blocks, 256, 0, h->stream>>>(b.runs, b.run_ptr, b.nruns, b.count, h->Kp,
                                                  h->Kc, h->Kv, h->xbar, h->rhat, h->row_eq,
                                                  ip, y);
  else
    k_dual_rows<L><<<blocks, 256, 0, h->stream>>>(b.ids, b.count, h->Kp, h->Kc, h->Kv,
                                                  h->xbar, h->rhat, h->row_eq, h->row_inst,
                                                  ip, y);
  h->launches++;
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_primal(GfCtx* h, const GfBucket& b, const GfIParam* ip,
                          const float* xo, float* xn, float* xbar, float* dlast, int adv,
                          GfIParam* ipn) {
  int64_t threads = (int64_t)b.count * L;
  int blocks = (int)((threads + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (L == 1 && b.runs && b.short_ok && !h->nnzQ) {
    const unsigned sb = (unsigned)std::max<int64_t>(
        1, (b.count + 256 * kShortRpt - 1) / (256 * kShortRpt));
    k_primal_short<<<sb, 256, 0, h->stream>>>(
        b.runs, b.run_ptr, b.nruns, b.count, h->Tp, h->Tr, h->Tv, h->y, xo, h->chat, ip, xn,
        xbar, dlast, adv, h->dstate, h->sched_d, h->normQhat_d, h->cap_d, ipn);
  } else if (b.runs)
    k_primal_runs<L><<<blocks, 256, 0, h->stream>>>(
        b.runs, b.run_ptr, b.nruns, b.count, h->Tp, h->Tr, h->Tv, h->nnzQ ? h->Qp : nullptr,
        h->Qc, h->Qv, h->y, xo, h->chat, ip, xn, xbar, dlast, adv, h->dstate, h->sched_d,
        h->normQhat_d, h->cap_d, ipn);
  else
    k_primal_cols<L><<<blocks, 256, 0, h->stream>>>(
        b.ids, b.count, h->Tp, h->Tr, h->Tv, h->nnzQ ? h->Qp : nullptr, h->Qc, h->Qv, h->y,
        xo, h->chat, h->var_inst, ip, xn, xbar, dlast, adv, h->dstate, h->sched_d,
        h->normQhat_d, h->cap_d, ipn);
  h->launches++;
  return cudaGetLastError();
}

// Bucket kernels with `lanes` threads per row / column (1, 2, 4, 8, 16, 32).
cudaError_t dual_bucket(GfCtx* h, const GfBucket& b, int lanes, const GfIParam* ip,
                        float* y) {
  switch (lanes) {
    case 1: return launch_dual<1>(h, b, ip, y);
    case 2: return launch_dual<2>(h, b, ip, y);
    case 4: return launch_dual<4>(h, b, ip, y);
    case 8: return launch_dual<8>(h, b, ip, y);
    case 16: return launch_dual<16>(h, b, ip, y);
    default: return launch_dual<32>(h, b, ip, y);
  }
}
cudaError_t primal_bucket(GfCtx* h, const GfBucket& b, int lanes, const GfIParam* ip,
                          const float* xo, float* xn, float* xbar, float* dlast, int adv,
                          GfIParam* ipn) {
  switch (lanes) {
    case 1: return launch_primal<1>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
    case 2: return launch_primal<2>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
    case 4: return launch_primal<4>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
    case 8: return launch_primal<8>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
    case 16: return launch_primal<16>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
    default: return launch_primal<32>(h, b, ip, xo, xn, xbar, dlast, adv, ipn);
  }
}

}  // namespace

static void dense_smem_attr(size_t smem) {
  static size_t done = 48 * 1024;
  if (smem > done) {
    cudaFuncSetAttribute(k_dense_primal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_dense_primal_i8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    done = smem;
  }
}

cudaError_t gf_launch_dense_gemv_q(GfCtx* h, const GfDenseQ& dq, const float* x,
                                   float* out) {
  size_t smem = sizeof(float) * (size_t)dq.ld;
  dense_smem_attr(smem);
  if (dq.W2i8) {
    const int blocks = (int)std::min<int64_t>(h->num_sms, (dq.n + 7) / 8);
    k_dense_primal_i8<<<blocks, kI8Warps * 32, smem, h->stream>>>(
        dq.W2i8, dq.ld, dq.n, h->ih[dq.inst].var_off, dq.qdiag, dq.qscale, nullptr, nullptr,
        nullptr, nullptr, x, h->chat, h->iprm, dq.inst, nullptr, nullptr, nullptr, 1, out, 0,
        nullptr, nullptr, nullptr, nullptr, nullptr);
    h->launches++;
    return cudaGetLastError();
  }
  int blocks = (int)std::min<int64_t>((dq.n + kDenseWarps - 1) / kDenseWarps, 296);
  k_dense_primal<<<blocks, kDenseWarps * 32, smem, h->stream>>>(
      dq.W2, dq.ld, dq.n, h->ih[dq.inst].var_off, dq.qdiag, dq.qscale, nullptr, nullptr,
      nullptr, nullptr, x, h->chat, h->iprm, dq.inst, nullptr, nullptr, nullptr, 1, out,
      0, nullptr, nullptr, nullptr, nullptr, nullptr);
  h->launches++;
  return cudaGetLastError();
}

// One PDHG iteration for every instance: dual buckets, long-row chunks,
// primal buckets, long-column chunks, dense-Q instances.  x_{k-1} is read
// from x[1-parity... ] -- iteration it = k+1 reads x[(it-1)&1], writes x[it&1].
cudaError_t gf_single_iter(GfCtx* h, int p);

cudaError_t gf_launch_pdhg_iter(GfCtx* h, int parity) {
  if (h->single_ok) return gf_single_iter(h, parity);
  const GfIParam* ip = h->iprm + (size_t)parity * h->ninst;
  GfIParam* ipn = h->iprm + (size_t)(1 - parity) * h->ninst;
  const float* xo = h->x[1 - parity];
  float* xn = h->x[parity];
  float* dl = h->light_iter ? nullptr : h->dlast;   // tau1 delta: full iterations only
  cudaError_t e;
  // ---- dual
  for (const GfBucket& b : h->rb) {
    if (!b.count) continue;
    if ((e = dual_bucket(h, b, b.lanes, ip, h->y)) != cudaSuccess) return e;
  }
  if (h->rlong.nlong) {
    k_long_partial<<<h->rlong.nchunks, 256, 0, h->stream>>>(
        h->rlong.chunks, h->rlong.nchunks, h->Kc, h->Kv, h->xbar, nullptr, nullptr,
        nullptr, h->rlong.partial);
    k_dual_long_final<<<(h->rlong.nlong + 127) / 128, 128, 0, h->stream>>>(
        h->rlong.ids, h->rlong.chunk_ptr, h->rlong.nlong, h->rlong.partial, h->rhat,
        h->row_eq, h->row_inst, ip, h->y);
    h->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // ---- primal (first launch advances the penalty state)
  int adv = 1;
  for (const GfDenseQ& dq : h->dense) {
    size_t smem = sizeof(float) * (size_t)dq.ld;
    dense_smem_attr(smem);
    const GfInstHost& I = h->ih[dq.inst];
    const bool hasK = (I.m1 + I.m2) > 0;
    if (dq.W2i8) {
      const int blocks = (int)std::min<int64_t>(h->num_sms, (dq.n + 7) / 8);
      k_dense_primal_i8<<<blocks, kI8Warps * 32, smem, h->stream>>>(
          dq.W2i8, dq.ld, dq.n, I.var_off, dq.qdiag, dq.qscale, hasK ? h->Tp : nullptr, h->Tr,
          h->Tv, h->y, xo, h->chat, ip, dq.inst, xn, h->xbar, dl, 0, nullptr, adv,
          h->dstate, h->sched_d, h->normQhat_d, h->cap_d, ipn);
      h->launches++;
      adv = 0;
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      continue;
    }
    int blocks = (int)std::min<int64_t>((dq.n + kDenseWarps - 1) / kDenseWarps, 296);
    k_dense_primal<<<blocks, kDenseWarps * 32, smem, h->stream>>>(
        dq.W2, dq.ld, dq.n, I.var_off, dq.qdiag, dq.qscale, hasK ? h->Tp : nullptr, h->Tr,
        h->Tv, h->y, xo, h->chat, ip, dq.inst, xn, h->xbar, dl, 0, nullptr, adv,
        h->dstate, h->sched_d, h->normQhat_d, h->cap_d, ipn);
    h->launches++;
    adv = 0;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (const GfBucket& b : h->cb) {
    if (!b.count) continue;
    e = primal_bucket(h, b, b.lanes, ip, xo, xn, h->xbar, dl, adv, ipn);
    adv = 0;
    if (e != cudaSuccess) return e;
  }
  if (h->clong.nlong) {
    if (h->csl.nblocks) {
      k_long_slices<<<h->csl.nblocks, 256, 0, h->stream>>>(
          h->csl.blk, h->csl.off, h->csl.len, h->csl.pbase, h->csl.sidx, h->csl.sval, h->y,
          h->clong.partial);
      h->launches++;
    }
    k_long_partial<<<h->clong.nchunks, 256, 0, h->stream>>>(
        h->clong.chunks, h->clong.nchunks, h->Tr, h->Tv, h->y, h->Qc, h->Qv, xo,
        h->clong.partial);
    k_primal_long_final<<<(h->clong.nlong + 255) / 256, 256, 0, h->stream>>>(
        h->clong.ids, h->clong.chunk_ptr, h->clong.nlong, h->clong.partial, xo, h->chat,
        h->var_inst, ip, xn, h->xbar, dl, adv, h->dstate, h->sched_d, h->normQhat_d,
        h->cap_d, ipn);
    h->launches += 2;
    adv = 0;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Autotuner of the bucket kernels: every (row or column) length bucket is run
// with 1, 2, 4, 8, 16 and 32 lanes per row / column on scratch outputs (the
// solver state is untouched) and the fastest lane count is kept.  The lane
// count changes only the FP32 summation order within a row / column.
// ---------------------------------------------------------------------------
// Best of 5 measurements of `inner` back-to-back launches (small kernels are
// timed in batches so that event resolution and launch jitter do not decide).
static float time_launches(GfCtx* h, const std::function<cudaError_t()>& f, cudaError_t* err) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  *err = f();                                    // warm-up
  int inner = 1;
  {
    // batch size: enough launches for ~200 us per measurement (at most 64)
    cudaEventRecord(a, h->stream);
    if (*err == cudaSuccess) *err = f();
    cudaEventRecord(b, h->stream);
    float ms = 0.f;
    if (*err == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess)
      cudaEventElapsedTime(&ms, a, b);
    if (ms > 0.f) inner = std::max(1, std::min(64, (int)(0.2f / ms)));
  }
  for (int rep = 0; rep < 5 && *err == cudaSuccess; ++rep) {
    cudaEventRecord(a, h->stream);
    for (int u = 0; u < inner && *err == cudaSuccess; ++u) *err = f();
    cudaEventRecord(b, h->stream);
    if (*err == cudaSuccess) *err = cudaEventSynchronize(b);
    float ms = 0.f;
    if (*err == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms / inner);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

cudaError_t gf_tune_lanes(GfCtx* h, int32_t lanes_out[10]) {
  static const int cand[6] = {1, 2, 4, 8, 16, 32};
  cudaError_t e = cudaSuccess;
  float* ys = gf_alloc_t<float>(h, std::max<int64_t>(1, h->M));
  float* xs = gf_alloc_t<float>(h, std::max<int64_t>(1, h->N));
  float* xb = gf_alloc_t<float>(h, std::max<int64_t>(1, h->N));
  if (!ys || !xs || !xb) {
    gf_free_one(h, ys); gf_free_one(h, xs); gf_free_one(h, xb);
    return cudaErrorMemoryAllocation;
  }
  if (h->M) e = cudaMemcpyAsync(ys, h->y, sizeof(float) * h->M, cudaMemcpyDeviceToDevice,
                                h->stream);
  const int p = (int)((h->k_host + 1) & 1);
  const GfIParam* ip = h->iprm + (size_t)p * h->ninst;
  const float* xo = h->x[1 - p];
  const long long saved = h->launches;
  // rows of bucket k are at most this long (bucket bounds of the loader)
  static const int64_t maxlen[5] = {2, 8, 32, 128, kLongLen};
  for (int side = 0; side < 2 && e == cudaSuccess; ++side) {
    std::vector<GfBucket>& bs = side ? h->cb : h->rb;
    for (size_t k = 0; k < bs.size() && e == cudaSuccess; ++k) {
      GfBucket& b = bs[k];
      if (!b.count) continue;
      // candidates in ascending lane count; a wider choice must beat the
      // best narrower one by 3% (timings of L2-resident buckets are close,
      // and the narrow form keeps more rows in flight when data are cold)
      float best = 1e30f;
      int pick = b.lanes;
      for (int c : cand) {
        if (c > maxlen[std::min<size_t>(k, 4)]) continue;
        float ms = time_launches(h, [&]() {
          return side ? primal_bucket(h, b, c, ip, xo, xs, xb, nullptr, 0, nullptr)
                      : dual_bucket(h, b, c, ip, ys);
        }, &e);
        if (e != cudaSuccess) break;
        if (ms < 0.97f * best) { best = ms; pick = c; }
      }
      b.lanes = pick;
    }
  }
  h->launches = saved;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  gf_free_one(h, ys);
  gf_free_one(h, xs);
  gf_free_one(h, xb);
  for (int k = 0; k < 5; ++k) {
    lanes_out[k] = k < (int)h->rb.size() ? h->rb[k].lanes : 0;
    lanes_out[5 + k] = k < (int)h->cb.size() ? h->cb[k].lanes : 0;
  }
  return e;
}

// Scaled values of the column slices from the CSC arrays (at load).
cudaError_t gf_fill_slices(GfCtx* h, const int64_t* src_d) {
  const dim3 grid(256, (unsigned)h->csl.nslices);
  k_fill_slices<<<grid, 256, 0, h->stream>>>(src_d, h->csl.off, h->csl.len, h->csl.nslices,
                                             h->Tv, h->csl.sval);
  return cudaGetLastError();
}
