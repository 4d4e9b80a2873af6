// k_small.cu -- PDHG iterations (Alg. 2) of instances small enough to keep
// their whole scaled matrix in one block's shared memory (set-cover-sized
// problems, alone or as large batches).
//
// One block per instance runs every iteration of a gfors_pdhg_steps call with
// block barriers only: K (CSR, for the dual step) and K^T (CSC, for the primal
// step) with 16-bit local indices, x, xbar, c_hat, y and r_hat stay in shared
// memory; global memory is read once at the start and written once at the
// end.  Rows whose coefficients are all equal (every row of a set-cover or
// assignment matrix) keep one value per row instead of one per nonzero.
// The penalty schedule advances inside every block from the same FP64 state.
// Arithmetic: 4-term plain FP32 chunks folded into compensated sums (8
// lanes per row, a thread per column), then the projected updates of Alg. 2.
#include <algorithm>

#include <cooperative_groups.h>

#include "internal.cuh"
#include "penalty.cuh"

struct GfSmallInst {                // one instance of the small-instance path
  int64_t v0, r0;                   // first variable / row (global ids)
  int64_t k0, t0;                   // first nonzero of its K rows / K^T columns
  int32_t n, m, nnz, uniform;       // uniform: every row has one value
};

namespace {

using gf::CSum;
constexpr int kThreads = 1024;
constexpr int kSchedThread = kThreads - 1;
constexpr int kRowLanes = 8;                    // lanes per row in the dual step

GF_DEV size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// The projected updates of Alg. 2 with every rounding explicit (nothing
// left to the compiler's contraction choices), shared by the one-block and
// the cluster kernels so that both give identical iterates.
GF_DEV float dual_update(float y, float tau2, float kx, float r, bool eq) {
  float v = __fadd_rn(y, __fmul_rn(tau2, __fadd_rn(kx, r)));
  if (!eq && v < 0.f) v = 0.f;
  return v;
}
GF_DEV float primal_delta(float c, float rho, float kty, float xi) {
  return __fsub_rn(__fadd_rn(__fadd_rn(c, rho), kty), __fmul_rn(__fmul_rn(2.0f, rho), xi));
}
GF_DEV float primal_x(float xi, float tau1, float delta) {
  return fminf(1.0f, fmaxf(0.0f, __fsub_rn(xi, __fmul_rn(tau1, delta))));
}

__global__ void __launch_bounds__(kThreads, 1)
k_pdhg_small(const GfSmallInst* __restrict__ insts, const int64_t* __restrict__ Kp,
             const int32_t* __restrict__ Kc, const float* __restrict__ Kv,
             const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
             const float* __restrict__ Tv, const uint16_t* __restrict__ perm_g,
             const float* __restrict__ rhat,
             const uint8_t* __restrict__ row_eq, const float* __restrict__ chat, float* x0,
             float* x1, float* __restrict__ xbar_g, float* __restrict__ y_g,
             float* __restrict__ dlast, GfIParam* iprm, int ninst,
             const long long* __restrict__ k0_snap, long long nsteps, GfDState* st,
             const GfSched* sc, const double* normQ, const int32_t* cap) {
  extern __shared__ __align__(16) uint8_t sm[];
  const int b = blockIdx.x;
  const GfSmallInst I = insts[b];
  const int n = I.n, m = I.m, nnz = I.nnz;
  // ---- shared-memory layout (4-byte arrays first)
  size_t off = 0;
  auto take = [&](size_t bytes) { uint8_t* p = sm + off; off = align16(off + bytes); return p; };
  int32_t* rp = reinterpret_cast<int32_t*>(take(4 * (size_t)(m + 1)));
  int32_t* cp = reinterpret_cast<int32_t*>(take(4 * (size_t)(n + 1)));
  float* xs0 = reinterpret_cast<float*>(take(4 * (size_t)n));
  float* xs1 = reinterpret_cast<float*>(take(4 * (size_t)n));
  float* xb = reinterpret_cast<float*>(take(4 * (size_t)n));
  float* cs = reinterpret_cast<float*>(take(4 * (size_t)n));
  float* ys = reinterpret_cast<float*>(take(4 * (size_t)m));
  float* rs = reinterpret_cast<float*>(take(4 * (size_t)m));
  float* rowval = reinterpret_cast<float*>(take(I.uniform ? 4 * (size_t)m : 0));
  float* kval = reinterpret_cast<float*>(take(I.uniform ? 0 : 4 * (size_t)nnz));
  float* tval = reinterpret_cast<float*>(take(I.uniform ? 0 : 4 * (size_t)nnz));
  uint16_t* kcol = reinterpret_cast<uint16_t*>(take(2 * (size_t)nnz));
  uint16_t* trow = reinterpret_cast<uint16_t*>(take(2 * (size_t)nnz));
  uint16_t* perm = reinterpret_cast<uint16_t*>(take(2 * (size_t)n));   // columns by length
  uint8_t* eq = take((size_t)m);
  __shared__ GfIParam qsm[2];
  __shared__ double rho_s;
  __shared__ int n_rho_s;
  // ---- stage the instance
  // iterations completed before this launch, from the device state as
  // snapshotted just before it (st->k itself is rewritten by block 0 at the
  // end, possibly before later blocks start), so a captured launch replays
  // with the current counter
  const long long it0 = *k0_snap + 1;
  const float* xo_g = (it0 & 1) ? x0 : x1;        // x_{k0} in x[k0 & 1]
  for (int j = threadIdx.x; j <= m; j += kThreads) rp[j] = (int32_t)(Kp[I.r0 + j] - I.k0);
  for (int i = threadIdx.x; i <= n; i += kThreads) cp[i] = (int32_t)(Tp[I.v0 + i] - I.t0);
  for (int i = threadIdx.x; i < n; i += kThreads) perm[i] = perm_g[I.v0 + i];
  for (int t = threadIdx.x; t < nnz; t += kThreads) {
    kcol[t] = (uint16_t)(Kc[I.k0 + t] - I.v0);
    trow[t] = (uint16_t)(Tr[I.t0 + t] - I.r0);
    if (!I.uniform) {
      kval[t] = Kv[I.k0 + t];
      tval[t] = Tv[I.t0 + t];
    }
  }
  for (int i = threadIdx.x; i < n; i += kThreads) {
    xs0[i] = xo_g[I.v0 + i];
    xb[i] = xbar_g[I.v0 + i];
    cs[i] = chat[I.v0 + i];
  }
  for (int j = threadIdx.x; j < m; j += kThreads) {
    ys[j] = y_g[I.r0 + j];
    rs[j] = rhat[I.r0 + j];
    eq[j] = row_eq[I.r0 + j];
  }
  if (threadIdx.x == kSchedThread) {
    n_rho_s = st->n_rho;
    rho_s = st->rho;
    qsm[0] = iprm[(size_t)(it0 & 1) * ninst + b];
  }
  __syncthreads();
  if (I.uniform)
    for (int j = threadIdx.x; j < m; j += kThreads)
      rowval[j] = rp[j + 1] > rp[j] ? Kv[I.k0 + rp[j]] : 0.0f;
  __syncthreads();
  long long s = 0;
  for (; s < nsteps; ++s) {
    const long long it = it0 + s;
    const GfIParam q = qsm[s & 1];
    float* xo = (s & 1) ? xs1 : xs0;                  // x_{it-1}
    float* xn = (s & 1) ? xs0 : xs1;                  // x_it
    // dual step: y <- Pi(y + tau2 (K xbar + r)), 8 lanes per row; each lane
    // sums chunks of 4 products in plain FP32 folded into a compensated sum
    for (int j = threadIdx.x / kRowLanes; j < m; j += kThreads / kRowLanes) {
      const int sl = threadIdx.x % kRowLanes;
      CSum acc;
      const float rv = I.uniform ? rowval[j] : 0.0f;
      const int te = rp[j + 1];
      for (int t = rp[j] + sl; t < te; t += 4 * kRowLanes) {
        float part = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int tt = t + u * kRowLanes;
          if (tt < te) part = __fadd_rn(part, __fmul_rn(I.uniform ? rv : kval[tt], xb[kcol[tt]]));
        }
        acc.add(part);
      }
      gf::csum_group_reduce<kRowLanes>(acc);
      if (sl == 0) ys[j] = dual_update(ys[j], q.tau2, acc.value(), rs[j], eq[j] != 0);
    }
    __syncthreads();
    // primal step: a thread per column, chunks of 4 products; columns are
    // taken in order of decreasing length, so the 32 columns of a warp have
    // nearly equal lengths and few lanes idle in the chunk loop
    const bool last = (s + 1 == nsteps);
    for (int ii = threadIdx.x; ii < n; ii += kThreads) {
      const int i = perm[ii];
      CSum acc;
      const int te = cp[i + 1];
      for (int t = cp[i]; t < te; t += 4) {
        float part = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t + u < te) {
            const int j = trow[t + u];
            part = __fadd_rn(part, __fmul_rn(I.uniform ? rowval[j] : tval[t + u], ys[j]));
          }
        }
        acc.add(part);
      }
      const float xi = xo[i];
      const float delta = primal_delta(cs[i], q.rho, acc.value(), xi);
      const float xv = primal_x(xi, q.tau1, delta);
      xn[i] = xv;
      xb[i] = __fsub_rn(__fmul_rn(2.0f, xv), xi);
      if (last && dlast) dlast[I.v0 + i] = __fmul_rn(q.tau1, delta);
    }
    if (threadIdx.x == kSchedThread) {
      // UpdatePenalty for iteration it+1 (counter advances once per k_int)
      const int n_next = (int)(it / sc->k_int);
      if (n_rho_s < n_next) {
        int n_rho = n_rho_s;
        double rho = rho_s;
        while (n_rho < n_next) {
          n_rho += 1;
          double rt = sc->rho_min * pow(1.0 + (double)n_rho / sc->T, sc->p);
          double lo = rho + sc->delta;
          double v = rt < lo ? lo : rt;
          rho = v > sc->rho_max ? sc->rho_max : v;
        }
        n_rho_s = n_rho;
        rho_s = rho;
        qsm[(s + 1) & 1] = step_params(sc->sigma, normQ[b], cap[b], rho);
      } else {
        qsm[(s + 1) & 1] = q;
      }
    }
    __syncthreads();
  }
  // ---- write back: x_last in x[last & 1], x_{last-1} in the other buffer
  if (s > 0) {
    const long long lastit = it0 + s - 1;
    float* xl_g = (lastit & 1) ? x1 : x0;
    float* xp_g = (lastit & 1) ? x0 : x1;
    const float* xl = ((s - 1) & 1) ? xs0 : xs1;
    const float* xp = ((s - 1) & 1) ? xs1 : xs0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      xl_g[I.v0 + i] = xl[i];
      xp_g[I.v0 + i] = xp[i];
      xbar_g[I.v0 + i] = xb[i];
    }
    for (int j = threadIdx.x; j < m; j += kThreads) y_g[I.r0 + j] = ys[j];
    if (threadIdx.x == kSchedThread) {
      iprm[(size_t)(lastit & 1) * ninst + b] = qsm[(s - 1) & 1];
      iprm[(size_t)((lastit + 1) & 1) * ninst + b] = qsm[s & 1];
      if (b == 0) {
        st->k = lastit;
        st->n_rho = n_rho_s;
        st->rho = rho_s;
      }
    }
  }
}

size_t small_smem(int64_t n, int64_t m, int64_t nnz, bool uniform) {
  auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
  size_t b = a16(4 * (m + 1)) + a16(4 * (n + 1)) + 4 * a16(4 * n) + 2 * a16(4 * m);
  b += uniform ? a16(4 * m) : 2 * a16(4 * nnz);
  b += 2 * a16(2 * nnz) + a16(2 * n) + a16(m);
  return b;
}

__global__ void k_snap_k(const GfDState* st, long long* snap) { *snap = st->k; }

// ---------------------------------------------------------------------------
// One instance per thread-block cluster of C CTAs (C = 16, or 8 where the
// device does not allow 16).  CTA q of the cluster owns rows [m q / C,
// m (q+1) / C) and the columns at positions [n q / C, n (q+1) / C) of the
// instance's length-sorted column order; every CTA keeps a full copy of
// y and of xbar, the latter stored in that column order, so every CTA's
// share of both is one contiguous slice.  An iteration: the dual step over
// the CTA's rows, then the whole block copies its slice of y into every
// other CTA of the cluster (distributed shared memory, coalesced stores),
// cluster barrier; the primal step over its columns, the slice of xbar
// likewise, cluster barrier.  (Every CTA running the dual step over all
// rows instead, with one barrier per iteration, measured slower: 6.6
// against 5.2 us per set-cover iteration.)  The row and column sums are
// those of k_pdhg_small (same lanes, chunks and compensated adds) and the
// updates share its explicitly rounded arithmetic, so the iterates equal
// the one-block kernel's.
namespace cg = cooperative_groups;

__global__ void __launch_bounds__(kThreads, 1)
k_pdhg_cluster(const GfSmallInst* __restrict__ insts, const int64_t* __restrict__ Kp,
               const int32_t* __restrict__ Kc, const float* __restrict__ Kv,
               const int64_t* __restrict__ Tp, const int32_t* __restrict__ Tr,
               const float* __restrict__ Tv, const uint16_t* __restrict__ perm_g,
               const float* __restrict__ rhat, const uint8_t* __restrict__ row_eq,
               const float* __restrict__ chat, float* x0, float* x1,
               float* __restrict__ xbar_g, float* __restrict__ y_g, float* __restrict__ dlast,
               GfIParam* iprm, int ninst, const long long* __restrict__ k0_snap,
               long long nsteps, GfDState* st, const GfSched* sc, const double* normQ,
               const int32_t* cap) {
  extern __shared__ __align__(16) uint8_t sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int b = (int)(blockIdx.x / C);
  const GfSmallInst I = insts[b];
  const int n = I.n, m = I.m;
  const int j0 = (int)((int64_t)m * q / C), j1 = (int)((int64_t)m * (q + 1) / C);
  const int p0 = (int)((int64_t)n * q / C), p1 = (int)((int64_t)n * (q + 1) / C);
  const int mr = j1 - j0, nc = p1 - p0;
  const int64_t rk0 = Kp[I.r0 + j0];                     // first nonzero of my rows
  const int nzr = (int)(Kp[I.r0 + j1] - rk0);
  // my columns' nonzero count
  __shared__ int nzc_s;
  if (threadIdx.x == 0) nzc_s = 0;
  __syncthreads();
  {
    int c = 0;
    for (int t = threadIdx.x; t < nc; t += kThreads) {
      const int i = perm_g[I.v0 + p0 + t];
      c += (int)(Tp[I.v0 + i + 1] - Tp[I.v0 + i]);
    }
    atomicAdd(&nzc_s, c);
  }
  __syncthreads();
  const int nzc = nzc_s;
  size_t off = 0;
  auto take = [&](size_t bytes) { uint8_t* p = sm + off; off = align16(off + bytes); return p; };
  float* xb = reinterpret_cast<float*>(take(4 * (size_t)n));          // replicated, by position
  float* ys = reinterpret_cast<float*>(take(4 * (size_t)m));          // replicated
  float* rowval = reinterpret_cast<float*>(take(I.uniform ? 4 * (size_t)m : 0));
  int32_t* rp = reinterpret_cast<int32_t*>(take(4 * (size_t)(mr + 1)));
  float* rs = reinterpret_cast<float*>(take(4 * (size_t)mr));
  float* kval = reinterpret_cast<float*>(take(I.uniform ? 0 : 4 * (size_t)nzr));
  uint16_t* kcol = reinterpret_cast<uint16_t*>(take(2 * (size_t)nzr));
  uint8_t* eq = take((size_t)mr);
  int32_t* cp = reinterpret_cast<int32_t*>(take(4 * (size_t)(nc + 1)));
  uint16_t* ci = reinterpret_cast<uint16_t*>(take(2 * (size_t)nc));
  float* xs0 = reinterpret_cast<float*>(take(4 * (size_t)nc));
  float* xs1 = reinterpret_cast<float*>(take(4 * (size_t)nc));
  float* cs = reinterpret_cast<float*>(take(4 * (size_t)nc));
  float* tval = reinterpret_cast<float*>(take(I.uniform ? 0 : 4 * (size_t)nzc));
  uint16_t* trow = reinterpret_cast<uint16_t*>(take(2 * (size_t)nzc));
  uint16_t* pos = reinterpret_cast<uint16_t*>(take(2 * (size_t)n));   // column -> position
  __shared__ GfIParam qsm[2];
  __shared__ double rho_s;
  __shared__ int n_rho_s;
  // ---- stage: replicated vectors, my rows, my columns (prefix of lengths
  // in order by one thread: the slices are small)
  const long long it0 = *k0_snap + 1;
  const float* xo_g = (it0 & 1) ? x0 : x1;               // x_{k0} in x[k0 & 1]
  for (int p = threadIdx.x; p < n; p += kThreads) {
    const int i = perm_g[I.v0 + p];
    pos[i] = (uint16_t)p;
    xb[p] = xbar_g[I.v0 + i];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += kThreads) {
    ys[j] = y_g[I.r0 + j];
    if (I.uniform) {
      const int64_t a = Kp[I.r0 + j];
      rowval[j] = Kp[I.r0 + j + 1] > a ? Kv[a] : 0.0f;
    }
  }
  for (int jj = threadIdx.x; jj <= mr; jj += kThreads)
    rp[jj] = (int32_t)(Kp[I.r0 + j0 + jj] - rk0);
  for (int jj = threadIdx.x; jj < mr; jj += kThreads) {
    rs[jj] = rhat[I.r0 + j0 + jj];
    eq[jj] = row_eq[I.r0 + j0 + jj];
  }
  for (int t = threadIdx.x; t < nzr; t += kThreads) {
    kcol[t] = pos[Kc[rk0 + t] - I.v0];                    // xbar is stored by position
    if (!I.uniform) kval[t] = Kv[rk0 + t];
  }
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < nc; ++t) {
      const int i = perm_g[I.v0 + p0 + t];
      ci[t] = (uint16_t)i;
      cp[t] = acc;
      acc += (int)(Tp[I.v0 + i + 1] - Tp[I.v0 + i]);
    }
    cp[nc] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nc; t += kThreads) {
    const int i = ci[t];
    xs0[t] = xo_g[I.v0 + i];
    cs[t] = chat[I.v0 + i];
    const int64_t a = Tp[I.v0 + i];
    for (int u = 0; u < cp[t + 1] - cp[t]; ++u) {
      trow[cp[t] + u] = (uint16_t)(Tr[a + u] - I.r0);
      if (!I.uniform) tval[cp[t] + u] = Tv[a + u];
    }
  }
  if (threadIdx.x == kSchedThread) {
    n_rho_s = st->n_rho;
    rho_s = st->rho;
    qsm[0] = iprm[(size_t)(it0 & 1) * ninst + b];
  }
  cl.sync();                                              // every copy staged
  long long s = 0;
  for (; s < nsteps; ++s) {
    const long long it = it0 + s;
    const GfIParam qq = qsm[s & 1];
    float* xo = (s & 1) ? xs1 : xs0;
    float* xn = (s & 1) ? xs0 : xs1;
    // dual step over my rows (k_pdhg_small's sums)
    for (int jj = threadIdx.x / kRowLanes; jj < mr; jj += kThreads / kRowLanes) {
      const int sl = threadIdx.x % kRowLanes;
      CSum acc;
      const int j = j0 + jj;
      const float rv = I.uniform ? rowval[j] : 0.0f;
      const int te = rp[jj + 1];
      for (int t = rp[jj] + sl; t < te; t += 4 * kRowLanes) {
        float part = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int tt = t + u * kRowLanes;
          if (tt < te) part = __fadd_rn(part, __fmul_rn(I.uniform ? rv : kval[tt], xb[kcol[tt]]));
        }
        acc.add(part);
      }
      gf::csum_group_reduce<kRowLanes>(acc);
      if (sl == 0) ys[j] = dual_update(ys[j], qq.tau2, acc.value(), rs[jj], eq[jj] != 0);
    }
    __syncthreads();
    // my slice of y into every other CTA's copy
    for (int e = threadIdx.x; e < mr * (C - 1); e += kThreads) {
      const int r = e / mr, jj = e - r * mr;
      *cl.map_shared_rank(ys + j0 + jj, r + (r >= q)) = ys[j0 + jj];
    }
    cl.sync();                                            // y complete everywhere
    // primal step over my columns; the new xbar_i goes to every CTA's copy
    const bool last = (s + 1 == nsteps);
    for (int t0 = threadIdx.x; t0 < nc; t0 += kThreads) {
      const int i = ci[t0];
      CSum acc;
      const int te = cp[t0 + 1];
      for (int t = cp[t0]; t < te; t += 4) {
        float part = 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (t + u < te) {
            const int j = trow[t + u];
            part = __fadd_rn(part, __fmul_rn(I.uniform ? rowval[j] : tval[t + u], ys[j]));
          }
        }
        acc.add(part);
      }
      const float xi = xo[t0];
      const float delta = primal_delta(cs[t0], qq.rho, acc.value(), xi);
      const float xv = primal_x(xi, qq.tau1, delta);
      xn[t0] = xv;
      xb[p0 + t0] = __fsub_rn(__fmul_rn(2.0f, xv), xi);
      if (last && dlast) dlast[I.v0 + i] = __fmul_rn(qq.tau1, delta);
    }
    if (threadIdx.x == kSchedThread) {
      // UpdatePenalty for iteration it+1 (counter advances once per k_int)
      const int n_next = (int)(it / sc->k_int);
      if (n_rho_s < n_next) {
        int n_rho = n_rho_s;
        double rho = rho_s;
        while (n_rho < n_next) {
          n_rho += 1;
          double rt = sc->rho_min * pow(1.0 + (double)n_rho / sc->T, sc->p);
          double lo = rho + sc->delta;
          double v = rt < lo ? lo : rt;
          rho = v > sc->rho_max ? sc->rho_max : v;
        }
        n_rho_s = n_rho;
        rho_s = rho;
        qsm[(s + 1) & 1] = step_params(sc->sigma, normQ[b], cap[b], rho);
      } else {
        qsm[(s + 1) & 1] = qq;
      }
    }
    __syncthreads();
    // my slice of xbar into every other CTA's copy
    for (int e = threadIdx.x; e < nc * (C - 1); e += kThreads) {
      const int r = e / nc, t = e - r * nc;
      *cl.map_shared_rank(xb + p0 + t, r + (r >= q)) = xb[p0 + t];
    }
    cl.sync();                                            // xbar complete everywhere
  }
  // ---- write back my columns (both parities), my rows, the schedule
  if (s > 0) {
    const long long lastit = it0 + s - 1;
    float* xl_g = (lastit & 1) ? x1 : x0;
    float* xp_g = (lastit & 1) ? x0 : x1;
    const float* xl = ((s - 1) & 1) ? xs0 : xs1;
    const float* xp = ((s - 1) & 1) ? xs1 : xs0;
    for (int t = threadIdx.x; t < nc; t += kThreads) {
      const int i = ci[t];
      xl_g[I.v0 + i] = xl[t];
      xp_g[I.v0 + i] = xp[t];
      xbar_g[I.v0 + i] = xb[p0 + t];
    }
    for (int jj = threadIdx.x; jj < mr; jj += kThreads) y_g[I.r0 + j0 + jj] = ys[j0 + jj];
    if (threadIdx.x == kSchedThread && q == 0) {
      iprm[(size_t)(lastit & 1) * ninst + b] = qsm[(s - 1) & 1];
      iprm[(size_t)((lastit + 1) & 1) * ninst + b] = qsm[s & 1];
      if (b == 0) {
        st->k = lastit;
        st->n_rho = n_rho_s;
        st->rho = rho_s;
      }
    }
  }
}

// Shared memory of one CTA of the cluster path for instance S (upper bound:
// every CTA's row / column slice is counted at its largest).
size_t cluster_smem(const GfSmallInst& S, int C, int64_t max_row_nnz, int64_t max_col_nnz) {
  auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
  const size_t mr = (size_t)S.m / C + 1, nc = (size_t)S.n / C + 1;
  size_t b = a16(4 * (size_t)S.n) + a16(4 * (size_t)S.m) + (S.uniform ? a16(4 * (size_t)S.m) : 0);
  b += a16(4 * (mr + 1)) + a16(4 * mr) + a16(mr);
  b += (S.uniform ? 0 : a16(4 * (size_t)max_row_nnz)) + a16(2 * (size_t)max_row_nnz);
  b += a16(4 * (nc + 1)) + a16(2 * nc) + 3 * a16(4 * nc);
  b += (S.uniform ? 0 : a16(4 * (size_t)max_col_nnz)) + a16(2 * (size_t)max_col_nnz);
  b += a16(2 * (size_t)S.n);                              // column -> position
  return b + 64;
}

}  // namespace

// Eligibility and tables of the small-instance path: every instance without
// Q, fewer than 2^16 variables and rows, its matrix and vectors within the
// shared-memory budget.  uniform[q]: every row of instance q has one value.
bool gf_small_setup(GfCtx* h, const std::vector<uint8_t>& uniform,
                    const std::vector<int64_t>& kp, const std::vector<int64_t>& tp) {
  if (h->prm.pdhg_mode == 1 || !h->dense.empty() || h->single_ok || h->M == 0) return false;
  std::vector<GfSmallInst> tab(h->ninst);
  size_t smem = 0;
  for (int q = 0; q < h->ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    if (I.qkind != 0 || I.n >= 65536 || I.m1 + I.m2 >= 65536 || I.m1 + I.m2 == 0) return false;
  }
  for (int q = 0; q < h->ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    GfSmallInst& S = tab[q];
    S.v0 = I.var_off;
    S.r0 = I.row_off;
    S.n = (int32_t)I.n;
    S.m = (int32_t)(I.m1 + I.m2);
    S.k0 = kp[I.row_off];
    S.t0 = tp[I.var_off];
    S.nnz = (int32_t)(kp[I.row_off + S.m] - S.k0);
    S.uniform = uniform[q] ? 1 : 0;
    if (tp[I.var_off + I.n] - S.t0 != S.nnz) return false;
    smem = std::max(smem, small_smem(S.n, S.m, S.nnz, S.uniform != 0));
  }
  if (smem > 200 * 1024) return false;
  // each instance's columns by decreasing length (ties in index order)
  std::vector<uint16_t> perm((size_t)h->N, 0);
  for (int q = 0; q < h->ninst; ++q) {
    const GfSmallInst& S = tab[q];
    std::vector<int32_t> ord(S.n);
    for (int32_t i = 0; i < S.n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t c) {
      return tp[S.v0 + a + 1] - tp[S.v0 + a] > tp[S.v0 + c + 1] - tp[S.v0 + c];
    });
    for (int32_t i = 0; i < S.n; ++i) perm[S.v0 + i] = (uint16_t)ord[i];
  }
  h->small_perm = gf_alloc_t<uint16_t>(h, perm.size());
  if (!h->small_perm) return false;
  if (cudaMemcpy(h->small_perm, perm.data(), sizeof(uint16_t) * perm.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaFuncSetAttribute(k_pdhg_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->small_tab = gf_alloc_t<GfSmallInst>(h, tab.size());
  h->small_k0 = gf_alloc_t<long long>(h, 1);
  if (!h->small_tab || !h->small_k0) return false;
  if (cudaMemcpyAsync(h->small_tab, tab.data(), sizeof(GfSmallInst) * tab.size(),
                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->small_smem = smem;
  // the cluster path: every instance in one wave of clusters (C CTAs each);
  // pdhg_mode 3 keeps one block per instance
  h->cluster_C = 0;
  if (h->prm.pdhg_mode != 3) {
    for (int C : {16, 8}) {
      if ((int64_t)h->ninst * C > h->num_sms) continue;
      size_t cs = 0;
      for (int q = 0; q < h->ninst; ++q) {
        const GfSmallInst& S = tab[q];
        int64_t mrow = 0, mcol = 0;
        for (int r = 0; r < C; ++r) {
          const int64_t a0 = (int64_t)S.m * r / C, a1 = (int64_t)S.m * (r + 1) / C;
          mrow = std::max(mrow, kp[S.r0 + a1] - kp[S.r0 + a0]);
          const int64_t c0 = (int64_t)S.n * r / C, c1 = (int64_t)S.n * (r + 1) / C;
          int64_t nz = 0;
          for (int64_t t = c0; t < c1; ++t) {
            const int64_t i = S.v0 + perm[S.v0 + t];
            nz += tp[i + 1] - tp[i];
          }
          mcol = std::max(mcol, nz);
        }
        cs = std::max(cs, cluster_smem(S, C, mrow, mcol));
      }
      if (cs > 200 * 1024) continue;
      if (cudaFuncSetAttribute(k_pdhg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)cs) != cudaSuccess ||
          (C > 8 && cudaFuncSetAttribute(k_pdhg_cluster,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                        cudaSuccess)) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(C * h->ninst));
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = cs;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, (void*)k_pdhg_cluster, &cfg) != cudaSuccess ||
          ncl < h->ninst) {
        cudaGetLastError();
        continue;
      }
      h->cluster_C = C;
      h->cluster_smem = cs;
      break;
    }
  }
  return true;
}

// nsteps iterations of every instance after the iterations completed so far
// (one launch, plus the one-thread snapshot of the device counter): one
// cluster per instance when the cluster path was chosen, else one block.
cudaError_t gf_launch_small(GfCtx* h, int64_t nsteps) {
  k_snap_k<<<1, 1, 0, h->stream>>>(h->dstate, h->small_k0);
  if (h->cluster_C > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)h->cluster_C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(h->cluster_C * h->ninst));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = h->cluster_smem;
    cfg.stream = h->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(
        &cfg, k_pdhg_cluster, (const GfSmallInst*)h->small_tab, (const int64_t*)h->Kp,
        (const int32_t*)h->Kc, (const float*)h->Kv, (const int64_t*)h->Tp,
        (const int32_t*)h->Tr, (const float*)h->Tv, (const uint16_t*)h->small_perm,
        (const float*)h->rhat, (const uint8_t*)h->row_eq, (const float*)h->chat, h->x[0],
        h->x[1], h->xbar, h->y, h->dlast, h->iprm, h->ninst, (const long long*)h->small_k0,
        (long long)nsteps, h->dstate, (const GfSched*)h->sched_d,
        (const double*)h->normQhat_d, (const int32_t*)h->cap_d);
    h->launches += 2;
    return e ? e : cudaGetLastError();
  }
  k_pdhg_small<<<h->ninst, kThreads, h->small_smem, h->stream>>>(
      h->small_tab, h->Kp, h->Kc, h->Kv, h->Tp, h->Tr, h->Tv, h->small_perm, h->rhat,
      h->row_eq, h->chat,
      h->x[0], h->x[1], h->xbar, h->y, h->dlast, h->iprm, h->ninst, h->small_k0, nsteps,
      h->dstate, h->sched_d, h->normQhat_d, h->cap_d);
  h->launches += 2;
  return cudaGetLastError();
}
