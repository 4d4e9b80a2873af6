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
      if (sl == 0) {
        float v = ys[j] + q.tau2 * (acc.value() + rs[j]);
        if (!eq[j] && v < 0.f) v = 0.f;
        ys[j] = v;
      }
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
      const float delta = cs[i] + q.rho + acc.value() - 2.0f * q.rho * xi;
      const float xv = fminf(1.0f, fmaxf(0.0f, xi - q.tau1 * delta));
      xn[i] = xv;
      xb[i] = 2.0f * xv - xi;
      if (last && dlast) dlast[I.v0 + i] = q.tau1 * delta;
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
  return true;
}

// nsteps iterations of every instance after the iterations completed so far
// (one launch, plus the one-thread snapshot of the device counter).
cudaError_t gf_launch_small(GfCtx* h, int64_t nsteps) {
  k_snap_k<<<1, 1, 0, h->stream>>>(h->dstate, h->small_k0);
  k_pdhg_small<<<h->ninst, kThreads, h->small_smem, h->stream>>>(
      h->small_tab, h->Kp, h->Kc, h->Kv, h->Tp, h->Tr, h->Tv, h->small_perm, h->rhat,
      h->row_eq, h->chat,
      h->x[0], h->x[1], h->xbar, h->y, h->dlast, h->iprm, h->ninst, h->small_k0, nsteps,
      h->dstate, h->sched_d, h->normQhat_d, h->cap_d);
  h->launches += 2;
  return cudaGetLastError();
}
