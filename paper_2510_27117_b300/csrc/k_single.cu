// k_single.cu -- PDHG iteration (Alg. 2) for batches in which every instance
// has exactly one constraint row and no Q (knapsack-type batches).
//
// With one row per instance, (K^T y)_i = k_i y and the dual step needs only
// the scalar K xbar.  One streaming kernel per iteration therefore does the
// whole primal step of every variable AND the partial sums of K xbar_k over
// fixed chunks of 2048 variables (compensated, deterministic order); a tiny
// kernel folds an instance's chunk partials in chunk order into the next dual
// step.  Per variable and iteration the kernels read x_{k-1}, k_i, c_hat_i
// and write x_k (16 bytes, the algorithmic minimum); xbar_k and tau1 delta_i
// are stored only by the last two iterations of a call -- the row is never
// re-read.
//
// Partial sums are double-buffered by iteration parity: iteration `it`
// (parity p = it & 1) reads part[1 - p] (K xbar_{it-1}) in its dual step and
// writes part[p] in its primal step.
#include "internal.cuh"
#include "penalty.cuh"

namespace {

using gf::CSum;

constexpr int kThreads = 256;      // 8 variables per thread per chunk

// Block-wide compensated sum of per-thread CSums (fixed order), to thread 0.
GF_DEV CSum block_csum(CSum a) {
  __shared__ float ss[kThreads / 32], scc[kThreads / 32];
  gf::csum_group_reduce<32>(a);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = a.s; scc[w] = a.c; }
  __syncthreads();
  CSum tot;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; ++q) tot.merge(ss[q], scc[q]);
  return tot;
}

// Dual step of every instance: y <- Pi(y + tau2 (K xbar + r)), K xbar the sum
// of the instance's chunk partials (lane-strided, then a fixed warp reduce).
__global__ void k_single_dual(const int32_t* __restrict__ ciptr, int ninst,
                              const float2* __restrict__ part, const float* __restrict__ r,
                              const uint8_t* __restrict__ row_eq,
                              const int64_t* __restrict__ row_of, const GfIParam* __restrict__ ip,
                              float* __restrict__ y) {
  const int q = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= ninst) return;
  CSum acc;
  for (int c = ciptr[q] + lane; c < ciptr[q + 1]; c += 32) acc.merge(part[c].x, part[c].y);
  gf::csum_group_reduce<32>(acc);
  if (lane == 0) {
    const int64_t j = row_of[q];
    float v = y[j] + ip[q].tau2 * (acc.value() + r[j]);
    if (!row_eq[j] && v < 0.f) v = 0.f;
    y[j] = v;
  }
}

// K xbar partials of every chunk from a stored xbar (before the first
// iteration after the state was set).
__global__ void __launch_bounds__(kThreads)
k_single_partials(const int32_t* __restrict__ ch, const float* __restrict__ kv,
                  const float* __restrict__ xbar, float2* __restrict__ part) {
  const int c = blockIdx.x;
  const int64_t v0 = ch[3 * c + 1], v1 = ch[3 * c + 2];
  CSum acc;
  for (int64_t i = v0 + threadIdx.x; i < v1; i += kThreads)
    acc.add(__fmul_rn(kv[i], xbar[i]));
  CSum tot = block_csum(acc);
  if (threadIdx.x == 0) part[c] = make_float2(tot.s, tot.c);
}

// Primal step of a chunk of variables, fused with the chunk's K xbar partial.
// FULL = false stores only x_k (xbar_k enters the partial directly).
template <bool FULL>
__global__ void __launch_bounds__(kThreads)
k_single_primal(const int32_t* __restrict__ ch, const float* __restrict__ kv,
                const float* __restrict__ x_old, const float* __restrict__ chat,
                const float* __restrict__ y, const int64_t* __restrict__ row_of,
                const GfIParam* __restrict__ ip, float* __restrict__ x_new,
                float* __restrict__ xbar, float* __restrict__ dlast,
                float2* __restrict__ part, int advance, GfDState* st, const GfSched* sc,
                const double* normQ, const int32_t* cap, GfIParam* ip_next) {
  const int c = blockIdx.x;
  const int q = ch[3 * c];
  const int64_t v0 = ch[3 * c + 1], v1 = ch[3 * c + 2];
  const GfIParam p = ip[q];
  const float yq = y[row_of[q]];
  CSum acc;
  for (int64_t i = v0 + threadIdx.x; i < v1; i += kThreads) {
    const float k = kv[i], xo = x_old[i];
    const float delta = chat[i] + p.rho + __fmul_rn(k, yq) - 2.0f * p.rho * xo;
    const float xn = fminf(1.0f, fmaxf(0.0f, xo - p.tau1 * delta));
    const float xb = 2.0f * xn - xo;
    x_new[i] = xn;
    if (FULL) {
      xbar[i] = xb;
      if (dlast) dlast[i] = p.tau1 * delta;
    }
    acc.add(__fmul_rn(k, xb));
  }
  CSum tot = block_csum(acc);
  if (threadIdx.x == 0) part[c] = make_float2(tot.s, tot.c);
  if (advance && blockIdx.x == 0) advance_penalty(st, sc, normQ, cap, ip, ip_next);
}

}  // namespace

// Partials of K xbar for the iteration after h->k_host (state just set).
cudaError_t gf_single_init(GfCtx* h) {
  const int pprev = (int)(h->k_host & 1);     // parity of the last iteration
  k_single_partials<<<(unsigned)h->sr_nchunk, kThreads, 0, h->stream>>>(
      h->sr_chunk, h->sr_kv, h->xbar, h->sr_part + (size_t)pprev * h->sr_nchunk);
  h->launches++;
  return cudaGetLastError();
}

// One iteration with parity p (dual step, then primal step + partials).
cudaError_t gf_single_iter(GfCtx* h, int p) {
  const GfIParam* ip = h->iprm + (size_t)p * h->ninst;
  GfIParam* ipn = h->iprm + (size_t)(1 - p) * h->ninst;
  k_single_dual<<<(unsigned)((h->ninst * 32 + 255) / 256), 256, 0, h->stream>>>(
      h->sr_ciptr, h->ninst, h->sr_part + (size_t)(1 - p) * h->sr_nchunk, h->rhat, h->row_eq,
      h->sr_row, ip, h->y);
  auto kern = h->light_iter ? k_single_primal<false> : k_single_primal<true>;
  kern<<<(unsigned)h->sr_nchunk, kThreads, 0, h->stream>>>(
      h->sr_chunk, h->sr_kv, h->x[1 - p], h->chat, h->y, h->sr_row, ip, h->x[p], h->xbar,
      h->dlast, h->sr_part + (size_t)p * h->sr_nchunk, 1, h->dstate, h->sched_d,
      h->normQhat_d, h->cap_d, ipn);
  h->launches += 2;
  return cudaGetLastError();
}

namespace {
// K entry of every variable: the single CSC entry of its column, 0 if none.
__global__ void k_single_kv(int64_t N, const int64_t* __restrict__ Tp,
                            const float* __restrict__ Tv, float* __restrict__ kv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) kv[i] = (Tp[i + 1] > Tp[i]) ? Tv[Tp[i]] : 0.0f;
}
}  // namespace

// Tables of the single-row path (after the FP32 scaled K exists on the
// device).  Returns false (path unused) unless every instance has one row,
// no Q and no dense operand.
bool gf_single_setup(GfCtx* h) {
  if (h->prm.pdhg_mode == 1 || !h->dense.empty() || h->M != h->ninst) return false;
  for (int q = 0; q < h->ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    if (I.m1 + I.m2 != 1 || I.qkind != 0) return false;
  }
  std::vector<int32_t> ch, cptr(h->ninst + 1);
  std::vector<int64_t> row(h->ninst);
  for (int q = 0; q < h->ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    cptr[q] = (int32_t)(ch.size() / 3);
    row[q] = I.row_off;
    for (int64_t a = 0; a < I.n; a += 2048) {
      ch.push_back(q);
      ch.push_back((int32_t)(I.var_off + a));
      ch.push_back((int32_t)(I.var_off + std::min<int64_t>(I.n, a + 2048)));
    }
  }
  cptr[h->ninst] = (int32_t)(ch.size() / 3);
  h->sr_nchunk = (int64_t)ch.size() / 3;
  h->sr_chunk = gf_alloc_t<int32_t>(h, ch.size());
  h->sr_ciptr = gf_alloc_t<int32_t>(h, cptr.size());
  h->sr_row = gf_alloc_t<int64_t>(h, row.size());
  h->sr_kv = gf_alloc_t<float>(h, h->N);
  h->sr_part = gf_alloc_t<float2>(h, 2 * h->sr_nchunk);
  if (!h->sr_chunk || !h->sr_ciptr || !h->sr_row || !h->sr_kv || !h->sr_part) return false;
  cudaMemcpyAsync(h->sr_chunk, ch.data(), sizeof(int32_t) * ch.size(), cudaMemcpyHostToDevice,
                  h->stream);
  cudaMemcpyAsync(h->sr_ciptr, cptr.data(), sizeof(int32_t) * cptr.size(),
                  cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->sr_row, row.data(), sizeof(int64_t) * row.size(), cudaMemcpyHostToDevice,
                  h->stream);
  k_single_kv<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(h->N, h->Tp, h->Tv,
                                                                    h->sr_kv);
  h->sr_valid = false;
  return cudaGetLastError() == cudaSuccess;
}
