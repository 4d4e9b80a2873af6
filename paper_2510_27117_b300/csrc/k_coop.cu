// k_coop.cu -- PDHG iterations (Alg. 2) of sparse problems whose matrices fit
// the L2 cache (e.g. the I = 64 axial assignment: 786k nonzeros), as ONE
// cooperative launch per gfors_pdhg_steps call: each iteration is the dual
// step over all rows, a grid barrier, the primal step over all columns, a
// grid barrier -- no launch gaps and no separate reduction kernels.
//
// Rows and columns are split by length into work lists: a block per long
// row / column (deterministic block reduction), a warp per medium one, a
// thread per short column.  Block 0 advances the penalty schedule during the
// primal step (as the first primal kernel of the per-iteration path does).
// Grid barriers are one release-add per block polled with acquire loads,
// bounded by a time limit (error flag in the device state on expiry).
#include "internal.cuh"
#include "penalty.cuh"

namespace {

using gf::CSum;
constexpr int kThreads = 1024;
constexpr int kMaxStagedY = 8192;                // y staged when it has <= this many rows

// arrive = false (test injection only) waits without arriving, so every
// block's bounded wait runs out.
GF_DEV bool coop_barrier(unsigned* bar, unsigned target, int* err, uint64_t limit_ns,
                         bool arrive = true) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    bool ok = true;
    if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    uint64_t t0 = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*(volatile int*)err) { ok = false; break; }
      const uint64_t now = gf::globaltimer_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) { atomicExch(err, 1); ok = false; break; }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Block-wide compensated sum (fixed order), result in every thread.
GF_DEV CSum block_sum(CSum a) {
  __shared__ float ss[kThreads / 32], sc[kThreads / 32];
  __shared__ float tot_s, tot_c;
  gf::csum_group_reduce<32>(a);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = a.s; sc[w] = a.c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum t;
    for (int q = 0; q < kThreads / 32; ++q) t.merge(ss[q], sc[q]);
    tot_s = t.s;
    tot_c = t.c;
  }
  __syncthreads();
  CSum r;
  r.s = tot_s;
  r.c = tot_c;
  __syncthreads();
  return r;
}

struct CoopLists {
  const int32_t *rblk, *rwarp;            // rows: block-per-row, warp-per-row
  const int32_t *cblk, *cwarp, *cthr;     // columns: block / warp / thread per column
  int32_t nrblk, nrwarp, ncblk, ncwarp, ncthr;
};

GF_DEV float dual_update(float yj, float tau2, float kx, float rj, bool eqrow) {
  float v = yj + tau2 * (kx + rj);
  if (!eqrow && v < 0.f) v = 0.f;
  return v;
}

__global__ void __launch_bounds__(kThreads, 1)
k_pdhg_coop(CoopLists L, const int64_t* __restrict__ Kp, const int32_t* __restrict__ Kc,
            const float* __restrict__ Kv, const int64_t* __restrict__ Tp,
            const int32_t* __restrict__ Tr, const float* __restrict__ Tv,
            const float* __restrict__ rhat, const uint8_t* __restrict__ row_eq,
            const int32_t* __restrict__ row_inst, const int32_t* __restrict__ var_inst,
            const float* __restrict__ chat, float* x0, float* x1, float* xbar, float* y,
            float* __restrict__ dlast, GfIParam* iprm, int ninst, long long k0,
            long long nsteps, GfDState* st, const GfSched* sc, const double* normQ,
            const int32_t* cap, unsigned* bar, uint64_t limit_ns, int stage_y,
            int skip_block) {
  extern __shared__ float ysm[];                // y staged for the primal step
  __shared__ double rho_s;                      // schedule state (block 0)
  __shared__ int n_rho_s, changed_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * (kThreads / 32) + warp, nwarps = gridDim.x * (kThreads / 32);
  const int gtid = blockIdx.x * kThreads + threadIdx.x, nthreads = gridDim.x * kThreads;
  const unsigned nb = gridDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    n_rho_s = st->n_rho;
    rho_s = st->rho;
  }
  int M = 0;                                    // rows (stage_y: y fits shared memory)
  if (stage_y) M = stage_y;
  long long s = 0;
  for (; s < nsteps; ++s) {
    const long long it = k0 + 1 + s;
    const int p = (int)(it & 1);
    const GfIParam* ip = iprm + (size_t)p * ninst;
    GfIParam* ipn = iprm + (size_t)(1 - p) * ninst;
    const float* xo = p ? x0 : x1;
    float* xn = p ? x1 : x0;
    // ---- dual step, Alg. 2
    for (int q = blockIdx.x; q < L.nrblk; q += gridDim.x) {
      const int j = L.rblk[q];
      CSum acc;
      for (int64_t t = Kp[j] + threadIdx.x; t < Kp[j + 1]; t += kThreads)
        acc.add(__fmul_rn(Kv[t], __ldcg(xbar + Kc[t])));
      const CSum tot = block_sum(acc);
      if (threadIdx.x == 0)
        y[j] = dual_update(y[j], ip[row_inst[j]].tau2, tot.value(), rhat[j], row_eq[j] != 0);
    }
    for (int q = gwarp; q < L.nrwarp; q += nwarps) {
      const int j = L.rwarp[q];
      CSum acc;
      for (int64_t t = Kp[j] + lane; t < Kp[j + 1]; t += 32)
        acc.add(__fmul_rn(Kv[t], __ldcg(xbar + Kc[t])));
      gf::csum_group_reduce<32>(acc);
      if (lane == 0)
        y[j] = dual_update(y[j], ip[row_inst[j]].tau2, acc.value(), rhat[j], row_eq[j] != 0);
    }
    if (!coop_barrier(bar, (unsigned)(2 * s + 1) * nb, &st->error, limit_ns,
                      !(s == 0 && (int)blockIdx.x == skip_block)))
      break;
    // ---- primal step, Alg. 2 (y of this iteration staged in shared memory)
    const float* yv = y;
    if (M > 0) {
      for (int j = threadIdx.x; j < M; j += kThreads) ysm[j] = __ldcg(y + j);
      __syncthreads();
      yv = ysm;
    }
    auto update = [&](int i, float kty) {
      const GfIParam pr = ip[var_inst[i]];
      const float xi = __ldcg(xo + i);
      const float delta = chat[i] + pr.rho + kty - 2.0f * pr.rho * xi;
      const float xv = fminf(1.0f, fmaxf(0.0f, xi - pr.tau1 * delta));
      xn[i] = xv;
      xbar[i] = 2.0f * xv - xi;
      if (dlast) dlast[i] = pr.tau1 * delta;
    };
    for (int q = blockIdx.x; q < L.ncblk; q += gridDim.x) {
      const int i = L.cblk[q];
      CSum acc;
      for (int64_t t = Tp[i] + threadIdx.x; t < Tp[i + 1]; t += kThreads)
        acc.add(__fmul_rn(Tv[t], M ? yv[Tr[t]] : __ldcg(y + Tr[t])));
      const CSum tot = block_sum(acc);
      if (threadIdx.x == 0) update(i, tot.value());
    }
    for (int q = gwarp; q < L.ncwarp; q += nwarps) {
      const int i = L.cwarp[q];
      CSum acc;
      for (int64_t t = Tp[i] + lane; t < Tp[i + 1]; t += 32)
        acc.add(__fmul_rn(Tv[t], M ? yv[Tr[t]] : __ldcg(y + Tr[t])));
      gf::csum_group_reduce<32>(acc);
      if (lane == 0) update(i, acc.value());
    }
    for (int q = gtid; q < L.ncthr; q += nthreads) {
      const int i = L.cthr[q];
      CSum acc;
      for (int64_t t = Tp[i]; t < Tp[i + 1]; ++t)
        acc.add(__fmul_rn(Tv[t], M ? yv[Tr[t]] : __ldcg(y + Tr[t])));
      update(i, acc.value());
    }
    if (blockIdx.x == 0) {
      // UpdatePenalty for iteration it+1 from block 0's shared state (no
      // global round trips on the barrier's critical path)
      if (threadIdx.x == 0) {
        const int n_next = (int)(it / sc->k_int);
        int changed = 0;
        while (n_rho_s < n_next) {
          n_rho_s += 1;
          double rt = sc->rho_min * pow(1.0 + (double)n_rho_s / sc->T, sc->p);
          double lo = rho_s + sc->delta;
          double v = rt < lo ? lo : rt;
          rho_s = v > sc->rho_max ? sc->rho_max : v;
          changed = 1;
        }
        changed_s = changed;
      }
      __syncthreads();
      for (int b = threadIdx.x; b < ninst; b += kThreads)
        ipn[b] = changed_s ? step_params(sc->sigma, normQ[b], cap[b], rho_s) : ip[b];
    }
    if (!coop_barrier(bar, (unsigned)(2 * s + 2) * nb, &st->error, limit_ns)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && s > 0) {
    st->k = k0 + s;
    st->n_rho = n_rho_s;
    st->rho = rho_s;
  }
}

}  // namespace

// Eligibility (pdhg_mode 2): sparse problems without Q whose K, K^T and
// vectors take at most 48 MB (L2-resident), not served by the small /
// one-row / dense paths.
bool gf_coop_setup(GfCtx* h, const std::vector<int64_t>& kp, const std::vector<int64_t>& tp) {
  // opt-in (pdhg_mode 2): on the I = 64 assignment it measured 13 us per
  // iteration against 12 us for CUDA graphs of the run-described kernels
  if (h->prm.pdhg_mode != 2 || h->small_ok || h->single_ok || h->persist_ok ||
      !h->dense.empty() || h->nnzQ > 0 || h->M == 0)
    return false;
  const double bytes = 16.0 * (double)h->nnzK + 28.0 * (double)h->N + 16.0 * (double)h->M;
  if (bytes > 48.0 * 1024 * 1024) return false;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev);
  if (!coop) return false;
  int nb = 0;
  const size_t smem = h->M <= kMaxStagedY ? sizeof(float) * (size_t)h->M : 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pdhg_coop, kThreads, smem) !=
          cudaSuccess || nb < 1) {
    cudaGetLastError();
    return false;
  }
  std::vector<int32_t> rblk, rwarp, cblk, cwarp, cthr;
  for (int64_t j = 0; j < h->M; ++j) (kp[j + 1] - kp[j] > 512 ? rblk : rwarp).push_back((int32_t)j);
  for (int q = 0; q < h->ninst; ++q) {
    const GfInstHost& I = h->ih[q];
    for (int64_t i = I.var_off; i < I.var_off + I.n; ++i) {
      const int64_t len = tp[i + 1] - tp[i];
      (len > 512 ? cblk : len > 16 ? cwarp : cthr).push_back((int32_t)i);
    }
  }
  auto up = [&](const std::vector<int32_t>& v) -> int32_t* {
    if (v.empty()) return nullptr;
    int32_t* d = gf_alloc_t<int32_t>(h, v.size());
    if (d) cudaMemcpyAsync(d, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice,
                           h->stream);
    return d;
  };
  h->coop_rblk = up(rblk);
  h->coop_rwarp = up(rwarp);
  h->coop_cblk = up(cblk);
  h->coop_cwarp = up(cwarp);
  h->coop_cthr = up(cthr);
  h->coop_n[0] = (int32_t)rblk.size();
  h->coop_n[1] = (int32_t)rwarp.size();
  h->coop_n[2] = (int32_t)cblk.size();
  h->coop_n[3] = (int32_t)cwarp.size();
  h->coop_n[4] = (int32_t)cthr.size();
  h->coop_bar = gf_alloc_t<unsigned>(h, 1);
  if (!h->coop_bar || cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

cudaError_t gf_launch_coop(GfCtx* h, int64_t nsteps) {
  cudaError_t e = cudaMemsetAsync(h->coop_bar, 0, sizeof(unsigned), h->stream);
  if (e) return e;
  CoopLists L{h->coop_rblk, h->coop_rwarp, h->coop_cblk, h->coop_cwarp, h->coop_cthr,
              h->coop_n[0], h->coop_n[1], h->coop_n[2], h->coop_n[3], h->coop_n[4]};
  const int64_t *Kp = h->Kp, *Tp = h->Tp;
  const int32_t *Kc = h->Kc, *Tr = h->Tr, *ri = h->row_inst, *vi = h->var_inst;
  const float *Kv = h->Kv, *Tv = h->Tv, *rhat = h->rhat, *chat = h->chat;
  const uint8_t* req = h->row_eq;
  float *x0 = h->x[0], *x1 = h->x[1], *xbar = h->xbar, *y = h->y, *dlast = h->dlast;
  GfIParam* iprm = h->iprm;
  int ninst = h->ninst;
  long long k0 = h->k_host, ns = nsteps;
  GfDState* st = h->dstate;
  const GfSched* sc = h->sched_d;
  const double* nq = h->normQhat_d;
  const int32_t* cap = h->cap_d;
  unsigned* bar = h->coop_bar;
  uint64_t limit = (uint64_t)(std::max(0.01, h->prm.wait_timeout_s) * 1e9);
  int stage_y = h->M <= kMaxStagedY ? (int)h->M : 0;
  int skip = h->inject_skip_block;
  h->inject_skip_block = -1;
  void* args[] = {&L, &Kp, &Kc, &Kv, &Tp, &Tr, &Tv, &rhat, &req, &ri, &vi, &chat, &x0, &x1,
                  &xbar, &y, &dlast, &iprm, &ninst, &k0, &ns, &st, &sc, &nq, &cap, &bar,
                  &limit, &stage_y, &skip};
  e = cudaLaunchCooperativeKernel((const void*)k_pdhg_coop, dim3(h->num_sms), dim3(kThreads),
                                  args, sizeof(float) * (size_t)stage_y, h->stream);
  h->launches += 2;
  return e;
}
