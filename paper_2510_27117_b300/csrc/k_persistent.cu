// k_persistent.cu -- PDHG iterations (Alg. 2) of a dense-Q instance in ONE
// cooperative launch: every block keeps its rows of W2 = offdiag(Q + Q^T)
// (int8, exact) resident in shared memory for the whole launch, so an
// iteration moves only x (n floats per block) instead of the n x n matrix.
// Iterations are separated by a grid-wide barrier whose wait is bounded by a
// time limit (on expiry: error flag in the device state, every block exits).
// Arithmetic is the one of k_pdhg.cu's dense step: 8-term plain FP32 chunks
// folded into a compensated sum, then the projected update.
#include "internal.cuh"

namespace {

using gf::CSum;

constexpr int kWarps = 32;

// UpdatePenalty for the next iteration (same rule as k_pdhg.cu), by block 0.
__device__ void advance_penalty_p(GfDState* st, const GfSched* sc, const double* normQ,
                                const int32_t* cap, const GfIParam* cur, GfIParam* next) {
  // The parameters of iteration it+1 equal those of iteration it unless the
  // penalty counter advances (once per k_int iterations): only then are rho
  // and the step sizes recomputed (FP64), otherwise the slot is copied.
  __shared__ double rho_s;
  __shared__ int changed_s;
  if (threadIdx.x == 0) {
    long long it = st->k + 1;               // the iteration now running
    int n_next = (int)(it / sc->k_int);     // counter used by iteration it+1
    double rho = st->rho;
    int changed = 0;
    while (st->n_rho < n_next) {
      st->n_rho += 1;
      double rt = sc->rho_min * pow(1.0 + (double)st->n_rho / sc->T, sc->p);
      double lo = rho + sc->delta;
      double v = rt < lo ? lo : rt;
      rho = v > sc->rho_max ? sc->rho_max : v;
      changed = 1;
    }
    st->rho = rho;
    st->k = it;
    rho_s = rho;
    changed_s = changed;
  }
  __syncthreads();
  const double rho = rho_s;
  const int changed = changed_s;
  for (int b = threadIdx.x; b < sc->ninst; b += blockDim.x) {
    if (!changed) {
      next[b] = cur[b];
      continue;
    }
    double t1 = sqrt(sc->sigma);
    if (cap[b]) {
      double L = 2.0 * (normQ[b] + rho);
      if (L > 0.0 && 1.0 / (2.0 * L) < t1) t1 = 1.0 / (2.0 * L);
    }
    double t2 = sc->sigma / t1;
    GfIParam q;
    q.tau1 = (float)t1; q.tau2 = (float)t2; q.rho = (float)rho; q.pad = 0.f;
    q.tau1d = t1; q.tau2d = t2; q.rhod = rho; q.normQ = normQ[b];
    next[b] = q;
  }
}

// Grid barrier: one arrival per block on a counter zeroed before the
// launch; the wait gives up after limit_ns (or when another block already
// gave up) and reports it.  Returns false when the launch must stop.
__device__ bool grid_barrier(unsigned* bar, unsigned target, uint64_t limit_ns, int* err,
                             volatile int* stop) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const uint64_t t0 = gf::globaltimer_ns();
    while (true) {
      if (*(volatile unsigned*)bar >= target) break;
      if (*(volatile int*)err) { *stop = 1; break; }
      if (gf::globaltimer_ns() - t0 > limit_ns) {
        atomicExch(err, 1);
        *stop = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *stop == 0;
}

__global__ void __launch_bounds__(kWarps * 32, 1)
k_pdhg_dense_persistent(const int8_t* __restrict__ W2, int64_t ld, int64_t n, int64_t v0,
                        const float* __restrict__ qdiag, float qscale, float* x0,
                        float* x1, float* __restrict__ xbar, const float* __restrict__ chat,
                        float* __restrict__ dlast, GfIParam* iprm, int inst, int ninst,
                        long long k0, long long nsteps, GfDState* st, const GfSched* sc,
                        const double* normQ, const int32_t* cap, unsigned* bar,
                        uint64_t limit_ns) {
  extern __shared__ float4 sm4[];
  float* xs = reinterpret_cast<float*>(sm4);                    // ld floats
  const uint32_t* Ws = reinterpret_cast<const uint32_t*>(xs + ld);   // my rows, int8
  __shared__ volatile int stop;
  if (threadIdx.x == 0) stop = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  // rows [r0, r1) of W2 into shared memory, once per launch
  {
    uint4* dst = reinterpret_cast<uint4*>(xs + ld);
    const uint4* src = reinterpret_cast<const uint4*>(W2 + r0 * ld);
    const int64_t cnt = (r1 > r0) ? (r1 - r0) * ld / 16 : 0;
    for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) dst[e] = src[e];
  }
  const int64_t nq = ld / 4;                      // 4-entry words per row
  for (long long s = 0; s < nsteps; ++s) {
    const long long it = k0 + 1 + s;
    const int p = (int)(it & 1);
    const float* xo = p ? x0 : x1;                // x_{it-1} in x[1 - p]
    float* xn = p ? x1 : x0;                      // x_it in x[p]
    const GfIParam q = iprm[(size_t)p * ninst + inst];
    // x_{it-1} into shared memory: the instance's padded range [v0, v0 + ld)
    // is 16-byte aligned and its padding entries are zero
    for (int64_t j4 = threadIdx.x; j4 < nq; j4 += blockDim.x)
      sm4[j4] = __ldcg(reinterpret_cast<const float4*>(xo + v0) + j4);
    __syncthreads();
    for (int64_t i = r0 + warp; i < r1; i += kWarps) {
      const uint32_t* row = Ws + (i - r0) * nq;
      CSum acc;
      // lane l takes words l, l+32, ... : conflict-free 4-byte W and
      // 16-byte x shared-memory reads; two words (8 terms) per chunk
      for (int64_t t = lane; t < nq; t += 64) {
        const uint32_t wa = row[t];
        const float4 xa = sm4[t];
        float part = (float)(int8_t)(wa) * xa.x;
        part = fmaf((float)(int8_t)(wa >> 8), xa.y, part);
        part = fmaf((float)(int8_t)(wa >> 16), xa.z, part);
        part = fmaf((float)(int8_t)(wa >> 24), xa.w, part);
        if (t + 32 < nq) {
          const uint32_t wb = row[t + 32];
          const float4 xb = sm4[t + 32];
          part = fmaf((float)(int8_t)(wb), xb.x, part);
          part = fmaf((float)(int8_t)(wb >> 8), xb.y, part);
          part = fmaf((float)(int8_t)(wb >> 16), xb.z, part);
          part = fmaf((float)(int8_t)(wb >> 24), xb.w, part);
        }
        acc.add(part);
      }
      gf::csum_group_reduce<32>(acc);
      if (lane == 0) {
        const float xo_i = xs[i];
        CSum sq;                                  // 2 (Q_hat x)_i
        sq.merge(__fmul_rn(2.0f * qscale, acc.s), __fmul_rn(2.0f * qscale, acc.c));
        sq.add(__fmul_rn(2.0f * qdiag[i], xo_i));
        const float delta = chat[v0 + i] + q.rho + sq.value() - 2.0f * q.rho * xo_i;
        const float xnew = fminf(1.0f, fmaxf(0.0f, xo_i - q.tau1 * delta));
        xn[v0 + i] = xnew;
        xbar[v0 + i] = 2.0f * xnew - xo_i;
        if (dlast) dlast[v0 + i] = q.tau1 * delta;
      }
    }
    if (blockIdx.x == 0) advance_penalty_p(st, sc, normQ, cap, iprm + (size_t)p * ninst,
                                          iprm + (size_t)(1 - p) * ninst);
    if (!grid_barrier(bar, (unsigned)((s + 1) * gridDim.x), limit_ns, &st->error, &stop)) break;
  }
}

}  // namespace

// Is the persistent path usable for this batch?  One dense instance without
// rows, int8 operand, its rows fit in shared memory, cooperative launch.
bool gf_persistent_setup(GfCtx* h) {
  if (h->ninst != 1 || h->dense.size() != 1 || h->M != 0) return false;
  const GfDenseQ& dq = h->dense[0];
  if (!dq.W2i8) return false;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev);
  if (!coop) return false;
  const int64_t per = (dq.n + h->num_sms - 1) / h->num_sms;
  const size_t smem = sizeof(float) * (size_t)dq.ld + (size_t)per * dq.ld;
  if (smem > 200 * 1024) return false;
  if (cudaFuncSetAttribute(k_pdhg_dense_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pdhg_dense_persistent, kWarps * 32,
                                                    smem) != cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    return false;
  }
  h->persist_smem = smem;
  h->persist_bar = gf_alloc_t<unsigned>(h, 1);
  return h->persist_bar != nullptr;
}

// nsteps iterations starting after iteration h->k_host (one launch).
cudaError_t gf_launch_persistent(GfCtx* h, int64_t nsteps) {
  const GfDenseQ& dq = h->dense[0];
  const GfInstHost& I = h->ih[dq.inst];
  cudaError_t e = cudaMemsetAsync(h->persist_bar, 0, sizeof(unsigned), h->stream);
  if (e) return e;
  const int8_t* W2 = dq.W2i8;
  int64_t ld = dq.ld, n = dq.n, v0 = I.var_off;
  const float* qdiag = dq.qdiag;
  float qscale = dq.qscale;
  float* x0 = h->x[0];
  float* x1 = h->x[1];
  float* xbar = h->xbar;
  const float* chat = h->chat;
  float* dlast = h->dlast;
  GfIParam* iprm = h->iprm;
  int inst = dq.inst, ninst = h->ninst;
  long long k0 = h->k_host, ns = nsteps;
  GfDState* st = h->dstate;
  const GfSched* sc = h->sched_d;
  const double* nq = h->normQhat_d;
  const int32_t* cap = h->cap_d;
  unsigned* bar = h->persist_bar;
  uint64_t limit = (uint64_t)(std::max(0.01, h->prm.wait_timeout_s) * 1e9);
  void* args[] = {&W2, &ld, &n, &v0, &qdiag, &qscale, &x0, &x1, &xbar, &chat, &dlast, &iprm,
                  &inst, &ninst, &k0, &ns, &st, &sc, &nq, &cap, &bar, &limit};
  e = cudaLaunchCooperativeKernel((const void*)k_pdhg_dense_persistent, dim3(h->num_sms),
                                  dim3(kWarps * 32), args, h->persist_smem, h->stream);
  h->launches += 2;
  return e;
}
