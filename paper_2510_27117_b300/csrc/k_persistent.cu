// k_persistent.cu -- PDHG iterations (Alg. 2) of a dense-Q instance in ONE
// cooperative launch: every block keeps its rows of W2 = offdiag(Q + Q^T)
// (int8, exact), the matching entries of c_hat and diag(Q_hat) in shared
// memory for the whole launch, so an iteration moves only x (n floats per
// block) instead of the n x n matrix.
//
// Iterations are separated by a grid barrier: one release-add per block on a
// counter, polled with acquire loads by one thread per block; every wait is
// bounded by a time limit (on expiry: error flag in the device state, every
// block exits).  The penalty schedule (UpdatePenalty) is advanced inside every
// block from the same FP64 state, so no block waits for another's parameter
// update.  Arithmetic: the row dot product of gf::i8_row_dot (shared with
// the per-iteration kernel of k_pdhg.cu), then the same projected update.
#include "internal.cuh"
#include "penalty.cuh"

namespace {

using gf::CSum;

constexpr int kWarps = 32;
constexpr int kSchedThread = kWarps * 32 - 1;   // advances the penalty schedule
constexpr int kMaxRows = 256;                   // rows per block (c_hat, diag cache)

// Arrive at the grid barrier of step s and wait until all nb blocks arrived
// (counter >= s * nb).  Called by one thread; false on timeout / error.
// arrive = false (test injection only) waits without arriving, so every
// block's bounded wait runs out.
GF_DEV bool grid_arrive_wait(unsigned* bar, unsigned target, int* err, uint64_t limit_ns,
                             bool arrive) {
  if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
  uint64_t t0 = 0;
  while (true) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
    if (v >= target) return true;
    if (*(volatile int*)err) return false;
    const uint64_t now = gf::globaltimer_ns();
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > limit_ns) {
      atomicExch(err, 1);
      return false;
    }
  }
}

__global__ void __launch_bounds__(kWarps * 32, 1)
k_pdhg_dense_persistent(const uint8_t* __restrict__ W2, int64_t ld, int64_t n, int64_t v0,
                        int64_t per, const float* __restrict__ qdiag, float qscale, float* x0,
                        float* x1, float* __restrict__ xbar, const float* __restrict__ chat,
                        float* __restrict__ dlast, GfIParam* iprm, int inst, int ninst,
                        long long k0, long long nsteps, GfDState* st, const GfSched* sc,
                        const double* normQ, const int32_t* cap, unsigned* bar,
                        uint64_t limit_ns, int skip_block) {
  extern __shared__ float4 sm4[];
  float* xs = reinterpret_cast<float*>(sm4);                          // [2][ld]
  const uint32_t* Ws = reinterpret_cast<const uint32_t*>(xs + 2 * ld);  // my rows, int8
  __shared__ GfIParam qsm[2];
  __shared__ float chat_s[kMaxRows], qd_s[kMaxRows];
  __shared__ double rho_s;
  __shared__ int n_rho_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = (r0 + per < n) ? r0 + per : n;
  // the host launches ceil(n / per) blocks, so every block owns >= 1 row
  {
    uint4* dst = reinterpret_cast<uint4*>(xs + 2 * ld);
    const uint4* src = reinterpret_cast<const uint4*>(W2 + r0 * ld);
    const int64_t cnt = (r1 - r0) * ld / 16;
    for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) dst[e] = src[e];
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      chat_s[i - r0] = chat[v0 + i];
      qd_s[i - r0] = qdiag[i];
    }
  }
  const long long it0 = k0 + 1;
  if (threadIdx.x == kSchedThread) {
    n_rho_s = st->n_rho;
    rho_s = st->rho;
    qsm[0] = iprm[(size_t)(it0 & 1) * ninst + inst];
  }
  const int64_t nq = ld / 4;                      // 4-entry words per row
  const unsigned nb = gridDim.x;
  long long s = 0;
  for (; s < nsteps; ++s) {
    const long long it = it0 + s;
    bool ok = true;
    if (s > 0) {
      __syncthreads();                            // this block's rows of step s-1 written
      if (threadIdx.x == 0)
        ok = grid_arrive_wait(bar, (unsigned)s * nb, &st->error, limit_ns,
                              !(s == 1 && (int)blockIdx.x == skip_block));
    }
    if (__syncthreads_or(!ok)) break;
    // x_{it-1} into shared memory (padding entries are zero, never written)
    float* xsb = xs + (s & 1) * ld;
    float4* xs4 = reinterpret_cast<float4*>(xsb);
    const float* xo = (it & 1) ? x0 : x1;         // x_{it-1} in x[(it-1) & 1]
    for (int64_t j4 = threadIdx.x; j4 < nq; j4 += blockDim.x)
      xs4[j4] = __ldcg(reinterpret_cast<const float4*>(xo + v0) + j4);
    __syncthreads();                              // x and q of this step published
    const GfIParam q = qsm[s & 1];
    float* xn = (it & 1) ? x1 : x0;               // x_it in x[it & 1]
    for (int64_t i = r0 + warp; i < r1; i += kWarps) {
      CSum acc = gf::i8_row_dot(Ws + (i - r0) * nq, xs4, nq, lane);
      gf::csum_group_reduce<32>(acc);
      if (lane == 0) {
        const float xo_i = xsb[i];
        CSum sq;                                  // 2 (Q_hat x)_i
        sq.merge(__fmul_rn(2.0f * qscale, acc.s), __fmul_rn(2.0f * qscale, acc.c));
        sq.add(__fmul_rn(2.0f * qd_s[i - r0], xo_i));
        const float delta = chat_s[i - r0] + q.rho + sq.value() - 2.0f * q.rho * xo_i;
        const float xnew = fminf(1.0f, fmaxf(0.0f, xo_i - q.tau1 * delta));
        xn[v0 + i] = xnew;
        xbar[v0 + i] = 2.0f * xnew - xo_i;
        if (dlast) dlast[v0 + i] = q.tau1 * delta;
      }
    }
    if (threadIdx.x == kSchedThread) {
      // UpdatePenalty for iteration it+1: the counter advances once per k_int
      // iterations; only then are rho and the step sizes recomputed
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
        qsm[(s + 1) & 1] = step_params(sc->sigma, normQ[inst], cap[inst], rho);
      } else {
        qsm[(s + 1) & 1] = q;
      }
    }
  }
  // device state after the last completed iteration (one block writes it)
  if (blockIdx.x == 0 && threadIdx.x == kSchedThread && s > 0) {
    const long long last = it0 + s - 1;
    st->k = last;
    st->n_rho = n_rho_s;
    st->rho = rho_s;
    iprm[(size_t)(last & 1) * ninst + inst] = qsm[(s - 1) & 1];
    iprm[(size_t)((last + 1) & 1) * ninst + inst] = qsm[s & 1];
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
  const size_t smem = 2 * sizeof(float) * (size_t)dq.ld + (size_t)per * dq.ld;
  if (smem > 200 * 1024 || per > kMaxRows) return false;
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
  h->persist_per = per;
  h->persist_grid = (int)((dq.n + per - 1) / per);
  h->persist_bar = gf_alloc_t<unsigned>(h, 1);   // grid-barrier counter
  return h->persist_bar != nullptr;
}

// nsteps iterations starting after iteration h->k_host (one launch).
cudaError_t gf_launch_persistent(GfCtx* h, int64_t nsteps) {
  const GfDenseQ& dq = h->dense[0];
  const GfInstHost& I = h->ih[dq.inst];
  cudaError_t e = cudaMemsetAsync(h->persist_bar, 0, sizeof(unsigned), h->stream);
  if (e) return e;
  const uint8_t* W2 = dq.W2i8;
  int64_t ld = dq.ld, n = dq.n, v0 = I.var_off, per = h->persist_per;
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
  int skip = h->inject_skip_block;
  h->inject_skip_block = -1;
  void* args[] = {&W2, &ld, &n, &v0, &per, &qdiag, &qscale, &x0, &x1, &xbar, &chat, &dlast,
                  &iprm, &inst, &ninst, &k0, &ns, &st, &sc, &nq, &cap, &bar, &limit, &skip};
  e = cudaLaunchCooperativeKernel((const void*)k_pdhg_dense_persistent, dim3(h->persist_grid),
                                  dim3(kWarps * 32), args, h->persist_smem, h->stream);
  h->launches += 2;
  return e;
}
