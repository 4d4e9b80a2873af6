// penalty.cuh -- UpdatePenalty on the device, shared by the PDHG kernels.
#pragma once
#include "common.cuh"

// UpdatePenalty for iteration k+1 (penalty counter advances once per k_int
// iterations), then the per-instance step sizes (tau1 = sqrt(sigma), capped
// at 1/(2L) with L = 2(||Q_hat|| + rho) when requested; tau2 = sigma/tau1).
// Executed by all threads of one block; `next` is the slot to write.
__device__ __forceinline__ void advance_penalty(GfDState* st, const GfSched* sc,
                                                const double* normQ, const int32_t* cap,
                                                const GfIParam* cur, GfIParam* next) {
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

// Step sizes of one instance for penalty rho (tau1 = min(sqrt(sigma), 1/(2L))
// when capped, tau2 = sigma / tau1), the per-instance half of advance_penalty
// for kernels that advance the schedule themselves.
__device__ __forceinline__ GfIParam step_params(double sigma, double normQ, int cap,
                                                double rho) {
  double t1 = sqrt(sigma);
  if (cap) {
    double L = 2.0 * (normQ + rho);
    if (L > 0.0 && 1.0 / (2.0 * L) < t1) t1 = 1.0 / (2.0 * L);
  }
  double t2 = sigma / t1;
  GfIParam q;
  q.tau1 = (float)t1; q.tau2 = (float)t2; q.rho = (float)rho; q.pad = 0.f;
  q.tau1d = t1; q.tau2d = t2; q.rhod = rho; q.normQ = normQ;
  return q;
}
