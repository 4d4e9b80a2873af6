// gfors_api.cu -- the GFORS loop (Alg. 1) around the device kernels, and
// the state-access entry points of gfors.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>

#include "internal.cuh"

void gf_set_slot(GfCtx* h, int parity, double rho);
cudaError_t gf_launch_dense_score(GfCtx* h, const GfDenseQ& dq, int s0, int len);

#define GF_ENTER(h)                                                          \
  do {                                                                       \
    if (!(h)) return GFORS_E_ARG;                                            \
    if ((h)->failed) return GFORS_E_STATE;                                   \
  } while (0)

namespace {

// bytes (sample-major k x n) -> variable-major bits for one instance
__global__ void k_pack_bits(const uint8_t* __restrict__ Xb, int k, int64_t n, int64_t v0,
                            int kws, uint32_t* __restrict__ X) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int kwu = (k + 31) / 32;
  if (gid >= n * kwu) return;
  const int64_t i = gid / kwu;
  const int w = (int)(gid % kwu);
  uint32_t m = 0;
  for (int t = 0; t < 32; ++t) {
    const int s = 32 * w + t;
    if (s < k && Xb[(int64_t)s * n + i]) m |= 1u << t;
  }
  X[(v0 + i) * kws + w] = m;
}

__global__ void k_unpack_bits(const uint32_t* __restrict__ X, int k, int64_t n, int64_t v0,
                              int kws, uint8_t* __restrict__ Xb) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= n * (int64_t)k) return;
  const int s = (int)(gid / n);
  const int64_t i = gid % n;
  Xb[gid] = (X[(v0 + i) * kws + (s >> 5)] >> (s & 31)) & 1u;
}

// Dense-Q candidate operand element: bf16 1.0 = 0x3F80, FP8 E4M3 1.0 = 0x38.
__device__ __forceinline__ void put_cand(void* Xs, int64_t idx, bool one, int f8) {
  if (f8) reinterpret_cast<uint8_t*>(Xs)[idx] = one ? 0x38u : 0u;
  else reinterpret_cast<uint16_t*>(Xs)[idx] = one ? 0x3F80u : 0u;
}

__global__ void k_pack_dense(const uint8_t* __restrict__ Xb, int k, int64_t n, int64_t ld,
                             void* __restrict__ Xs, int f8) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)k * ld) return;
  const int s = (int)(gid / ld);
  const int64_t i = gid % ld;
  put_cand(Xs, gid, i < n && Xb[(int64_t)s * n + i], f8);
}

// candidate bytes from the bit words Xb[s * ld/32 + w]
__global__ void k_unpack_dense(const uint32_t* __restrict__ Xw, int k, int64_t n, int64_t ld,
                               uint8_t* __restrict__ Xb) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)k * n) return;
  const int s = (int)(gid / n);
  const int64_t i = gid % n;
  Xb[gid] = (Xw[(int64_t)s * (ld / 32) + i / 32] >> (i & 31)) & 1u;
}

// round(x_k) as candidate 0 (bits and dense operands)
__global__ void k_round_bits(const float* __restrict__ x, const uint8_t* __restrict__ live,
                             int64_t N, int kws, uint32_t* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  X[i * kws] = (live[i] && x[i] > 0.5f) ? 1u : 0u;
}
__global__ void k_round_dense(const float* __restrict__ x, int64_t v0, int64_t n, int64_t ld,
                              void* __restrict__ Xs, int f8) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ld) return;
  put_cand(Xs, i, i < n && x[v0 + i] > 0.5f, f8);
}
__global__ void k_set_round(GfDState* st, unsigned v) { st->round_id = v; }
// proposal 3: after the plain round (which advanced the id to r + 1), the
// network's round takes id r | 2^31; after it (id (r | 2^31) + 1) the plain
// sequence resumes at r + 1.  Done on the device so a captured trigger
// replays with the right ids.
__global__ void k_round_to_learned(GfDState* st) {
  st->round_id = (st->round_id - 1u) | 0x80000000u;
}
__global__ void k_round_to_plain(GfDState* st) { st->round_id &= 0x7FFFFFFFu; }

__global__ void k_x0_random(float* __restrict__ x, const int32_t* __restrict__ var_inst,
                            const int64_t* __restrict__ var_off, const uint8_t* __restrict__ live,
                            int64_t N, uint64_t seed, int inst_base) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (!live[i]) { x[i] = 0.0f; return; }
  const int b = var_inst[i];
  const int64_t loc = i - var_off[b];
  const uint4 u = gf::philox_call(seed, gf::kStreamX0, (uint32_t)(inst_base + b), 0u, 0u,
                                  (uint64_t)(loc >> 2));
  x[i] = (float)(gf::lane_of(u, (uint32_t)(loc & 3)) >> 8) * (1.0f / 16777216.0f);
}

}  // namespace

cudaError_t gf_launch_x0_random(GfCtx* h) {
  k_x0_random<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(
      h->x[0], h->var_inst, h->var_off_d, h->var_live, h->N, h->prm.seed, h->prm.inst_base);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// phase profiling
static cudaEvent_t prof_event(GfCtx* h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int gf_prof_begin(GfCtx* h, int phase) {
  if (!h->prof) return -1;
  GfCtx::ProfRec r{phase, 0, prof_event(h), prof_event(h)};
  cudaEventRecord(r.a, h->stream);
  h->prof_recs.push_back(r);
  return (int)h->prof_recs.size() - 1;
}

void gf_prof_end(GfCtx* h, int idx, int count) {
  if (idx < 0) return;
  h->prof_recs[idx].count = count;
  cudaEventRecord(h->prof_recs[idx].b, h->stream);
}

static void prof_clear(GfCtx* h) {
  for (auto& r : h->prof_recs) {
    h->prof_pool.push_back(r.a);
    h->prof_pool.push_back(r.b);
  }
  h->prof_recs.clear();
}

extern "C" gfors_status gfors_profile(gfors_handle h, int32_t enable) {
  GF_ENTER(h);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "profile sync");
  prof_clear(h);
  h->prof = enable != 0;
  return GFORS_OK;
}

extern "C" gfors_status gfors_profile_read(gfors_handle h, int32_t nphases, double* ms,
                                           int64_t* counts) {
  GF_ENTER(h);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "profile sync");
  for (int q = 0; q < nphases; ++q) {
    if (ms) ms[q] = 0.0;
    if (counts) counts[q] = 0;
  }
  for (auto& r : h->prof_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { cudaGetLastError(); continue; }
    if (r.phase < nphases) {
      if (ms) ms[r.phase] += t;
      if (counts) counts[r.phase] += r.count;
    }
  }
  return GFORS_OK;
}

// After a synchronisation: a device wait that ran out of time left an error
// in the device state; the handle becomes failed.
static gfors_status check_device_error(GfCtx* h) {
  int err = 0;
  cudaError_t e = cudaMemcpy(&err, &h->dstate->error, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return gf_cuda(h, e, "device state");
  if (err) return gf_fail(h, GFORS_E_TIMEOUT, "a bounded device-side wait gave up");
  return GFORS_OK;
}

// ---------------------------------------------------------------------------
// host mirror of UpdatePenalty (same recursion as the device)
static void host_advance(GfCtx* h, long long it) {
  const gfors_params& P = h->prm;
  const int n_next = (int)(it / P.k_int);
  while (h->n_rho_host < n_next) {
    h->n_rho_host++;
    double rt = P.rho_min * pow(1.0 + (double)h->n_rho_host / P.T, P.p);
    double lo = h->rho_host + P.delta;
    double v = rt < lo ? lo : rt;
    h->rho_host = v > P.rho_max ? P.rho_max : v;
  }
}

cudaError_t gf_launch_persistent(GfCtx* h, int64_t nsteps);

cudaError_t gf_single_init(GfCtx* h);
cudaError_t gf_launch_small(GfCtx* h, int64_t nsteps);
cudaError_t gf_launch_coop(GfCtx* h, int64_t nsteps);

static cudaError_t enqueue_steps(GfCtx* h, int64_t nsteps) {
  cudaError_t e;
  int64_t done = 0;
  if (h->single_ok && !h->sr_valid && nsteps > 0) {
    // K xbar partials of the current state, read by the next dual step
    if ((e = gf_single_init(h))) return e;
    h->sr_valid = true;
  }
  if ((h->small_ok || h->coop_ok) && nsteps > 0) {
    // one launch: every instance's iterations in its own block (small), or
    // the whole batch as one cooperative grid (L2-resident)
    while (done < nsteps) {
      const int64_t cnt = std::min<int64_t>(nsteps - done, (int64_t)1 << 20);
      const int pi = gf_prof_begin(h, 0);
      if ((e = h->small_ok ? gf_launch_small(h, cnt) : gf_launch_coop(h, cnt))) return e;
      gf_prof_end(h, pi, (int)cnt);
      for (int64_t s = 0; s < cnt; ++s) host_advance(h, h->k_host + 1 + s);
      h->k_host += cnt;
      done += cnt;
    }
    return cudaSuccess;
  }
  if (h->persist_ok && nsteps > 0) {
    // one cooperative launch runs all nsteps iterations
    // (at most 2^20 iterations per launch keeps the barrier counter in range)
    while (done < nsteps) {
      const int64_t cnt = std::min<int64_t>(nsteps - done, (int64_t)1 << 20);
      const int pi = gf_prof_begin(h, 0);
      if ((e = gf_launch_persistent(h, cnt))) return e;
      gf_prof_end(h, pi, (int)cnt);
      for (int64_t s = 0; s < cnt; ++s) host_advance(h, h->k_host + 1 + s);
      h->k_host += cnt;
      done += cnt;
    }
    return cudaSuccess;
  }
  // light pairs while more than two iterations remain
  while (h->use_graphs && nsteps - done >= 3) {
    const int p = (int)((h->k_host + 1) & 1);
    if (h->capturing) {
      // inside the capture of a whole trigger (no nested capture, no graph
      // launch): the pair's two light iterations as direct launches
      h->light_iter = true;
      e = gf_launch_pdhg_iter(h, p);
      if (e == cudaSuccess) e = gf_launch_pdhg_iter(h, 1 - p);
      h->light_iter = false;
      if (e) return e;
      host_advance(h, h->k_host + 1);
      host_advance(h, h->k_host + 2);
      h->k_host += 2;
      done += 2;
      continue;
    }
    if (!h->g_light2[p]) {
      cudaGraph_t g;
      if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal))) return e;
      long long saved = h->launches;
      h->light_iter = true;
      cudaError_t e1 = gf_launch_pdhg_iter(h, p);
      cudaError_t e2 = (e1 == cudaSuccess) ? gf_launch_pdhg_iter(h, 1 - p) : e1;
      h->light_iter = false;
      h->pair_launches = h->launches - saved;
      h->launches = saved;
      e = cudaStreamEndCapture(h->stream, &g);
      if (e2 != cudaSuccess) return e2;
      if (e) return e;
      e = cudaGraphInstantiate(&h->g_light2[p], g, 0);
      cudaGraphDestroy(g);
      if (e) return e;
    }
    const int pi = gf_prof_begin(h, 0);
    if ((e = cudaGraphLaunch(h->g_light2[p], h->stream))) return e;
    gf_prof_end(h, pi, 2);
    h->launches += h->pair_launches;
    host_advance(h, h->k_host + 1);
    host_advance(h, h->k_host + 2);
    h->k_host += 2;
    done += 2;
  }
  // replay a captured pair of iterations while at least two remain
  while (h->use_graphs && nsteps - done >= 2) {
    const int p = (int)((h->k_host + 1) & 1);   // parity of the first iteration
    if (h->capturing) {                          // as above, full iterations
      e = gf_launch_pdhg_iter(h, p);
      if (e == cudaSuccess) e = gf_launch_pdhg_iter(h, 1 - p);
      if (e) return e;
      host_advance(h, h->k_host + 1);
      host_advance(h, h->k_host + 2);
      h->k_host += 2;
      done += 2;
      continue;
    }
    if (!h->g_iter2[p]) {
      cudaGraph_t g;
      if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal))) return e;
      long long saved = h->launches;
      cudaError_t e1 = gf_launch_pdhg_iter(h, p);
      cudaError_t e2 = (e1 == cudaSuccess) ? gf_launch_pdhg_iter(h, 1 - p) : e1;
      h->pair_launches = h->launches - saved;
      h->launches = saved;
      e = cudaStreamEndCapture(h->stream, &g);
      if (e2 != cudaSuccess) return e2;
      if (e) return e;
      e = cudaGraphInstantiate(&h->g_iter2[p], g, 0);
      cudaGraphDestroy(g);
      if (e) return e;
    }
    const int pi = gf_prof_begin(h, 0);
    if ((e = cudaGraphLaunch(h->g_iter2[p], h->stream))) return e;
    gf_prof_end(h, pi, 2);
    h->launches += h->pair_launches;
    host_advance(h, h->k_host + 1);
    host_advance(h, h->k_host + 2);
    h->k_host += 2;
    done += 2;
  }
  for (; done < nsteps; ++done) {
    const long long it = h->k_host + 1;
    const int pi = gf_prof_begin(h, 0);
    if ((e = gf_launch_pdhg_iter(h, (int)(it & 1)))) return e;
    gf_prof_end(h, pi, 1);
    host_advance(h, it);
    h->k_host = it;
  }
  return cudaSuccess;
}

extern "C" gfors_status gfors_pdhg_steps(gfors_handle h, int64_t nsteps) {
  GF_ENTER(h);
  if (nsteps < 0) return gf_fail(h, GFORS_E_ARG, "nsteps < 0");
  cudaError_t e = enqueue_steps(h, nsteps);
  if (e != cudaSuccess) return gf_cuda(h, e, "gfors_pdhg_steps");
  return GFORS_OK;
}

// One round: candidates [sb, se) of the round's k_b (processed in chunks);
// candidates below `split` are drawn from p_a, the others from p_b (split =
// k_b: a single proposal).  Candidate indices are global within the round, so
// disjoint ranges of one round (on several devices) draw exactly the
// candidates of the whole round.
static cudaError_t enqueue_round(GfCtx* h, const float* p_a, const float* p_b, int split,
                                 int sb, int se) {
  const int kb = se;
  cudaError_t e;
  for (int s0 = sb; s0 < kb;) {
    const int seg_end = (s0 < split) ? std::min(split, kb) : kb;
    const float* p = (s0 < split) ? p_a : p_b;
    const int len = std::min(h->chunk, seg_end - s0);
    const bool last = (s0 + len >= kb);
    h->last_p = p;
    h->last_s0 = s0;
    h->last_chunk_len = len;
    h->last_round = h->host_round;
    int pi;
    if (h->fused_ok) {
      pi = gf_prof_begin(h, 5);
      if ((e = gf_launch_fused(h, p, s0, len))) return e;
      gf_prof_end(h, pi, 1);
      h->last_mode = 1;
      pi = gf_prof_begin(h, 4);
      if ((e = gf_launch_incumbent(h, s0, len, 1, last))) return e;
      gf_prof_end(h, pi, 1);
    } else {
      pi = gf_prof_begin(h, 1);
      bool pick_obj = false;
      if ((e = gf_launch_sample(h, p, s0, len, !h->dense.empty(), &pick_obj))) return e;
      gf_prof_end(h, pi, 1);
      pi = gf_prof_begin(h, 2);
      if ((e = gf_launch_eval(h, s0, len, pick_obj))) return e;
      gf_prof_end(h, pi, 1);
      for (const GfDenseQ& dq : h->dense) {
        pi = gf_prof_begin(h, 3);
        if ((e = gf_launch_dense_score(h, dq, s0, len))) return e;
        gf_prof_end(h, pi, 1);
      }
      h->last_mode = 0;
      pi = gf_prof_begin(h, 4);
      if ((e = gf_launch_incumbent(h, s0, len, 0, last))) return e;
      gf_prof_end(h, pi, 1);
    }
    s0 += len;
  }
  return cudaSuccess;
}

static gfors_status sample_rounds(GfCtx* h, int32_t nrounds, int32_t proposal, int sb,
                                  int se) {
  if (!h->all_integral)
    return gf_fail(h, GFORS_E_UNSUPPORTED,
                   "exact evaluation needs integral data (|value| < 2^31)");
  if (proposal != 0 && !h->mlp_W)
    return gf_fail(h, GFORS_E_STATE, "learned proposal requested but none attached");
  cudaError_t e;
  const float* xk = h->x[h->k_host & 1];
  // the group samplers' cumulative weights depend on p alone, which stays
  // fixed for the whole call: each source's weights are formed once
  if (!h->capturing && (e = gf_ensure_pick_obj(h))) return gf_cuda(h, e, "pick objective tables");
  struct CwCache {
    GfCtx* h;
    explicit CwCache(GfCtx* c) : h(c) {
      h->cw_src[0] = h->cw_src[1] = nullptr;
      h->cw_cache = true;
    }
    ~CwCache() { h->cw_cache = false; }
  } cw_cache(h);
  if (proposal != 0 && nrounds > 0) {
    // features of this trigger, then the network's probabilities
    if ((e = gf_launch_features(h))) return gf_cuda(h, e, "features");
    if ((e = gf_launch_mlp_proposal(h))) return gf_cuda(h, e, "learned proposal");
  }
  const int kb = h->prm.k_b;
  if (proposal == 3) {
    // every round twice: from x_k under its own id (the candidates of
    // proposal 0), then from the network under id | 2^31 (disjoint Philox
    // counters); the plain sampler stays complete in every round
    for (int r = 0; r < nrounds; ++r) {
      const unsigned rid = h->host_round;
      if ((e = enqueue_round(h, xk, xk, kb, sb, se))) return gf_cuda(h, e, "sampling round");
      k_round_to_learned<<<1, 1, 0, h->stream>>>(h->dstate);
      h->host_round = rid | 0x80000000u;
      if ((e = enqueue_round(h, h->p_learn, xk, kb, sb, se)))
        return gf_cuda(h, e, "sampling round");
      k_round_to_plain<<<1, 1, 0, h->stream>>>(h->dstate);
      h->host_round = rid + 1;
      h->launches += 2;
    }
    return GFORS_OK;
  }
  // proposal 2: first half of every round from the network, second half
  // from x_k (rounded to the 32-candidate word)
  const int split = (proposal == 2) ? std::max(32, (kb / 2) / 32 * 32) : kb;
  for (int r = 0; r < nrounds; ++r) {
    const float* pa = (proposal == 0) ? xk : h->p_learn;
    if ((e = enqueue_round(h, pa, xk, split, sb, se))) return gf_cuda(h, e, "sampling round");
    h->host_round++;
  }
  return GFORS_OK;
}

extern "C" gfors_status gfors_sample_eval(gfors_handle h, int32_t nrounds,
                                          uint32_t first_round_id, int32_t proposal) {
  GF_ENTER(h);
  if (nrounds < 0 || proposal < 0 || proposal > 3)
    return gf_fail(h, GFORS_E_ARG, "bad nrounds / proposal");
  k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, first_round_id);
  h->launches++;
  h->host_round = first_round_id;
  return sample_rounds(h, nrounds, proposal, 0, h->prm.k_b);
}

extern "C" gfors_status gfors_dense_info(gfors_handle h, int32_t inst, int64_t out[4]) {
  if (!h || !out || inst < 0 || inst >= h->ninst) return GFORS_E_ARG;
  out[0] = out[1] = out[2] = out[3] = 0;
  const GfInstHost& I = h->ih[inst];
  if (I.qkind == 1) {
    const GfDenseQ& dq = h->dense[I.dense_idx];
    out[0] = 1;
    out[1] = dq.tc_ok && h->prm.eval_mode != 4;
    out[2] = dq.f8;
    out[3] = dq.w2max;
  }
  return GFORS_OK;
}

extern "C" gfors_status gfors_pdhg_path(gfors_handle h, int32_t* path) {
  if (!h || !path) return GFORS_E_ARG;
  *path = h->persist_ok ? GFORS_PATH_PERSISTENT
        : (h->small_ok && h->cluster_C > 0) ? GFORS_PATH_CLUSTER
        : h->small_ok   ? GFORS_PATH_SMALL
        : h->coop_ok    ? GFORS_PATH_COOPERATIVE
        : h->single_ok  ? GFORS_PATH_ONE_ROW
                        : GFORS_PATH_BUCKETS;
  return GFORS_OK;
}

extern "C" gfors_status gfors_sample_eval_range(gfors_handle h, int32_t nrounds,
                                                uint32_t first_round_id, int32_t proposal,
                                                int32_t s_begin, int32_t s_end) {
  GF_ENTER(h);
  if (nrounds < 0 || proposal < 0 || proposal > 3)
    return gf_fail(h, GFORS_E_ARG, "bad nrounds / proposal");
  if (s_begin < 0 || s_end > h->prm.k_b || s_begin >= s_end || s_begin % 32 || s_end % 32)
    return gf_fail(h, GFORS_E_ARG, "need 0 <= s_begin < s_end <= k_b, multiples of 32");
  k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, first_round_id);
  h->launches++;
  h->host_round = first_round_id;
  return sample_rounds(h, nrounds, proposal, s_begin, s_end);
}

namespace {
__global__ void k_inc_key(const GfInc* __restrict__ inc, int q, long long* __restrict__ out) {
  const GfInc v = inc[q];
  out[0] = v.found ? v.obj : 0x7FFFFFFFFFFFFFFFll;
  out[1] = v.found ? (long long)v.round_id : 0x7FFFFFFFFFFFFFFFll;
  out[2] = v.found ? (long long)v.sample : 0x7FFFFFFFFFFFFFFFll;
}
}  // namespace

extern "C" gfors_status gfors_incumbent_key_async(gfors_handle h, int32_t inst,
                                                  int64_t* key_dev) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst || !key_dev) return gf_fail(h, GFORS_E_ARG, "bad inst / key");
  k_inc_key<<<1, 1, 0, h->stream>>>(h->inc, inst, reinterpret_cast<long long*>(key_dev));
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (e) return gf_cuda(h, e, "gfors_incumbent_key_async");
  return GFORS_OK;
}

extern "C" gfors_status gfors_incumbent_async(gfors_handle h, int32_t inst, int64_t* key_host) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst || !key_host) return gf_fail(h, GFORS_E_ARG, "bad inst / key");
  if (!h->key_stage) {
    h->key_stage = gf_alloc_t<long long>(h, 3 * (size_t)h->ninst);
    if (!h->key_stage) return gf_fail(h, GFORS_E_OOM, "key staging");
  }
  long long* kd = h->key_stage + 3 * (size_t)inst;
  k_inc_key<<<1, 1, 0, h->stream>>>(h->inc, inst, kd);
  h->launches++;
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(key_host, kd, 3 * sizeof(long long), cudaMemcpyDeviceToHost,
                              h->stream);
  if (e) return gf_cuda(h, e, "gfors_incumbent_async");
  return GFORS_OK;
}

extern "C" gfors_status gfors_debug_inject(gfors_handle h, int32_t kind, int32_t block) {
  GF_ENTER(h);
  if (kind == 0) {
    h->inject_skip_block = -1;
    return GFORS_OK;
  }
  if (kind != 1 || block < 0) return gf_fail(h, GFORS_E_ARG, "gfors_debug_inject: bad kind/block");
  h->inject_skip_block = block;
  return GFORS_OK;
}

extern "C" gfors_status gfors_synchronize(gfors_handle h) {
  GF_ENTER(h);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "gfors_synchronize");
  return GFORS_OK;
}

static cudaError_t enqueue_final_round(GfCtx* h) {
  cudaError_t e;
  const float* xk = h->x[h->k_host & 1];
  k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, 0xFFFFFFFFu);
  h->last_round = 0xFFFFFFFFu;
  k_round_bits<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(xk, h->var_live, h->N,
                                                                     h->kw, h->X);
  for (const GfDenseQ& dq : h->dense)
  {
    k_round_dense<<<(unsigned)((dq.ld + 255) / 256), 256, 0, h->stream>>>(
        xk, h->ih[dq.inst].var_off, dq.n, dq.ld, dq.Xs, (int)dq.f8);
    k_dense_bits<<<(unsigned)((dq.ld / 32 + 255) / 256), 256, 0, h->stream>>>(dq.Xs, 1, dq.ld,
                                                                               dq.Xb, (int)dq.f8);
  }
  h->launches += 2 + (long long)h->dense.size();
  if ((e = gf_launch_eval(h, 0, 1))) return e;
  for (const GfDenseQ& dq : h->dense)
    if ((e = gf_launch_dense_score(h, dq, 0, 1))) return e;
  h->last_mode = 0;
  h->last_s0 = 0;
  h->last_chunk_len = 1;
  if ((e = gf_launch_incumbent(h, 0, 1, 0, false))) return e;
  k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, h->host_round);
  return cudaGetLastError();
}

extern "C" gfors_status gfors_final_round(gfors_handle h) {
  GF_ENTER(h);
  if (!h->all_integral)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "exact evaluation needs integral data");
  cudaError_t e = enqueue_final_round(h);
  if (e) return gf_cuda(h, e, "gfors_final_round");
  return GFORS_OK;
}

// CheckHalt (Section 3), host side, on the device's FP64 sums.
static void stats_of(GfCtx* h, int b, const double* s1, const double* s2, double* out) {
  const GfInstHost& I = h->ih[b];
  const double pres = sqrt(s1[0]) / (1.0 + sqrt(s1[1]));
  const double pobj = s2[3] + s2[4];
  const double D = s1[2] + s2[6];
  const double sx = sqrt(s2[7]);
  out[0] = pres;
  out[1] = (I.qkind == 0) ? fabs(pobj - D) / (1.0 + fabs(pobj) + fabs(D)) : sx;
  out[2] = s2[5] / (double)I.n;
  out[3] = pobj;
  out[4] = (I.qkind == 0) ? D : NAN;
  out[5] = sx;
  out[6] = h->rho_host;
  out[7] = (double)h->k_host;
}

static gfors_status fetch_stats(GfCtx* h, std::vector<double>& out) {
  cudaError_t e = gf_launch_stats(h);
  if (e) return gf_cuda(h, e, "stats");
  std::vector<double> a(8 * h->ninst), b2(8 * h->ninst);
  if ((e = cudaMemcpyAsync(a.data(), h->stats, sizeof(double) * 8 * h->ninst,
                           cudaMemcpyDeviceToHost, h->stream)))
    return gf_cuda(h, e, "stats copy");
  if ((e = cudaMemcpyAsync(b2.data(), h->stats2, sizeof(double) * 8 * h->ninst,
                           cudaMemcpyDeviceToHost, h->stream)))
    return gf_cuda(h, e, "stats copy");
  if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "stats sync");
  if (gfors_status ds = check_device_error(h)) return ds;
  out.assign(8 * h->ninst, 0.0);
  for (int b = 0; b < h->ninst; ++b) stats_of(h, b, &a[8 * b], &b2[8 * b], &out[8 * b]);
  return GFORS_OK;
}

extern "C" gfors_status gfors_lp_stats(gfors_handle h, int32_t inst, double out[8]) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst || !out) return gf_fail(h, GFORS_E_ARG, "bad instance");
  std::vector<double> v;
  gfors_status st = fetch_stats(h, v);
  if (st) return st;
  memcpy(out, &v[8 * inst], sizeof(double) * 8);
  return GFORS_OK;
}

// value-stalling detector: indicator q of instance b is done when <= tol or
// its best value has not improved by 1e-3 (relative) for stall_window triggers
static bool halt_update(GfCtx* h, const std::vector<double>& st) {
  h->h_trig++;
  bool all = true;
  for (int b = 0; b < h->ninst; ++b) {
    bool done = true;
    for (int q = 0; q < 3; ++q) {
      const double v = st[8 * b + q];
      double& best = h->h_best[3 * b + q];
      long long& last = h->h_last[3 * b + q];
      if (std::isinf(best) || v < best * (1.0 - 1e-3)) { best = v; last = h->h_trig; }
      done &= (v <= h->prm.halt_tol) || (h->h_trig - last >= h->prm.stall_window);
    }
    all &= done;
  }
  return all;
}

extern "C" gfors_status gfors_run(gfors_handle h, int64_t max_iters, double time_budget_s,
                                  int32_t proposal, int64_t* iters_out) {
  GF_ENTER(h);
  if (max_iters < 0 || proposal < 0 || proposal > 3)
    return gf_fail(h, GFORS_E_ARG, "bad max_iters / proposal");
  const auto t0 = std::chrono::steady_clock::now();
  const int kint = h->prm.k_int;
  gfors_status st;
  while (h->k_host < max_iters) {
    int64_t to_trig = kint - (h->k_host % kint);
    int64_t n = std::min<int64_t>(to_trig, max_iters - h->k_host);
    cudaError_t e = enqueue_steps(h, n);
    if (e) return gf_cuda(h, e, "gfors_run steps");
    if (h->k_host % kint == 0) {
      const long long trig = h->k_host / kint - 1;
      k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, (unsigned)(trig * h->prm.k_r));
      h->host_round = (unsigned)(trig * h->prm.k_r);
      if ((st = sample_rounds(h, h->prm.k_r, proposal, 0, h->prm.k_b))) return st;
      std::vector<double> sv;
      if ((st = fetch_stats(h, sv))) return st;
      if (halt_update(h, sv)) break;
    }
    if (time_budget_s > 0.0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > time_budget_s) break;
    }
  }
  if ((st = gfors_final_round(h))) return st;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "gfors_run sync");
  if (iters_out) *iters_out = h->k_host;
  return GFORS_OK;
}

// ---------------------------------------------------------------------------
// Alg. 1 as one CUDA-graph launch: the body of a while node is one trigger
// (k_int iterations, k_r rounds, the FP64 CheckHalt sums) and ends with the
// halt kernel, which evaluates CheckHalt (the host loop's halt_update, same
// FP64 formulas and stall rule), the trigger budget and the optional
// objective targets, and sets the loop's condition.  Everything that
// differs between runs (budget, first trigger, targets) lives in device
// memory, so one instantiated graph per proposal serves every run of the
// handle until its structure changes.
namespace {
__global__ void k_trigger_round(GfDState* st, const long long* ctl, int kr) {
  st->round_id = (unsigned)((ctl[4] + ctl[0]) * (long long)kr);
}

__global__ void k_halt_step(const double* __restrict__ s_rows, const double* __restrict__ s_vars,
                            const int32_t* __restrict__ nvar, const int32_t* __restrict__ qk,
                            double* best, long long* last, long long* ctl,
                            const long long* __restrict__ tgt, const GfInc* __restrict__ inc,
                            int ninst, double tol, int window,
                            cudaGraphConditionalHandle cond) {
  __shared__ int all_done, all_hit;
  const bool use_tgt = ctl[5] != 0;
  if (threadIdx.x == 0) {
    all_done = 1;
    all_hit = use_tgt ? 1 : 0;
  }
  __syncthreads();
  const long long t = ctl[1] + 1;               // CheckHalt trigger count
  for (int b = threadIdx.x; b < ninst; b += blockDim.x) {
    const double* s1 = s_rows + 8 * b;
    const double* s2 = s_vars + 8 * b;
    double v[3];
    v[0] = sqrt(s1[0]) / (1.0 + sqrt(s1[1]));
    const double pobj = s2[3] + s2[4], D = s1[2] + s2[6], sx = sqrt(s2[7]);
    v[1] = (qk[b] == 0) ? fabs(pobj - D) / (1.0 + fabs(pobj) + fabs(D)) : sx;
    v[2] = s2[5] / (double)nvar[b];
    bool done = true;
    for (int q = 0; q < 3; ++q) {
      double& bq = best[3 * b + q];
      long long& lq = last[3 * b + q];
      if (isinf(bq) || v[q] < bq * (1.0 - 1e-3)) {
        bq = v[q];
        lq = t;
      }
      done &= (v[q] <= tol) || (t - lq >= window);
    }
    if (!done) all_done = 0;
    if (use_tgt && !(inc[b].found && inc[b].obj <= tgt[b])) all_hit = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[1] = t;
    const long long ran = ctl[0] + 1;
    ctl[0] = ran;
    const long long reason = all_done ? 1 : all_hit ? 2 : (ran >= ctl[3] ? 0 : -1);
    ctl[2] = reason;
    cudaGraphSetConditional(cond, reason < 0 ? 1u : 0u);
  }
}
}  // namespace

// Checks and lazy state shared by the build and the run of the graph.
static gfors_status run_graph_ready(GfCtx* h, int32_t proposal) {
  if (proposal < 0 || proposal > 3) return gf_fail(h, GFORS_E_ARG, "bad proposal");
  if (!h->all_integral)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "exact evaluation needs integral data");
  if (proposal != 0 && !h->mlp_W)
    return gf_fail(h, GFORS_E_STATE, "learned proposal requested but none attached");
  if (h->prm.k_int % 2 != 0 || h->k_host % h->prm.k_int != 0)
    return gf_fail(h, GFORS_E_UNSUPPORTED,
                   "gfors_run_graph needs an even k_int and k at a trigger boundary");
  if (h->persist_ok || h->coop_ok)
    return gf_fail(h, GFORS_E_UNSUPPORTED,
                   "gfors_run_graph: cooperative PDHG launches are not captured; use gfors_run");
  cudaStream_t s = h->stream;
  cudaError_t e;
  // everything a trigger allocates, uploads or synchronises on, done first
  if (h->single_ok && !h->sr_valid) {
    if ((e = gf_single_init(h))) return gf_cuda(h, e, "one-row init");
    h->sr_valid = true;
  }
  if (proposal != 0 && (e = gf_prepare_features(h))) return gf_cuda(h, e, "feature buffers");
  if ((e = gf_ensure_pick_obj(h))) return gf_cuda(h, e, "pick objective tables");
  if (!h->fused_ok && (e = gf_ensure_bit_list(h))) return gf_cuda(h, e, "sampling list");
  const int nb = h->ninst;
  if (!h->halt_ctl) {
    h->halt_n = gf_alloc_t<int32_t>(h, nb);
    h->halt_q = gf_alloc_t<int32_t>(h, nb);
    h->halt_best = gf_alloc_t<double>(h, 3 * nb);
    h->halt_last = gf_alloc_t<long long>(h, 3 * nb);
    h->halt_tgt = gf_alloc_t<long long>(h, nb);
    h->halt_ctl = gf_alloc_t<long long>(h, 6);
    if (!h->halt_n || !h->halt_q || !h->halt_best || !h->halt_last || !h->halt_tgt ||
        !h->halt_ctl)
      return gf_fail(h, GFORS_E_OOM, "halt state");
    std::vector<int32_t> nv(nb), qv(nb);
    for (int b = 0; b < nb; ++b) {
      nv[b] = (int32_t)h->ih[b].n;
      qv[b] = h->ih[b].qkind;
    }
    if ((e = cudaMemcpyAsync(h->halt_n, nv.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaMemcpyAsync(h->halt_q, qv.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice,
                             s)) ||
        (e = cudaStreamSynchronize(s)))
      return gf_cuda(h, e, "halt constants");
  }
  return GFORS_OK;
}

// Capture one trigger into the body of a while node and instantiate it
// (cached per proposal until the handle's structure changes).
static gfors_status run_graph_build(GfCtx* h, int32_t proposal) {
  GfCtx::RunGraph& rg = h->run_graph[proposal];
  if (rg.exec && rg.sv == h->struct_version && rg.gv == h->grp_version) return GFORS_OK;
  if (rg.exec) {
    cudaGraphExecDestroy(rg.exec);
    rg.exec = nullptr;
  }
  cudaStream_t s = h->stream;
  const int kint = h->prm.k_int, kr = h->prm.k_r;
  const long long k0 = h->k_host;
  const int n_rho0 = h->n_rho_host;
  const double rho0 = h->rho_host;
  const long long l0 = h->launches;
  const unsigned hr0 = h->host_round;
  const bool prof0 = h->prof;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle hc;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e) return gf_cuda(h, e, "graph");
  e = cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  if (!e) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  gfors_status st = GFORS_OK;
  if (!e) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (!e) {
      h->capturing = true;
      h->prof = false;                  // no event nodes inside the body
      cudaError_t ec = enqueue_steps(h, kint);
      if (!ec) {
        k_trigger_round<<<1, 1, 0, s>>>(h->dstate, h->halt_ctl, kr);
        h->launches++;
        st = sample_rounds(h, kr, proposal, 0, h->prm.k_b);
      }
      if (!ec && st == GFORS_OK) ec = gf_launch_stats(h);
      if (!ec && st == GFORS_OK) {
        k_halt_step<<<1, 256, 0, s>>>(h->stats, h->stats2, h->halt_n, h->halt_q, h->halt_best,
                                      h->halt_last, h->halt_ctl, h->halt_tgt, h->inc, h->ninst,
                                      h->prm.halt_tol, h->prm.stall_window, hc);
        h->launches++;
        ec = cudaGetLastError();
      }
      h->capturing = false;
      h->prof = prof0;
      cudaGraph_t out = nullptr;
      cudaError_t ee = cudaStreamEndCapture(s, &out);
      e = ec ? ec : ee;
    }
  }
  rg.per_trig = h->launches - l0;
  // the capture advanced the host mirrors by one trigger: undo
  h->k_host = k0;
  h->n_rho_host = n_rho0;
  h->rho_host = rho0;
  h->launches = l0;
  h->host_round = hr0;
  if (!e && st == GFORS_OK) e = cudaGraphInstantiate(&rg.exec, g, 0);
  // upload now (set-up), so the first run does not pay for it
  if (!e && st == GFORS_OK) e = cudaGraphUpload(rg.exec, s);
  if (!e && st == GFORS_OK) e = cudaStreamSynchronize(s);
  cudaGraphDestroy(g);
  if (st != GFORS_OK) return st;
  if (e) {
    rg.exec = nullptr;
    return gf_cuda(h, e, "gfors_run_graph build");
  }
  rg.sv = h->struct_version;
  rg.gv = h->grp_version;
  return GFORS_OK;
}

extern "C" gfors_status gfors_run_graph_prepare(gfors_handle h, int32_t proposal) {
  GF_ENTER(h);
  gfors_status st = run_graph_ready(h, proposal);
  if (st) return st;
  return run_graph_build(h, proposal);
}

extern "C" gfors_status gfors_run_graph(gfors_handle h, int64_t max_iters, int32_t proposal,
                                        const int64_t* target_obj, int64_t* iters_out,
                                        int64_t* triggers_out) {
  GF_ENTER(h);
  if (max_iters < 0) return gf_fail(h, GFORS_E_ARG, "bad max_iters");
  gfors_status st = run_graph_ready(h, proposal);
  if (st) return st;
  const int kint = h->prm.k_int, kr = h->prm.k_r, nb = h->ninst;
  cudaStream_t s = h->stream;
  cudaError_t e;
  const long long ntrig = (max_iters - h->k_host) / kint;
  long long ran = 0, reason = 0;
  if (ntrig > 0) {
    if ((st = run_graph_build(h, proposal))) return st;
    const GfCtx::RunGraph& rg = h->run_graph[proposal];
    const long long k0 = h->k_host;
    long long ctl[6] = {0, h->h_trig, -1, ntrig, k0 / kint, target_obj ? 1 : 0};
    if ((e = cudaMemcpyAsync(h->halt_best, h->h_best.data(), sizeof(double) * 3 * nb,
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(h->halt_last, h->h_last.data(), sizeof(long long) * 3 * nb,
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(h->halt_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s)) ||
        (target_obj && (e = cudaMemcpyAsync(h->halt_tgt, target_obj, sizeof(long long) * nb,
                                            cudaMemcpyHostToDevice, s))))
      return gf_cuda(h, e, "halt state upload");
    long long ctl_out[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> bst(3 * nb);
    std::vector<long long> lst(3 * nb);
    if ((e = cudaGraphLaunch(rg.exec, s)) ||
        (e = cudaMemcpyAsync(ctl_out, h->halt_ctl, sizeof(ctl_out), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(bst.data(), h->halt_best, sizeof(double) * 3 * nb,
                             cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(lst.data(), h->halt_last, sizeof(long long) * 3 * nb,
                             cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
      return gf_cuda(h, e, "gfors_run_graph");
    if (gfors_status ds = check_device_error(h)) return ds;
    // host mirrors after `ran` triggers
    ran = ctl_out[0];
    reason = ctl_out[2];
    for (long long it = k0 + 1; it <= k0 + ran * kint; ++it) host_advance(h, it);
    h->k_host = k0 + ran * kint;
    h->launches += ran * rg.per_trig;
    h->h_trig = ctl_out[1];
    h->h_best = bst;
    h->h_last = lst;
    const unsigned last_plain = (unsigned)((k0 / kint + ran) * kr - 1);
    h->host_round = last_plain + 1;
    h->last_round = (proposal == 3) ? (last_plain | 0x80000000u) : last_plain;
  }
  // CheckHalt or the targets stop Alg. 1 at once; the iteration budget runs
  // the iterations after the last trigger, as gfors_run does
  if (ntrig <= 0 || reason == 0) {
    const int64_t rest = max_iters - h->k_host;
    if (rest > 0 && (e = enqueue_steps(h, rest))) return gf_cuda(h, e, "gfors_run_graph steps");
  }
  gfors_status st2 = gfors_final_round(h);
  if (st2) return st2;
  if ((e = cudaStreamSynchronize(s))) return gf_cuda(h, e, "gfors_run_graph sync");
  if (iters_out) *iters_out = h->k_host;
  if (triggers_out) *triggers_out = ran;
  return GFORS_OK;
}

extern "C" gfors_status gfors_incumbent(gfors_handle h, int32_t inst, int32_t* found,
                                        int64_t* obj_i, double* obj_f, uint32_t* round_id,
                                        int32_t* sample, uint8_t* x_out) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  GfInc I;
  cudaError_t e = cudaMemcpyAsync(&I, h->inc + inst, sizeof(GfInc), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e) return gf_cuda(h, e, "incumbent copy");
  const GfInstHost& H = h->ih[inst];
  if (x_out && (e = cudaMemcpyAsync(x_out, h->xbest + H.var_off, H.n, cudaMemcpyDeviceToHost,
                                    h->stream)))
    return gf_cuda(h, e, "incumbent copy");
  if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "incumbent sync");
  if (gfors_status ds = check_device_error(h)) return ds;
  if (found) *found = I.found;
  if (obj_i) *obj_i = I.obj;
  if (obj_f) *obj_f = I.objf;
  if (round_id) *round_id = I.round_id;
  if (sample) *sample = I.sample;
  return GFORS_OK;
}

extern "C" gfors_status gfors_get_scales(gfors_handle h, int32_t inst, double out[8]) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst || !out) return gf_fail(h, GFORS_E_ARG, "bad instance");
  const GfInstHost& I = h->ih[inst];
  GfIParam q;
  cudaError_t e = cudaMemcpyAsync(&q, h->iprm + (size_t)((h->k_host + 1) & 1) * h->ninst + inst,
                                  sizeof(q), cudaMemcpyDeviceToHost, h->stream);
  if (e || (e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "scales");
  out[0] = I.normQ_raw; out[1] = I.s_obj; out[2] = I.normK; out[3] = I.normQhat;
  out[4] = I.itQ; out[5] = I.itK; out[6] = q.tau1d; out[7] = q.tau2d;
  return GFORS_OK;
}

extern "C" gfors_status gfors_get_iterate(gfors_handle h, int32_t inst, float* x, float* xbar,
                                          float* x_prev, float* y) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  const GfInstHost& I = h->ih[inst];
  const int par = (int)(h->k_host & 1);
  cudaError_t e = cudaSuccess;
  if (x && !e) e = cudaMemcpyAsync(x, h->x[par] + I.var_off, sizeof(float) * I.n,
                                   cudaMemcpyDeviceToHost, h->stream);
  if (xbar && !e) e = cudaMemcpyAsync(xbar, h->xbar + I.var_off, sizeof(float) * I.n,
                                      cudaMemcpyDeviceToHost, h->stream);
  if (x_prev && !e) e = cudaMemcpyAsync(x_prev, h->x[1 - par] + I.var_off, sizeof(float) * I.n,
                                        cudaMemcpyDeviceToHost, h->stream);
  if (y && I.m1 + I.m2 && !e)
    e = cudaMemcpyAsync(y, h->y + I.row_off, sizeof(float) * (I.m1 + I.m2),
                        cudaMemcpyDeviceToHost, h->stream);
  if (!e) e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "gfors_get_iterate");
  return GFORS_OK;
}

static gfors_status set_iterate_impl(gfors_handle h, int32_t inst, const float* x,
                                     const float* xbar, const float* y, bool sync);

extern "C" gfors_status gfors_set_iterate(gfors_handle h, int32_t inst, const float* x,
                                          const float* xbar, const float* y) {
  return set_iterate_impl(h, inst, x, xbar, y, true);
}

extern "C" gfors_status gfors_set_iterate_async(gfors_handle h, int32_t inst, const float* x,
                                                const float* xbar, const float* y) {
  return set_iterate_impl(h, inst, x, xbar, y, false);
}

static gfors_status set_iterate_impl(gfors_handle h, int32_t inst, const float* x,
                                     const float* xbar, const float* y, bool sync) {
  GF_ENTER(h);
  h->sr_valid = false;                    // K xbar partials recomputed
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  const GfInstHost& I = h->ih[inst];
  const int par = (int)(h->k_host & 1);
  cudaError_t e = cudaSuccess;
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice;
  if (x) {
    e = cudaMemcpyAsync(h->x[par] + I.var_off, x, sizeof(float) * I.n, H2D, h->stream);
    if (!e) e = cudaMemcpyAsync(h->x[1 - par] + I.var_off, x, sizeof(float) * I.n, H2D,
                                h->stream);
  }
  if (xbar && !e)
    e = cudaMemcpyAsync(h->xbar + I.var_off, xbar, sizeof(float) * I.n, H2D, h->stream);
  if (y && I.m1 + I.m2 && !e)
    e = cudaMemcpyAsync(h->y + I.row_off, y, sizeof(float) * (I.m1 + I.m2), H2D, h->stream);
  if (!e && sync) e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "gfors_set_iterate");
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_counters(gfors_handle h, int64_t k, double rho) {
  GF_ENTER(h);
  h->sr_valid = false;                    // K xbar partials recomputed
  if (k < 0) return gf_fail(h, GFORS_E_ARG, "k < 0");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "set_counters sync");
  if ((k & 1) != (h->k_host & 1)) {       // keep x_k in x[k & 1]
    std::swap(h->x[0], h->x[1]);
    h->struct_version++;                  // captured launches name these buffers
    for (int q = 0; q < 2; ++q)
      if (h->g_iter2[q]) { cudaGraphExecDestroy(h->g_iter2[q]); h->g_iter2[q] = nullptr; }
    for (int q = 0; q < 2; ++q)
      if (h->g_light2[q]) { cudaGraphExecDestroy(h->g_light2[q]); h->g_light2[q] = nullptr; }
  }
  const gfors_params& P = h->prm;
  h->n_rho_host = 0;
  h->rho_host = std::min(P.rho_min, P.rho_max);
  h->k_host = 0;
  host_advance(h, k);
  if (rho >= 0.0) h->rho_host = rho;
  h->k_host = k;
  GfDState ds;
  if ((e = cudaMemcpy(&ds, h->dstate, sizeof(ds), cudaMemcpyDeviceToHost)))
    return gf_cuda(h, e, "set_counters");
  ds.k = k;
  ds.n_rho = h->n_rho_host;
  ds.rho = h->rho_host;
  if ((e = cudaMemcpy(h->dstate, &ds, sizeof(ds), cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "set_counters");
  gf_set_slot(h, (int)((k + 1) & 1), h->rho_host);
  gf_set_slot(h, (int)(k & 1), h->rho_host);
  if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "set_counters");
  return GFORS_OK;
}

extern "C" gfors_status gfors_eval_candidates(gfors_handle h, int32_t inst, int32_t k,
                                              const uint8_t* X, int32_t* viol, int64_t* obj_i,
                                              double* obj_f) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst || k < 0 || (k > 0 && !X))
    return gf_fail(h, GFORS_E_ARG, "bad arguments");
  if (!h->all_integral) return gf_fail(h, GFORS_E_UNSUPPORTED, "needs integral data");
  const GfInstHost& I = h->ih[inst];
  cudaError_t e;
  uint8_t* Xd = gf_alloc_t<uint8_t>(h, (size_t)h->chunk * I.n);
  if (!Xd) return gf_fail(h, GFORS_E_OOM, "eval_candidates buffer");
  std::vector<int32_t> v(h->chunk);
  std::vector<long long> o(h->chunk);
  for (int s0 = 0; s0 < k; s0 += h->chunk) {
    const int len = std::min(h->chunk, k - s0);
    if ((e = cudaMemcpyAsync(Xd, X + (size_t)s0 * I.n, (size_t)len * I.n,
                             cudaMemcpyHostToDevice, h->stream)))
      return gf_cuda(h, e, "eval_candidates upload");
    if (I.qkind == 1) {
      const GfDenseQ& dq = h->dense[I.dense_idx];
      k_pack_dense<<<(unsigned)(((int64_t)len * dq.ld + 255) / 256), 256, 0, h->stream>>>(
          Xd, len, I.n, dq.ld, dq.Xs, (int)dq.f8);
      k_dense_bits<<<(unsigned)(((int64_t)len * (dq.ld / 32) + 255) / 256), 256, 0,
                     h->stream>>>(dq.Xs, len, dq.ld, dq.Xb, (int)dq.f8);
    } else {
      const int kwu = (len + 31) / 32;
      k_pack_bits<<<(unsigned)((I.n * kwu + 255) / 256), 256, 0, h->stream>>>(Xd, len, I.n,
                                                                              I.var_off, h->kw,
                                                                              h->X);
    }
    if ((e = gf_launch_eval(h, 0, len))) return gf_cuda(h, e, "eval_candidates");
    if (I.qkind == 1 && (e = gf_launch_dense_score(h, h->dense[I.dense_idx], 0, len)))
      return gf_cuda(h, e, "eval_candidates dense");
    if ((e = cudaMemcpyAsync(v.data(), h->viol + (size_t)inst * h->chunk, sizeof(int32_t) * len,
                             cudaMemcpyDeviceToHost, h->stream)))
      return gf_cuda(h, e, "eval_candidates copy");
    if ((e = cudaMemcpyAsync(o.data(), h->obj + (size_t)inst * h->chunk,
                             sizeof(long long) * len, cudaMemcpyDeviceToHost, h->stream)))
      return gf_cuda(h, e, "eval_candidates copy");
    if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "eval_candidates sync");
    if (gfors_status ds = check_device_error(h)) return ds;
    for (int t = 0; t < len; ++t) {
      if (viol) viol[s0 + t] = v[t];
      if (obj_i) obj_i[s0 + t] = o[t];
      if (obj_f) obj_f[s0 + t] = (double)o[t];
    }
  }
  gf_free_one(h, Xd);
  return GFORS_OK;
}

extern "C" gfors_status gfors_get_samples(gfors_handle h, int32_t inst, uint8_t* X_out,
                                          int32_t* viol, int64_t* obj_i, int32_t* count) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  const GfInstHost& I = h->ih[inst];
  const int len = h->last_chunk_len;
  cudaError_t e;
  if (count) *count = len;
  if (len == 0) return GFORS_OK;
  if (X_out) {
    uint8_t* Xd = gf_alloc_t<uint8_t>(h, (size_t)len * I.n);
    if (!Xd) return gf_fail(h, GFORS_E_OOM, "get_samples buffer");
    if (I.qkind == 1) {
      const GfDenseQ& dq = h->dense[I.dense_idx];
      k_unpack_dense<<<(unsigned)(((int64_t)len * I.n + 255) / 256), 256, 0, h->stream>>>(
          dq.Xb, len, I.n, dq.ld, Xd);
    } else {
      if (h->last_mode == 1) {
        // fused chunks are not materialised: regenerate the same draws
        k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, h->last_round);
        if ((e = gf_launch_sample(h, h->last_p, h->last_s0, len, false)))
          return gf_cuda(h, e, "get_samples regenerate");
        k_set_round<<<1, 1, 0, h->stream>>>(h->dstate, h->host_round);
      }
      k_unpack_bits<<<(unsigned)(((int64_t)len * I.n + 255) / 256), 256, 0, h->stream>>>(
          h->X, len, I.n, I.var_off, h->kw, Xd);
    }
    if ((e = cudaMemcpyAsync(X_out, Xd, (size_t)len * I.n, cudaMemcpyDeviceToHost, h->stream)))
      return gf_cuda(h, e, "get_samples copy");
    if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "get_samples sync");
    gf_free_one(h, Xd);
  }
  std::vector<int32_t> v(len);
  std::vector<long long> o(len);
  if ((e = cudaMemcpyAsync(v.data(), h->viol + (size_t)inst * h->chunk, sizeof(int32_t) * len,
                           cudaMemcpyDeviceToHost, h->stream)))
    return gf_cuda(h, e, "get_samples copy");
  if ((e = cudaMemcpyAsync(o.data(), h->obj + (size_t)inst * h->chunk, sizeof(long long) * len,
                           cudaMemcpyDeviceToHost, h->stream)))
    return gf_cuda(h, e, "get_samples copy");
  if ((e = cudaStreamSynchronize(h->stream))) return gf_cuda(h, e, "get_samples sync");
  if (gfors_status ds = check_device_error(h)) return ds;
  for (int t = 0; t < len; ++t) {
    if (viol) viol[t] = v[t];
    if (obj_i) obj_i[t] = o[t];
  }
  return GFORS_OK;
}

// ---------------------------------------------------------------------------
// groups and closure
extern "C" gfors_status gfors_set_groups(gfors_handle h, int32_t inst, int32_t mode,
                                         int64_t ngroups, const int64_t* grp_ptr,
                                         const int64_t* grp_idx, int32_t axial_I) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  GfInstHost& I = h->ih[inst];
  if (I.qkind == 1 && mode != 0)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "groups on a dense tensor-core instance");
  if (h->fused_ok && mode != 0)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "groups on a fused single-row batch");
  if (I.group_mode != 0) return gf_fail(h, GFORS_E_STATE, "groups already set");
  cudaError_t e;
  std::vector<uint8_t> grouped(I.npad, 0);
  if (mode == 0) return GFORS_OK;
  if (mode == 2) {
    if (axial_I < 1 || axial_I > 256 || (int64_t)axial_I * axial_I * axial_I != I.n)
      return gf_fail(h, GFORS_E_ARG, "axial mode needs n = I^3 with 1 <= I <= 256");
    I.group_mode = 2;
    I.axial_I = axial_I;
    for (int64_t i = 0; i < I.n; ++i) grouped[i] = 1;
  } else if (mode == 1) {
    if (ngroups < 0 || (ngroups > 0 && (!grp_ptr || !grp_idx)) || (ngroups && grp_ptr[0] != 0))
      return gf_fail(h, GFORS_E_ARG, "bad group arrays");
    for (int64_t g = 0; g < ngroups; ++g) {
      if (grp_ptr[g + 1] < grp_ptr[g]) return gf_fail(h, GFORS_E_ARG, "group ptr not monotone");
      for (int64_t t = grp_ptr[g]; t < grp_ptr[g + 1]; ++t) {
        const int64_t v = grp_idx[t];
        if (v < 0 || v >= I.n) return gf_fail(h, GFORS_E_ARG, "group index out of range");
        if (grouped[v]) return gf_fail(h, GFORS_E_ARG, "groups must be disjoint");
        grouped[v] = 1;
      }
    }
    I.group_mode = 1;
    I.ngroups = ngroups;
    const int64_t base = (int64_t)h->h_grp_idx.size();
    if (h->h_grp_ptr.empty()) h->h_grp_ptr.push_back(0);
    for (int64_t g = 0; g < ngroups; ++g) {
      for (int64_t t = grp_ptr[g]; t < grp_ptr[g + 1]; ++t)
        h->h_grp_idx.push_back(I.var_off + grp_idx[t]);
      h->h_grp_ptr.push_back(base + grp_ptr[g + 1]);
      h->h_grp_inst.push_back(inst);
      h->h_grp_local.push_back((int32_t)g);
    }
    h->ngroups_tot = (int64_t)h->h_grp_inst.size();
    // (re)upload the global group tables
    h->grp_ptr = gf_alloc_t<int64_t>(h, h->h_grp_ptr.size());
    h->grp_idx = gf_alloc_t<int64_t>(h, h->h_grp_idx.size());
    h->grp_inst = gf_alloc_t<int32_t>(h, h->h_grp_inst.size());
    h->grp_local = gf_alloc_t<int32_t>(h, h->h_grp_local.size());
    h->grp_cw = gf_alloc_t<unsigned long long>(h, h->h_grp_idx.size());
    h->grp_cw2 = gf_alloc_t<unsigned long long>(h, h->h_grp_idx.size());
    h->grp_step = gf_alloc_t<int64_t>(h, h->h_grp_inst.size());
    if (!h->grp_ptr || !h->grp_idx || !h->grp_inst || !h->grp_local || !h->grp_cw ||
        !h->grp_cw2 || !h->grp_step)
      return gf_fail(h, GFORS_E_OOM, "group tables");
    // member lists in constant steps (e.g. a customer's x_ij over i) are
    // generated in the samplers instead of read
    {
      std::vector<int64_t> step(h->h_grp_inst.size(), 0);
      for (size_t g = 0; g < step.size(); ++g) {
        const int64_t a = h->h_grp_ptr[g], b = h->h_grp_ptr[g + 1];
        if (b - a < 2) continue;
        const int64_t d = h->h_grp_idx[a + 1] - h->h_grp_idx[a];
        if (d <= 0) continue;
        bool ok = true;
        for (int64_t t = a + 2; t < b && ok; ++t) ok = h->h_grp_idx[t] - h->h_grp_idx[t - 1] == d;
        if (ok) step[g] = d;
      }
      if ((e = cudaMemcpy(h->grp_step, step.data(), sizeof(int64_t) * step.size(),
                          cudaMemcpyHostToDevice)))
        return gf_cuda(h, e, "group upload");
    }
    if ((e = cudaMemcpy(h->grp_ptr, h->h_grp_ptr.data(), sizeof(int64_t) * h->h_grp_ptr.size(),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->grp_idx, h->h_grp_idx.data(), sizeof(int64_t) * h->h_grp_idx.size(),
                        cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->grp_inst, h->h_grp_inst.data(),
                        sizeof(int32_t) * h->h_grp_inst.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->grp_local, h->h_grp_local.data(),
                        sizeof(int32_t) * h->h_grp_local.size(), cudaMemcpyHostToDevice)))
      return gf_cuda(h, e, "group upload");
  } else {
    return gf_fail(h, GFORS_E_ARG, "mode must be 0, 1 or 2");
  }
  h->n_bit_g4 = -1;                      // Bernoulli group list rebuilt
  h->grp_version++;                      // static features rebuilt
  if ((e = cudaMemcpy(h->var_grouped + I.var_off, grouped.data(), I.npad,
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->var_grouped_feat + I.var_off, grouped.data(), I.npad,
                      cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "group flags");
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_assign3d_custom(gfors_handle h, int32_t inst, int32_t I3,
                                                  int32_t gamma, int32_t L) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  GfInstHost& I = h->ih[inst];
  if (I.qkind == 1 || h->fused_ok)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "Algorithm 4 needs a sparse, sampled instance");
  if (I.group_mode != 0) return gf_fail(h, GFORS_E_STATE, "groups already set");
  if (I3 < 1 || I3 > 64 || (int64_t)I3 * I3 * I3 != I.n)
    return gf_fail(h, GFORS_E_ARG, "Algorithm 4 needs n = I^3 with 1 <= I <= 64");
  if (gamma < 0 || gamma > I3 || I3 * gamma * I3 > 16384 || L < 0)
    return gf_fail(h, GFORS_E_ARG, "need 0 <= gamma <= I, I * gamma * I <= 16384, L >= 0");
  if (!I.integral) return gf_fail(h, GFORS_E_UNSUPPORTED, "Algorithm 4 needs integral costs");
  if (!h->a4_cand) {
    h->a4_cand = gf_alloc_t<unsigned long long>(h, 16384);
    h->a4_J0 = gf_alloc_t<int32_t>(h, 64);
    h->a4_K0 = gf_alloc_t<int32_t>(h, 64);
    if (!h->a4_cand || !h->a4_J0 || !h->a4_K0)
      return gf_fail(h, GFORS_E_OOM, "Algorithm 4 scratch");
  }
  {
    // gains are differences of two pairs of costs: int32 holds them when
    // 4 max|c| < 2^31
    std::vector<long long> cost((size_t)I.n);
    if (cudaError_t e0 = cudaMemcpy(cost.data(), h->cint + I.var_off, sizeof(long long) * I.n,
                                    cudaMemcpyDeviceToHost))
      return gf_cuda(h, e0, "Algorithm 4 costs");
    long long cmax = 0;
    for (long long v : cost) cmax = std::max(cmax, v < 0 ? -v : v);
    I.a4_gain32 = cmax < (1ll << 29);
  }
  I.group_mode = 3;
  I.axial_I = I3;
  I.a4_gamma = gamma;
  I.a4_L = L;
  std::vector<uint8_t> grouped(I.npad, 0);
  for (int64_t i = 0; i < I.n; ++i) grouped[i] = 1;
  cudaError_t e;
  h->n_bit_g4 = -1;                      // Bernoulli group list rebuilt
  h->grp_version++;                      // static features rebuilt
  if ((e = cudaMemcpy(h->var_grouped + I.var_off, grouped.data(), I.npad,
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->var_grouped_feat + I.var_off, grouped.data(), I.npad,
                      cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "group flags");
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_repair_groups(gfors_handle h, int32_t inst, int64_t ngroups,
                                                const int64_t* grp_ptr, const int64_t* grp_idx) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  const GfInstHost& I = h->ih[inst];
  if (ngroups <= 0) return GFORS_OK;
  if (!grp_ptr || !grp_idx || grp_ptr[0] != 0) return gf_fail(h, GFORS_E_ARG, "bad group arrays");
  if (I.qkind == 1 || h->fused_ok)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "repair groups on a dense / fused instance");
  if (!I.integral) return gf_fail(h, GFORS_E_UNSUPPORTED, "repair groups need integral costs");
  // the instance's integer costs: members are stored in (cost, listing
  // position) order, so the repair kernel keeps the first selected member
  std::vector<long long> cost((size_t)I.n);
  if (cudaError_t e0 = cudaMemcpy(cost.data(), h->cint + I.var_off, sizeof(long long) * I.n,
                                  cudaMemcpyDeviceToHost))
    return gf_cuda(h, e0, "repair group costs");
  std::vector<uint8_t> seen(I.n, 0);
  if (h->h_rg_ptr.empty()) h->h_rg_ptr.push_back(0);
  const int64_t base = (int64_t)h->h_rg_idx.size();
  for (int64_t g = 0; g < ngroups; ++g) {
    if (grp_ptr[g + 1] < grp_ptr[g]) return gf_fail(h, GFORS_E_ARG, "group ptr not monotone");
    for (int64_t t = grp_ptr[g]; t < grp_ptr[g + 1]; ++t) {
      const int64_t v = grp_idx[t];
      if (v < 0 || v >= I.n) return gf_fail(h, GFORS_E_ARG, "group index out of range");
      if (seen[v]) return gf_fail(h, GFORS_E_ARG, "groups must be disjoint");
      seen[v] = 1;
      h->h_rg_idx.push_back(I.var_off + v);
    }
    std::stable_sort(h->h_rg_idx.begin() + base + grp_ptr[g], h->h_rg_idx.end(),
                     [&](int64_t x, int64_t y) {
                       return cost[x - I.var_off] < cost[y - I.var_off];
                     });
    h->h_rg_ptr.push_back(base + grp_ptr[g + 1]);
  }
  h->nrg = (int64_t)h->h_rg_ptr.size() - 1;
  h->repair_version++;
  h->struct_version++;
  h->rg_ptr = gf_alloc_t<int64_t>(h, h->h_rg_ptr.size());
  h->rg_idx = gf_alloc_t<int64_t>(h, std::max<size_t>(1, h->h_rg_idx.size()));
  if (!h->rg_ptr || !h->rg_idx) return gf_fail(h, GFORS_E_OOM, "repair groups");
  cudaError_t e;
  if ((e = cudaMemcpy(h->rg_ptr, h->h_rg_ptr.data(), sizeof(int64_t) * h->h_rg_ptr.size(),
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->rg_idx, h->h_rg_idx.data(), sizeof(int64_t) * h->h_rg_idx.size(),
                      cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "repair group upload");
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_repair_rows(gfors_handle h, int32_t inst, int64_t nrows,
                                              const int64_t* row_ptr, const int64_t* row_idx) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  GfInstHost& I = h->ih[inst];
  if (nrows <= 0) return GFORS_OK;
  if (!row_ptr || !row_idx || row_ptr[0] != 0) return gf_fail(h, GFORS_E_ARG, "bad row arrays");
  if (I.qkind == 1 || h->fused_ok)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "repair rows on a dense / fused instance");
  if (!I.integral) return gf_fail(h, GFORS_E_UNSUPPORTED, "repair rows need integral costs");
  if (I.rr_set) return gf_fail(h, GFORS_E_STATE, "repair rows already set for this instance");
  std::vector<long long> cost((size_t)I.n);
  if (cudaError_t e0 = cudaMemcpy(cost.data(), h->cint + I.var_off, sizeof(long long) * I.n,
                                  cudaMemcpyDeviceToHost))
    return gf_cuda(h, e0, "repair row costs");
  // rows (local ids checked) and the rows of each variable
  std::vector<std::vector<int64_t>> vr((size_t)I.n);
  for (int64_t r = 0; r < nrows; ++r) {
    if (row_ptr[r + 1] < row_ptr[r]) return gf_fail(h, GFORS_E_ARG, "row ptr not monotone");
    for (int64_t t = row_ptr[r]; t < row_ptr[r + 1]; ++t)
      if (row_idx[t] < 0 || row_idx[t] >= I.n)
        return gf_fail(h, GFORS_E_ARG, "row index out of range");
  }
  if (h->h_rr_ptr.empty()) h->h_rr_ptr.push_back(0);
  if (h->h_rr_optr.empty()) h->h_rr_optr.push_back(0);
  if (h->h_rr_vptr.empty()) h->h_rr_vptr.push_back(0);
  const int64_t r0 = (int64_t)h->h_rr_ptr.size() - 1;        // global id of row 0
  for (int64_t r = 0; r < nrows; ++r) {
    for (int64_t t = row_ptr[r]; t < row_ptr[r + 1]; ++t) {
      h->h_rr_idx.push_back(I.var_off + row_idx[t]);
      vr[(size_t)row_idx[t]].push_back(r0 + r);
    }
    h->h_rr_ptr.push_back((int64_t)h->h_rr_idx.size());
  }
  // the row variables in decreasing cost, ties to the larger index first
  std::vector<int64_t> order;
  for (int64_t v = 0; v < I.n; ++v)
    if (!vr[(size_t)v].empty()) order.push_back(v);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return cost[a] != cost[b] ? cost[a] > cost[b] : a > b;
  });
  for (int64_t v : order) {
    h->h_rr_order.push_back(I.var_off + v);
    for (int64_t r : vr[(size_t)v]) h->h_rr_vrow.push_back(r);
    h->h_rr_vptr.push_back((int64_t)h->h_rr_vrow.size());
  }
  h->h_rr_optr.push_back((int64_t)h->h_rr_order.size());
  h->nrr = (int64_t)h->h_rr_ptr.size() - 1;
  h->nrr_seg = (int64_t)h->h_rr_optr.size() - 1;
  I.rr_set = true;
  h->repair_version++;
  h->struct_version++;
  auto up = [&](int64_t*& d, const std::vector<int64_t>& v) {
    d = gf_alloc_t<int64_t>(h, std::max<size_t>(1, v.size()));
    return d && cudaMemcpy(d, v.data(), sizeof(int64_t) * v.size(), cudaMemcpyHostToDevice) ==
                    cudaSuccess;
  };
  if (!up(h->rr_ptr, h->h_rr_ptr) || !up(h->rr_idx, h->h_rr_idx) ||
      !up(h->rr_optr, h->h_rr_optr) || !up(h->rr_order, h->h_rr_order) ||
      !up(h->rr_vptr, h->h_rr_vptr) || !up(h->rr_vrow, h->h_rr_vrow))
    return gf_fail(h, GFORS_E_OOM, "repair rows");
  h->rr_cnt = gf_alloc_t<int32_t>(h, (size_t)h->nrr * h->chunk);
  if (!h->rr_cnt) return gf_fail(h, GFORS_E_OOM, "repair row counts");
  return GFORS_OK;
}

extern "C" gfors_status gfors_set_closure(gfors_handle h, int32_t inst, int64_t nrep,
                                          const int64_t* rep_var, const int64_t* rep_ptr,
                                          const int64_t* rep_idx) {
  GF_ENTER(h);
  if (inst < 0 || inst >= h->ninst) return gf_fail(h, GFORS_E_ARG, "bad instance");
  GfInstHost& I = h->ih[inst];
  if (nrep <= 0) return GFORS_OK;
  if (!rep_var || !rep_ptr || !rep_idx || rep_ptr[0] != 0)
    return gf_fail(h, GFORS_E_ARG, "bad closure arrays");
  if (I.qkind == 1 || h->fused_ok)
    return gf_fail(h, GFORS_E_UNSUPPORTED, "closure on a dense / fused instance");
  if (h->h_rep_ptr.empty()) h->h_rep_ptr.push_back(0);
  const int64_t base = (int64_t)h->h_rep_idx.size();
  for (int64_t q = 0; q < nrep; ++q) {
    if (rep_var[q] < 0 || rep_var[q] >= I.n || rep_ptr[q + 1] < rep_ptr[q])
      return gf_fail(h, GFORS_E_ARG, "closure index out of range");
    h->h_rep_var.push_back(I.var_off + rep_var[q]);
    for (int64_t t = rep_ptr[q]; t < rep_ptr[q + 1]; ++t) {
      if (rep_idx[t] < 0 || rep_idx[t] >= I.n)
        return gf_fail(h, GFORS_E_ARG, "closure index out of range");
      h->h_rep_idx.push_back(I.var_off + rep_idx[t]);
    }
    h->h_rep_ptr.push_back(base + rep_ptr[q + 1]);
  }
  h->nrep_tot = (int64_t)h->h_rep_var.size();
  h->repair_version++;
  h->struct_version++;
  h->rep_var = gf_alloc_t<int64_t>(h, h->h_rep_var.size());
  h->rep_ptr = gf_alloc_t<int64_t>(h, h->h_rep_ptr.size());
  h->rep_idx = gf_alloc_t<int64_t>(h, h->h_rep_idx.size());
  h->rep_step = gf_alloc_t<int64_t>(h, h->h_rep_var.size());
  if (!h->rep_var || !h->rep_ptr || !h->rep_idx || !h->rep_step)
    return gf_fail(h, GFORS_E_OOM, "closure");
  // lists in constant steps (e.g. x_ij over j for one y_i) are generated in
  // the kernel instead of read
  std::vector<int64_t> step(h->h_rep_var.size(), 0);
  for (size_t q = 0; q < step.size(); ++q) {
    const int64_t a = h->h_rep_ptr[q], b = h->h_rep_ptr[q + 1];
    if (b - a < 2) continue;
    const int64_t d = h->h_rep_idx[a + 1] - h->h_rep_idx[a];
    if (d <= 0) continue;
    bool ok = true;
    for (int64_t t = a + 2; t < b && ok; ++t) ok = h->h_rep_idx[t] - h->h_rep_idx[t - 1] == d;
    if (ok) step[q] = d;
  }
  cudaError_t e;
  if ((e = cudaMemcpy(h->rep_step, step.data(), sizeof(int64_t) * step.size(),
                      cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "closure upload");
  if ((e = cudaMemcpy(h->rep_var, h->h_rep_var.data(), sizeof(int64_t) * h->h_rep_var.size(),
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->rep_ptr, h->h_rep_ptr.data(), sizeof(int64_t) * h->h_rep_ptr.size(),
                      cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->rep_idx, h->h_rep_idx.data(), sizeof(int64_t) * h->h_rep_idx.size(),
                      cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "closure upload");
  return GFORS_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume
namespace {
struct Blob {
  std::vector<uint8_t> b;
  template <class T> void put(const T& v) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
  void put_raw(const void* p, size_t n) {
    const uint8_t* q = static_cast<const uint8_t*>(p);
    b.insert(b.end(), q, q + n);
  }
};
const uint64_t kMagic = 0x47464F5253303031ull;  // "GFORS001"
}  // namespace

static gfors_status export_blob(GfCtx* h, Blob& B) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "export sync");
  const int64_t N = h->N, M = h->M;
  std::vector<float> x0(N), x1(N), xb(N), y(std::max<int64_t>(M, 1));
  std::vector<GfIParam> ip(2 * h->ninst);
  std::vector<GfInc> inc(h->ninst);
  std::vector<uint8_t> xbest(N);
  GfDState ds;
  if ((e = cudaMemcpy(x0.data(), h->x[0], sizeof(float) * N, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(x1.data(), h->x[1], sizeof(float) * N, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(xb.data(), h->xbar, sizeof(float) * N, cudaMemcpyDeviceToHost)) ||
      (M && (e = cudaMemcpy(y.data(), h->y, sizeof(float) * M, cudaMemcpyDeviceToHost))) ||
      (e = cudaMemcpy(ip.data(), h->iprm, sizeof(GfIParam) * 2 * h->ninst,
                      cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(inc.data(), h->inc, sizeof(GfInc) * h->ninst, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(xbest.data(), h->xbest, N, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(&ds, h->dstate, sizeof(ds), cudaMemcpyDeviceToHost)))
    return gf_cuda(h, e, "export copy");
  B.put(kMagic);
  B.put((int64_t)h->ninst);
  B.put(N);
  B.put(M);
  B.put(h->k_host);
  B.put(h->n_rho_host);
  B.put(h->rho_host);
  B.put(h->h_trig);
  B.put(ds);
  B.put_raw(x0.data(), sizeof(float) * N);
  B.put_raw(x1.data(), sizeof(float) * N);
  B.put_raw(xb.data(), sizeof(float) * N);
  B.put_raw(y.data(), sizeof(float) * M);
  B.put_raw(ip.data(), sizeof(GfIParam) * ip.size());
  B.put_raw(inc.data(), sizeof(GfInc) * inc.size());
  B.put_raw(xbest.data(), N);
  B.put_raw(h->h_best.data(), sizeof(double) * h->h_best.size());
  B.put_raw(h->h_last.data(), sizeof(long long) * h->h_last.size());
  return GFORS_OK;
}

extern "C" gfors_status gfors_state_export(gfors_handle h, void* buf, size_t* len) {
  GF_ENTER(h);
  if (!len) return gf_fail(h, GFORS_E_ARG, "len is NULL");
  Blob B;
  gfors_status st = export_blob(h, B);
  if (st) return st;
  if (!buf) { *len = B.b.size(); return GFORS_OK; }
  if (*len < B.b.size()) return gf_fail(h, GFORS_E_ARG, "buffer too small");
  memcpy(buf, B.b.data(), B.b.size());
  *len = B.b.size();
  return GFORS_OK;
}

extern "C" gfors_status gfors_state_import(gfors_handle h, const void* buf, size_t len) {
  GF_ENTER(h);
  h->sr_valid = false;                    // K xbar partials recomputed
  if (!buf) return gf_fail(h, GFORS_E_ARG, "buffer is NULL");
  const uint8_t* p = static_cast<const uint8_t*>(buf);
  size_t off = 0;
  auto get = [&](void* dst, size_t n) -> bool {
    if (off + n > len) return false;
    memcpy(dst, p + off, n);
    off += n;
    return true;
  };
  uint64_t magic;
  int64_t ninst, N, M;
  long long k;
  int nr;
  double rho;
  long long trig;
  GfDState ds;
  if (!get(&magic, 8) || magic != kMagic || !get(&ninst, 8) || !get(&N, 8) || !get(&M, 8) ||
      ninst != h->ninst || N != h->N || M != h->M)
    return gf_fail(h, GFORS_E_ARG, "checkpoint does not match this handle");
  if (!get(&k, sizeof k) || !get(&nr, sizeof nr) || !get(&rho, sizeof rho) ||
      !get(&trig, sizeof trig) || !get(&ds, sizeof ds))
    return gf_fail(h, GFORS_E_ARG, "truncated checkpoint");
  std::vector<float> x0(N), x1(N), xb(N), y(std::max<int64_t>(M, 1));
  std::vector<GfIParam> ip(2 * h->ninst);
  std::vector<GfInc> inc(h->ninst);
  std::vector<uint8_t> xbest(N);
  std::vector<double> best(h->h_best.size());
  std::vector<long long> last(h->h_last.size());
  if (!get(x0.data(), sizeof(float) * N) || !get(x1.data(), sizeof(float) * N) ||
      !get(xb.data(), sizeof(float) * N) || !get(y.data(), sizeof(float) * M) ||
      !get(ip.data(), sizeof(GfIParam) * ip.size()) || !get(inc.data(), sizeof(GfInc) * inc.size()) ||
      !get(xbest.data(), N) || !get(best.data(), sizeof(double) * best.size()) ||
      !get(last.data(), sizeof(long long) * last.size()))
    return gf_fail(h, GFORS_E_ARG, "truncated checkpoint");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "import sync");
  if ((e = cudaMemcpy(h->x[0], x0.data(), sizeof(float) * N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->x[1], x1.data(), sizeof(float) * N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->xbar, xb.data(), sizeof(float) * N, cudaMemcpyHostToDevice)) ||
      (M && (e = cudaMemcpy(h->y, y.data(), sizeof(float) * M, cudaMemcpyHostToDevice))) ||
      (e = cudaMemcpy(h->iprm, ip.data(), sizeof(GfIParam) * ip.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->inc, inc.data(), sizeof(GfInc) * inc.size(), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->xbest, xbest.data(), N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->dstate, &ds, sizeof ds, cudaMemcpyHostToDevice)))
    return gf_cuda(h, e, "import copy");
  h->k_host = k;
  h->n_rho_host = nr;
  h->rho_host = rho;
  h->h_trig = trig;
  h->h_best = best;
  h->h_last = last;
  return GFORS_OK;
}
