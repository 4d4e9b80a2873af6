// k_power.cu -- FP64 work of the hot path: the spectral norms of Preprocess
// (Section 3) by power iteration on M^T M, the FP64 -> FP32 scaling of the
// preprocessed data, and the FP64 reductions behind CheckHalt (Section 3).
// Per-instance sums are deterministic: every instance's vectors are cut into
// fixed chunks, each chunk reduced by one block in a fixed tree order, and
// the chunk partials added in chunk order.
#include "internal.cuh"

namespace {

constexpr int kRedThreads = 256;
constexpr int kRowChunk = 2048;    // rows per statistics chunk (the load's row chunks)
constexpr int kStatLong = 256;     // longer rows are summed by a whole block

__device__ double block_sum(double v) {
  __shared__ double sh[kRedThreads];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Power-iteration start vector: ((u + 0.5) 2^-31 - 1), u = Philox lane
// (stream 3, sample = which, round 0, local index); padding gets 0.
__global__ void k_pw_start(double* __restrict__ v, const int32_t* __restrict__ var_inst,
                           const int64_t* __restrict__ var_off,
                           const uint8_t* __restrict__ live, int64_t N, uint64_t seed,
                           int inst_base, int which) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (!live[i]) { v[i] = 0.0; return; }
  const int b = var_inst[i];
  const int64_t loc = i - var_off[b];
  const uint4 u = gf::philox_call(seed, gf::kStreamPower, (uint32_t)(inst_base + b), 0u,
                                  (uint32_t)which, (uint64_t)(loc >> 2));
  v[i] = ((double)gf::lane_of(u, (uint32_t)(loc & 3)) + 0.5) * (1.0 / 2147483648.0) - 1.0;
}

// sum of squares of vec over chunks (inst, a, b) -> partial[c]
__global__ void __launch_bounds__(kRedThreads)
k_chunk_sumsq(const double* __restrict__ vec, const int32_t* __restrict__ ch, int64_t nch,
              double* __restrict__ partial) {
  const int64_t c = blockIdx.x;
  if (c >= nch) return;
  const int a = ch[3 * c + 1], b = ch[3 * c + 2];
  double s = 0.0;
  for (int i = a + threadIdx.x; i < b; i += kRedThreads) s += vec[i] * vec[i];
  s = block_sum(s);
  if (threadIdx.x == 0) partial[c] = s;
}

// per instance: out[b] = sum of partial[c] for c in [iptr[b], iptr[b+1])
__global__ void k_inst_sum(const double* __restrict__ partial, const int32_t* __restrict__ iptr,
                           int ninst, int stride, int comps, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ninst) return;
  for (int q = 0; q < comps; ++q) {
    double s = 0.0;
    for (int c = iptr[b]; c < iptr[b + 1]; ++c) s += partial[(int64_t)c * stride + q];
    out[(int64_t)b * comps + q] = s;
  }
}

// FP64 CSR product out = M vec, LANES threads per row; rows longer than
// kPwLong entries are left to k_spmv64_long.
constexpr int64_t kPwLong = 256;
template <int LANES>
__global__ void __launch_bounds__(256)
k_spmv64(const int64_t* __restrict__ Mp, const int32_t* __restrict__ Mc,
         const double* __restrict__ Mv, const double* __restrict__ vec, int64_t rows,
         double* __restrict__ out) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = gid / LANES;
  const int lane = (int)(gid % LANES);
  if (r >= rows) return;
  if (Mp[r + 1] - Mp[r] > kPwLong) return;      // the whole group skips it
  double s = 0.0;
  for (int64_t t = Mp[r] + lane; t < Mp[r + 1]; t += LANES) s += Mv[t] * vec[Mc[t]];
  if (LANES > 1) {
    const unsigned lid = threadIdx.x & 31u;
    const unsigned mask = (LANES == 32) ? 0xFFFFFFFFu
                                        : (((1u << LANES) - 1u) << (lid & ~(unsigned)(LANES - 1)));
    for (int off = LANES / 2; off > 0; off >>= 1) s += __shfl_down_sync(mask, s, off, LANES);
  }
  if (lane == 0) out[r] = s;
}

// The long rows (ids[]) of the same product, one block each, block_sum in a
// fixed order.
__global__ void __launch_bounds__(kRedThreads)
k_spmv64_long(const int64_t* __restrict__ Mp, const int32_t* __restrict__ Mc,
              const double* __restrict__ Mv, const double* __restrict__ vec,
              const int64_t* __restrict__ ids, double* __restrict__ out) {
  const int64_t r = ids[blockIdx.x];
  double s = 0.0;
  for (int64_t t = Mp[r] + threadIdx.x; t < Mp[r + 1]; t += kRedThreads)
    s += Mv[t] * vec[Mc[t]];
  s = block_sum(s);
  if (threadIdx.x == 0) out[r] = s;
}

// FP64 dense symmetric product for one dense-Q instance:
// out_i = 0.5 sum_j W2_ij vec_j + D_i vec_i   (Q_sym = W2/2 + diag(D)).
__global__ void __launch_bounds__(256)
k_dense64(const __nv_bfloat16* __restrict__ W2, int64_t ld, int64_t n, int64_t v0,
          const double* __restrict__ diag, const double* __restrict__ vec,
          double* __restrict__ out) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  const __nv_bfloat16* wr = W2 + row * ld;
  for (int64_t j = lane; j < n; j += 32) s += (double)__bfloat162float(wr[j]) * vec[v0 + j];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
  if (lane == 0) out[v0 + row] = 0.5 * s + diag[row] * vec[v0 + row];
}

struct PwState {
  double lam, lam_prev, result;
  int done, iters, upd, pad;
};

// Per-instance bookkeeping of one power-iteration step t (the oracle's
// order): lambda_t = ||M v_t||^2, zn = ||M^T M v_t||; zn = 0 ends;
// otherwise v_{t+1} = z / zn and the relative-change test ends it.  t is
// the device step counter (the loop runs as one graph launch).
__global__ void k_pw_step(PwState* __restrict__ ps, const double* __restrict__ lam,
                          const double* __restrict__ zn2, int ninst, const int* __restrict__ tc,
                          double tol, int maxit, int* __restrict__ ndone) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ninst) return;
  const int t = *tc;
  PwState S = ps[b];
  S.upd = 0;
  if (!S.done) {
    const double L = lam[b];
    const double zn = sqrt(zn2[b]);
    S.lam = L;
    if (zn == 0.0) {
      S.done = 1; S.result = L; S.iters = t + 1;
    } else {
      S.upd = 1;
      if (t >= 1 && fabs(L - S.lam_prev) <= tol * L) {
        S.done = 1; S.result = L; S.iters = t + 1;
      } else if (t == maxit - 1) {
        S.done = 1; S.result = L; S.iters = maxit;
      } else {
        S.lam_prev = L;
      }
    }
    if (S.done) atomicAdd(ndone, 1);
  }
  ps[b] = S;
}

// v = z / |z| per instance; v and z may be the same vector (in-place start)
__global__ void k_pw_normalize(double* v, const double* z,
                               const double* __restrict__ zn2,
                               const int32_t* __restrict__ var_inst,
                               const PwState* __restrict__ ps, int64_t N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = var_inst[i];
  if (ps[b].upd) v[i] = z[i] / sqrt(zn2[b]);
}

// End of a loop step: t <- t + 1, and the loop goes on while an instance is
// still iterating and t < maxit.
__global__ void k_pw_next(int* tc, const int* __restrict__ ndone, int ninst, int maxit,
                          cudaGraphConditionalHandle cond) {
  const int t = *tc + 1;
  *tc = t;
  cudaGraphSetConditional(cond, (*ndone < ninst && t < maxit) ? 1u : 0u);
}

__global__ void k_scale_f32(const double* __restrict__ src, float* __restrict__ dst,
                            const int32_t* __restrict__ inst_of, const int64_t* __restrict__ ptr,
                            int64_t nlines, const double* __restrict__ scale) {
  // line l (row or column) owns entries [ptr[l], ptr[l+1]); inst_of[l] its
  // instance; dst = src / scale[inst]
  const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= nlines) return;
  const double s = scale[inst_of[l]];
  for (int64_t t = ptr[l] + lane; t < ptr[l + 1]; t += 32) dst[t] = (float)(src[t] / s);
}

__global__ void k_scale_vec(const double* __restrict__ src, float* __restrict__ dst,
                            const int32_t* __restrict__ inst_of, int64_t n,
                            const double* __restrict__ scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = (float)(src[i] / scale[inst_of[i]]);
}

// ---- CheckHalt statistics ---------------------------------------------------
// rows: per chunk sums of [0] primal violation^2, [1] r^2, [2] r y
__global__ void __launch_bounds__(kRedThreads)
k_stats_rows(const int32_t* __restrict__ ch, int64_t nch, const int64_t* __restrict__ Kp,
             const int32_t* __restrict__ Kc, const float* __restrict__ Kv,
             const float* __restrict__ r, const uint8_t* __restrict__ row_eq,
             const float* __restrict__ x, const float* __restrict__ y,
             double* __restrict__ partial) {
  const int64_t c = blockIdx.x;
  if (c >= nch) return;
  const int a = ch[3 * c + 1], e = ch[3 * c + 2];
  double s0 = 0, s1 = 0, s2 = 0;
  // rows longer than kStatLong entries are marked here and summed by the
  // whole block below, in row order (a single thread would walk them alone)
  __shared__ uint32_t lmask[kRowChunk / 32];
  for (int q = threadIdx.x; q < kRowChunk / 32; q += kRedThreads) lmask[q] = 0u;
  __syncthreads();
  for (int j = a + threadIdx.x; j < e; j += kRedThreads) {
    if (Kp[j + 1] - Kp[j] > kStatLong) {
      atomicOr(&lmask[(j - a) >> 5], 1u << ((j - a) & 31));
      continue;
    }
    double v = 0.0;
    for (int64_t t = Kp[j]; t < Kp[j + 1]; ++t) v += (double)Kv[t] * (double)x[Kc[t]];
    v += (double)r[j];
    if (!row_eq[j] && v < 0.0) v = 0.0;
    s0 += v * v;
    s1 += (double)r[j] * (double)r[j];
    s2 += (double)r[j] * (double)y[j];
  }
  __syncthreads();
  for (int q = 0; q < (e - a + 31) / 32; ++q) {
    uint32_t m = lmask[q];                      // the same word in every thread
    while (m) {
      const int j = a + 32 * q + __ffs(m) - 1;
      m &= m - 1u;
      double v = 0.0;
      for (int64_t t = Kp[j] + threadIdx.x; t < Kp[j + 1]; t += kRedThreads)
        v += (double)Kv[t] * (double)x[Kc[t]];
      v = block_sum(v);
      if (threadIdx.x == 0) {
        v += (double)r[j];
        if (!row_eq[j] && v < 0.0) v = 0.0;
        s0 += v * v;
        s1 += (double)r[j] * (double)r[j];
        s2 += (double)r[j] * (double)y[j];
      }
    }
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    partial[c * 8 + 0] = s0; partial[c * 8 + 1] = s1; partial[c * 8 + 2] = s2;
  }
}

// vars: per chunk sums of [3] c x, [4] x (Q x), [5] min(x, 1-x),
// [6] min(0, c + K^T y), [7] ||s^x||^2 with s^x = -dx/tau1 + 2 Q dx - 2 rho dx
__global__ void __launch_bounds__(kRedThreads)
k_stats_vars(const int32_t* __restrict__ ch, int64_t nch, const int64_t* __restrict__ Tp,
             const int32_t* __restrict__ Tr, const float* __restrict__ Tv,
             const int64_t* __restrict__ Qp, const int32_t* __restrict__ Qc,
             const float* __restrict__ Qv, const float* __restrict__ qx_dense,
             const float* __restrict__ qdx_dense, const uint8_t* __restrict__ is_dense,
             const float* __restrict__ chat, const float* __restrict__ x,
             const float* __restrict__ xp, const float* __restrict__ y,
             const uint8_t* __restrict__ live, const GfIParam* __restrict__ ip,
             double* __restrict__ partial) {
  const int64_t c = blockIdx.x;
  if (c >= nch) return;
  const int b = ch[3 * c], a = ch[3 * c + 1], e = ch[3 * c + 2];
  const double tau1 = ip[b].tau1d, rho = ip[b].rhod;
  double s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
  for (int i = a + threadIdx.x; i < e; i += kRedThreads) {
    if (!live[i]) continue;
    const double xi = x[i], dx = (double)x[i] - (double)xp[i];
    double qx = 0.0, qdx = 0.0;
    if (is_dense[b]) {
      qx = qx_dense[i];
      qdx = qdx_dense[i];
    } else if (Qp) {
      for (int64_t t = Qp[i]; t < Qp[i + 1]; ++t) {
        qx += (double)Qv[t] * (double)x[Qc[t]];
        qdx += (double)Qv[t] * ((double)x[Qc[t]] - (double)xp[Qc[t]]);
      }
    }
    double g = (double)chat[i];
    for (int64_t t = Tp[i]; t < Tp[i + 1]; ++t) g += (double)Tv[t] * (double)y[Tr[t]];
    s3 += (double)chat[i] * xi;
    s4 += xi * qx;
    s5 += (xi < 1.0 - xi) ? xi : 1.0 - xi;
    s6 += (g < 0.0) ? g : 0.0;
    const double sx = -dx / tau1 + 2.0 * qdx - 2.0 * rho * dx;
    s7 += sx * sx;
  }
  s3 = block_sum(s3); s4 = block_sum(s4); s5 = block_sum(s5);
  s6 = block_sum(s6); s7 = block_sum(s7);
  if (threadIdx.x == 0) {
    partial[c * 8 + 3] = s3; partial[c * 8 + 4] = s4; partial[c * 8 + 5] = s5;
    partial[c * 8 + 6] = s6; partial[c * 8 + 7] = s7;
  }
}

__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b,
                      float* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host driver of the FP64 power iterations.  which = 0: M = K (CSR rows Kp,
// CSC Tp); which = 1: M = Q_sym (CSR Kp = rows of Q; dense instances use
// their W2 operand).  norms[b] = ||M_b||_2, iters[b] = iterations used.
// Synchronises (host polls the per-instance done counter).
// ---------------------------------------------------------------------------
struct PowerScratch {
  double *v, *w, *z, *lam, *zn2, *partial;
  PwState* ps;
  int* ndone;
  int* tc;                          // step counter of the graph loop
};

// ids of the lines of a CSR (ptr, lines) longer than kPwLong, on the device
static int64_t* long_lines(GfCtx* h, const int64_t* ptr_dev, int64_t lines, int64_t* count,
                           cudaError_t* err) {
  *count = 0;
  *err = cudaSuccess;
  if (lines <= 0) return nullptr;
  std::vector<int64_t> p(lines + 1), ids;
  if ((*err = cudaMemcpy(p.data(), ptr_dev, sizeof(int64_t) * (lines + 1),
                         cudaMemcpyDeviceToHost)))
    return nullptr;
  for (int64_t l = 0; l < lines; ++l)
    if (p[l + 1] - p[l] > kPwLong) ids.push_back(l);
  *count = (int64_t)ids.size();
  if (ids.empty()) return nullptr;
  int64_t* d = gf_alloc_t<int64_t>(h, ids.size());
  if (!d) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  *err = cudaMemcpy(d, ids.data(), sizeof(int64_t) * ids.size(), cudaMemcpyHostToDevice);
  return d;
}

extern "C++" cudaError_t gf_power_run(GfCtx* h, int which, const int64_t* Mp,
                                      const int32_t* Mc, const double* Mv,
                                      const int64_t* Tp, const int32_t* Tr,
                                      const double* Tv, int64_t mrows,
                                      const int32_t* rch, int64_t nrch, const int32_t* rptr,
                                      const double* const* dense_diag,
                                      double* norms, int* iters) {
  cudaStream_t s = h->stream;
  const int64_t N = h->N;
  const int nb = h->ninst;
  PowerScratch S;
  S.v = gf_alloc_t<double>(h, N);
  S.z = gf_alloc_t<double>(h, N);
  S.w = gf_alloc_t<double>(h, which == 0 ? std::max<int64_t>(mrows, 1) : N);
  S.lam = gf_alloc_t<double>(h, nb);
  S.zn2 = gf_alloc_t<double>(h, nb);
  S.partial = gf_alloc_t<double>(h, std::max(nrch, h->nvchunk) + 1);
  S.ps = gf_alloc_t<PwState>(h, nb);
  S.ndone = gf_alloc_t<int>(h, 1);
  S.tc = gf_alloc_t<int>(h, 1);
  if (!S.v || !S.z || !S.w || !S.lam || !S.zn2 || !S.partial || !S.ps || !S.ndone || !S.tc)
    return cudaErrorMemoryAllocation;
  cudaError_t e;
  // long lines of the two products (one block each)
  int64_t nlr = 0, nlc = 0;
  const int64_t* lr = nullptr;
  const int64_t* lc = nullptr;
  if (which == 0) {
    lr = long_lines(h, Mp, mrows, &nlr, &e);
    if (e) return e;
    lc = long_lines(h, Tp, N, &nlc, &e);
    if (e) return e;
  } else if (Mp) {
    lr = long_lines(h, Mp, N, &nlr, &e);
    if (e) return e;
  }
  // instances without the matrix are done from the start
  std::vector<PwState> init(nb);
  int pre_done = 0;
  for (int b = 0; b < nb; ++b) {
    const GfInstHost& I = h->ih[b];
    bool has = (which == 0) ? (I.m1 + I.m2 > 0) : (I.qkind != 0);
    init[b] = PwState{0, 0, 0, has ? 0 : 1, 0, 0, 0};
    pre_done += has ? 0 : 1;
  }
  if ((e = cudaMemcpyAsync(S.ps, init.data(), sizeof(PwState) * nb, cudaMemcpyHostToDevice, s)))
    return e;
  if ((e = cudaMemcpyAsync(S.ndone, &pre_done, sizeof(int), cudaMemcpyHostToDevice, s))) return e;
  k_pw_start<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(S.v, h->var_inst, h->var_off_d,
                                                         h->var_live, N, h->prm.seed,
                                                         h->prm.inst_base, which);
  // normalise the start vector: v /= ||v|| per instance
  k_chunk_sumsq<<<(unsigned)h->nvchunk, kRedThreads, 0, s>>>(S.v, h->vchunk, h->nvchunk,
                                                              S.partial);
  k_inst_sum<<<(nb + 127) / 128, 128, 0, s>>>(S.partial, h->vchunk_iptr, nb, 1, 1, S.zn2);
  {
    // all instances normalise their start vector
    std::vector<PwState> up(init);
    for (auto& u : up) u.upd = 1;
    PwState* tmp = gf_alloc_t<PwState>(h, nb);
    if (!tmp) return cudaErrorMemoryAllocation;
    cudaMemcpyAsync(tmp, up.data(), sizeof(PwState) * nb, cudaMemcpyHostToDevice, s);
    k_pw_normalize<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(S.v, S.v, S.zn2, h->var_inst,
                                                               tmp, N);
    if ((e = cudaStreamSynchronize(s))) return e;
  }
  const int maxit = h->prm.power_maxit > 0 ? h->prm.power_maxit : 5000;
  const double tol = h->prm.power_tol > 0 ? h->prm.power_tol : 1e-12;
  // lanes per row of M from its mean row length (rows of two nonzeros get
  // one thread, rows of hundreds a warp)
  const double mean_len = mrows > 0 ? (double)h->nnzK / (double)mrows : 0.0;
  const int rl = mean_len <= 4 ? 1 : mean_len <= 16 ? 4 : mean_len <= 64 ? 8 : 32;
  auto product = [&](const double* in, double* out, bool transpose) {
    if (which == 0) {
      if (!transpose) {
        const unsigned nblk = (unsigned)((mrows * rl + 255) / 256);
        if (rl == 1) k_spmv64<1><<<nblk, 256, 0, s>>>(Mp, Mc, Mv, in, mrows, out);
        else if (rl == 4) k_spmv64<4><<<nblk, 256, 0, s>>>(Mp, Mc, Mv, in, mrows, out);
        else if (rl == 8) k_spmv64<8><<<nblk, 256, 0, s>>>(Mp, Mc, Mv, in, mrows, out);
        else k_spmv64<32><<<nblk, 256, 0, s>>>(Mp, Mc, Mv, in, mrows, out);
        if (nlr) k_spmv64_long<<<(unsigned)nlr, kRedThreads, 0, s>>>(Mp, Mc, Mv, in, lr, out);
      } else {
        k_spmv64<4><<<(unsigned)((N * 4 + 255) / 256), 256, 0, s>>>(Tp, Tr, Tv, in, N, out);
        if (nlc) k_spmv64_long<<<(unsigned)nlc, kRedThreads, 0, s>>>(Tp, Tr, Tv, in, lc, out);
      }
    } else {
      if (Mp) {
        k_spmv64<4><<<(unsigned)((N * 4 + 255) / 256), 256, 0, s>>>(Mp, Mc, Mv, in, N, out);
        if (nlr) k_spmv64_long<<<(unsigned)nlr, kRedThreads, 0, s>>>(Mp, Mc, Mv, in, lr, out);
      } else {
        cudaMemsetAsync(out, 0, sizeof(double) * N, s);
      }
      for (size_t q = 0; q < h->dense.size(); ++q) {
        const GfDenseQ& dq = h->dense[q];
        k_dense64<<<(unsigned)((dq.n * 32 + 255) / 256), 256, 0, s>>>(
            dq.W2, dq.ld, dq.n, h->ih[dq.inst].var_off, dense_diag[q], in, out);
      }
    }
  };
  // the iteration loop as ONE graph launch: a while node whose body is one
  // step (products, reductions, bookkeeping, normalisation, counter)
  if (pre_done < nb) {
    if ((e = cudaMemsetAsync(S.tc, 0, sizeof(int), s))) return e;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaGraphConditionalHandle hc;
    if ((e = cudaGraphCreate(&g, 0))) return e;
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
    if (!e) e = cudaStreamBeginCaptureToGraph(s, np.conditional.phGraph_out[0], nullptr, nullptr,
                                              0, cudaStreamCaptureModeRelaxed);
    if (!e) {
      product(S.v, S.w, false);
      if (which == 0) {
        k_chunk_sumsq<<<(unsigned)nrch, kRedThreads, 0, s>>>(S.w, rch, nrch, S.partial);
        k_inst_sum<<<(nb + 127) / 128, 128, 0, s>>>(S.partial, rptr, nb, 1, 1, S.lam);
      } else {
        k_chunk_sumsq<<<(unsigned)h->nvchunk, kRedThreads, 0, s>>>(S.w, h->vchunk, h->nvchunk,
                                                                    S.partial);
        k_inst_sum<<<(nb + 127) / 128, 128, 0, s>>>(S.partial, h->vchunk_iptr, nb, 1, 1,
                                                     S.lam);
      }
      product(S.w, S.z, true);
      k_chunk_sumsq<<<(unsigned)h->nvchunk, kRedThreads, 0, s>>>(S.z, h->vchunk, h->nvchunk,
                                                                  S.partial);
      k_inst_sum<<<(nb + 127) / 128, 128, 0, s>>>(S.partial, h->vchunk_iptr, nb, 1, 1, S.zn2);
      k_pw_step<<<(nb + 127) / 128, 128, 0, s>>>(S.ps, S.lam, S.zn2, nb, S.tc, tol, maxit,
                                                  S.ndone);
      k_pw_normalize<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(S.v, S.z, S.zn2, h->var_inst,
                                                                 S.ps, N);
      k_pw_next<<<1, 1, 0, s>>>(S.tc, S.ndone, nb, maxit, hc);
      cudaError_t ec = cudaGetLastError();
      cudaGraph_t out = nullptr;
      cudaError_t ee = cudaStreamEndCapture(s, &out);
      e = ec ? ec : ee;
    }
    if (!e) e = cudaGraphInstantiate(&ge, g, 0);
    if (!e) e = cudaGraphLaunch(ge, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (ge) cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    if (e) return e;
    h->launches += 1;
  }
  std::vector<PwState> fin(nb);
  if ((e = cudaMemcpyAsync(fin.data(), S.ps, sizeof(PwState) * nb, cudaMemcpyDeviceToHost, s)))
    return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  for (int b = 0; b < nb; ++b) {
    norms[b] = sqrt(fin[b].result);
    iters[b] = fin[b].iters;
  }
  return cudaSuccess;
}

cudaError_t gf_scale_to_f32(GfCtx* h, const double* Kd, const double* Td, const double* rd,
                            const double* cd, const double* Qd, const double* sK,
                            const double* sobj) {
  cudaStream_t s = h->stream;
  if (h->M) {
    k_scale_f32<<<(unsigned)((h->M * 32 + 255) / 256), 256, 0, s>>>(Kd, h->Kv, h->row_inst,
                                                                    h->Kp, h->M, sK);
    k_scale_vec<<<(unsigned)((h->M + 255) / 256), 256, 0, s>>>(rd, h->rhat, h->row_inst, h->M,
                                                               sK);
  }
  k_scale_f32<<<(unsigned)((h->N * 32 + 255) / 256), 256, 0, s>>>(Td, h->Tv, h->var_inst, h->Tp,
                                                                  h->N, sK);
  k_scale_vec<<<(unsigned)((h->N + 255) / 256), 256, 0, s>>>(cd, h->chat, h->var_inst, h->N,
                                                             sobj);
  if (h->nnzQ)
    k_scale_f32<<<(unsigned)((h->N * 32 + 255) / 256), 256, 0, s>>>(Qd, h->Qv, h->var_inst,
                                                                    h->Qp, h->N, sobj);
  return cudaGetLastError();
}

// FP64 CheckHalt sums of every instance at x_k (x[k&1]), x_{k-1}, y_k into
// h->stats[b][8] (device).
cudaError_t gf_launch_stats(GfCtx* h) {
  cudaStream_t s = h->stream;
  const int par = (int)(h->k_host & 1);
  const float* x = h->x[par];
  const float* xp = h->x[1 - par];
  // iteration k's parameters live in slot k & 1
  const GfIParam* ip = h->iprm + (size_t)par * h->ninst;
  cudaError_t e;
  for (const GfDenseQ& dq : h->dense) {
    const int64_t v0 = h->ih[dq.inst].var_off;
    if ((e = gf_launch_dense_gemv_q(h, dq, x, h->qbuf + v0))) return e;
    k_sub<<<(unsigned)((h->N + 255) / 256), 256, 0, s>>>(x, xp, h->dxbuf, h->N);
    if ((e = gf_launch_dense_gemv_q(h, dq, h->dxbuf, h->qbuf2 + v0))) return e;
  }
  if ((e = cudaMemsetAsync(h->stats_part, 0,
                           sizeof(double) * 8 * (h->nrchunk + h->nvchunk + 1), s)))
    return e;
  if (h->nrchunk) {
    k_stats_rows<<<(unsigned)h->nrchunk, kRedThreads, 0, s>>>(
        h->rchunk, h->nrchunk, h->Kp, h->Kc, h->Kv, h->rhat, h->row_eq, x, h->y,
        h->stats_part);
  }
  k_stats_vars<<<(unsigned)h->nvchunk, kRedThreads, 0, s>>>(
      h->vchunk, h->nvchunk, h->Tp, h->Tr, h->Tv, h->nnzQ ? h->Qp : nullptr, h->Qc, h->Qv,
      h->qbuf, h->qbuf2, h->inst_dense, h->chat, x, xp, h->y, h->var_live, ip,
      h->stats_part + 8 * h->nrchunk);
  h->launches += 2;
  // rows: chunks of instance b are [rchunk_iptr[b], ...); vars likewise
  k_inst_sum<<<(h->ninst + 127) / 128, 128, 0, s>>>(h->stats_part, h->rchunk_iptr, h->ninst, 8,
                                                     8, h->stats);
  k_inst_sum<<<(h->ninst + 127) / 128, 128, 0, s>>>(h->stats_part + 8 * h->nrchunk,
                                                     h->vchunk_iptr, h->ninst, 8, 8,
                                                     h->stats2);
  h->launches += 2;
  return cudaGetLastError();
}
