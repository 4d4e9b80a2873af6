// k_mlp.cu -- learned proposal: per-variable features, a 2-hidden-layer MLP
// (F = 8 -> H = 128 -> 128 -> 1) mapping them to sampling probabilities,
// and its training kernels (mean BCE on the logit, backward, Adam).  The
// paper has no such network; it is an added pattern whose output replaces
// p = x_k as the input of RandSampleStep (Alg. 3 / Section 2.4.2), with the
// plain form kept as fallback and reference.
//
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3,
//   p  = clip(sigmoid(z), 2^-24, 1 - 2^-24).
// Weights (not biases, not activations) are rounded to bf16 (round to
// nearest even) when staged; arithmetic is FP32.  Gradients are taken with
// respect to the FP32 masters, the rounding passed straight through.  The
// forward pass used for sampling runs on the tensor cores (k_mlp_tc.cu)
// with the same numerics; the gradient pass here recomputes its own forward.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "internal.cuh"

cudaError_t gf_mlp_forward_tc(const float* W, int64_t nv, const float* feat, float* z,
                              float* p, const uint8_t* live, uint64_t limit_ns, int* err,
                              cudaStream_t s);

namespace {

constexpr int kF = 8, kH = 128;
constexpr int64_t kNP = (int64_t)kH * kF + kH + (int64_t)kH * kH + kH + kH + 1;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH;

GF_DEV float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Stage weights (bf16-rounded) and biases in shared memory.
struct alignas(16) MlpSmem {   // every array 16-byte aligned (float4 reads)
  alignas(16) float W1[kH * kF];
  alignas(16) float b1[kH];
  alignas(16) float W2[kH * kH];
  alignas(16) float b2[kH];
  alignas(16) float w3[kH];
  float b3;
};

GF_DEV void stage_weights(MlpSmem& S, const float* __restrict__ W) {
  for (int t = threadIdx.x; t < kH * kF; t += blockDim.x) S.W1[t] = bf16r(W[oW1 + t]);
  for (int t = threadIdx.x; t < kH * kH; t += blockDim.x) S.W2[t] = bf16r(W[oW2 + t]);
  for (int t = threadIdx.x; t < kH; t += blockDim.x) {
    S.b1[t] = W[oB1 + t];
    S.b2[t] = W[oB2 + t];
    S.w3[t] = bf16r(W[oW3 + t]);
  }
  if (threadIdx.x == 0) S.b3 = W[oB3];
  __syncthreads();
}

// Loss and gradient over a block of 128 variables (one per thread).  The
// block keeps h1 and h2 (then dh2, dh1) as [128 variables x 128 units] tiles
// in shared memory, so the weight gradients are sums over the tile computed
// unit by unit; each block writes its partial gradient, reduced afterwards
// in block order (deterministic).
struct alignas(16) GradSmem {
  MlpSmem w;
  alignas(16) float H1[128 * kH];     // h1, later dh1
  alignas(16) float H2[128 * kH];     // pre-activation h2, later dh2
  alignas(16) float F[128 * kF];
  alignas(16) float dz[128];
};

__global__ void __launch_bounds__(128, 1)
k_mlp_grad(const float* __restrict__ W, int64_t nv, const float* __restrict__ feat,
           const float* __restrict__ label, float* __restrict__ part, double* __restrict__ lpart) {
  extern __shared__ float4 smem4[];
  GradSmem& S = *reinterpret_cast<GradSmem*>(smem4);
  stage_weights(S.w, W);
  const int t = threadIdx.x;
  const int64_t v = (int64_t)blockIdx.x * 128 + t;
  const bool act = v < nv;
  float f[kF];
#pragma unroll
  for (int q = 0; q < kF; ++q) {
    f[q] = act ? feat[v * kF + q] : 0.0f;
    S.F[t * kF + q] = f[q];
  }
  // forward, keeping h1 and the pre-activations of h2 in shared memory
  float z = S.w.b3;
  {
    float h1[kH];
#pragma unroll
    for (int a = 0; a < kH; ++a) {
      float s = S.w.b1[a];
#pragma unroll
      for (int q = 0; q < kF; ++q) s = fmaf(S.w.W1[a * kF + q], f[q], s);
      h1[a] = fmaxf(s, 0.0f);
      S.H1[t * kH + a] = h1[a];
    }
    for (int a = 0; a < kH; ++a) {
      const float4* w = reinterpret_cast<const float4*>(S.w.W2 + a * kH);
      float s = S.w.b2[a];
#pragma unroll
      for (int q4 = 0; q4 < kH / 4; ++q4) {
        const float4 ww = w[q4];
        s = fmaf(ww.x, h1[4 * q4], s);
        s = fmaf(ww.y, h1[4 * q4 + 1], s);
        s = fmaf(ww.z, h1[4 * q4 + 2], s);
        s = fmaf(ww.w, h1[4 * q4 + 3], s);
      }
      S.H2[t * kH + a] = s;
      z = fmaf(S.w.w3[a], fmaxf(s, 0.0f), z);
    }
  }
  // mean BCE on the logit: softplus(z) - y z;  dL/dz = (sigmoid(z) - y) / nv
  double lossv = 0.0;
  float dz = 0.0f;
  if (act) {
    const float y = label[v];
    const double zd = z;
    lossv = (zd > 0.0 ? zd + log1p(exp(-zd)) : log1p(exp(zd))) - (double)y * zd;
    dz = (1.0f / (1.0f + expf(-z)) - y) / (float)nv;
  }
  S.dz[t] = dz;
  __syncthreads();
  float* g = part + (int64_t)blockIdx.x * kNP;
  // thread t owns unit a = t: dw3, db2, dW2 row a (needs h2 and dh2 columns)
  {
    const int a = t;
    float gw3 = 0.0f, gb2 = 0.0f;
    float acc[kH];
#pragma unroll
    for (int q = 0; q < kH; ++q) acc[q] = 0.0f;
    for (int u = 0; u < 128; ++u) {
      const float pre = S.H2[u * kH + a];
      const float d = S.dz[u];
      gw3 = fmaf(d, fmaxf(pre, 0.0f), gw3);
      const float dh2 = (pre > 0.0f) ? d * S.w.w3[a] : 0.0f;
      if (dh2 != 0.0f) {
        gb2 += dh2;
        const float4* h = reinterpret_cast<const float4*>(S.H1 + u * kH);
#pragma unroll
        for (int q4 = 0; q4 < kH / 4; ++q4) {
          const float4 hh = h[q4];
          acc[4 * q4] = fmaf(dh2, hh.x, acc[4 * q4]);
          acc[4 * q4 + 1] = fmaf(dh2, hh.y, acc[4 * q4 + 1]);
          acc[4 * q4 + 2] = fmaf(dh2, hh.z, acc[4 * q4 + 2]);
          acc[4 * q4 + 3] = fmaf(dh2, hh.w, acc[4 * q4 + 3]);
        }
      }
    }
    g[oW3 + a] = gw3;
    g[oB2 + a] = gb2;
#pragma unroll
    for (int q = 0; q < kH; ++q) g[oW2 + a * kH + q] = acc[q];
  }
  __syncthreads();
  // dh2 in place of the pre-activations
  for (int e = t; e < 128 * kH; e += 128) {
    const int u = e / kH, a = e % kH;
    S.H2[e] = (S.H2[e] > 0.0f) ? S.dz[u] * S.w.w3[a] : 0.0f;
  }
  __syncthreads();
  // thread t = variable: dh1 = (W2^T dh2) * [h1 > 0]
  {
    float dh1[kH];
#pragma unroll
    for (int q = 0; q < kH; ++q) dh1[q] = 0.0f;
    for (int a = 0; a < kH; ++a) {
      const float d = S.H2[t * kH + a];
      if (d == 0.0f) continue;
      const float4* w = reinterpret_cast<const float4*>(S.w.W2 + a * kH);
#pragma unroll
      for (int q4 = 0; q4 < kH / 4; ++q4) {
        const float4 ww = w[q4];
        dh1[4 * q4] = fmaf(d, ww.x, dh1[4 * q4]);
        dh1[4 * q4 + 1] = fmaf(d, ww.y, dh1[4 * q4 + 1]);
        dh1[4 * q4 + 2] = fmaf(d, ww.z, dh1[4 * q4 + 2]);
        dh1[4 * q4 + 3] = fmaf(d, ww.w, dh1[4 * q4 + 3]);
      }
    }
    __syncthreads();   // every thread done reading H1 as h1 (dW2 pass above)
#pragma unroll
    for (int q = 0; q < kH; ++q) S.H1[t * kH + q] = (S.H1[t * kH + q] > 0.0f) ? dh1[q] : 0.0f;
  }
  __syncthreads();
  // thread t owns unit a = t: dW1 row a, db1
  {
    const int a = t;
    float gb1 = 0.0f, gw[kF];
#pragma unroll
    for (int q = 0; q < kF; ++q) gw[q] = 0.0f;
    for (int u = 0; u < 128; ++u) {
      const float d = S.H1[u * kH + a];
      gb1 += d;
#pragma unroll
      for (int q = 0; q < kF; ++q) gw[q] = fmaf(d, S.F[u * kF + q], gw[q]);
    }
    g[oB1 + a] = gb1;
#pragma unroll
    for (int q = 0; q < kF; ++q) g[oW1 + a * kF + q] = gw[q];
  }
  // loss partial and db3
  __shared__ double lred[128];
  __shared__ float dred[128];
  lred[t] = lossv;
  dred[t] = dz;
  __syncthreads();
  for (int off = 64; off > 0; off >>= 1) {
    if (t < off) {
      lred[t] += lred[t + off];
      dred[t] += dred[t + off];
    }
    __syncthreads();
  }
  if (t == 0) {
    g[oB3] = dred[0];
    lpart[blockIdx.x] = lred[0];
  }
}

// grad[p] = sum over blocks (in block order) of part[b][p]; loss likewise.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk,
                             const double* __restrict__ lpart, float* __restrict__ grad,
                             double* __restrict__ loss, int64_t nv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNP) {
    float s = 0.0f, c = 0.0f;            // compensated
    for (int b = 0; b < nblk; ++b) {
      const float v = part[(int64_t)b * kNP + p];
      const float tt = s + v;
      const float zz = tt - s;
      c += (s - (tt - zz)) + (v - zz);
      s = tt;
    }
    grad[p] = s + c;
  }
  if (p == 0 && loss) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += lpart[b];
    *loss = s / (double)nv;
  }
}

__global__ void k_adam(int64_t np, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, double c1, double c2,
                       float lr, float b1, float b2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = (float)(mi / c1), vh = (float)(vi / c2);
  w[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ---- features -----------------------------------------------------------
// 1 standardised cost (c_hat - mean) / sd over the instance, 2 column degree
// / max degree, 3 x_k, 4 x_k - x at the previous trigger, 5 the standardised
// cost above the cheapest member of the variable's group (one-hot group or
// axial slab x_i**; the whole instance when ungrouped), 6 x / max of x over
// the variable's group (x itself when ungrouped), 7 tau1 delta of the last
// primal step, 8 rho / rho_max.
__global__ void k_group_max(const int64_t* __restrict__ gp, const int64_t* __restrict__ gi,
                            int64_t ngroups, const float* __restrict__ x,
                            float* __restrict__ gmax) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= ngroups) return;
  float m = 0.0f;
  for (int64_t t = gp[g] + lane; t < gp[g + 1]; t += 32) m = fmaxf(m, x[gi[t]]);
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
  for (int64_t t = gp[g] + lane; t < gp[g + 1]; t += 32) gmax[gi[t]] = m;
}

__global__ void k_slab_max(const float* __restrict__ x, int64_t v0, int I,
                           float* __restrict__ gmax) {
  const int i = blockIdx.x;               // slab x_i** of an axial instance
  const int64_t P = (int64_t)I * I;
  float m = 0.0f;
  for (int64_t q = threadIdx.x; q < P; q += blockDim.x) m = fmaxf(m, x[v0 + i * P + q]);
  __shared__ float red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  for (int64_t q = threadIdx.x; q < P; q += blockDim.x) gmax[v0 + i * P + q] = red[0];
}

__global__ void k_features(int64_t N, const float* __restrict__ x, const float* __restrict__ xprev_trig,
                           const float* __restrict__ crel,
                           const float* __restrict__ cstd, const float* __restrict__ degn,
                           const float* __restrict__ gmax, const uint8_t* __restrict__ grouped,
                           const float* __restrict__ dlast, const uint8_t* __restrict__ live,
                           const GfDState* __restrict__ st, double rho_max,
                           float* __restrict__ feat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // rho of the next iteration from the device state (a captured launch
  // replays with the current penalty)
  const float rho_frac = (float)(rho_max > 0.0 ? st->rho / rho_max : 0.0);
  float f[kF];
  if (!live[i]) {
#pragma unroll
    for (int q = 0; q < kF; ++q) f[q] = 0.0f;
  } else {
    const float xi = x[i];
    f[0] = cstd[i];
    f[1] = degn[i];
    f[2] = xi;
    f[3] = xi - xprev_trig[i];
    f[4] = crel[i];
    f[5] = grouped[i] ? (gmax[i] > 0.0f ? xi / gmax[i] : 0.0f) : xi;
    f[6] = dlast[i];
    f[7] = rho_frac;
  }
#pragma unroll
  for (int q = 0; q < kF; ++q) feat[i * kF + q] = f[q];
}

static_assert(offsetof(MlpSmem, W2) % 16 == 0, "W2 must be 16-byte aligned");
static_assert(offsetof(GradSmem, H1) % 16 == 0 && offsetof(GradSmem, H2) % 16 == 0,
              "tiles must be 16-byte aligned");
size_t grad_smem() { return sizeof(GradSmem) + 16; }

cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)grad_smem());
  if (!e) done = true;
  return e;
}

// Forward pass on the tensor cores (k_mlp_tc.cu); err: device error word
// of a handle, or NULL (outputs NaN if the tensor cores never answered).
cudaError_t mlp_forward(const float* W, int64_t nv, const float* feat, float* z, float* p,
                        const uint8_t* live, cudaStream_t s, uint64_t limit_ns = 2000000000ull,
                        int* err = nullptr) {
  return gf_mlp_forward_tc(W, nv, feat, z, p, live, limit_ns, err, s);
}

}  // namespace

extern "C" int64_t gfors_mlp_nparams(int32_t F, int32_t H) {
  if (F <= 0 || H <= 0) return 0;
  return (int64_t)H * F + H + (int64_t)H * H + H + H + 1;
}

extern "C" gfors_status gfors_mlp_forward(int32_t F, int32_t H, const float* W_dev, int64_t nv,
                                          const float* feat_dev, float* z_dev, float* p_dev,
                                          void* cuda_stream) {
  if (F != kF || H != kH) {
    gf_fail(nullptr, GFORS_E_UNSUPPORTED, "MLP kernels are built for F = 8, H = 128");
    return GFORS_E_UNSUPPORTED;
  }
  if (nv < 0 || !W_dev || (nv > 0 && (!feat_dev || !z_dev))) {
    gf_fail(nullptr, GFORS_E_ARG, "gfors_mlp_forward: bad arguments");
    return GFORS_E_ARG;
  }
  if (nv == 0) return GFORS_OK;
  cudaError_t e = mlp_forward(W_dev, nv, feat_dev, z_dev, p_dev, nullptr,
                              (cudaStream_t)cuda_stream);
  if (e) {
    gf_fail(nullptr, GFORS_E_CUDA, std::string("gfors_mlp_forward: ") + cudaGetErrorString(e));
    return GFORS_E_CUDA;
  }
  return GFORS_OK;
}

// The gradient pass needs block partials; they live in a per-call scratch
// taken from the allocation hook / cudaMalloc and freed stream-ordered.
extern "C" gfors_status gfors_mlp_loss_grad(int32_t F, int32_t H, const float* W_dev, int64_t nv,
                                            const float* feat_dev, const float* label_dev,
                                            float* grad_dev, double* loss_dev,
                                            void* cuda_stream) {
  if (F != kF || H != kH) {
    gf_fail(nullptr, GFORS_E_UNSUPPORTED, "MLP kernels are built for F = 8, H = 128");
    return GFORS_E_UNSUPPORTED;
  }
  if (nv <= 0 || !W_dev || !feat_dev || !label_dev || !grad_dev) {
    gf_fail(nullptr, GFORS_E_ARG, "gfors_mlp_loss_grad: bad arguments");
    return GFORS_E_ARG;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = set_attrs();
  const int nblk = (int)((nv + 127) / 128);
  float* part = nullptr;
  double* lpart = nullptr;
  if (!e) e = cudaMallocAsync((void**)&part, sizeof(float) * kNP * (size_t)nblk, s);
  if (!e) e = cudaMallocAsync((void**)&lpart, sizeof(double) * (size_t)nblk, s);
  if (!e) {
    k_mlp_grad<<<nblk, 128, grad_smem(), s>>>(W_dev, nv, feat_dev, label_dev, part, lpart);
    k_mlp_reduce<<<(unsigned)((kNP + 255) / 256), 256, 0, s>>>(part, nblk, lpart, grad_dev,
                                                               loss_dev, nv);
    e = cudaGetLastError();
  }
  if (part) cudaFreeAsync(part, s);
  if (lpart) cudaFreeAsync(lpart, s);
  if (e) {
    gf_fail(nullptr, GFORS_E_CUDA, std::string("gfors_mlp_loss_grad: ") + cudaGetErrorString(e));
    return GFORS_E_CUDA;
  }
  return GFORS_OK;
}

extern "C" gfors_status gfors_mlp_adam(int64_t np, float* W_dev, const float* grad_dev,
                                       float* m_dev, float* v_dev, int64_t t, double lr,
                                       double beta1, double beta2, double eps,
                                       void* cuda_stream) {
  if (np <= 0 || t < 1 || !W_dev || !grad_dev || !m_dev || !v_dev) {
    gf_fail(nullptr, GFORS_E_ARG, "gfors_mlp_adam: bad arguments");
    return GFORS_E_ARG;
  }
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  k_adam<<<(unsigned)((np + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      np, W_dev, grad_dev, m_dev, v_dev, c1, c2, (float)lr, (float)beta1, (float)beta2,
      (float)eps);
  cudaError_t e = cudaGetLastError();
  if (e) {
    gf_fail(nullptr, GFORS_E_CUDA, std::string("gfors_mlp_adam: ") + cudaGetErrorString(e));
    return GFORS_E_CUDA;
  }
  return GFORS_OK;
}

// ---- solver integration ---------------------------------------------------
static cudaError_t ensure_feature_buffers(GfCtx* h) {
  if (h->feat && h->feat_grp_version == h->grp_version) return cudaSuccess;
  const int64_t N = h->N;
  if (!h->feat) {
    h->feat = gf_alloc_t<float>(h, (size_t)N * kF);
    h->x_trig_prev = gf_alloc_t<float>(h, N);
    h->p_learn = gf_alloc_t<float>(h, N);
    h->degnorm = gf_alloc_t<float>(h, N);
    h->cstd = gf_alloc_t<float>(h, N);
    h->crel = gf_alloc_t<float>(h, N);
    h->grpmax = gf_alloc_t<float>(h, N);
    if (!h->feat || !h->x_trig_prev || !h->p_learn || !h->degnorm || !h->cstd || !h->crel ||
        !h->grpmax)
      return cudaErrorMemoryAllocation;
  }
  // static features: standardised cost, normalised column degree, and the
  // standardised cost above its group's cheapest member
  std::vector<float> cs(N, 0.0f), dg(N, 0.0f), cr(N, 0.0f);
  std::vector<float> chat(N);
  std::vector<int64_t> Tp(N + 1), Qp(N + 1);
  cudaError_t e;
  if ((e = cudaMemcpy(chat.data(), h->chat, sizeof(float) * N, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(Tp.data(), h->Tp, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(Qp.data(), h->Qp, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost)))
    return e;
  for (int b = 0; b < h->ninst; ++b) {
    const GfInstHost& I = h->ih[b];
    double mu = 0.0, sd = 0.0;
    int64_t dmax = 1;
    for (int64_t i = 0; i < I.n; ++i) mu += chat[I.var_off + i];
    mu /= (double)I.n;
    for (int64_t i = 0; i < I.n; ++i) {
      const double d = chat[I.var_off + i] - mu;
      sd += d * d;
      const int64_t v = I.var_off + i;
      const int64_t deg = (Tp[v + 1] - Tp[v]) + (Qp[v + 1] - Qp[v]) + (I.qkind == 1 ? I.n : 0);
      dmax = std::max(dmax, deg);
    }
    sd = sqrt(sd / (double)I.n);
    float cmin = INFINITY;
    for (int64_t i = 0; i < I.n; ++i) {
      const int64_t v = I.var_off + i;
      cs[v] = sd > 0.0 ? (float)((chat[v] - mu) / sd) : 0.0f;
      cmin = std::min(cmin, cs[v]);
      const int64_t deg = (Tp[v + 1] - Tp[v]) + (Qp[v + 1] - Qp[v]) + (I.qkind == 1 ? I.n : 0);
      dg[v] = (float)deg / (float)dmax;
    }
    for (int64_t i = 0; i < I.n; ++i) cr[I.var_off + i] = cs[I.var_off + i] - cmin;
    if ((I.group_mode == 2 || I.group_mode == 3) && I.axial_I > 0) {
      const int64_t P = (int64_t)I.axial_I * I.axial_I;        // slab x_i** of the axial form
      for (int64_t a = 0; a < I.axial_I; ++a) {
        const int64_t v0 = I.var_off + a * P;
        float m = INFINITY;
        for (int64_t q = 0; q < P; ++q) m = std::min(m, cs[v0 + q]);
        for (int64_t q = 0; q < P; ++q) cr[v0 + q] = cs[v0 + q] - m;
      }
    }
  }
  for (int64_t g = 0; g < h->ngroups_tot; ++g) {             // one-hot groups
    float m = INFINITY;
    for (int64_t t = h->h_grp_ptr[g]; t < h->h_grp_ptr[g + 1]; ++t)
      m = std::min(m, cs[h->h_grp_idx[t]]);
    for (int64_t t = h->h_grp_ptr[g]; t < h->h_grp_ptr[g + 1]; ++t)
      cr[h->h_grp_idx[t]] = cs[h->h_grp_idx[t]] - m;
  }
  if ((e = cudaMemcpy(h->cstd, cs.data(), sizeof(float) * N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->degnorm, dg.data(), sizeof(float) * N, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->crel, cr.data(), sizeof(float) * N, cudaMemcpyHostToDevice)))
    return e;
  if (h->feat_grp_version < 0) {
    const float* xk = h->x[h->k_host & 1];
    if ((e = cudaMemcpyAsync(h->x_trig_prev, xk, sizeof(float) * N, cudaMemcpyDeviceToDevice,
                             h->stream)))
      return e;
  }
  h->feat_grp_version = h->grp_version;
  return cudaSuccess;
}

cudaError_t gf_prepare_features(GfCtx* h) { return ensure_feature_buffers(h); }

// Features at the current iterate; called once per sampling trigger, it also
// pushes x_k into the trigger history.
cudaError_t gf_launch_features(GfCtx* h) {
  cudaError_t e = ensure_feature_buffers(h);
  if (e) return e;
  const int64_t N = h->N;
  cudaStream_t s = h->stream;
  const float* xk = h->x[h->k_host & 1];
  if (h->ngroups_tot)
    k_group_max<<<(unsigned)((h->ngroups_tot * 32 + 255) / 256), 256, 0, s>>>(
        h->grp_ptr, h->grp_idx, h->ngroups_tot, xk, h->grpmax);
  for (int b = 0; b < h->ninst; ++b)
    if (h->ih[b].group_mode == 2 || h->ih[b].group_mode == 3)
      k_slab_max<<<h->ih[b].axial_I, 256, 0, s>>>(xk, h->ih[b].var_off, h->ih[b].axial_I,
                                                  h->grpmax);
  k_features<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
      N, xk, h->x_trig_prev, h->crel, h->cstd, h->degnorm, h->grpmax,
      h->var_grouped_feat, h->dlast, h->var_live, h->dstate, h->prm.rho_max, h->feat);
  h->launches += 1 + (h->ngroups_tot ? 1 : 0);
  if ((e = cudaGetLastError())) return e;
  // remember x_k for the next trigger's trajectory feature
  return cudaMemcpyAsync(h->x_trig_prev, xk, sizeof(float) * N, cudaMemcpyDeviceToDevice, s);
}

cudaError_t gf_launch_mlp_proposal(GfCtx* h) {
  if (!h->mlp_W || !h->feat) return cudaErrorInvalidValue;
  h->launches++;
  const uint64_t limit = (uint64_t)(std::max(0.01, h->prm.wait_timeout_s) * 1e9);
  return mlp_forward(h->mlp_W, h->N, h->feat, h->p_learn_z, h->p_learn, h->var_live, h->stream,
                     limit, &h->dstate->error);
}

extern "C" gfors_status gfors_set_proposal(gfors_handle h, const float* W, int64_t nW) {
  if (!h) return GFORS_E_ARG;
  if (h->failed) return GFORS_E_STATE;
  if (!W || nW != kNP) return gf_fail(h, GFORS_E_ARG, "weights must hold gfors_mlp_nparams(8,128)");
  if (!h->mlp_W) {
    h->mlp_W = gf_alloc_t<float>(h, kNP);
    h->p_learn_z = gf_alloc_t<float>(h, h->N);
    if (!h->mlp_W || !h->p_learn_z) return gf_fail(h, GFORS_E_OOM, "proposal weights");
  }
  cudaError_t e = cudaMemcpyAsync(h->mlp_W, W, sizeof(float) * kNP, cudaMemcpyHostToDevice,
                                  h->stream);
  if (!e) e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "gfors_set_proposal");
  h->mlp_np = kNP;
  cudaError_t e2 = ensure_feature_buffers(h);
  if (e2) return gf_cuda(h, e2, "feature buffers");
  return GFORS_OK;
}

extern "C" gfors_status gfors_get_features(gfors_handle h, int32_t inst, float* feat) {
  if (!h) return GFORS_E_ARG;
  if (h->failed) return GFORS_E_STATE;
  if (inst < 0 || inst >= h->ninst || !feat) return gf_fail(h, GFORS_E_ARG, "bad arguments");
  cudaError_t e = gf_launch_features(h);
  if (e) return gf_cuda(h, e, "features");
  const GfInstHost& I = h->ih[inst];
  e = cudaMemcpyAsync(feat, h->feat + I.var_off * kF, sizeof(float) * kF * I.n,
                      cudaMemcpyDeviceToHost, h->stream);
  if (!e) e = cudaStreamSynchronize(h->stream);
  if (e) return gf_cuda(h, e, "get_features");
  return GFORS_OK;
}
