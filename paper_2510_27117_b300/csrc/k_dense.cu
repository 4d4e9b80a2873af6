// k_dense.cu -- EvalBest for a dense Q with small-integer off-diagonal part:
//   obj_s = X_s^T Q X_s + c^T X_s = (1/2) X_s^T W2 X_s + (c + diag Q)^T X_s,
// W2 = offdiag(Q + Q^T).  This file holds the CUDA-core scorer (one block per
// candidate), used for checking and for shapes the tensor-core kernel does
// not take; k_score_tc.cu holds the tcgen05 kernel.
#include "internal.cuh"

namespace {

__global__ void __launch_bounds__(256)
k_dense_score_simt(const __nv_bfloat16* __restrict__ W2, int64_t ld, int64_t n,
                   const long long* __restrict__ lin, const __nv_bfloat16* __restrict__ Xs,
                   int len, long long* __restrict__ obj) {
  const int s = blockIdx.x;
  if (s >= len) return;
  extern __shared__ uint32_t xb[];           // ld / 32 words
  const int nw = (int)(ld / 32);
  const __nv_bfloat16* xr = Xs + (int64_t)s * ld;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    uint32_t m = 0;
    for (int t = 0; t < 32; ++t)
      if (__bfloat162float(xr[32 * w + t]) != 0.0f) m |= 1u << t;
    xb[w] = m;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  long long acc = 0;                          // sum_i x_i (W2 x)_i, per warp
  for (int64_t i = warp; i < n; i += blockDim.x / 32) {
    if (!((xb[i >> 5] >> (i & 31)) & 1u)) continue;
    const __nv_bfloat16* wr = W2 + i * ld;
    int part = 0;
    for (int64_t j = lane; j < n; j += 32)
      if ((xb[j >> 5] >> (j & 31)) & 1u) part += (int)__bfloat162float(wr[j]);
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, off);
    if (lane == 0) acc += part;
  }
  long long l = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if ((xb[i >> 5] >> (i & 31)) & 1u) l += lin[i];
  __shared__ long long red[256];            // acc is non-zero in lane 0 only
  red[threadIdx.x] = acc;
  __shared__ long long redl[256];
  redl[threadIdx.x] = l;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      red[threadIdx.x] += red[threadIdx.x + off];
      redl[threadIdx.x] += redl[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) obj[s] = red[0] / 2 + redl[0];
}

}  // namespace

cudaError_t gf_launch_dense_score_tc(GfCtx* h, const GfDenseQ& dq, int s0, int len);

cudaError_t gf_launch_dense_score(GfCtx* h, const GfDenseQ& dq, int s0, int len) {
  if (dq.tc_ok && h->prm.eval_mode != 4) return gf_launch_dense_score_tc(h, dq, s0, len);
  long long* out = h->obj + (int64_t)dq.inst * h->chunk;
  k_dense_score_simt<<<len, 256, sizeof(uint32_t) * (dq.ld / 32), h->stream>>>(
      dq.W2, dq.ld, dq.n, dq.lin, dq.Xs, len, out);
  h->launches++;
  return cudaGetLastError();
}
