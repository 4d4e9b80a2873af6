// k_mlp_tc.cu -- forward pass of the learned proposal's MLP on the
// 5th-generation tensor cores (tcgen05):
//
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3,
//   p  = clip(sigmoid(z), 2^-24, 1 - 2^-24)    (F = 8, H = 128),
//
// with the numerics of the CUDA-core kernel in k_mlp.cu: weights rounded to
// bf16, every other quantity FP32.  The FP32 inputs of the two GEMMs (the
// features f and the hidden layer h1) are split exactly into three bf16
// pieces, x = x_hi + x_mid + x_lo (8 + 8 + 8 significand bits), so every
// tensor-core product w * piece is exact and the sums accumulate in FP32 in
// TMEM -- the GEMMs carry FP32 activations, not bf16 ones.
//
// One persistent CTA per SM, tiles of 128 variables, 9 warps:
//   warps 0-7  row warps: warp w serves TMEM lanes 32 (w mod 4) .. + 31 (one
//              variable per lane) and hidden units 64 (w / 4) .. + 63: features
//              -> pieces -> A1 (warps 0-3); TMEM D1 -> +b1, relu -> pieces ->
//              A2; TMEM D2 -> +b2, relu, half of the w3 dot; the two halves of
//              z meet in shared memory -> z, p
//   warp 8     MMA issuer (lane 0): layer 1 = 3 MMAs (M=N=128, K=16, one per
//              feature piece against W1 replicated at K offsets 0/16/32),
//              layer 2 = 24 MMAs (3 pieces x 8 K-steps of 16) into D2
// Operands are K-major, 128-byte swizzled, in shared memory; W1 and W2 are
// staged once per CTA.  Waits on MMA completion are bounded by a time limit;
// on expiry the kernel records an error (or writes NaN outputs when no error
// word is given), waits for its MMAs and frees TMEM.
#include "internal.cuh"
#include "tc_util.cuh"

namespace {

using namespace gf_tc;

constexpr int kF = 8, kH = 128, TM = 128;
constexpr int kThreads = 288;           // 8 row warps + 1 MMA warp
constexpr int kRowThreads = 256;
constexpr int kMmaWarp = 8;
constexpr uint32_t kIdesc = idesc_bf16(128, 128);
constexpr uint32_t TMEM_COLS = 256;          // D1 = columns [0, 128), D2 = [128, 256)
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH;
// shared-memory layout (offsets from a 1024-byte aligned base)
constexpr int PANEL = 128 * 128;             // 128 rows x 128 bytes (64 bf16 per row)
constexpr int A1_OFF = 0;                    // features: pieces at K = 0, 16, 32
constexpr int B1_OFF = A1_OFF + PANEL;       // W1 at K = 0, 16, 32
constexpr int A2_OFF = B1_OFF + PANEL;       // h1: 3 pieces x 2 panels (K 0-63, 64-127)
constexpr int B2_OFF = A2_OFF + 6 * PANEL;   // W2: 2 panels
constexpr int VEC_OFF = B2_OFF + 2 * PANEL;  // b1, b2, w3 (FP32), b3
constexpr int ZP_OFF = VEC_OFF + 3 * kH * 4 + 16;   // z half sums [2][128]
constexpr int BAR_OFF = ZP_OFF + 2 * 128 * 4;
constexpr int SMEM_BYTES = BAR_OFF + 64 + 1024;

// Byte offset of element (row r, k) of a K-major 128-byte-swizzled panel
// (k < 64): 8-row atoms of 1024 bytes, 16-byte chunk index XOR (r mod 8).
GF_DEV uint32_t sw_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
}

GF_DEV uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Exact split of 8 FP32 values into three bf16 pieces; writes one 16-byte
// chunk per piece (row r, K offset k0 of the piece's panel base).
GF_DEV void split8_store(uint8_t* base0, uint8_t* base1, uint8_t* base2, int r, int k0,
                         const float* v) {
  uint32_t hi[4], mid[4], lo[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a = v[2 * q], b = v[2 * q + 1];
    const float ah = __bfloat162float(__float2bfloat16_rn(a));
    const float bh = __bfloat162float(__float2bfloat16_rn(b));
    const float a1 = __fsub_rn(a, ah), b1 = __fsub_rn(b, bh);
    const float am = __bfloat162float(__float2bfloat16_rn(a1));
    const float bm = __bfloat162float(__float2bfloat16_rn(b1));
    hi[q] = pack_bf16x2(ah, bh);
    mid[q] = pack_bf16x2(am, bm);
    lo[q] = pack_bf16x2(__fsub_rn(a1, am), __fsub_rn(b1, bm));
  }
  const uint32_t o = sw_off(r, k0);
  *reinterpret_cast<uint4*>(base0 + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(base1 + o) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
  *reinterpret_cast<uint4*>(base2 + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

GF_DEV float clip_sigmoid(float z) {
  const float p = 1.0f / (1.0f + expf(-z));
  // bounds: the sampler's resolution (threshold floor(p 2^24) >= 1)
  return fminf(fmaxf(p, 0x1p-24f), 1.0f - 0x1p-24f);
}

GF_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1)
k_mlp_fwd_tc(const float* __restrict__ W, int64_t nv, const float* __restrict__ feat,
             float* __restrict__ z_out, float* __restrict__ p_out,
             const uint8_t* __restrict__ live, uint64_t limit_ns, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* A1 = base + A1_OFF;
  uint8_t* B1 = base + B1_OFF;
  uint8_t* A2 = base + A2_OFF;
  uint8_t* B2 = base + B2_OFF;
  float* b1s = reinterpret_cast<float*>(base + VEC_OFF);
  float* b2s = b1s + kH;
  float* w3s = b2s + kH;
  float* b3s = w3s + kH;
  float* zpart = reinterpret_cast<float*>(base + ZP_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + BAR_OFF);
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mb1 = smem_u32(bars), mb2 = smem_u32(bars + 1);

  // ---- stage weights (bf16-rounded) and biases; zero the operand tiles
  for (int e = threadIdx.x; e < 8 * PANEL / 16; e += kThreads)
    reinterpret_cast<uint4*>(base)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int e = threadIdx.x; e < kH * 8; e += kThreads) {      // W1 rows, chunk at K 0/16/32
    const int a = e >> 3, q = e & 7;
    if (q) continue;
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = W[oW1 + a * kF + t];
    const uint4 w = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                               pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
#pragma unroll
    for (int p = 0; p < 3; ++p) *reinterpret_cast<uint4*>(B1 + sw_off(a, 16 * p)) = w;
  }
  for (int e = threadIdx.x; e < kH * (kH / 8); e += kThreads) {  // W2 rows, 8 at a time
    const int a = e / (kH / 8), k0 = (e % (kH / 8)) * 8;
    const float* src = W + oW2 + a * kH + k0;
    const uint4 w = make_uint4(pack_bf16x2(src[0], src[1]), pack_bf16x2(src[2], src[3]),
                               pack_bf16x2(src[4], src[5]), pack_bf16x2(src[6], src[7]));
    *reinterpret_cast<uint4*>(B2 + (k0 >> 6) * PANEL + sw_off(a, k0 & 63)) = w;
  }
  for (int a = threadIdx.x; a < kH; a += kThreads) {
    b1s[a] = W[oB1 + a];
    b2s[a] = W[oB2 + a];
    w3s[a] = __bfloat162float(__float2bfloat16_rn(W[oW3 + a]));
  }
  if (threadIdx.x == 0) {
    b3s[0] = W[oB3];
    abort_flag = 0;
    mbar_init(mb1, 1);
    mbar_init(mb2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();                         // weight tiles visible to the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const int64_t ntiles = (nv + TM - 1) / TM;
  int j = 0;                                  // tiles done by this CTA
  int issued = 0;                             // commits issued (MMA warp)
  // features of the next tile, loaded one tile ahead by warps 0-3 so that
  // their global-memory latency overlaps the current tile
  float4 fn0 = make_float4(0.f, 0.f, 0.f, 0.f), fn1 = fn0;
  auto load_feat = [&](int64_t tile) {
    const int64_t v = tile * TM + threadIdx.x;
    if (tile < ntiles && v < nv) {
      fn0 = __ldg(reinterpret_cast<const float4*>(feat + v * kF));
      fn1 = __ldg(reinterpret_cast<const float4*>(feat + v * kF) + 1);
    } else {
      fn0 = fn1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (warp < 4) load_feat(blockIdx.x);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
    const uint32_t ph = (uint32_t)j & 1u;
    const int qq = warp & 3, half = warp >> 2;  // TMEM lane quarter, hidden-unit half
    if (warp < 4) {
      // ---- features -> three bf16 pieces at K = 0, 16, 32 of A1
      const int r = threadIdx.x;
      float f[kF];
      f[0] = fn0.x; f[1] = fn0.y; f[2] = fn0.z; f[3] = fn0.w;
      f[4] = fn1.x; f[5] = fn1.y; f[6] = fn1.z; f[7] = fn1.w;
      load_feat(t + gridDim.x);
      // the three pieces share one panel: hi at K 0, mid at K 16, lo at K 32
      {
        uint32_t hi[4], mid[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float a = f[2 * q], b = f[2 * q + 1];
          const float ah = __bfloat162float(__float2bfloat16_rn(a));
          const float bh = __bfloat162float(__float2bfloat16_rn(b));
          const float a1 = __fsub_rn(a, ah), b1 = __fsub_rn(b, bh);
          const float am = __bfloat162float(__float2bfloat16_rn(a1));
          const float bm = __bfloat162float(__float2bfloat16_rn(b1));
          hi[q] = pack_bf16x2(ah, bh);
          mid[q] = pack_bf16x2(am, bm);
          lo[q] = pack_bf16x2(__fsub_rn(a1, am), __fsub_rn(b1, bm));
        }
        *reinterpret_cast<uint4*>(A1 + sw_off(r, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(A1 + sw_off(r, 16)) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
        *reinterpret_cast<uint4*>(A1 + sw_off(r, 32)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_async_smem();
    }
    // A1 written (and the last tile's TMEM reads done); a wait that gave up
    // anywhere ends the loop for every thread alike
    if (named_bar_or(1, kThreads, abort_flag != 0)) break;
    if (warp == kMmaWarp) {
      if (lane == 0) {
        tc_fence_after();
#pragma unroll
        for (int p = 0; p < 3; ++p)
          mma_f16(tmem, sw128_desc(smem_u32(A1) + 32 * p), sw128_desc(smem_u32(B1) + 32 * p),
                  kIdesc, p > 0 ? 1u : 0u);
        mma_commit(mb1);
        ++issued;
      }
      __syncwarp();
    } else {
      // ---- D1 -> +b1, relu -> three bf16 pieces of h1 into A2 (this warp's
      // 64 hidden units = one K panel)
      const int r = qq * 32 + lane;
      if (!mbar_wait(mb1, ph, limit_ns, &abort_flag)) abort_flag = 1;
      tc_fence_after();
#pragma unroll 1
      for (int c = 2 * half; c < 2 * half + 2; ++c) {
        uint32_t d[32];
        tmem_ld32(tmem + ((uint32_t)(qq * 32) << 16) + (uint32_t)(c * 32), d);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          float h[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            h[q] = fmaxf(__fadd_rn(__uint_as_float(d[8 * g + q]), b1s[32 * c + 8 * g + q]), 0.0f);
          const int k = 32 * c + 8 * g;
          const int pan = k >> 6;
          split8_store(A2 + (0 * 2 + pan) * PANEL, A2 + (1 * 2 + pan) * PANEL,
                       A2 + (2 * 2 + pan) * PANEL, r, k & 63, h);
        }
      }
      fence_async_smem();
      tc_fence_before();
    }
    named_bar(2, kThreads);                   // A2 written, D1 read
    if (warp == kMmaWarp) {
      if (lane == 0) {
        tc_fence_after();
        const uint32_t d2 = tmem + 128u;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int s = 0; s < 8; ++s)
            mma_f16(d2, sw128_desc(smem_u32(A2 + (2 * p + (s >> 2)) * PANEL) + 32 * (s & 3)),
                    sw128_desc(smem_u32(B2 + (s >> 2) * PANEL) + 32 * (s & 3)), kIdesc,
                    (p | s) != 0 ? 1u : 0u);
        mma_commit(mb2);
        ++issued;
      }
      __syncwarp();
    } else {
      // ---- D2 -> +b2, relu, w3 dot over this warp's 64 units -> z, p
      const int r = qq * 32 + lane;
      const int64_t v = t * TM + r;
      bool ok = mbar_wait(mb2, ph, limit_ns, &abort_flag);
      if (!ok) abort_flag = 1;
      tc_fence_after();
      float zh = half ? 0.0f : b3s[0];
#pragma unroll 1
      for (int c = 2 * half; c < 2 * half + 2; ++c) {
        uint32_t d[32];
        tmem_ld32(tmem + ((uint32_t)(qq * 32) << 16) + 128u + (uint32_t)(c * 32), d);
#pragma unroll
        for (int q = 0; q < 32; ++q)
          zh = fmaf(w3s[32 * c + q],
                    fmaxf(__fadd_rn(__uint_as_float(d[q]), b2s[32 * c + q]), 0.0f), zh);
      }
      tc_fence_before();
      zpart[half * 128 + r] = zh;
      named_bar(3, kRowThreads);              // both halves of z in shared memory
      const float z = __fadd_rn(zpart[r], zpart[128 + r]);
      if (half == 0 && v < nv) {
        if (!ok || abort_flag) {
          if (!err) {
            if (z_out) z_out[v] = __int_as_float(0x7FC00000);
            if (p_out) p_out[v] = __int_as_float(0x7FC00000);
          }
        } else {
          if (z_out) z_out[v] = z;
          if (p_out) p_out[v] = (live && !live[v]) ? 0.0f : clip_sigmoid(z);
        }
      }
    }
  }
  __syncthreads();
  if (warp == kMmaWarp) {
    // no MMA may still write TMEM when it is freed: wait (bounded) for the
    // last commit of each barrier
    if (lane == 0 && issued > 0) {
      volatile int drain = 0;
      const int l1 = (issued + 1) / 2, l2 = issued / 2;   // commits on mb1 / mb2
      if (l1 > 0) mbar_wait(mb1, (uint32_t)(l1 - 1) & 1u, limit_ns, &drain);
      if (l2 > 0) mbar_wait(mb2, (uint32_t)(l2 - 1) & 1u, limit_ns, &drain);
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
  if (abort_flag && threadIdx.x == 0 && err) atomicExch(err, 1);
}

}  // namespace

// Launch of the tensor-core forward (one CTA per SM); err (device, may be
// NULL) receives 1 if a wait on the tensor cores gave up.
cudaError_t gf_mlp_forward_tc(const float* W, int64_t nv, const float* feat, float* z,
                              float* p, const uint8_t* live, uint64_t limit_ns, int* err,
                              cudaStream_t s) {
  static int done = 0, sms = 0;
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    done = 1;
  }
  const int64_t tiles = (nv + TM - 1) / TM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, sms > 0 ? sms : 148));
  k_mlp_fwd_tc<<<grid, kThreads, SMEM_BYTES, s>>>(W, nv, feat, z, p, live, limit_ns, err);
  return cudaGetLastError();
}
