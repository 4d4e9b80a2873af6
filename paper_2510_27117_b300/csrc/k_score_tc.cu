// k_score_tc.cu -- EvalBest for a dense small-integer Q on the 5th-generation
// tensor cores (tcgen05, sm_103a):
//
//   S = W2 . X^T      (bf16 operands, FP32 accumulation in TMEM)
//   obj_s = (1/2) sum_i X_si (S_is + 2 lin_i),   lin = c + diag(Q),
//
// W2 = offdiag(Q + Q^T).  Exactness: every entry of W2 and X is an integer
// representable in bf16 and |S_is| <= n max|W2| < 2^24, so each FP32 sum is
// exact in any order; the epilogue converts to int and reduces in int32/int64.
//
// Structure (one persistent CTA per SM, 6 warps):
//   warp 0      TMA producer: 128x64 tile of W2 and 256x64 tile of X per
//               k-step, 128-byte swizzle, 4-stage mbarrier ring
//   warp 1      TMEM owner and MMA issuer: 4 x tcgen05.mma (M=128, N=256,
//               K=16) per k-step into one of two TMEM accumulators
//               (2 x 256 columns)
//   warps 2-5   epilogue: tcgen05.ld 32 columns at a time, multiply by the
//               candidate bits, warp butterfly reduce-scatter over rows,
//               cross-warp sum, one atomic per (tile, candidate)
// Every mbarrier wait is bounded by a time limit; on expiry the kernel
// records an error in the device state, drains, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "tc_util.cuh"

namespace {

using namespace gf_tc;

// BK: bf16 elements per 128-byte operand row of a stage (FP8 stages hold
// 2 x BK elements in the same bytes)
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
constexpr int TMEM_COLS = 512;                  // two 256-column accumulators
constexpr int kThreads = 192;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 4 * BN * 4 /*partials*/ +
                           4 * BN * 4 /*candidate bits*/ + 256 /*barriers*/;

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = gf_tc::idesc_bf16(BM, BN);
// FP8 (E4M3) operands: the same 128-byte rows hold 128 elements, every MMA
// takes K = 32 (32 bytes of each row, as K = 16 in bf16).
constexpr uint32_t kIdescF8 = gf_tc::idesc_e4m3(BM, BN);

template <bool F8>
GF_DEV void mma_op(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  if constexpr (F8) gf_tc::mma_f8f6f4(d_tmem, a, b, kIdescF8, accum);
  else gf_tc::mma_f16(d_tmem, a, b, kIdesc, accum);
}

// One CTA per 128 x 256 output tile; every CTA loads its own operand tiles.
template <bool F8>
__global__ void __launch_bounds__(kThreads, 1)
k_score_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           int n, int64_t ld, int len, int num_m, int num_n, int num_k,
           const uint32_t* __restrict__ Xb, const long long* __restrict__ lin,
           unsigned long long* __restrict__ obj, uint64_t limit_ns, GfDState* st) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* stA = base;                                   // STAGES x 16 KB
  uint8_t* stB = base + STAGES * A_BYTES;                // STAGES x 32 KB
  int* partial = reinterpret_cast<int*>(base + STAGES * STAGE_BYTES);   // [4][BN]
  uint32_t* xbits = reinterpret_cast<uint32_t*>(partial + 4 * BN);      // [BN][4]
  uint64_t* bars = reinterpret_cast<uint64_t*>(xbits + 4 * BN);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2]
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ volatile int drain_flag;      // private flag of the drain waits
  __shared__ int ep_ok[4];                 // per-epilogue-warp wait results

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int KE = F8 ? 2 * BK : BK;     // K elements per stage (128-byte rows)
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    drain_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull0 + 8 * a, 1);
      mbar_init(tempty0 + 8 * a, 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const int num_tiles = num_m * num_n;
  const int cid = blockIdx.x, ncl = gridDim.x;
  auto tile_m0 = [&](int t) { return (t % num_m) * BM; };
  auto tile_n0 = [&](int t) { return (t / num_m) * BN; };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = cid; t < num_tiles && ok; t += ncl) {
        const int m0 = tile_m0(t), n0 = tile_n0(t);
        for (int kb = 0; kb < num_k && ok; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!(ok = mbar_wait(empty0 + 8 * s, ph ^ 1u, limit_ns, &abort_flag))) break;
          mbar_arrive_expect_tx(full0 + 8 * s, STAGE_BYTES);
          tma_load_2d(smem_u32(stA + s * A_BYTES), &tmA, full0 + 8 * s, kb * KE, m0);
          tma_load_2d(smem_u32(stB + s * B_BYTES), &tmB, full0 + 8 * s, kb * KE, n0);
        }
      }
      if (!ok) {
        // drain: wait (bounded, ignoring the abort flag) for issued copies
        for (int q = 0; q < STAGES && q < it; ++q) {
          const int j = it - 1 - q;
          mbar_wait(full0 + 8 * (j % STAGES), (uint32_t)(j / STAGES) & 1u, limit_ns,
                    &drain_flag);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int it = 0, j = 0;
      bool ok = true;
      for (int t = cid; t < num_tiles && ok; t += ncl, ++j) {
        const int acc = j & 1;
        const uint32_t aph = (uint32_t)(j >> 1) & 1u;
        if (!(ok = mbar_wait(tempty0 + 8 * acc, aph ^ 1u, limit_ns, &abort_flag))) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        for (int kb = 0; kb < num_k; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
          if (!(ok = mbar_wait(full0 + 8 * s, ph, limit_ns, &abort_flag))) break;
          tc_fence_after();
          const uint32_t a0 = smem_u32(stA + s * A_BYTES), b0 = smem_u32(stB + s * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k)
            mma_op<F8>(d, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k),
                       (kb | k) != 0 ? 1u : 0u);
          mma_commit(empty0 + 8 * s);
        }
        if (ok) mma_commit(tfull0 + 8 * acc);
      }
      // make sure no MMA is still writing TMEM before it is freed
      if (it > 0) {
        const int j2 = it - 1;
        mbar_wait(empty0 + 8 * (j2 % STAGES), (uint32_t)(j2 / STAGES) & 1u, limit_ns,
                  &abort_flag);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lane quarter of this warp
    const int et = threadIdx.x - 64;         // 0..127 within the epilogue group
    int j = 0;
    for (int t = cid; t < num_tiles; t += ncl, ++j) {
      const int acc = j & 1;
      const uint32_t aph = (uint32_t)(j >> 1) & 1u;
      bool ok = true;
      if (lane == 0) ep_ok[q] = mbar_wait(tfull0 + 8 * acc, aph, limit_ns, &abort_flag) ? 1 : 0;
      // all four epilogue warps take the same decision (no warp may be left
      // alone at a named barrier)
      named_bar(1, 128);
      ok = ep_ok[0] && ep_ok[1] && ep_ok[2] && ep_ok[3];
      if (!ok) break;
      tc_fence_after();
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      // the tile's candidate bits (256 candidates x the 4 words of rows
      // m0..m0+127) into shared memory once; read back as broadcast words
      {
        const int ldw = (int)(ld / 32);
        for (int e = et; e < BN * 4; e += 128) {
          const int sl = e >> 2, w = m0 / 32 + (e & 3), s = n0 + sl;
          xbits[e] = (s < len && w < ldw) ? Xb[(int64_t)s * ldw + w] : 0u;
        }
        named_bar(1, 128);
      }
      const int i = m0 + q * 32 + lane;
      const bool row_ok = i < n;
      const int lin2 = row_ok ? (int)(2 * lin[i]) : 0;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32), r);
        int v[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const uint32_t word = xbits[(c * 32 + jj) * 4 + q];
          const bool bit = row_ok && ((word >> lane) & 1u);
          v[jj] = bit ? (__float2int_rn(__uint_as_float(r[jj])) + lin2) : 0;
        }
        // butterfly reduce-scatter: lane t ends with the sum of column t
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          const bool up = (lane & off) != 0;
#pragma unroll
          for (int jj = 0; jj < off; ++jj) {
            const int send = up ? v[jj] : v[jj + off];
            const int keep = up ? v[jj + off] : v[jj];
            v[jj] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, off);
          }
        }
        partial[q * BN + c * 32 + lane] = v[0];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
      named_bar(1, 128);
      for (int col = et; col < BN; col += 128) {
        const int s = n0 + col;
        if (s < len) {
          const long long tot = (long long)partial[col] + partial[BN + col] +
                                partial[2 * BN + col] + partial[3 * BN + col];
          if (tot != 0) atomicAdd(obj + s, (unsigned long long)tot);
        }
      }
      named_bar(1, 128);
    }
  }
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) atomicExch(&st->error, 1);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

__global__ void k_halve(long long* __restrict__ obj, int len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < len) obj[s] /= 2;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D tiled map over a row-major [rows x ld] operand of 2-byte (bf16) or
// 1-byte (FP8) elements; boxes of box_inner x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
              uint32_t box_inner, uint32_t box_rows, bool f8) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld * (f8 ? 1 : 2)};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct TcCache {
  const void* W2 = nullptr;
  const void* Xs = nullptr;
  CUtensorMap a, b;
  int sms = 0;
  bool attr = false;
};

}  // namespace

// Launch the tensor-core scorer for candidates [0, len) of the chunk;
// obj (zeroed by the evaluation pass) receives the exact objectives.
cudaError_t gf_launch_dense_score_tc(GfCtx* h, const GfDenseQ& dq, int s0, int len) {
  (void)s0;
  static thread_local std::vector<TcCache> caches;
  if (caches.size() < 64) caches.resize(64);
  TcCache& C = caches[dq.inst % 64];
  const bool f8 = dq.f8;
  const void* Wop = f8 ? (const void*)dq.W2f8 : (const void*)dq.W2;
  const uint32_t ke = f8 ? 2 * BK : BK;      // elements in a 128-byte box row
  if (C.W2 != Wop || C.Xs != dq.Xs) {
    if (!make_map(&C.a, Wop, (uint64_t)dq.ld, (uint64_t)dq.n, (uint64_t)dq.ld, ke, BM, f8) ||
        !make_map(&C.b, dq.Xs, (uint64_t)dq.ld, (uint64_t)dq.chunk, (uint64_t)dq.ld, ke, BN,
                  f8))
      return cudaErrorInvalidValue;
    C.W2 = Wop;
    C.Xs = dq.Xs;
  }
  if (!C.attr) {
    cudaError_t e = cudaSuccess;
    for (const void* fn : {(const void*)k_score_tc<false>, (const void*)k_score_tc<true>})
      if (!e) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&C.sms, cudaDevAttrMultiProcessorCount, dev);
    C.attr = true;
  }
  const int num_m = (int)((dq.n + BM - 1) / BM);
  const int num_n = (len + BN - 1) / BN;
  const int num_k = (int)((dq.ld + ke - 1) / ke);
  long long* out = h->obj + (int64_t)dq.inst * h->chunk;
  unsigned long long* outu = reinterpret_cast<unsigned long long*>(out);
  const uint64_t limit = (uint64_t)(std::max(0.01, h->prm.wait_timeout_s) * 1e9);
  const uint32_t* Xb = dq.Xb;
  const long long* lin = dq.lin;
  int nn = (int)dq.n, ll = len;
  int64_t ld = dq.ld;
  GfDState* st = h->dstate;
  const int tiles = num_m * num_n;
  const int grid = std::min(tiles, C.sms > 0 ? C.sms : 148);
  if (f8)
    k_score_tc<true><<<grid, kThreads, SMEM_BYTES, h->stream>>>(
        C.a, C.b, nn, ld, ll, num_m, num_n, num_k, Xb, lin, outu, limit, st);
  else
    k_score_tc<false><<<grid, kThreads, SMEM_BYTES, h->stream>>>(
        C.a, C.b, nn, ld, ll, num_m, num_n, num_k, Xb, lin, outu, limit, st);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_halve<<<(len + 255) / 256, 256, 0, h->stream>>>(out, len);
  h->launches += 2;
  return cudaGetLastError();
}
