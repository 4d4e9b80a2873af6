// k_noalloc.cu -- allocation-free variant of the fused single-row
// sampling + evaluation pass (the knapsack-form kernel of k_eval.cu).
//
// Some callers cannot allocate device memory at the moment they need this
// pass: code that runs while a CUDA graph is being captured on its thread
// (cudaMalloc is not allowed there), serving loops that must never touch
// the allocator after start-up, and hosts whose whole device budget is
// owned by their own memory pool.  This entry point takes every input and
// output from the caller and keeps its only scratch -- one int64 row sum
// per candidate -- in a fixed, file-scope device array, so it performs no
// allocation of any kind.
//
// Set-up: the first call on a device looks the array's device address up
// (cudaGetSymbolAddress, with that device current) and caches it; make
// that first call before any stream capture.  The cached address belongs
// to the device's primary context: after cudaDeviceReset it is stale, so
// this entry point must not be used after a reset in the same process.  Every device that loads the
// library holds the array (GFORS_NOALLOC_MAX_SAMPLES x 8 bytes) until the
// process exits.  All calls share it: each call clears the part it uses
// first, and calls whose work overlaps on the GPU (different streams, no
// ordering) race on it.
#include <mutex>

#include "internal.cuh"

static __device__ __align__(256) long long g_noalloc_rowsum[GFORS_NOALLOC_MAX_SAMPLES];

namespace {

constexpr int kMaxDevices = 64;
long long* g_rowsum_ptr[kMaxDevices] = {};
std::mutex g_rowsum_mu;

__global__ void k_na_clear(long long* __restrict__ rowsum, long long* __restrict__ obj,
                           int len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < len) {
    rowsum[s] = 0;
    obj[s] = 0;
  }
}

// One thread per candidate (128 per block); blockIdx.x walks slices of 8192
// variables, four per Philox call.  Same draws as the handle path:
// X_si = [(u >> 8) < floor(p_i 2^24)], u = lane i&3 of Philox(i>>2, s, round,
// inst | stream 0).
__global__ void __launch_bounds__(128)
k_na_fused(const float* __restrict__ p, const int32_t* __restrict__ a,
           const long long* __restrict__ c, int64_t n, uint64_t seed, uint32_t inst,
           uint32_t round, int s0, int len, long long* __restrict__ rowsum,
           long long* __restrict__ obj) {
  const int sidx = blockIdx.y * 128 + threadIdx.x;
  if (sidx >= len) return;
  const int64_t v0 = (int64_t)blockIdx.x * 8192;
  const int64_t v1 = (v0 + 8192 < n) ? v0 + 8192 : n;
  const uint32_t s = (uint32_t)(s0 + sidx);
  long long rs = 0, ob = 0;
  for (int64_t v = v0; v < v1; v += 4) {
    const uint4 u = gf::philox_call(seed, gf::kStreamBern, inst, round, s, (uint64_t)(v >> 2));
    const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int64_t i = v + l;
      if (i < v1 && (uu[l] >> 8) < gf::prob_threshold(p[i])) {
        rs += a[i];
        ob += c[i];
      }
    }
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(rowsum + sidx), (unsigned long long)rs);
  atomicAdd(reinterpret_cast<unsigned long long*>(obj + sidx), (unsigned long long)ob);
}

__global__ void k_na_viol(const long long* __restrict__ rowsum, long long rhs, int len,
                          int32_t* __restrict__ viol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < len) viol[s] = rowsum[s] < rhs ? 1 : 0;
}

}  // namespace

extern "C" gfors_status gfors_fused_eval_noalloc(const float* p_dev, const int32_t* a_dev,
                                                 const int64_t* c_dev, int64_t n, int64_t rhs,
                                                 uint64_t seed, uint32_t inst_id,
                                                 uint32_t round_id, int32_t first_sample,
                                                 int32_t nsamples, int32_t* viol_dev,
                                                 int64_t* obj_dev, void* cuda_stream) {
  if (nsamples < 0 || nsamples > GFORS_NOALLOC_MAX_SAMPLES) {
    gf_fail(nullptr, GFORS_E_ARG,
            "gfors_fused_eval_noalloc: nsamples must lie in [0, " +
                std::to_string(GFORS_NOALLOC_MAX_SAMPLES) + "]");
    return GFORS_E_ARG;
  }
  if (n < 0 || first_sample < 0 || (n > 0 && (!p_dev || !a_dev || !c_dev)) ||
      (nsamples > 0 && (!viol_dev || !obj_dev))) {
    gf_fail(nullptr, GFORS_E_ARG, "gfors_fused_eval_noalloc: bad pointer or size");
    return GFORS_E_ARG;
  }
  // candidate indices first_sample + s must stay within int32
  if (first_sample > INT32_MAX - nsamples) {
    gf_fail(nullptr, GFORS_E_ARG,
            "gfors_fused_eval_noalloc: first_sample + nsamples exceeds INT32_MAX");
    return GFORS_E_ARG;
  }
  if (nsamples == 0) return GFORS_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    gf_fail(nullptr, GFORS_E_CUDA, "gfors_fused_eval_noalloc: no usable device");
    return GFORS_E_CUDA;
  }
  long long* rowsum;
  {
    std::lock_guard<std::mutex> lk(g_rowsum_mu);
    if (!g_rowsum_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_rowsum);
      if (e != cudaSuccess) {
        cudaGetLastError();
        gf_fail(nullptr, GFORS_E_CUDA,
                std::string("gfors_fused_eval_noalloc: cudaGetSymbolAddress: ") +
                    cudaGetErrorString(e));
        return GFORS_E_CUDA;
      }
      g_rowsum_ptr[dev] = static_cast<long long*>(ptr);
    }
    rowsum = g_rowsum_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  long long* obj = reinterpret_cast<long long*>(obj_dev);
  k_na_clear<<<(nsamples + 255) / 256, 256, 0, st>>>(rowsum, obj, nsamples);
  if (n > 0) {
    dim3 grid((unsigned)((n + 8191) / 8192), (unsigned)((nsamples + 127) / 128));
    k_na_fused<<<grid, 128, 0, st>>>(p_dev, a_dev, reinterpret_cast<const long long*>(c_dev), n,
                                     seed, inst_id, round_id, first_sample, nsamples, rowsum,
                                     obj);
  }
  k_na_viol<<<(nsamples + 255) / 256, 256, 0, st>>>(rowsum, (long long)rhs, nsamples, viol_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    gf_fail(nullptr, GFORS_E_CUDA,
            std::string("gfors_fused_eval_noalloc: launch: ") + cudaGetErrorString(e));
    return GFORS_E_CUDA;
  }
  return GFORS_OK;
}
