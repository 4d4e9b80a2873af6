// common.cuh -- device helpers shared by the GFORS kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define GF_DEV __device__ __forceinline__

namespace gf {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds; each round
// takes the 32x32->64 products of the multipliers with counter words 0 and 2
// and mixes their halves with words 1, 3 and the round key; the key grows
// by the golden-ratio / sqrt(3)-1 Weyl increments between rounds.
// ---------------------------------------------------------------------------
GF_DEV uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a0 = 0xD2511F53u, a1 = 0xCD9E8D57u;
    uint32_t lo0 = a0 * c.x, hi0 = __umulhi(a0, c.x);
    uint32_t lo1 = a1 * c.z, hi1 = __umulhi(a1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Counter layout of every random draw: (idx >> 2, sample, round, inst |
// stream << 28) under key (seed lo, seed hi); the draw for idx is lane idx&3.
enum : uint32_t { kStreamBern = 0, kStreamGroup = 1, kStreamAxial = 2,
                  kStreamPower = 3, kStreamX0 = 5 };

GF_DEV uint4 philox_call(uint64_t seed, uint32_t stream, uint32_t inst,
                         uint32_t round, uint32_t s, uint64_t idx4) {
  return philox(make_uint4((uint32_t)idx4, s, round,
                           (inst & 0x0FFFFFFFu) | (stream << 28)),
                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

GF_DEV uint32_t lane_of(uint4 v, uint32_t l) {
  return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

// Bernoulli threshold floor(p 2^24) of an FP32 probability (exact).
GF_DEV uint32_t prob_threshold(float p) {
  if (!(p > 0.0f)) return 0u;
  if (p >= 1.0f) return 16777216u;
  return (uint32_t)(p * 16777216.0f);
}

// ---------------------------------------------------------------------------
// Compensated FP32 summation (Neumaier / TwoSum).  Every add is an
// error-free transformation, written with non-contractible intrinsics so the
// compiler cannot fuse them into FMAs.  Error of a sum of n products:
// about eps * sum|terms| (product rounding) + 2 eps * sum|terms|.
// ---------------------------------------------------------------------------
struct CSum {
  float s, c;
  GF_DEV CSum() : s(0.f), c(0.f) {}
  GF_DEV void add(float v) {
    float t = __fadd_rn(s, v);
    float z = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(v, z));
    c = __fadd_rn(c, e);
    s = t;
  }
  GF_DEV void merge(float os, float oc) {
    add(os);
    c = __fadd_rn(c, oc);
  }
  GF_DEV float value() const { return __fadd_rn(s, c); }
};

// Sum-reduce a CSum over aligned groups of W lanes (W a power of two <= 32);
// the result lands in the group's first lane.
template <int W>
GF_DEV void csum_group_reduce(CSum& a) {
  if (W == 1) return;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = (W == 32) ? 0xFFFFFFFFu
                                  : (((1u << W) - 1u) << (lane & ~(unsigned)(W - 1)));
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) {
    float os = __shfl_down_sync(mask, a.s, off, W);
    float oc = __shfl_down_sync(mask, a.c, off, W);
    a.merge(os, oc);
  }
}

// ---------------------------------------------------------------------------
// Time source for bounded device waits.
// ---------------------------------------------------------------------------
GF_DEV uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace gf

// ---------------------------------------------------------------------------
// Device-resident solver state (one per handle).
// ---------------------------------------------------------------------------
struct GfDState {
  long long k;          // PDHG iterations completed
  int n_rho;            // penalty counter used by iteration k+1
  int error;            // nonzero: a device wait gave up (timeout)
  double rho;           // penalty of iteration k+1
  unsigned round_id;    // Philox round id of the next sampling round
  int pad;
};

// Per-instance scalars of one iteration (double-buffered by iteration parity).
struct GfIParam {
  float tau1, tau2, rho, pad;
  double tau1d, tau2d, rhod, normQ;
};

// Schedule constants needed on the device to advance the penalty.
struct GfSched {
  double sigma, rho_min, rho_max, T, p, delta;
  int k_int, ninst;
};

// Incumbent of one instance (EvalBest).
struct GfInc {
  long long obj;        // exact objective (integer data)
  double objf;          // objective in FP64
  unsigned round_id;
  int sample;
  int found;
  int changed;          // set when the last update replaced it
};
