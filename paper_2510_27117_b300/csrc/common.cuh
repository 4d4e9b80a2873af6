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

// The same generator with the ten round keys computed once (they depend on
// the seed only): for threads that draw many counters under one key.
struct PhiloxKeys {
  uint32_t kx[10], ky[10];
};
GF_DEV PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t kx = (uint32_t)seed, ky = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.kx[r] = kx;
    K.ky[r] = ky;
    kx += 0x9E3779B9u;
    ky += 0xBB67AE85u;
  }
  return K;
}
GF_DEV uint4 philox_k(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a0 = 0xD2511F53u, a1 = 0xCD9E8D57u;
    uint32_t lo0 = a0 * c.x, hi0 = __umulhi(a0, c.x);
    uint32_t lo1 = a1 * c.z, hi1 = __umulhi(a1, c.z);
    c = make_uint4(hi1 ^ c.y ^ K.kx[r], lo1, hi0 ^ c.w ^ K.ky[r], lo0);
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

// acc += val[t] * vec[idx[t]] for t = t, t + S, t + 2S, ... < t1, added in
// that order; U consecutive terms have their index and value loads issued,
// then their gathers, before any is added (U independent gathers in flight
// instead of one dependent chain), so the sum equals the plain loop's.
template <int U>
GF_DEV void gather_dot(CSum& acc, const int32_t* __restrict__ idx,
                       const float* __restrict__ val, const float* __restrict__ vec,
                       int64_t t, int64_t t1, int S) {
  for (; t + (int64_t)(U - 1) * S < t1; t += (int64_t)U * S) {
    int32_t c[U];
    float v[U], g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = idx[t + (int64_t)u * S];
      v[u] = val[t + (int64_t)u * S];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) g[u] = vec[c[u]];
#pragma unroll
    for (int u = 0; u < U; ++u) acc.add(__fmul_rn(v[u], g[u]));
  }
  for (; t < t1; t += S) acc.add(__fmul_rn(val[t], vec[idx[t]]));
}

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
// Packed FP32 pair arithmetic (two IEEE round-to-nearest operations per
// instruction) on 64-bit registers holding (lo, hi) floats.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;
GF_DEV f32x2 f2_pack(uint32_t lo, uint32_t hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}
GF_DEV f32x2 f2_add(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
GF_DEV f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
GF_DEV f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
GF_DEV float f2_sum(f32x2 a) {
  return __fadd_rn(__uint_as_float((uint32_t)a), __uint_as_float((uint32_t)(a >> 32)));
}
// Signed bytes k, k+1 of a word as an exact float pair.  `wbias` holds the
// bytes biased by +128 (as the matrix is stored): the biased byte becomes the
// low mantissa bits of 2^23, and 2^23 + 128 is subtracted afterwards.
GF_DEV f32x2 f2_i8pair(uint32_t wbias, int k) {
  return f2_pack(__byte_perm(wbias, 0x4B000000u, 0x7650u + k),
                 __byte_perm(wbias, 0x4B000000u, 0x7651u + k));
}

// One lane's share of an int8 row (stored as biased bytes, w + 128) times an
// FP32 vector (the dense Q GEMV of
// the primal step).  Lane l reads the 4-entry words l, l + 32, l + 64, ...
// of the row; words (t, t + 32) form one 8-term chunk summed in plain FP32
// (packed pairs).  Chunks starting at t = l + 128 j go to a first compensated
// sum, chunks starting at t = l + 64 + 128 j to a second (two independent
// dependency chains), merged at the end.  `row` may point to shared or global
// memory; `x4` holds the vector as float4 words in shared memory.  Both PDHG
// paths of a dense instance use this one routine, so their sums are
// identical.
GF_DEV f32x2 i8_chunk_x(const uint32_t* row, int64_t t, bool has_b, ulonglong2 xa,
                        ulonglong2 xb, f32x2 bias) {
  const uint32_t wa = row[t];
  f32x2 pr = f2_mul(f2_add(f2_i8pair(wa, 0), bias), xa.x);
  pr = f2_fma(f2_add(f2_i8pair(wa, 2), bias), xa.y, pr);
  if (has_b) {
    const uint32_t wb = row[t + 32];
    pr = f2_fma(f2_add(f2_i8pair(wb, 0), bias), xb.x, pr);
    pr = f2_fma(f2_add(f2_i8pair(wb, 2), bias), xb.y, pr);
  }
  return pr;
}
GF_DEV f32x2 i8_chunk(const uint32_t* row, const ulonglong2* xv, int64_t t, int64_t nq,
                      f32x2 bias) {
  const bool has_b = t + 32 < nq;
  return i8_chunk_x(row, t, has_b, xv[t], has_b ? xv[t + 32] : make_ulonglong2(0, 0), bias);
}
// Rows whose word count is a multiple of 128: the same chunks, chains and
// order as the general loop below, without its bounds tests and with
// 32-bit offsets (so the two give identical sums).
GF_DEV CSum i8_row_dot_full(const uint32_t* row, const ulonglong2* xv, int nq, int lane,
                            f32x2 bias) {
  CSum acc, acc2;
  const uint32_t* r = row + lane;
  const ulonglong2* xp = xv + lane;
  for (int it = nq >> 7; it > 0; --it, r += 128, xp += 128) {
    const f32x2 pa = i8_chunk_x(r, 0, true, xp[0], xp[32], bias);
    const f32x2 pb = i8_chunk_x(r, 64, true, xp[64], xp[96], bias);
    acc2.add(f2_sum(pb));
    acc.add(f2_sum(pa));
  }
  acc.merge(acc2.s, acc2.c);
  return acc;
}
GF_DEV CSum i8_row_dot(const uint32_t* row, const float4* x4, int64_t nq, int lane) {
  const f32x2 bias = f2_pack(__float_as_uint(-8388736.0f), __float_as_uint(-8388736.0f));
  const ulonglong2* xv = reinterpret_cast<const ulonglong2*>(x4);
  if ((nq & 127) == 0 && nq < (1ll << 30)) return i8_row_dot_full(row, xv, (int)nq, lane, bias);
  CSum acc, acc2;
  for (int64_t t = lane; t < nq; t += 128) {
    const f32x2 p1 = i8_chunk(row, xv, t, nq, bias);
    if (t + 64 < nq) acc2.add(f2_sum(i8_chunk(row, xv, t + 64, nq, bias)));
    acc.add(f2_sum(p1));
  }
  acc.merge(acc2.s, acc2.c);
  return acc;
}

// ---------------------------------------------------------------------------
// 32 x 32 bit transpose across a warp: lane l holds word A_l; afterwards
// lane b holds the word whose bit l is bit b of A_l.  Five block-swap
// stages; in the stage of distance j a lane keeps its own bits outside the
// mask M and takes its partner's word rotated by j (lower lane) or 32 - j
// (upper lane) inside it.  The per-lane rotations and masks depend on the
// lane only (TransposeLane, computed once).
struct TransposeLane {
  uint32_t rot[5], mask[5];
};
GF_DEV TransposeLane transpose_lane(int lane) {
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
  TransposeLane t;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const bool low = (lane & j) == 0;
    t.rot[k] = low ? (uint32_t)j : (uint32_t)(32 - j);
    t.mask[k] = low ? (m[k] << j) : m[k];
  }
  return t;
}
GF_DEV uint32_t warp_transpose32(uint32_t x, const TransposeLane& t) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, 16 >> k);
    const uint32_t r = __funnelshift_l(y, y, t.rot[k]);
    x = (x & ~t.mask[k]) | (r & t.mask[k]);
  }
  return x;
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
