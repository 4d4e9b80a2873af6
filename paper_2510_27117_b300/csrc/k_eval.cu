// k_eval.cu -- EvalBest (Alg. 1, Section 3) on the device, on the ORIGINAL
// integer data of Eq. (1):
//   viol_s = #{j : A_j X_s < b_j} + #{j : B_j X_s != d_j},
//   obj_s  = X_s^T Q X_s + c^T X_s,
// exact (int64) for every candidate of a chunk, then the incumbent update:
// the least objective among feasible candidates (earliest sample on ties)
// replaces the incumbent only when strictly better.
//
// Rows are classified when the instance is loaded:
//   U rows: all coefficients equal -> the count of chosen columns must lie
//           in [L, U]; counted 32 candidates at a time in bit-sliced form.
//   P rows: at most two nonzeros -> 4-entry violation truth table.
//   G rows: anything else -> 32 per-candidate int64 accumulators.
#include "internal.cuh"

namespace {

// Add per-candidate violation flags (one 32-bit mask per thread, all lanes
// of the warp on the same word w) into viol[inst][32 w + t].
__device__ void add_violations(uint32_t vmask, int inst, int w, int chunk,
                               int32_t* __restrict__ viol, bool valid) {
  const int lane = threadIdx.x & 31;
  const unsigned act = __activemask();
  const int lead_inst = __shfl_sync(act, inst, __ffs(act) - 1);
  const int lead_w = __shfl_sync(act, w, __ffs(act) - 1);
  const bool uniform = __all_sync(act, (!valid) || (inst == lead_inst && w == lead_w));
  if (uniform) {
    // lane t accumulates the count of candidate t over the warp's rows
    int cnt = 0;
    for (int t = 0; t < 32; ++t) {
      const unsigned bal = __ballot_sync(act, valid && ((vmask >> t) & 1u));
      if (lane == t) cnt = __popc(bal);
    }
    if (cnt && ((act >> lane) & 1u))
      atomicAdd(&viol[(int64_t)lead_inst * chunk + 32 * lead_w + lane], cnt);
  } else if (valid) {
    while (vmask) {
      const int t = __ffs(vmask) - 1;
      vmask &= vmask - 1;
      atomicAdd(&viol[(int64_t)inst * chunk + 32 * w + t], 1);
    }
  }
}

// U rows: one warp per (row, group of up to 8 candidate words); the lanes
// stride over the row's columns (consecutive lanes, consecutive columns) and
// keep per-word state, combined across the warp at the end:
//   covering rows (L <= 1, no upper bound): OR of the chosen columns;
//   at-most/exactly-one rows (U == 1): ones / twos masks;
//   others: a 16-slice bit-sliced counter per word (up to 2^16 - 1), summed
//   across lanes by bit-sliced addition, then count in [L, U].
constexpr int kUG = 8;                   // candidate words per warp task

GF_DEV void load_words(const uint32_t* __restrict__ X, int64_t v, int kws, int w0, int nw,
                       bool vec, uint32_t* m) {
  const uint32_t* src = X + v * kws + w0;
  if (vec && nw == kUG) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(src));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(src) + 1);
    m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
    m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < kUG; ++j) m[j] = (j < nw) ? __ldg(src + j) : 0u;
  }
}

// Violations of one row for candidates of word w: lane t adds bit t.
GF_DEV void add_row_violations(uint32_t vmask, int inst, int w, int len, int chunk,
                               int32_t* __restrict__ viol) {
  const int lane = threadIdx.x & 31;
  const int nt = len - 32 * w;
  if (nt < 32) vmask &= (1u << nt) - 1u;
  if ((vmask >> lane) & 1u) atomicAdd(&viol[(int64_t)inst * chunk + 32 * w + lane], 1);
}

// CLS: the rows' class (0: L <= 1 without upper bound, an OR; 1: U = 1,
// L <= 1, ones and twos; 2: general bounds), so that each class compiles to
// its own register budget.
template <int CLS>
__global__ void __launch_bounds__(256)
k_eval_urows(const GfURow* __restrict__ rows, int64_t nrows,
             const int32_t* __restrict__ ucols, const uint32_t* __restrict__ X, int kws,
             int kwu, int len, int chunk, int32_t* __restrict__ viol) {
  const int lane = threadIdx.x & 31;
  const int ng = (kwu + kUG - 1) / kUG;
  const int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (task >= nrows * ng) return;                 // whole warps exit together
  const int64_t r = task / ng;
  const int w0 = (int)(task - r * ng) * kUG;
  const int nw = min(kUG, kwu - w0);
  const bool vec = (kws % 4) == 0;
  const GfURow R = rows[r];
  const int32_t* cols = ucols + R.t0;
  const bool no_upper = (R.U < 0 || R.U >= R.len);
  uint32_t m[kUG];
  if (CLS == 0) {
    uint32_t any[kUG] = {0, 0, 0, 0, 0, 0, 0, 0};
    // two columns per lane and step, both loads issued before either is used
    int t = lane;
    for (; t + 32 < R.len; t += 64) {
      const int32_t ca = cols[t], cb = cols[t + 32];
      uint32_t m2[kUG];
      load_words(X, ca, kws, w0, nw, vec, m);
      load_words(X, cb, kws, w0, nw, vec, m2);
#pragma unroll
      for (int j = 0; j < kUG; ++j) any[j] |= m[j] | m2[j];
    }
    if (t < R.len) {
      load_words(X, cols[t], kws, w0, nw, vec, m);
#pragma unroll
      for (int j = 0; j < kUG; ++j) any[j] |= m[j];
    }
#pragma unroll
    for (int j = 0; j < kUG; ++j) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) any[j] |= __shfl_xor_sync(0xFFFFFFFFu, any[j], off);
      if (j < nw && R.L == 1) add_row_violations(~any[j], R.inst, w0 + j, len, chunk, viol);
    }
  } else if (CLS == 1) {
    uint32_t ones[kUG] = {0, 0, 0, 0, 0, 0, 0, 0}, twos[kUG] = {0, 0, 0, 0, 0, 0, 0, 0};
    // two columns per lane and step, both loads issued before either is used
    int t = lane;
    for (; t + 32 < R.len; t += 64) {
      const int32_t ca = cols[t], cb = cols[t + 32];
      uint32_t m2[kUG];
      load_words(X, ca, kws, w0, nw, vec, m);
      load_words(X, cb, kws, w0, nw, vec, m2);
#pragma unroll
      for (int j = 0; j < kUG; ++j) {
        twos[j] |= (ones[j] & m[j]) | (m[j] & m2[j]) | (ones[j] & m2[j]);
        ones[j] |= m[j] | m2[j];
      }
    }
    if (t < R.len) {
      load_words(X, cols[t], kws, w0, nw, vec, m);
#pragma unroll
      for (int j = 0; j < kUG; ++j) {
        twos[j] |= ones[j] & m[j];
        ones[j] |= m[j];
      }
    }
#pragma unroll
    for (int j = 0; j < kUG; ++j) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, ones[j], off);
        const uint32_t tw = __shfl_xor_sync(0xFFFFFFFFu, twos[j], off);
        twos[j] |= tw | (ones[j] & o);
        ones[j] |= o;
      }
      if (j < nw)
        add_row_violations(twos[j] | (R.L == 1 ? ~ones[j] : 0u), R.inst, w0 + j, len, chunk,
                           viol);
    }
  } else {
    // general count bounds: one word at a time (16 slices per word)
    for (int j = 0; j < nw; ++j) {
      uint32_t sl[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) sl[q] = 0u;
      for (int t = lane; t < R.len; t += 32) {
        uint32_t c = __ldg(X + (int64_t)cols[t] * kws + w0 + j);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const uint32_t carry = sl[q] & c;
          sl[q] ^= c;
          c = carry;
        }
      }
      // bit-sliced sum across the warp (counts < 2^16: R.len < 65536)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        uint32_t carry = 0u;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, sl[q], off);
          const uint32_t x = sl[q] ^ o;
          const uint32_t nc = (sl[q] & o) | (carry & x);
          sl[q] = x ^ carry;
          carry = nc;
        }
      }
      // ge = (count >= L), gt = (count > U), MSB-first bit-sliced compares
      uint32_t eqL = 0xFFFFFFFFu, gtL = 0u, eqU = 0xFFFFFFFFu, gtU = 0u;
      const uint32_t L = (uint32_t)max(R.L, 0), U = (uint32_t)max(R.U, 0);
#pragma unroll
      for (int q = 15; q >= 0; --q) {
        if ((L >> q) & 1u) { eqL &= sl[q]; } else { gtL |= eqL & sl[q]; eqL &= ~sl[q]; }
        if ((U >> q) & 1u) { eqU &= sl[q]; } else { gtU |= eqU & sl[q]; eqU &= ~sl[q]; }
      }
      uint32_t vmask = ~(gtL | eqL);
      if (!no_upper) vmask |= gtU;
      add_row_violations(vmask, R.inst, w0 + j, len, chunk, viol);
    }
  }
}

// P rows: at most two variables; `table` bit (x1 + 2 x2) marks a violation.
// One thread per row, all candidate words of the row in groups of 8 (16-byte
// loads of the two variables' consecutive words), per-word warp aggregation.
__global__ void __launch_bounds__(256)
k_eval_prows(const GfPRow* __restrict__ rows, int64_t nrows,
             const uint32_t* __restrict__ X, int kws, int kwu, int len, int chunk,
             int32_t* __restrict__ viol) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < nrows;
  const bool vec = (kws % 4) == 0;
  GfPRow R;
  R.inst = 0; R.v1 = 0; R.v2 = -1; R.table = 0;
  if (valid) R = rows[r];
  for (int w0 = 0; w0 < kwu; w0 += kUG) {          // uniform across the warp
    const int nw = min(kUG, kwu - w0);
    uint32_t a[kUG], b[kUG];
    if (valid) {
      load_words(X, R.v1, kws, w0, nw, vec, a);
      if (R.v2 >= 0) {
        load_words(X, R.v2, kws, w0, nw, vec, b);
      } else {
#pragma unroll
        for (int j = 0; j < kUG; ++j) b[j] = 0u;
      }
    }
#pragma unroll
    for (int j = 0; j < kUG; ++j) {
      if (j >= nw) break;
      uint32_t vmask = 0u;
      if (valid) {
        const uint32_t T = R.table;
        vmask = ((T & 1u) ? (~a[j] & ~b[j]) : 0u) | ((T & 2u) ? (a[j] & ~b[j]) : 0u) |
                ((T & 4u) ? (~a[j] & b[j]) : 0u) | ((T & 8u) ? (a[j] & b[j]) : 0u);
        const int nt = len - 32 * (w0 + j);
        if (nt < 32) vmask &= (1u << nt) - 1u;
      }
      if (__any_sync(0xFFFFFFFFu, vmask != 0u))
        add_violations(vmask, R.inst, w0 + j, chunk, viol, valid);
    }
  }
}

// Runs of P rows (v1 + e stride, v2), e < len: one warp per chunk; lane l
// takes rows l, l + 32, ..., kPRowsU of them loaded together.  The words of
// v2 are loaded once per chunk, and each row's words are one contiguous
// segment of X.
constexpr int kPRowsU = 4;
// A row's violation masks over all candidate words are formed first, and
// the per-word aggregation runs only when some lane has a violation.
__global__ void __launch_bounds__(256)
k_eval_pchunks(const GfPChunk* __restrict__ chunks, int64_t nchunks,
               const uint32_t* __restrict__ X, int kws, int kwu, int len, int chunk,
               int32_t* __restrict__ viol) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;                       // uniform across the warp
  const GfPChunk C = chunks[c];
  const bool vec = (kws % 4) == 0;
  const uint32_t T = C.table;
  for (int w0 = 0; w0 < kwu; w0 += kUG) {
    const int nw = min(kUG, kwu - w0);
    uint32_t b[kUG];
    load_words(X, (int64_t)C.v2, kws, w0, nw, vec, b);     // the hub: once per chunk
    for (int e0 = 0; e0 < C.len; e0 += 32 * kPRowsU) {      // uniform across the warp
      // the words of kPRowsU rows per lane are loaded before any is used
      uint32_t a[kPRowsU][kUG];
#pragma unroll
      for (int r = 0; r < kPRowsU; ++r) {
        const int e = e0 + 32 * r + lane;
        if (e < C.len) {
          load_words(X, (int64_t)C.v1 + (int64_t)e * C.stride, kws, w0, nw, vec, a[r]);
        } else {
#pragma unroll
          for (int j = 0; j < kUG; ++j) a[r][j] = 0u;
        }
      }
#pragma unroll
      for (int r = 0; r < kPRowsU; ++r) {
        const int e = e0 + 32 * r + lane;
        const bool valid = e < C.len;
        uint32_t vm[kUG];
        uint32_t any = 0u;
#pragma unroll
        for (int j = 0; j < kUG; ++j) {
          uint32_t vmask = 0u;
          if (valid && j < nw) {
            const uint32_t x = a[r][j], y = b[j];
            vmask = ((T & 1u) ? (~x & ~y) : 0u) | ((T & 2u) ? (x & ~y) : 0u) |
                    ((T & 4u) ? (~x & y) : 0u) | ((T & 8u) ? (x & y) : 0u);
            const int nt = len - 32 * (w0 + j);
            if (nt < 32) vmask &= (1u << nt) - 1u;
          }
          vm[j] = vmask;
          any |= vmask;
        }
        if (!__any_sync(0xFFFFFFFFu, any != 0u)) continue;
#pragma unroll
        for (int j = 0; j < kUG; ++j) {
          if (j >= nw) break;
          if (__any_sync(0xFFFFFFFFu, vm[j] != 0u))
            add_violations(vm[j], C.inst, w0 + j, chunk, viol, valid);
        }
      }
    }
  }
}

// Slices of P-row runs: one warp per slice, lane l the run of hub v2 + l
// (its words loaded once) over rows v1 + l + e stride, kPRowsU rows in
// flight; a warp's loads of one row index e are adjacent variables.
__global__ void __launch_bounds__(256)
k_eval_pslices(const GfPSlice* __restrict__ sl, int64_t nsl, const uint32_t* __restrict__ X,
               int kws, int kwu, int len, int chunk, int32_t* __restrict__ viol) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nsl) return;                           // uniform across the warp
  const GfPSlice S = sl[c];
  const bool vec = (kws % 4) == 0;
  const uint32_t T = S.table;
  const bool lv = lane < S.lanes;
  for (int w0 = 0; w0 < kwu; w0 += kUG) {
    const int nw = min(kUG, kwu - w0);
    uint32_t b[kUG];
    if (lv) {
      load_words(X, (int64_t)S.v2 + lane, kws, w0, nw, vec, b);
    } else {
#pragma unroll
      for (int j = 0; j < kUG; ++j) b[j] = 0u;
    }
    for (int e0 = 0; e0 < S.len; e0 += kPRowsU) {  // uniform across the warp
      uint32_t a[kPRowsU][kUG];
#pragma unroll
      for (int r = 0; r < kPRowsU; ++r) {
        const int e = e0 + r;
        if (lv && e < S.len) {
          load_words(X, (int64_t)S.v1 + lane + (int64_t)e * S.stride, kws, w0, nw, vec, a[r]);
        } else {
#pragma unroll
          for (int j = 0; j < kUG; ++j) a[r][j] = 0u;
        }
      }
#pragma unroll
      for (int r = 0; r < kPRowsU; ++r) {
        const bool valid = lv && e0 + r < S.len;
        uint32_t vm[kUG];
        uint32_t any = 0u;
#pragma unroll
        for (int j = 0; j < kUG; ++j) {
          uint32_t vmask = 0u;
          if (valid && j < nw) {
            const uint32_t x = a[r][j], y = b[j];
            vmask = ((T & 1u) ? (~x & ~y) : 0u) | ((T & 2u) ? (x & ~y) : 0u) |
                    ((T & 4u) ? (~x & y) : 0u) | ((T & 8u) ? (x & y) : 0u);
            const int nt = len - 32 * (w0 + j);
            if (nt < 32) vmask &= (1u << nt) - 1u;
          }
          vm[j] = vmask;
          any |= vmask;
        }
        if (!__any_sync(0xFFFFFFFFu, any != 0u)) continue;
#pragma unroll
        for (int j = 0; j < kUG; ++j) {
          if (j >= nw) break;
          if (__any_sync(0xFFFFFFFFu, vm[j] != 0u))
            add_violations(vm[j], S.inst, w0 + j, chunk, viol, valid);
        }
      }
    }
  }
}

// G rows: 32 per-candidate accumulators.
__global__ void __launch_bounds__(128)
k_eval_grows(const GfGRow* __restrict__ rows, int64_t nrows,
             const int32_t* __restrict__ gcols, const int32_t* __restrict__ gvals,
             const uint32_t* __restrict__ X, int kws, int kwu, int len, int chunk,
             int32_t* __restrict__ viol) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = (int)(gid / nrows);
  const int64_t r = gid - (int64_t)w * nrows;
  const bool valid = (w < kwu);
  uint32_t vmask = 0;
  int inst = 0;
  if (valid) {
    const GfGRow R = rows[r];
    inst = R.inst;
    long long acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0;
    for (int q = 0; q < R.len; ++q) {
      const uint32_t m = X[(int64_t)gcols[R.t0 + q] * kws + w];
      if (!m) continue;
      const long long a = gvals[R.t0 + q];
#pragma unroll
      for (int t = 0; t < 32; ++t) acc[t] += ((m >> t) & 1u) ? a : 0ll;
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const bool bad = R.eq ? (acc[t] != R.rhs) : (acc[t] < R.rhs);
      vmask |= (uint32_t)bad << t;
    }
    const int nt = len - 32 * w;
    if (nt < 32) vmask &= (1u << nt) - 1u;
  }
  add_violations(vmask, inst, w, chunk, viol, valid);
}

// Long G rows: one 256-thread block per (row, candidate word); each thread
// sums its entries for the 32 candidates, a warp reduction hands lane t the
// warp's sum for candidate t, and the warps' sums are added in shared
// memory.  Integer sums, so the counts equal the one-thread kernel's.
__global__ void __launch_bounds__(256)
k_eval_grows_long(const GfGRow* __restrict__ rows, const int32_t* __restrict__ gcols,
                  const int32_t* __restrict__ gvals, const uint32_t* __restrict__ X, int kws,
                  int len, int chunk, int32_t* __restrict__ viol) {
  const GfGRow R = rows[blockIdx.x];
  const int w = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long acc[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) acc[t] = 0;
  for (int q = threadIdx.x; q < R.len; q += blockDim.x) {
    const uint32_t m = X[(int64_t)gcols[R.t0 + q] * kws + w];
    if (!m) continue;
    const long long a = gvals[R.t0 + q];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] += ((m >> t) & 1u) ? a : 0ll;
  }
  long long mine = 0;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    long long v = acc[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    if (lane == t) mine = v;
  }
  __shared__ long long red[8][32];
  red[warp][lane] = mine;
  __syncthreads();
  if (warp == 0) {
    long long tot = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += red[q][lane];
    const bool bad = R.eq ? (tot != R.rhs) : (tot < R.rhs);
    if (bad && 32 * w + lane < len)
      atomicAdd(&viol[(int64_t)R.inst * chunk + 32 * w + lane], 1);
  }
}

constexpr int kQW = 4;

// Weighted counts of a warp's 32 items for the 32 candidates of each of kQW
// words: acc[k] of lane b gains sum_l w_l * bit b of m_l[k] (lane l: item
// l's weight w_l and candidate words m_l).  A bit transpose hands lane b the
// word T of its candidate; with the weights shifted to u_l = w_l + bias >= 0
// (P bit planes by ballot) the sum is sum_p 2^p popc(T & plane_p) -
// bias popc(T).
template <int P>
GF_DEV void weighted_counts(const uint32_t (&m)[kQW], uint32_t u, long long bias, int nw,
                            const gf::TransposeLane& tl, long long (&acc)[kQW]) {
  uint32_t plane[P > 0 ? P : 1];
#pragma unroll
  for (int q = 0; q < P; ++q) plane[q] = __ballot_sync(0xFFFFFFFFu, (u >> q) & 1u);
#pragma unroll
  for (int k = 0; k < kQW; ++k) {
    if (k >= nw) break;
    const uint32_t T = gf::warp_transpose32(m[k], tl);
    int sum = 0;                                 // <= 32 (2^P - 1) < 2^18
#pragma unroll
    for (int q = 0; q < P; ++q) sum += __popc(T & plane[q]) * (1 << q);
    acc[k] += (long long)sum - bias * (long long)__popc(T);
  }
}

// The same sums item by item (broadcast of each nonzero word and its
// weight): cheaper when few items have a nonzero word, and the form for
// weight spans wider than the bit-plane kernels take.
GF_DEV void weighted_counts_sparse(const uint32_t (&m)[kQW], long long w, int nw, int lane,
                                   long long (&acc)[kQW]) {
#pragma unroll
  for (int k = 0; k < kQW; ++k) {
    if (k >= nw) break;
    unsigned nz = __ballot_sync(0xFFFFFFFFu, m[k] != 0u && w != 0);
    while (nz) {
      const int src = __ffs(nz) - 1;
      nz &= nz - 1;
      const uint32_t word = __shfl_sync(0xFFFFFFFFu, m[k], src);
      const long long wv = __shfl_sync(0xFFFFFFFFu, w, src);
      if ((word >> lane) & 1u) acc[k] += wv;
    }
  }
}

// Bit-plane form for P <= 12 planes (uniform across the warp), else item by
// item.
GF_DEV void weighted_counts_p(int P, const uint32_t (&m)[kQW], long long w, long long bias,
                              int nw, int lane, const gf::TransposeLane& tl,
                              long long (&acc)[kQW]) {
  const uint32_t u = (uint32_t)(w + bias);
  switch (P) {
    case 0: weighted_counts<0>(m, u, bias, nw, tl, acc); break;
    case 1: weighted_counts<1>(m, u, bias, nw, tl, acc); break;
    case 2: weighted_counts<2>(m, u, bias, nw, tl, acc); break;
    case 3: weighted_counts<3>(m, u, bias, nw, tl, acc); break;
    case 4: weighted_counts<4>(m, u, bias, nw, tl, acc); break;
    case 5: weighted_counts<5>(m, u, bias, nw, tl, acc); break;
    case 6: weighted_counts<6>(m, u, bias, nw, tl, acc); break;
    case 7: weighted_counts<7>(m, u, bias, nw, tl, acc); break;
    case 8: weighted_counts<8>(m, u, bias, nw, tl, acc); break;
    case 9: weighted_counts<9>(m, u, bias, nw, tl, acc); break;
    case 10: weighted_counts<10>(m, u, bias, nw, tl, acc); break;
    case 11: weighted_counts<11>(m, u, bias, nw, tl, acc); break;
    case 12: weighted_counts<12>(m, u, bias, nw, tl, acc); break;
    default: weighted_counts_sparse(m, w, nw, lane, acc); break;
  }
}

constexpr int kSparseLanes = 16;

// Linear objective c^T x_s of every candidate: a warp takes 32 variables
// (lane = variable; 32-variable groups never straddle instances, whose
// offsets are multiples of 64) and kQW candidate words; per group the bias
// -min c and the bit width P of the cost span are precomputed.  Block sums
// go to obj with one atomic per candidate.
__global__ void __launch_bounds__(256)
k_eval_obj_lin(const GfObjChunk* __restrict__ ch, int64_t nch,
               const long long* __restrict__ cint, const long long* __restrict__ gbias,
               const uint8_t* __restrict__ gP, const uint32_t* __restrict__ X, int kws,
               int kwu, int len, int chunk, const uint32_t* __restrict__ gmask,
               long long* __restrict__ obj) {
  const int64_t c = blockIdx.x;
  if (c >= nch) return;
  const GfObjChunk C = ch[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const gf::TransposeLane tl = gf::transpose_lane(lane);
  __shared__ long long red[8][kQW][32];
  for (int w0 = 0; w0 < kwu; w0 += kQW) {
    const int nw = min(kQW, kwu - w0);
    const bool vec = (kws % 4) == 0 && nw == kQW;
    long long acc[kQW] = {0, 0, 0, 0};
    for (int v = C.v0 + warp * 32; v < C.v1; v += 256) {
      const int myv = v + lane;
      uint32_t mw[kQW] = {0u, 0u, 0u, 0u};
      long long mc = 0;
      if (myv < C.v1) {
        mc = cint[myv];
        const uint32_t* src = X + (int64_t)myv * kws + w0;
        if (vec) {
          const uint4 q = __ldg(reinterpret_cast<const uint4*>(src));
          mw[0] = q.x; mw[1] = q.y; mw[2] = q.z; mw[3] = q.w;
        } else {
#pragma unroll
          for (int j = 0; j < kQW; ++j)
            if (j < nw) mw[j] = __ldg(src + j);
        }
      }
      // lanes whose variable's objective came with the one-hot picks
      if (gmask && ((gmask[v >> 5] >> lane) & 1u)) {
#pragma unroll
        for (int j = 0; j < kQW; ++j) mw[j] = 0u;
      }
      // item by item when at most kSparseLanes (variable, word) pairs of the
      // four words are nonzero (sparse candidates, e.g. one-hot groups)
      int dense = 0;
#pragma unroll
      for (int j = 0; j < kQW; ++j) dense += __popc(__ballot_sync(0xFFFFFFFFu, mw[j] != 0u));
      if (dense <= kSparseLanes) weighted_counts_sparse(mw, mc, nw, lane, acc);
      else weighted_counts_p(gP[v >> 5], mw, mc, gbias[v >> 5], nw, lane, tl, acc);
    }
#pragma unroll
    for (int j = 0; j < kQW; ++j) red[warp][j][lane] = acc[j];
    __syncthreads();
    if (warp < nw) {
      long long s = 0;
      for (int q = 0; q < 8; ++q) s += red[q][warp][lane];
      const int cand = 32 * (w0 + warp) + lane;
      if (s != 0 && cand < len)
        atomicAdd(reinterpret_cast<unsigned long long*>(&obj[(int64_t)C.inst * chunk + cand]),
                  (unsigned long long)s);
    }
    __syncthreads();
  }
}

// Sparse Q term: sum over the pairs (i < j) of w_ij x_i x_j per candidate
// (w_ij = q_ij + q_ji).  A warp takes a block of 32 pairs (lane l: m_l =
// X_i & X_j of pair l, weight w_l) and kQW candidate words; the block's
// bias -min w and bit width P of the weight span are precomputed.
__global__ void __launch_bounds__(256)
k_eval_obj_q(const GfQChunk* __restrict__ ch, int64_t nch, const int32_t* __restrict__ Pi,
             const int32_t* __restrict__ Pj, const long long* __restrict__ Pv,
             const long long* __restrict__ Pb, const uint8_t* __restrict__ Pw,
             const uint32_t* __restrict__ X, int kws, int kwu, int len, int chunk,
             long long* __restrict__ obj) {
  const int64_t c = blockIdx.x;
  const int w0 = blockIdx.y * kQW;
  if (c >= nch || w0 >= kwu) return;
  const GfQChunk C = ch[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = min(kQW, kwu - w0);
  const bool vec = (kws % 4) == 0 && nw == kQW;
  const gf::TransposeLane tl = gf::transpose_lane(lane);
  long long acc[kQW] = {0, 0, 0, 0};
  for (int pb = C.r0 + warp; pb < C.r1; pb += 8) {
    const int64_t t = (int64_t)pb * 32 + lane;
    const int64_t i = Pi[t], j = Pj[t];
    uint32_t m[kQW] = {0u, 0u, 0u, 0u};
    {
      const uint32_t* si = X + i * kws + w0;
      const uint32_t* sj = X + j * kws + w0;
      if (vec) {
        const uint4 a4 = __ldg(reinterpret_cast<const uint4*>(si));
        const uint4 b4 = __ldg(reinterpret_cast<const uint4*>(sj));
        m[0] = a4.x & b4.x; m[1] = a4.y & b4.y; m[2] = a4.z & b4.z; m[3] = a4.w & b4.w;
      } else {
#pragma unroll
        for (int k = 0; k < kQW; ++k)
          if (k < nw) m[k] = __ldg(si + k) & __ldg(sj + k);
      }
    }
    weighted_counts_p(Pw[pb], m, Pv[t], Pb[pb], nw, lane, tl, acc);
  }
  __shared__ long long red[8][kQW][32];
#pragma unroll
  for (int k = 0; k < kQW; ++k) red[warp][k][lane] = acc[k];
  __syncthreads();
  if (warp < nw) {
    long long sm = 0;
    for (int q = 0; q < 8; ++q) sm += red[q][warp][lane];
    const int s = 32 * (w0 + warp) + lane;
    if (sm != 0 && s < len)
      atomicAdd(reinterpret_cast<unsigned long long*>(&obj[(int64_t)C.inst * chunk + s]),
                (unsigned long long)sm);
  }
}

// Fused sampling + evaluation for single-row instances (knapsack form
// -w^T x >= -cap): a thread takes kFusedCpt candidates (128 threads, 128 kFusedCpt
// candidates per block), the block walks a slice [v0, v1) of one instance's
// variables four at a time (one Philox call per four Bernoulli draws of one
// candidate; the thresholds and row data are loaded once for all of a
// thread's candidates), accumulating the row sum and the objective;
// nothing is materialised.
constexpr int kFusedCpt = 4;

template <typename Acc>
__global__ void __launch_bounds__(128)
k_fused_single_row(const int32_t* __restrict__ blk, const uint32_t* __restrict__ thr,
                   const int32_t* __restrict__ wrow, const long long* __restrict__ cint,
                   const int32_t* __restrict__ c32, const int64_t* __restrict__ var_off,
                   int s0, int len, int chunk, uint64_t seed, int inst_base,
                   const GfDState* __restrict__ st, long long* __restrict__ fsum,
                   long long* __restrict__ obj) {
  const int b = blk[3 * blockIdx.x], v0 = blk[3 * blockIdx.x + 1], v1 = blk[3 * blockIdx.x + 2];
  const int sbase = blockIdx.y * (128 * kFusedCpt) + threadIdx.x;
  if (sbase >= len) return;
  uint32_t s[kFusedCpt];
  bool on[kFusedCpt];
#pragma unroll
  for (int q = 0; q < kFusedCpt; ++q) {
    on[q] = sbase + 128 * q < len;
    s[q] = (uint32_t)(s0 + sbase + 128 * q);
  }
  const uint32_t round = st->round_id;
  const int64_t off = var_off[b];
  const gf::PhiloxKeys K = gf::philox_keys(seed);
  const uint32_t c3 = ((uint32_t)(inst_base + b) & 0x0FFFFFFFu) | (gf::kStreamBern << 28);
  Acc rs[kFusedCpt], ob[kFusedCpt];       // int32 when every sum provably fits
#pragma unroll
  for (int q = 0; q < kFusedCpt; ++q) rs[q] = ob[q] = 0;
  // pointers advance by increments (no per-load index multiply), and the
  // selected terms are masked in with logic ops: the integer multiply pipe
  // is left to the generator, which bounds this kernel
  const uint4* tp = reinterpret_cast<const uint4*>(thr + v0);
  const int4* wp = reinterpret_cast<const int4*>(wrow + v0);
  // (the int64 form reads cint instead; cp then walks wrow unused)
  const int4* cp = reinterpret_cast<const int4*>((sizeof(Acc) == 4 ? c32 : wrow) + v0);
  uint32_t q4 = (uint32_t)((v0 - off) >> 2);
  for (int v = v0; v < v1; v += 4, ++tp, ++wp, ++cp, ++q4) {
    const uint4 t = *tp;
    const int4 ww = *wp;
    int4 cc = make_int4(0, 0, 0, 0);
    if constexpr (sizeof(Acc) == 4) cc = *cp;
#pragma unroll
    for (int q = 0; q < kFusedCpt; ++q) {
      if (!on[q]) continue;                      // warp-uniform (len: whole words)
      const uint4 u = gf::philox_k(make_uint4(q4, s[q], round, c3), K);
      const int m0 = -(int)((u.x >> 8) < t.x), m1 = -(int)((u.y >> 8) < t.y);
      const int m2 = -(int)((u.z >> 8) < t.z), m3 = -(int)((u.w >> 8) < t.w);
      rs[q] += (ww.x & m0) + (ww.y & m1) + (ww.z & m2) + (ww.w & m3);
      if constexpr (sizeof(Acc) == 4) {
        ob[q] += (cc.x & m0) + (cc.y & m1) + (cc.z & m2) + (cc.w & m3);
      } else {
        if (m0) ob[q] += cint[v];
        if (m1) ob[q] += cint[v + 1];
        if (m2) ob[q] += cint[v + 2];
        if (m3) ob[q] += cint[v + 3];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kFusedCpt; ++q) {
    if (!on[q]) continue;
    const int sidx = sbase + 128 * q;
    atomicAdd(reinterpret_cast<unsigned long long*>(&fsum[(int64_t)b * chunk + sidx]),
              (unsigned long long)(long long)rs[q]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&obj[(int64_t)b * chunk + sidx]),
              (unsigned long long)(long long)ob[q]);
  }
}

// Thresholds floor(p 2^24) of every variable (0 for padding), once per chunk.
__global__ void k_thresholds_all(const float* __restrict__ p, const uint8_t* __restrict__ live,
                                 int64_t N, uint32_t* __restrict__ thr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) thr[i] = live[i] ? gf::prob_threshold(p[i]) : 0u;
}

__global__ void k_fused_viol(const long long* __restrict__ fsum, const long long* __restrict__ rhs,
                             int ninst, int len, int chunk, int32_t* __restrict__ viol) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (int64_t)ninst * len) return;
  const int b = (int)(gid / len), s = (int)(gid % len);
  viol[(int64_t)b * chunk + s] = (fsum[(int64_t)b * chunk + s] < rhs[b]) ? 1 : 0;
}

// Incumbent update of one instance per block: least feasible objective,
// earliest candidate on ties; replaces only when strictly better.
// (obj, sample) pair ordering: feasible first, then smaller objective, then
// earlier sample.
GF_DEV bool better(long long oa, int sa, long long ob, int sb) {
  if (sb < 0) return false;
  if (sa < 0) return true;
  return ob < oa || (ob == oa && sb < sa);
}

constexpr int kIncThreads = 1024;

__global__ void __launch_bounds__(kIncThreads)
k_incumbent(const int32_t* __restrict__ viol, const long long* __restrict__ obj, int len,
            int chunk, int s0, const GfDState* __restrict__ st, GfInc* __restrict__ inc) {
  const int b = blockIdx.x;
  const int32_t* vb = viol + (int64_t)b * chunk;
  const long long* ob = obj + (int64_t)b * chunk;
  long long best = 0;
  int bs = -1;
  // four independent loads in flight per thread
  for (int s = threadIdx.x; s < len; s += 4 * kIncThreads) {
    int vv[4];
    long long oo[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int su = s + u * kIncThreads;
      vv[u] = (su < len) ? vb[su] : 1;
      oo[u] = (su < len) ? ob[su] : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (vv[u] == 0 && better(best, bs, oo[u], s + u * kIncThreads)) {
        best = oo[u];
        bs = s + u * kIncThreads;
      }
  }
  // warp argmin by shuffles, then across the 32 warps
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long o2 = __shfl_down_sync(0xFFFFFFFFu, best, off);
    const int s2 = __shfl_down_sync(0xFFFFFFFFu, bs, off);
    if (better(best, bs, o2, s2)) { best = o2; bs = s2; }
  }
  __shared__ long long wb[32];
  __shared__ int ws[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { wb[warp] = best; ws[warp] = bs; }
  __syncthreads();
  if (warp == 0) {
    best = (lane < kIncThreads / 32) ? wb[lane] : 0;
    bs = (lane < kIncThreads / 32) ? ws[lane] : -1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const long long o2 = __shfl_down_sync(0xFFFFFFFFu, best, off);
      const int s2 = __shfl_down_sync(0xFFFFFFFFu, bs, off);
      if (better(best, bs, o2, s2)) { best = o2; bs = s2; }
    }
    if (lane == 0) {
      GfInc I = inc[b];
      I.changed = 0;
      if (bs >= 0 && (!I.found || best < I.obj)) {
        I.found = 1;
        I.obj = best;
        I.objf = (double)best;
        I.round_id = st->round_id;
        I.sample = s0 + bs;
        I.changed = 1;
      }
      inc[b] = I;
    }
  }
}

// x_best extraction after an update (mode 0: bits, 1: Philox regeneration
// of a fused candidate, dense instances read their bf16 operand).
__global__ void __launch_bounds__(256)
k_extract(const GfInc* __restrict__ inc, const int32_t* __restrict__ var_inst,
          const int64_t* __restrict__ var_off, const uint8_t* __restrict__ live, int64_t N,
          const uint32_t* __restrict__ X, int kws, int s0, int mode, const float* __restrict__ p,
          uint64_t seed, int inst_base, uint8_t* __restrict__ xbest) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int b = var_inst[i];
  const GfInc I = inc[b];
  if (!I.changed) return;
  if (!live[i]) { xbest[i] = 0; return; }
  const int sl = I.sample - s0;
  uint8_t bit;
  if (mode == 1) {
    const int64_t loc = i - var_off[b];
    const uint4 u = gf::philox_call(seed, gf::kStreamBern, (uint32_t)(inst_base + b), I.round_id,
                                    (uint32_t)I.sample, (uint64_t)(loc >> 2));
    bit = (gf::lane_of(u, (uint32_t)(loc & 3)) >> 8) < gf::prob_threshold(p[i]);
  } else {
    bit = (X[i * kws + (sl >> 5)] >> (sl & 31)) & 1u;
  }
  xbest[i] = bit;
}

// The same per instance: block row b covers instance b's variables and
// returns at once when its incumbent did not change (no per-variable reads).
__global__ void __launch_bounds__(256)
k_extract_inst(const GfInc* __restrict__ inc, const int64_t* __restrict__ var_off,
               const uint8_t* __restrict__ live, const uint32_t* __restrict__ X, int kws,
               int s0, int mode, const float* __restrict__ p, uint64_t seed, int inst_base,
               uint8_t* __restrict__ xbest) {
  const int b = blockIdx.y;
  const GfInc I = inc[b];
  if (!I.changed) return;
  const int64_t v0 = var_off[b], n = var_off[b + 1] - v0;
  const int sl = I.sample - s0;
  for (int64_t loc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; loc < n;
       loc += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = v0 + loc;
    if (!live[i]) { xbest[i] = 0; continue; }
    uint8_t bit;
    if (mode == 1) {
      const uint4 u = gf::philox_call(seed, gf::kStreamBern, (uint32_t)(inst_base + b),
                                      I.round_id, (uint32_t)I.sample, (uint64_t)(loc >> 2));
      bit = (gf::lane_of(u, (uint32_t)(loc & 3)) >> 8) < gf::prob_threshold(p[i]);
    } else {
      bit = (X[i * kws + (sl >> 5)] >> (sl & 31)) & 1u;
    }
    xbest[i] = bit;
  }
}

__global__ void k_extract_dense(const GfInc* __restrict__ inc, int b, int64_t v0, int64_t n,
                                int64_t ld, const uint32_t* __restrict__ Xw, int s0,
                                uint8_t* __restrict__ xbest) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GfInc I = inc[b];
  if (!I.changed) return;
  const int sl = I.sample - s0;
  xbest[v0 + i] = (Xw[(int64_t)sl * (ld / 32) + i / 32] >> (i & 31)) & 1u;
}

__global__ void k_round_end(GfDState* st) { st->round_id += 1u; }

}  // namespace

// Exact evaluation of the materialised chunk (bits in h->X) of every
// non-dense instance into viol / obj (zeroed here).
cudaError_t gf_launch_eval(GfCtx* h, int s0, int len, bool pick_obj) {
  (void)s0;
  cudaError_t e;
  const int kwu = (len + 31) / 32;
  if ((e = cudaMemsetAsync(h->viol, 0, sizeof(int32_t) * h->ninst * h->chunk, h->stream)))
    return e;
  // the objective starts from the one-hot picks' costs when the sampler left them
  if (pick_obj) {
    if ((e = cudaMemcpyAsync(h->obj, h->objp, sizeof(long long) * h->ninst * h->chunk,
                             cudaMemcpyDeviceToDevice, h->stream)))
      return e;
  } else if ((e = cudaMemsetAsync(h->obj, 0, sizeof(long long) * h->ninst * h->chunk,
                                  h->stream))) {
    return e;
  }
  for (int c = 0, r0 = 0; c < 3; r0 += (int)h->nurows_cls[c], ++c) {
    const int64_t nr = h->nurows_cls[c];
    if (!nr) continue;
    const int64_t warps = nr * ((kwu + kUG - 1) / kUG);
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    const GfURow* rows = h->urows + r0;
    if (c == 0)
      k_eval_urows<0><<<blocks, 256, 0, h->stream>>>(rows, nr, h->ucols, h->X, h->kw, kwu, len,
                                                     h->chunk, h->viol);
    else if (c == 1)
      k_eval_urows<1><<<blocks, 256, 0, h->stream>>>(rows, nr, h->ucols, h->X, h->kw, kwu, len,
                                                     h->chunk, h->viol);
    else
      k_eval_urows<2><<<blocks, 256, 0, h->stream>>>(rows, nr, h->ucols, h->X, h->kw, kwu, len,
                                                     h->chunk, h->viol);
    h->launches++;
  }
  if (h->npslices) {
    k_eval_pslices<<<(unsigned)((h->npslices * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->pslices, h->npslices, h->X, h->kw, kwu, len, h->chunk, h->viol);
    h->launches++;
  }
  if (h->npchunks) {
    k_eval_pchunks<<<(unsigned)((h->npchunks * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->pchunks, h->npchunks, h->X, h->kw, kwu, len, h->chunk, h->viol);
    h->launches++;
  }
  if (h->nprows) {
    k_eval_prows<<<(unsigned)((h->nprows + 255) / 256), 256, 0, h->stream>>>(
        h->prows, h->nprows, h->X, h->kw, kwu, len, h->chunk, h->viol);
    h->launches++;
  }
  if (h->ngrows_short) {
    const int64_t th = h->ngrows_short * kwu;
    k_eval_grows<<<(unsigned)((th + 127) / 128), 128, 0, h->stream>>>(
        h->grows, h->ngrows_short, h->gcols, h->gvals, h->X, h->kw, kwu, len, h->chunk,
        h->viol);
    h->launches++;
  }
  if (h->ngrows > h->ngrows_short) {
    dim3 grid((unsigned)(h->ngrows - h->ngrows_short), (unsigned)kwu);
    k_eval_grows_long<<<grid, 256, 0, h->stream>>>(h->grows + h->ngrows_short, h->gcols,
                                                   h->gvals, h->X, h->kw, len, h->chunk,
                                                   h->viol);
    h->launches++;
  }
  if (h->nochunks) {
    const GfObjChunk* ocs = pick_obj ? h->ochunks_ng : h->ochunks;
    const int64_t noc = pick_obj ? h->nochunks_ng : h->nochunks;
    if (noc > 0) {
      k_eval_obj_lin<<<(unsigned)noc, 256, 0, h->stream>>>(
          ocs, noc, h->clin ? h->clin : h->cint, h->cgbias, h->cgP, h->X, h->kw, kwu, len,
          h->chunk, pick_obj ? h->slab_gmask : nullptr, h->obj);
      h->launches++;
    }
  }
  if (h->nqchunks) {
    dim3 grid((unsigned)h->nqchunks, (unsigned)((kwu + kQW - 1) / kQW));
    const int pq = gf_prof_begin(h, 8);         // inside phase 2
    k_eval_obj_q<<<grid, 256, 0, h->stream>>>(h->qchunks, h->nqchunks, h->QIi, h->QIc, h->QIv,
                                              h->QIb, h->QIw, h->X, h->kw, kwu, len, h->chunk,
                                              h->obj);
    gf_prof_end(h, pq, 1);
    h->launches++;
  }
  return cudaGetLastError();
}

cudaError_t gf_launch_fused(GfCtx* h, const float* p, int s0, int len) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->fsum, 0, sizeof(long long) * h->ninst * h->chunk, h->stream)))
    return e;
  if ((e = cudaMemsetAsync(h->obj, 0, sizeof(long long) * h->ninst * h->chunk, h->stream)))
    return e;
  dim3 grid((unsigned)h->nfblk, (unsigned)((len + 128 * kFusedCpt - 1) / (128 * kFusedCpt)));
  k_thresholds_all<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(p, h->var_live, h->N,
                                                                           h->fthr);
  if (h->f_c32)
    k_fused_single_row<int><<<grid, 128, 0, h->stream>>>(
        h->fblk, h->fthr, h->frow_w, h->cint, h->f_c32, h->var_off_d, s0, len, h->chunk,
        h->prm.seed, h->prm.inst_base, h->dstate, h->fsum, h->obj);
  else
    k_fused_single_row<long long><<<grid, 128, 0, h->stream>>>(
        h->fblk, h->fthr, h->frow_w, h->cint, nullptr, h->var_off_d, s0, len, h->chunk,
        h->prm.seed, h->prm.inst_base, h->dstate, h->fsum, h->obj);
  h->launches++;
  const int64_t th = (int64_t)h->ninst * len;
  k_fused_viol<<<(unsigned)((th + 255) / 256), 256, 0, h->stream>>>(h->fsum, h->frhs, h->ninst,
                                                                   len, h->chunk, h->viol);
  h->launches += 2;
  return cudaGetLastError();
}

// mode: 0 materialised bits, 1 fused (Philox regeneration), 2 dense.
cudaError_t gf_launch_incumbent(GfCtx* h, int s0, int len, int mode, bool last_chunk) {
  k_incumbent<<<h->ninst, kIncThreads, 0, h->stream>>>(h->viol, h->obj, len, h->chunk, s0, h->dstate,
                                               h->inc);
  h->launches++;
  if (h->N > 0 && mode != 2) {
    int64_t span = 0;                        // the largest instance's variable range
    for (int b = 0; b < h->ninst; ++b) {
      const int64_t end = (b + 1 < h->ninst) ? h->ih[b + 1].var_off : h->N;
      span = std::max(span, end - h->ih[b].var_off);
    }
    if (h->ninst <= 65535) {
      const dim3 grid((unsigned)std::min<int64_t>((span + 255) / 256, 4096), (unsigned)h->ninst);
      k_extract_inst<<<grid, 256, 0, h->stream>>>(h->inc, h->var_off_d, h->var_live, h->X,
                                                   h->kw, s0, mode, h->last_p, h->prm.seed,
                                                   h->prm.inst_base, h->xbest);
    } else {
      k_extract<<<(unsigned)((h->N + 255) / 256), 256, 0, h->stream>>>(
          h->inc, h->var_inst, h->var_off_d, h->var_live, h->N, h->X, h->kw, s0, mode,
          h->last_p, h->prm.seed, h->prm.inst_base, h->xbest);
    }
    h->launches++;
  }
  for (const GfDenseQ& dq : h->dense) {
    k_extract_dense<<<(unsigned)((dq.n + 255) / 256), 256, 0, h->stream>>>(
        h->inc, dq.inst, h->ih[dq.inst].var_off, dq.n, dq.ld, dq.Xb, s0, h->xbest);
    h->launches++;
  }
  if (last_chunk) {
    k_round_end<<<1, 1, 0, h->stream>>>(h->dstate);
    h->launches++;
  }
  return cudaGetLastError();
}
