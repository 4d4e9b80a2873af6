// k_sample.cu -- RandSampleStep (Alg. 3) and the customised samplers of
// Section 2.4.2 / 2.4.3 on the device.  Candidates are stored
// variable-major and bit-packed: word X[i * kw + w] holds samples
// s0 + 32 w + t (bit t) of variable i.  Every draw comes from Philox4x32-10
// with counter (local index >> 2, sample, round, instance | stream << 28).
#include "internal.cuh"

namespace {

// Repair after the monotone relaxation (Section 2.4.3): an equality group
// relaxed to "sum >= 1" may hold several selected members; each candidate
// keeps its selected member of least cost (ties to the member listed first).
// The members of every group are stored in (cost, listing position) order,
// so that member is simply the first one selected in storage order.  One
// warp per (group, word), kRepairU chunks of 32 members per step with all
// their loads in flight: pass 1 transposes each chunk's words so that lane b
// sees candidate b's selections and keeps the first, stopping once every
// candidate has one; pass 2 transposes the kept bits back and rewrites the
// members' words that change.
constexpr int kRepairU = 4;

__global__ void __launch_bounds__(256)
k_repair_min(const int64_t* __restrict__ gp, const int64_t* __restrict__ gi, int64_t ng,
             int kws, int kwu, uint32_t* __restrict__ X) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= ng * kwu) return;                       // whole warps
  const int64_t g = wid / kwu;
  const int w = (int)(wid % kwu);
  const int64_t a = gp[g], e = gp[g + 1];
  const gf::TransposeLane tl = gf::transpose_lane(lane);
  int64_t bt = -1;                                   // storage position of the kept member
  for (int64_t t0 = a; t0 < e; t0 += 32 * kRepairU) {
    uint32_t word[kRepairU];
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const int64_t t = t0 + 32 * u + lane;
      word[u] = t < e ? X[gi[t] * kws + w] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const uint32_t T = gf::warp_transpose32(word[u], tl);
      if (bt < 0 && T) bt = t0 + 32 * u + (__ffs(T) - 1);
    }
    if (__all_sync(0xFFFFFFFFu, bt >= 0)) break;
  }
  for (int64_t t0 = a; t0 < e; t0 += 32 * kRepairU) {
    int64_t m[kRepairU];
    uint32_t cur[kRepairU];
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const int64_t t = t0 + 32 * u + lane;
      m[u] = t < e ? gi[t] : -1;
      cur[u] = t < e ? X[m[u] * kws + w] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const int64_t c0 = t0 + 32 * u;
      const uint32_t mine = (bt >= c0 && bt < c0 + 32) ? (1u << (uint32_t)(bt - c0)) : 0u;
      const uint32_t keep =
          __any_sync(0xFFFFFFFFu, mine != 0u) ? gf::warp_transpose32(mine, tl) : 0u;
      if (m[u] >= 0 && cur[u] != keep) X[m[u] * kws + w] = keep;
    }
  }
}

// General repair after a monotone relaxation (reverse delete over relaxed
// covering rows).  k_rr_count: one warp per (row, candidate word), the
// members' words in chunks of 32 transposed so that lane b counts candidate
// b's selected members.  k_rr_delete: one warp per (instance segment, word);
// the segment's row variables in decreasing cost, four 32-variable chunks
// of loads in flight; for every variable some candidate selected, each lane
// (candidate) drops it when all its rows keep another selected member, and
// the counts follow.  Every lane follows the sequential rule of its own
// candidate, so the result equals the one-candidate-at-a-time repair.
__global__ void __launch_bounds__(256)
k_rr_count(const int64_t* __restrict__ rp, const int64_t* __restrict__ ri, int64_t nr,
           int kws, int kwu, int chunk, const uint32_t* __restrict__ X,
           int32_t* __restrict__ cnt) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nr * kwu) return;                       // whole warps
  const int64_t r = wid / kwu;
  const int w = (int)(wid % kwu);
  const gf::TransposeLane tl = gf::transpose_lane(lane);
  int c = 0;
  for (int64_t t0 = rp[r]; t0 < rp[r + 1]; t0 += 32 * kRepairU) {
    uint32_t word[kRepairU];
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const int64_t t = t0 + 32 * u + lane;
      word[u] = t < rp[r + 1] ? X[ri[t] * kws + w] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) c += __popc(gf::warp_transpose32(word[u], tl));
  }
  cnt[r * chunk + 32 * w + lane] = c;
}

__global__ void __launch_bounds__(256)
k_rr_delete(const int64_t* __restrict__ optr, const int64_t* __restrict__ order,
            const int64_t* __restrict__ vptr, const int64_t* __restrict__ vrow, int64_t nseg,
            int kws, int kwu, int chunk, uint32_t* __restrict__ X, int32_t* __restrict__ cnt) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nseg * kwu) return;                     // whole warps
  const int64_t seg = wid / kwu;
  const int w = (int)(wid % kwu);
  const int64_t o0 = optr[seg], o1 = optr[seg + 1];
  const int cand = 32 * w + lane;
  for (int64_t p0 = o0; p0 < o1; p0 += 32 * kRepairU) {
    int64_t v[kRepairU];
    uint32_t m[kRepairU];
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      const int64_t p = p0 + 32 * u + lane;
      v[u] = p < o1 ? order[p] : -1;
      m[u] = v[u] >= 0 ? X[v[u] * kws + w] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kRepairU; ++u) {
      uint32_t nz = __ballot_sync(0xFFFFFFFFu, m[u] != 0u);
      while (nz) {                                   // warp-uniform
        const int l = __ffs(nz) - 1;
        nz &= nz - 1u;
        const int64_t vv = __shfl_sync(0xFFFFFFFFu, v[u], l);
        const uint32_t mm = __shfl_sync(0xFFFFFFFFu, m[u], l);
        const int64_t p = p0 + 32 * u + l;
        const int64_t t0 = vptr[p], t1 = vptr[p + 1];
        bool rem = (mm >> lane) & 1u;
        for (int64_t t = t0; t < t1; ++t)
          if (rem && cnt[vrow[t] * chunk + cand] < 2) rem = false;
        if (rem)
          for (int64_t t = t0; t < t1; ++t) cnt[vrow[t] * chunk + cand] -= 1;
        const uint32_t gone = __ballot_sync(0xFFFFFFFFu, rem);
        if (gone && lane == 0) X[vv * kws + w] = mm & ~gone;
      }
    }
  }
}

// Indices of the 4-variable groups holding a variable that no group sampler
// draws (order irrelevant: every entry writes its own words).
__global__ void k_bit_list(const uint8_t* __restrict__ grouped, int64_t N4,
                           int32_t* __restrict__ list, int32_t* __restrict__ count) {
  const int64_t g4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g4 >= N4) return;
  const uint32_t w = *reinterpret_cast<const uint32_t*>(grouped + 4 * g4);
  if (w != 0x01010101u) list[atomicAdd(count, 1)] = (int32_t)g4;
}

// Generic Bernoulli: X_si = [(u_si >> 8) < floor(p_i 2^24)].  One thread
// per (4 consecutive variables, 32-sample word): 32 Philox calls fill four
// words.  Grouped variables (drawn by a group sampler) and padding are
// skipped / zeroed.
__global__ void __launch_bounds__(256)
k_bern_bits(const float* __restrict__ p, const int32_t* __restrict__ var_inst,
            const int64_t* __restrict__ var_off, const uint8_t* __restrict__ grouped,
            const uint8_t* __restrict__ live, const int32_t* __restrict__ g4list, int64_t N4,
            int kws, int kwu, int s0, int len, uint64_t seed, int inst_base,
            const GfDState* __restrict__ st, uint32_t* __restrict__ X) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= N4 * kwu) return;
  const int64_t g4 = g4list[gid / kwu];
  const int w = (int)(gid % kwu);
  const int64_t i0 = g4 * 4;
  const int b = var_inst[i0];
  const int64_t loc4 = (i0 - var_off[b]) >> 2;
  const uint32_t round = st->round_id;
  uint32_t thr[4];
  bool skip[4];
  bool any = false;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    skip[l] = grouped[i0 + l] != 0;
    thr[l] = live[i0 + l] ? gf::prob_threshold(p[i0 + l]) : 0u;
    any |= (!skip[l] && thr[l] != 0u);
  }
  uint32_t word[4] = {0u, 0u, 0u, 0u};
  if (any) {
    const int nt = min(32, len - 32 * w);
    const gf::PhiloxKeys K = gf::philox_keys(seed);
    const uint32_t c3 = ((uint32_t)(inst_base + b) & 0x0FFFFFFFu) | (gf::kStreamBern << 28);
    for (int t = 0; t < nt; ++t) {
      const uint32_t s = (uint32_t)(s0 + 32 * w + t);
      const uint4 u = gf::philox_k(make_uint4((uint32_t)loc4, s, round, c3), K);
      word[0] |= (uint32_t)((u.x >> 8) < thr[0]) << t;
      word[1] |= (uint32_t)((u.y >> 8) < thr[1]) << t;
      word[2] |= (uint32_t)((u.z >> 8) < thr[2]) << t;
      word[3] |= (uint32_t)((u.w >> 8) < thr[3]) << t;
    }
  }
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (!skip[l]) X[(i0 + l) * kws + w] = word[l];
}

// Cumulative weights floor(p 2^24) of each group's members (in list order),
// one warp per group: warp-wide inclusive scans of 32-member slices.  A
// member list in constant steps (gstep > 0) is generated from its first
// entry.
__global__ void k_group_cw(const int64_t* __restrict__ gp, const int64_t* __restrict__ gi,
                           const int64_t* __restrict__ gstep, int64_t ngroups,
                           const float* __restrict__ p, unsigned long long* __restrict__ cw) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= ngroups) return;
  const int64_t a = gp[g], d = gstep[g];
  const int64_t v0 = d ? gi[a] : 0;         // d > 0 only for lists of 2 or more
  unsigned long long carry = 0;
  for (int64_t t0 = a; t0 < gp[g + 1]; t0 += 32) {
    const int64_t t = t0 + lane;
    const int64_t v = d ? v0 + (t - a) * d : (t < gp[g + 1] ? gi[t] : 0);
    unsigned long long w = (t < gp[g + 1]) ? gf::prob_threshold(p[v]) : 0ull;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, w, off);
      if (lane >= off) w += o;
    }
    if (t < gp[g + 1]) cw[t] = carry + w;
    carry += __shfl_sync(0xFFFFFFFFu, w, 31);
  }
}

// One-hot group draw, one warp per (group, word); a block takes one word of
// kPickWarps consecutive groups: lane t draws sample s0 + 32 w + t.  With W = total weight > 0 the pick is the first
// member whose inclusive prefix exceeds floor(u W / 2^32) (exact 128-bit
// product, binary search); with W = 0 it is member floor(u len / 2^32).
// The group's words start zeroed (one memset of the instance's range per
// chunk); each distinct pick is written once with the mask of lanes that
// chose it.  With cost != NULL the picks' costs are also summed per
// candidate over the block's warps (same word and instance) into objp.
constexpr int kPickWarps = 16;

__global__ void __launch_bounds__(32 * kPickWarps)
k_group_pick(const int64_t* __restrict__ gp, const int64_t* __restrict__ gi,
             const int64_t* __restrict__ gstep,
             const int32_t* __restrict__ ginst, const int32_t* __restrict__ glocal,
             int64_t ngroups, const unsigned long long* __restrict__ cw, int kws, int kwu,
             int s0, int len, uint64_t seed, int inst_base,
             const GfDState* __restrict__ st, uint32_t* __restrict__ X,
             const long long* __restrict__ cost, unsigned long long* __restrict__ objp,
             int chunk) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // block b: candidate word b mod kwu of the kPickWarps groups of block row
  // b / kwu (the kwu blocks of one set of groups run back to back)
  const int w = (int)(blockIdx.x % (unsigned)kwu);
  const int64_t g0 = (int64_t)(blockIdx.x / (unsigned)kwu) * kPickWarps + warp;
  const bool wvalid = g0 < ngroups;
  const int64_t g = wvalid ? g0 : 0;
  int64_t pick = -1;
  int inst = -1;
  if (wvalid) {
    inst = ginst[g];
    const int64_t a = gp[g], e = gp[g + 1];
    const int64_t glen = e - a;
    const int sidx = 32 * w + lane;
    if (glen > 0 && sidx < len) {
      const uint32_t gl = (uint32_t)glocal[g];
      const uint4 u4 = gf::philox_call(seed, gf::kStreamGroup, (uint32_t)(inst_base + inst),
                                       st->round_id, (uint32_t)(s0 + sidx), gl >> 2);
      const uint32_t u = gf::lane_of(u4, gl & 3u);
      const unsigned long long W = cw[e - 1];
      int64_t pos;
      if (W == 0ull) {
        pos = (int64_t)(((unsigned long long)u * (unsigned long long)glen) >> 32);
      } else {
        const unsigned long long lo = (unsigned long long)u * W;
        const unsigned long long hi = __umul64hi((unsigned long long)u, W);
        const unsigned long long r = (hi << 32) | (lo >> 32);
        int64_t lo_i = 0, hi_i = glen - 1;      // first position with cw > r
        while (lo_i < hi_i) {
          const int64_t mid = (lo_i + hi_i) >> 1;
          if (cw[a + mid] > r) hi_i = mid; else lo_i = mid + 1;
        }
        pos = lo_i;
      }
      const int64_t d = gstep[g];
      pick = d ? gi[a] + pos * d : gi[a + pos];
    }
  }
  const unsigned active = __ballot_sync(0xFFFFFFFFu, pick >= 0);
  const unsigned same = __match_any_sync(0xFFFFFFFFu, pick);
  if (pick >= 0 && lane == __ffs(same & active) - 1)
    X[pick * kws + w] = same & active;
  if (cost == nullptr) return;                  // the same for the whole grid
  __shared__ long long red[kPickWarps][32];
  __shared__ int key_inst[kPickWarps], key_w[kPickWarps];
  red[warp][lane] = pick >= 0 ? cost[pick] : 0;
  if (lane == 0) {
    key_inst[warp] = wvalid ? inst : -1;
    key_w[warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
    // lane t: candidate 32 w + t; warps with the first warp's (instance,
    // word) are summed here, any other warp adds its own
    const int i0 = key_inst[0], w0 = key_w[0];
    long long sum = 0;
    for (int q = 0; q < kPickWarps; ++q) {
      const int iq = key_inst[q];
      if (iq < 0) continue;
      const long long x = red[q][lane];
      if (iq == i0 && key_w[q] == w0) {
        sum += x;
      } else {
        const int cand = 32 * key_w[q] + lane;
        if (x != 0 && cand < len)
          atomicAdd(&objp[(int64_t)iq * chunk + cand], (unsigned long long)x);
      }
    }
    const int cand = 32 * w0 + lane;
    if (i0 >= 0 && sum != 0 && cand < len)
      atomicAdd(&objp[(int64_t)i0 * chunk + cand], (unsigned long long)sum);
  }
}

// Axial 3D assignment, one block per (instance, sample): for i = 0..I-1 the
// pair (j,k) is drawn among pairs with j and k both unused by the rule of
// k_group_pick over x_ijk in (j,k) row-major order (u: Philox stream 2,
// index i).  Bits are OR-ed into X (zeroed beforehand).
constexpr int kAxThreads = 256;
__global__ void __launch_bounds__(kAxThreads)
k_axial(const float* __restrict__ p, int64_t v0, int I, int inst, int s0, int len,
        int kw, uint64_t seed, int inst_base, const GfDState* __restrict__ st,
        uint32_t* __restrict__ X) {
  const int sidx = blockIdx.x;
  if (sidx >= len) return;
  const uint32_t s = (uint32_t)(s0 + sidx);
  __shared__ uint8_t usedJ[256], usedK[256];
  __shared__ unsigned long long wsum[kAxThreads / 32];
  __shared__ unsigned long long sh_r, sh_W;
  __shared__ int sh_pick;
  for (int q = threadIdx.x; q < I; q += blockDim.x) { usedJ[q] = 0; usedK[q] = 0; }
  __syncthreads();
  const int P = I * I;
  const int per = (P + kAxThreads - 1) / kAxThreads;
  const int q0 = threadIdx.x * per, q1 = min(P, q0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < I; ++i) {
    const float* pi = p + v0 + (int64_t)i * P;
    unsigned long long mine = 0;
    for (int q = q0; q < q1; ++q) {
      const int j = q / I, k = q - j * I;
      if (!usedJ[j] && !usedK[k]) mine += gf::prob_threshold(pi[q]);
    }
    // block exclusive scan of `mine`
    unsigned long long v = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, v, off);
      if (lane >= off) v += o;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    unsigned long long wbase = 0, tot = 0;
    for (int q = 0; q < kAxThreads / 32; ++q) {
      if (q < warp) wbase += wsum[q];
      tot += wsum[q];
    }
    const unsigned long long excl = wbase + v - mine;
    if (threadIdx.x == 0) {
      const uint4 u4 = gf::philox_call(seed, gf::kStreamAxial, (uint32_t)(inst_base + inst),
                                       st->round_id, s, (uint64_t)(i >> 2));
      const uint32_t u = gf::lane_of(u4, (uint32_t)(i & 3));
      sh_W = tot;
      if (tot > 0) {
        const unsigned long long lo = (unsigned long long)u * tot;
        const unsigned long long hi = __umul64hi((unsigned long long)u, tot);
        sh_r = (hi << 32) | (lo >> 32);
      } else {
        const int free = I - i;
        sh_r = ((unsigned long long)u * (unsigned long long)(free * free)) >> 32;
      }
      sh_pick = -1;
    }
    __syncthreads();
    const unsigned long long r = sh_r;
    if (sh_W > 0) {
      if (mine > 0 && excl <= r && r < excl + mine) {
        unsigned long long acc = excl;
        for (int q = q0; q < q1; ++q) {
          const int j = q / I, k = q - j * I;
          if (usedJ[j] || usedK[k]) continue;
          acc += gf::prob_threshold(pi[q]);
          if (acc > r) { sh_pick = q; break; }
        }
      }
    } else if (threadIdx.x == 0) {
      // r-th allowed pair in row-major order: (a-th free j, b-th free k)
      const int free = I - i;
      int a = (int)(r / free), bb = (int)(r % free), j = -1, k = -1;
      for (int q = 0, c = 0; q < I; ++q) if (!usedJ[q]) { if (c == a) { j = q; break; } ++c; }
      for (int q = 0, c = 0; q < I; ++q) if (!usedK[q]) { if (c == bb) { k = q; break; } ++c; }
      sh_pick = j * I + k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int q = sh_pick;
      const int j = q / I, k = q - j * I;
      usedJ[j] = 1;
      usedK[k] = 1;
      const int64_t var = v0 + (int64_t)i * P + q;
      atomicOr(&X[var * kw + (sidx >> 5)], 1u << (sidx & 31));
    }
    __syncthreads();
  }
}

// Same draws as k_axial for I <= 64: a group of four warps (128 threads) per
// candidate, four candidates per block.  Per step i the block stages
// floor(p 2^24) of slab i once in shared memory; thread t of a group owns the
// 32 pairs q in [32t, 32t + 32) (row-major; slots XOR-swizzled so that the
// group reads them conflict-free).  When 32 divides I those pairs lie in one
// row j, so the thread skips a used row at once and visits only the set bits
// of its 32 available columns.  A scan across the group gives the prefixes and
// the thread holding the crossing point finds the pick.  Identical picks to
// k_axial (first pair, row-major, whose inclusive prefix exceeds r).
GF_DEV void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
constexpr int kAxMaxP = 4096;
constexpr int kAxGroup = 128;                         // threads per candidate
constexpr int kAxCands = 4;                           // candidates per block
GF_DEV int ax_slot(int q) { return (q & ~31) | ((q & 31) ^ ((q >> 5) & 31)); }

__global__ void __launch_bounds__(kAxGroup * kAxCands, 2)
k_axial_grp(const float* __restrict__ p, int64_t v0, int I, int inst, int s0, int len,
            int kw, uint64_t seed, int inst_base, const GfDState* __restrict__ st,
            uint32_t* __restrict__ X) {
  __shared__ uint32_t wt[kAxMaxP];
  __shared__ unsigned long long gsum[kAxCands][kAxGroup / 32];
  __shared__ unsigned long long sh_r[kAxCands];
  __shared__ int sh_pick[kAxCands];
  const int g = threadIdx.x / kAxGroup;               // candidate slot in the block
  const int t = threadIdx.x % kAxGroup;               // thread in the group
  const int lane = threadIdx.x & 31, gw = t >> 5;
  const int sidx = blockIdx.x * kAxCands + g;
  const bool active = sidx < len;
  const uint32_t s = (uint32_t)(s0 + sidx);
  const int P = I * I;
  const uint32_t round = st->round_id;
  unsigned long long usedJ = 0ull, usedK = 0ull;      // uniform in the group
  const int qa = 32 * t;                              // first pair of this thread
  const int ja = qa / I, ka = qa - (qa / I) * I;
  const bool rowwise = (I % 32) == 0;                 // the 32 pairs share row ja
  const int nq = max(0, min(32, P - qa));             // pairs of this thread
  const int bar = 1 + g;                              // named barrier of the group
  for (int i = 0; i < I; ++i) {
    const float* pi = p + v0 + (int64_t)i * P;
    constexpr int kStage = kAxMaxP / (kAxGroup * kAxCands);
    float pv[kStage];
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int q = threadIdx.x + u * kAxGroup * kAxCands;
      pv[u] = q < P ? __ldg(pi + q) : 0.0f;
    }
    __syncthreads();                                  // previous step's reads done
#pragma unroll
    for (int u = 0; u < kStage; ++u) {
      const int q = threadIdx.x + u * kAxGroup * kAxCands;
      wt[ax_slot(q)] = q < P ? gf::prob_threshold(pv[u]) : 0u;
    }
    __syncthreads();
    if (!active) continue;                            // whole group alike
    // available pairs of this thread as a bit mask (bit m: pair qa + m)
    uint32_t avail = 0u;
    if (nq > 0) {
      if (rowwise) {
        if (!((usedJ >> ja) & 1ull)) avail = ~(uint32_t)(usedK >> ka);
      } else {
        int j = ja, k = ka;
        for (int m = 0; m < nq; ++m) {
          if (!(((usedJ >> j) | (usedK >> k)) & 1ull)) avail |= 1u << m;
          if (++k == I) { k = 0; ++j; }
        }
      }
      if (nq < 32) avail &= (1u << nq) - 1u;
    }
    unsigned long long mine = 0;
    for (uint32_t a2 = avail; a2; a2 &= a2 - 1) mine += wt[ax_slot(qa + __ffs(a2) - 1)];
    unsigned long long incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) gsum[g][gw] = incl;
    named_barrier(bar, kAxGroup);
    unsigned long long before = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kAxGroup / 32; ++q) {
      const unsigned long long v = gsum[g][q];
      if (q < gw) before += v;
      tot += v;
    }
    const unsigned long long excl = before + incl - mine;
    if (t == 0) {
      const uint4 u4 = gf::philox_call(seed, gf::kStreamAxial, (uint32_t)(inst_base + inst),
                                       round, s, (uint64_t)(i >> 2));
      const uint32_t u = gf::lane_of(u4, (uint32_t)(i & 3));
      unsigned long long r;
      if (tot > 0) {
        const unsigned long long lo = (unsigned long long)u * tot;
        const unsigned long long hi = __umul64hi((unsigned long long)u, tot);
        r = (hi << 32) | (lo >> 32);
      } else {
        const int free = I - i;
        r = ((unsigned long long)u * (unsigned long long)(free * free)) >> 32;
      }
      sh_r[g] = r;
      sh_pick[g] = -1;
      if (tot == 0) {
        // r-th allowed pair in row-major order: (a-th free j, b-th free k)
        const int free = I - i;
        const int a = (int)(r / free), bb = (int)(r % free);
        int jj = -1, kk = -1;
        for (int q = 0, c = 0; q < I; ++q)
          if (!((usedJ >> q) & 1ull)) { if (c == a) { jj = q; break; } ++c; }
        for (int q = 0, c = 0; q < I; ++q)
          if (!((usedK >> q) & 1ull)) { if (c == bb) { kk = q; break; } ++c; }
        sh_pick[g] = jj * I + kk;
      }
    }
    named_barrier(bar, kAxGroup);
    const unsigned long long r = sh_r[g];
    if (tot > 0 && mine > 0 && excl <= r && r < excl + mine) {
      unsigned long long acc = excl;
      for (uint32_t a2 = avail; a2; a2 &= a2 - 1) {
        const int m = __ffs(a2) - 1;
        const uint32_t w = wt[ax_slot(qa + m)];
        acc += w;
        if (w && acc > r) { sh_pick[g] = qa + m; break; }
      }
    }
    named_barrier(bar, kAxGroup);
    const int pick = sh_pick[g];
    if (pick < 0 || pick >= P) continue;              // unreachable: r < tot
    const int jj = pick / I, kk = pick - jj * I;
    usedJ |= 1ull << jj;
    usedK |= 1ull << kk;
    if (t == 0) {
      const int64_t var = v0 + (int64_t)i * P + pick;
      atomicOr(&X[var * kw + (sidx >> 5)], 1u << (sidx & 31));
    }
  }
}

// Closure repair (Section 2.4.3): rep_var[q] |= OR of its list, per word.
// One block per repaired variable; thread tid owns word tid % kw.  A list
// in constant steps (rstep[q] > 0) is generated from its first entry.
__global__ void k_closure(const int64_t* __restrict__ rv, const int64_t* __restrict__ rp,
                          const int64_t* __restrict__ ri, const int64_t* __restrict__ rstep,
                          int64_t nrep, int kws, int kw, uint32_t* __restrict__ X) {
  const int64_t q = blockIdx.x;
  if (q >= nrep) return;
  extern __shared__ uint32_t red[];
  const int per = blockDim.x / kw;           // threads per word
  const int w = threadIdx.x % kw;
  const int slot = threadIdx.x / kw;
  uint32_t acc = 0;
  if (slot < per) {
    const int64_t a = rp[q], e = rp[q + 1], d = rstep[q];
    if (d > 0) {
      const int64_t v0 = ri[a];
      for (int64_t t = slot; t < e - a; t += per) acc |= X[(v0 + t * d) * kws + w];
    } else {
      for (int64_t t = a + slot; t < e; t += per) acc |= X[ri[t] * kws + w];
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < kw) {
    uint32_t v = X[rv[q] * kws + threadIdx.x];
    for (int s = 0; s < per; ++s) v |= red[s * kw + threadIdx.x];
    X[rv[q] * kws + threadIdx.x] = v;
  }
}

// Bernoulli thresholds floor(p 2^24) of a dense instance's variables (0 past
// n), computed once per chunk instead of once per draw.
__global__ void k_thresholds(const float* __restrict__ p, int64_t v0, int64_t n, int64_t ld,
                             uint32_t* __restrict__ thr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) thr[i] = i < n ? gf::prob_threshold(p[v0 + i]) : 0u;
}

// Bernoulli draws of a dense-Q instance written sample-major as FP8 / bf16
// 0/1 (the tensor-core operand) and as bit words Xb[s * ld/32 + w] (bit t =
// variable 32 w + t, read by the scorer's epilogue).  A thread takes 4
// variables and kBernCands consecutive samples (round keys and thresholds
// loaded once); 8 consecutive lanes assemble one word.
constexpr int kBernCands = 8;

__global__ void __launch_bounds__(256)
k_bern_bf16(const uint32_t* __restrict__ thr, int64_t n, int64_t ld,
            int s0, int len, uint64_t seed, int inst, const GfDState* __restrict__ st,
            void* __restrict__ Xs, uint32_t* __restrict__ Xb, int f8) {
  const int64_t n4 = ld / 4;
  const int64_t g4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g4 >= n4) return;
  const int64_t i0 = g4 * 4;
  const bool live = i0 < n;
  // thresholds floor(p 2^24) of the round (0 for padding entries)
  const uint4 t = live ? __ldg(reinterpret_cast<const uint4*>(thr) + g4) : make_uint4(0, 0, 0, 0);
  const gf::PhiloxKeys K = gf::philox_keys(seed);
  const uint32_t round = st->round_id;
  const uint32_t c3 = ((uint32_t)inst & 0x0FFFFFFFu) | (gf::kStreamBern << 28);
  // ld/4 is a multiple of 16, so the 8 lanes holding one 32-variable word
  // are always active together and belong to the same candidate
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m8 = 0xFFu << (lane & ~7u);
  const int c0 = blockIdx.y * kBernCands;
#pragma unroll 2
  for (int c = 0; c < kBernCands; ++c) {
    const int sidx = c0 + c;
    if (sidx >= len) break;
    uint32_t b[4] = {0, 0, 0, 0};
    if (live) {
      const uint4 u = gf::philox_k(make_uint4((uint32_t)g4, (uint32_t)(s0 + sidx), round, c3), K);
      b[0] = (u.x >> 8) < t.x;
      b[1] = (u.y >> 8) < t.y;
      b[2] = (u.z >> 8) < t.z;
      b[3] = (u.w >> 8) < t.w;
    }
    if (f8) {
      // FP8 E4M3 one = 0x38
      const uint32_t out = (b[0] ? 0x38u : 0u) | ((b[1] ? 0x38u : 0u) << 8) |
                           ((b[2] ? 0x38u : 0u) << 16) | ((b[3] ? 0x38u : 0u) << 24);
      reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(Xs) + (int64_t)sidx * ld)[g4] = out;
    } else {
      // bf16 one = 0x3F80
      uint2 out;
      out.x = (b[0] ? 0x3F80u : 0u) | ((b[1] ? 0x3F80u : 0u) << 16);
      out.y = (b[2] ? 0x3F80u : 0u) | ((b[3] ? 0x3F80u : 0u) << 16);
      reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(Xs) + (int64_t)sidx * ld)[g4] = out;
    }
    uint32_t v = (b[0] | (b[1] << 1) | (b[2] << 2) | (b[3] << 3)) << (4 * (lane & 7u));
    v |= __shfl_xor_sync(m8, v, 1, 8);
    v |= __shfl_xor_sync(m8, v, 2, 8);
    v |= __shfl_xor_sync(m8, v, 4, 8);
    if ((lane & 7u) == 0) Xb[(int64_t)sidx * (ld / 32) + g4 / 8] = v;
  }
}

}  // namespace

// Bit words of bf16 / FP8 candidate rows (for writers other than the sampler).
__global__ void k_dense_bits(const void* __restrict__ Xs, int len, int64_t ld,
                             uint32_t* __restrict__ Xb, int f8) {
  const int64_t nw = ld / 32;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nw * len) return;
  const int s = (int)(gid / nw);
  const int64_t w = gid % nw;
  uint32_t m = 0;
  if (f8) {
    const uint8_t* row = reinterpret_cast<const uint8_t*>(Xs) + (int64_t)s * ld;
    for (int t = 0; t < 32; ++t) m |= (uint32_t)(row[32 * w + t] != 0) << t;
  } else {
    const uint16_t* row = reinterpret_cast<const uint16_t*>(Xs) + (int64_t)s * ld;
    for (int t = 0; t < 32; ++t) m |= (uint32_t)(row[32 * w + t] != 0) << t;
  }
  Xb[gid] = m;
}

namespace {

}  // namespace

// Sample `len` candidates (samples s0 .. s0+len-1 of the current round) of
// every instance from proposal p.  for_dense: dense-Q instances get their
// bf16 sample-major operand instead of bits.

// The list of 4-variable groups that Bernoulli draws cover (those holding a
// variable no group sampler draws); built once after the groups change.
// Synchronises when it builds, so callers that capture a graph build it first.
cudaError_t gf_ensure_bit_list(GfCtx* h) {
  if (h->n_bit_g4 >= 0) return cudaSuccess;
  cudaError_t e;
  const int64_t N4 = h->N / 4;
  if ((e = cudaMemsetAsync(h->bit_count, 0, sizeof(int32_t), h->stream))) return e;
  k_bit_list<<<(unsigned)((N4 + 255) / 256), 256, 0, h->stream>>>(h->var_grouped, N4,
                                                                   h->bit_g4, h->bit_count);
  int32_t cnt = 0;
  if ((e = cudaMemcpyAsync(&cnt, h->bit_count, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return e;
  h->n_bit_g4 = cnt;
  return cudaSuccess;
}

cudaError_t gf_launch_sample(GfCtx* h, const float* p, int s0, int len, bool for_dense,
                             bool* pick_obj) {
  if (pick_obj) *pick_obj = false;
  const gfors_params& P = h->prm;
  cudaError_t e;
  const int kw = (len + 31) / 32;
  // group-sampled instances start from zeroed words (axial picks are OR-ed
  // in; one-hot picks write only the chosen members' words); the Bernoulli
  // sampler then overwrites the words of the other variables
  for (int b = 0; b < h->ninst; ++b) {
    const GfInstHost& I = h->ih[b];
    if (I.group_mode == 1 || I.group_mode == 2 || I.group_mode == 3) {
      e = cudaMemsetAsync(h->X + I.var_off * h->kw, 0, sizeof(uint32_t) * I.npad * h->kw,
                          h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  // Bernoulli bits only for the 4-variable groups that hold a variable no
  // group sampler draws (the list is rebuilt after the groups change)
  if ((e = gf_ensure_bit_list(h))) return e;
  if (h->n_bit_g4 > 0) {
    const int64_t N4 = h->n_bit_g4;
    const int64_t threads = N4 * kw;
    k_bern_bits<<<(unsigned)((threads + 255) / 256), 256, 0, h->stream>>>(
        p, h->var_inst, h->var_off_d, h->var_grouped, h->var_live, h->bit_g4, N4, h->kw, kw,
        s0, len, P.seed, P.inst_base, h->dstate, h->X);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (h->ngroups_tot > 0) {
    // within one sampling call the weights of a p already formed are reused
    unsigned long long* cw = h->grp_cw;
    bool fresh = true;
    if (h->cw_cache) {
      int slot = (h->cw_src[0] == p) ? 0 : (h->cw_src[1] == p) ? 1 : -1;
      if (slot >= 0) {
        fresh = false;
      } else {
        slot = (h->cw_src[0] == nullptr) ? 0 : (h->cw_src[1] == nullptr) ? 1 : 0;
        h->cw_src[slot] = p;
      }
      cw = slot ? h->grp_cw2 : h->grp_cw;
    }
    if (fresh) {
      k_group_cw<<<(unsigned)((h->ngroups_tot * 32 + 255) / 256), 256, 0, h->stream>>>(
          h->grp_ptr, h->grp_idx, h->grp_step, h->ngroups_tot, p, cw);
      h->launches++;
    }
    // the picks' costs, when no later repair changes a grouped variable
    const bool po = pick_obj && h->pick_obj_valid && h->pick_obj_rv == h->repair_version &&
                    h->pick_obj_gv == h->grp_version;
    if (po) {
      if ((e = cudaMemsetAsync(h->objp, 0, sizeof(long long) * h->ninst * h->chunk, h->stream)))
        return e;
      *pick_obj = true;
    }
    const int64_t gblocks = (h->ngroups_tot + kPickWarps - 1) / kPickWarps;
    k_group_pick<<<(unsigned)(gblocks * kw), 32 * kPickWarps, 0,
                   h->stream>>>(h->grp_ptr, h->grp_idx, h->grp_step, h->grp_inst, h->grp_local,
                                h->ngroups_tot, cw, h->kw, kw, s0, len, P.seed, P.inst_base,
                                h->dstate, h->X, po ? (h->clin ? h->clin : h->cint) : nullptr,
                                reinterpret_cast<unsigned long long*>(h->objp), h->chunk);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int b = 0; b < h->ninst; ++b) {
    const GfInstHost& I = h->ih[b];
    if (I.group_mode == 3) {
      extern cudaError_t gf_launch_assign_custom(GfCtx * h, int b, const float* p, int s0,
                                                 int len);
      if ((e = gf_launch_assign_custom(h, b, p, s0, len)) != cudaSuccess) return e;
      continue;
    }
    if (I.group_mode != 2) continue;
    if (I.axial_I <= 64 && I.axial_I * I.axial_I <= kAxMaxP)
      k_axial_grp<<<(len + kAxCands - 1) / kAxCands, kAxGroup * kAxCands, 0, h->stream>>>(
          p, I.var_off, I.axial_I, b, s0, len, h->kw, P.seed, P.inst_base, h->dstate, h->X);
    else
      k_axial<<<len, kAxThreads, 0, h->stream>>>(p, I.var_off, I.axial_I, b, s0, len, h->kw,
                                                 P.seed, P.inst_base, h->dstate, h->X);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (h->nrg > 0) {
    const int64_t warps = h->nrg * kw;
    k_repair_min<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->rg_ptr, h->rg_idx, h->nrg, h->kw, kw, h->X);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (h->nrr > 0) {
    const int64_t wc = h->nrr * kw, wd = h->nrr_seg * kw;
    k_rr_count<<<(unsigned)((wc * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->rr_ptr, h->rr_idx, h->nrr, h->kw, kw, h->chunk, h->X, h->rr_cnt);
    k_rr_delete<<<(unsigned)((wd * 32 + 255) / 256), 256, 0, h->stream>>>(
        h->rr_optr, h->rr_order, h->rr_vptr, h->rr_vrow, h->nrr_seg, h->kw, kw, h->chunk, h->X,
        h->rr_cnt);
    h->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (h->nrep_tot > 0) {
    int per = std::max(1, 256 / kw);
    int threads = per * kw;
    k_closure<<<(unsigned)h->nrep_tot, threads, sizeof(uint32_t) * threads, h->stream>>>(
        h->rep_var, h->rep_ptr, h->rep_idx, h->rep_step, h->nrep_tot, h->kw, kw, h->X);
    h->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (for_dense) {
    for (const GfDenseQ& dq : h->dense) {
      k_thresholds<<<(unsigned)((dq.ld + 255) / 256), 256, 0, h->stream>>>(
          p, h->ih[dq.inst].var_off, dq.n, dq.ld, dq.thr);
      h->launches++;
      // kBernCands candidates per block row, at most 32768 block rows per launch
      for (int a = 0; a < len; a += 32768 * kBernCands) {
        const int cnt = std::min(32768 * kBernCands, len - a);
        const dim3 grid((unsigned)((dq.ld / 4 + 255) / 256),
                        (unsigned)((cnt + kBernCands - 1) / kBernCands));
        k_bern_bf16<<<grid, 256, 0, h->stream>>>(
            dq.thr, dq.n, dq.ld, s0 + a, cnt, P.seed, P.inst_base + dq.inst,
            h->dstate,
            dq.f8 ? (void*)(reinterpret_cast<uint8_t*>(dq.Xs) + (int64_t)a * dq.ld)
                  : (void*)(dq.Xs + (int64_t)a * dq.ld),
            dq.Xb + (int64_t)a * (dq.ld / 32), (int)dq.f8);
        h->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

// The objective of one-hot groups' variables can come from the picks when no
// repair that runs after them (least-cost repair groups, reverse delete over
// repair rows, the closure) changes a grouped variable, and no grouped
// variable belongs to a dense tensor-core instance.  Then evaluation covers
// the 32-variable slabs with an ungrouped variable (grouped lanes masked).
cudaError_t gf_ensure_pick_obj(GfCtx* h) {
  if (h->pick_obj_rv == h->repair_version && h->pick_obj_gv == h->grp_version)
    return cudaSuccess;
  h->pick_obj_valid = false;
  h->pick_obj_rv = h->repair_version;
  h->pick_obj_gv = h->grp_version;
  if (h->ngroups_tot <= 0 || !h->all_integral) return cudaSuccess;
  const int64_t N = h->N;
  std::vector<uint32_t> gm((size_t)(N / 32), 0u);
  for (int64_t v : h->h_grp_idx) gm[(size_t)(v >> 5)] |= 1u << (v & 31);
  auto grouped = [&](int64_t v) { return (gm[(size_t)(v >> 5)] >> (v & 31)) & 1u; };
  for (int64_t v : h->h_rep_var)
    if (grouped(v)) return cudaSuccess;
  for (int64_t v : h->h_rg_idx)
    if (grouped(v)) return cudaSuccess;
  for (int64_t v : h->h_rr_idx)
    if (grouped(v)) return cudaSuccess;
  for (int b = 0; b < h->ninst; ++b) {
    const GfInstHost& I = h->ih[b];
    if (I.qkind != 1) continue;
    for (int64_t v = I.var_off; v < I.var_off + I.npad; v += 32)
      if (gm[(size_t)(v >> 5)]) return cudaSuccess;
  }
  // objective chunks (<= 256 variables: these slabs are few, and denser
  // than grouped ones) over slabs with an ungrouped lane
  std::vector<GfObjChunk> oc;
  for (int b = 0; b < h->ninst; ++b) {
    const GfInstHost& I = h->ih[b];
    if (I.qkind == 1) continue;
    int64_t start = -1;
    const int64_t aend = (I.n + 31) / 32 * 32;   // one step past the last slab
    for (int64_t a = 0; a <= aend; a += 32) {
      const bool open = a < I.n && gm[(size_t)((I.var_off + a) >> 5)] != 0xFFFFFFFFu;
      if (open && start < 0) start = a;
      const bool close = start >= 0 && (!open || a - start >= 256);
      if (close) {
        oc.push_back(GfObjChunk{b, (int32_t)(I.var_off + start),
                                (int32_t)(I.var_off + std::min<int64_t>(a, I.n)), 0});
        start = open ? a : -1;
      }
    }
  }
  h->ochunks_ng = gf_alloc_t<GfObjChunk>(h, std::max<size_t>(1, oc.size()));
  h->slab_gmask = gf_alloc_t<uint32_t>(h, std::max<size_t>(1, gm.size()));
  if (!h->ochunks_ng || !h->slab_gmask) return cudaErrorMemoryAllocation;
  cudaError_t e;
  if (!oc.empty() &&
      (e = cudaMemcpy(h->ochunks_ng, oc.data(), sizeof(GfObjChunk) * oc.size(),
                      cudaMemcpyHostToDevice)))
    return e;
  if (!gm.empty() && (e = cudaMemcpy(h->slab_gmask, gm.data(), sizeof(uint32_t) * gm.size(),
                                     cudaMemcpyHostToDevice)))
    return e;
  h->nochunks_ng = (int64_t)oc.size();
  h->pick_obj_valid = true;
  return cudaSuccess;
}
