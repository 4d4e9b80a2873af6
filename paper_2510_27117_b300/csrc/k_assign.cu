// k_assign.cu -- Algorithm 4 (customized sampling for the 3D assignment,
// Section 2.4.2) on the device.  Readings (the paper gives the outline):
//   (a) the gamma*I largest entries of p, ordered by p descending, then by
//       variable index ascending;
//   (b) greedy partial assignment: an entry (i,j,k) is accepted when i, j
//       and k are all unused;
//   (c) every candidate completes it: the free j's and the free k's (each
//       ascending) are shuffled by Fisher-Yates (q = F-1 down to 1,
//       r = floor(u (q+1) / 2^32), u = Philox lane of stream 6, index t of
//       the t-th draw, j's first) and handed in turn to the free i's;
//   (d) then up to L steps, each applying the single best strictly improving
//       pairwise interchange between the triples of i = a < i = b (type 0:
//       exchange j, type 1: exchange k; exact integer costs; ties to the
//       smallest (a, b, type)); a step without improvement ends the search.
// Kernels: per-slab top-K by a bitonic sort of 64-bit keys (p bits, then the
// complemented index) in shared memory; one block merges the slab lists
// (the global top K lie in the union of the slabs' top K) and runs (b);
// one block per candidate runs (c) and (d).
#include "internal.cuh"

namespace {

// Descending bitonic sort of N (power of two) keys in shared memory.
GF_DEV void bitonic_desc(unsigned long long* key, int N) {
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
        const int ixj = idx ^ j;
        if (ixj > idx) {
          const unsigned long long a = key[idx], b = key[ixj];
          const bool desc = (idx & k) == 0;
          if (desc ? (a < b) : (a > b)) { key[idx] = b; key[ixj] = a; }
        }
      }
      __syncthreads();
    }
}

GF_DEV unsigned long long pkey(float p, uint32_t v) {
  // p in [0, 1]: its IEEE bits order like its value (-0 and negatives as 0);
  // ties by index ascending
  return ((unsigned long long)__float_as_uint(p > 0.0f ? p : 0.0f) << 32) |
         (unsigned long long)(0xFFFFFFFFu - v);
}

__global__ void __launch_bounds__(1024)
k_a4_slabtop(const float* __restrict__ p, int64_t v0, int I, int K,
             unsigned long long* __restrict__ out) {
  extern __shared__ unsigned long long key[];
  const int i = blockIdx.x;
  const int P = I * I;
  int N = 1;
  while (N < P) N <<= 1;
  for (int q = threadIdx.x; q < N; q += blockDim.x)
    key[q] = q < P ? pkey(p[v0 + (int64_t)i * P + q], (uint32_t)(i * P + q)) : 0ull;
  __syncthreads();
  bitonic_desc(key, N);
  for (int q = threadIdx.x; q < K; q += blockDim.x) out[(int64_t)i * K + q] = key[q];
}

__global__ void __launch_bounds__(1024)
k_a4_partial(const unsigned long long* __restrict__ cand, int I, int K,
             int32_t* __restrict__ J0, int32_t* __restrict__ K0) {
  extern __shared__ unsigned long long key[];
  const int total = I * K;
  int N = 1;
  while (N < total) N <<= 1;
  for (int q = threadIdx.x; q < N; q += blockDim.x) key[q] = q < total ? cand[q] : 0ull;
  __syncthreads();
  bitonic_desc(key, N);
  if (threadIdx.x == 0) {
    unsigned long long uj = 0ull, uk = 0ull;
    for (int a = 0; a < I; ++a) { J0[a] = -1; K0[a] = -1; }
    for (int e = 0; e < K; ++e) {
      const uint32_t v = 0xFFFFFFFFu - (uint32_t)(key[e] & 0xFFFFFFFFull);
      const int i = (int)(v / (uint32_t)(I * I)), j = (int)((v / I) % I), k = (int)(v % I);
      if (J0[i] < 0 && !((uj >> j) & 1ull) && !((uk >> k) & 1ull)) {
        J0[i] = j;
        K0[i] = k;
        uj |= 1ull << j;
        uk |= 1ull << k;
      }
    }
  }
}

constexpr int kA4Threads = 256;
constexpr int kA4MaxPairs = 64 * 63 / 2;

// Index of the pair (a, b), a < b, in lexicographic order.
GF_DEV int pair_index(int a, int b, int I) { return a * (2 * I - a - 1) / 2 + (b - a - 1); }

// One block per candidate.  The interchange search keeps the gain of every
// (pair, type) in shared memory: an applied interchange at (a, b) changes
// only the gains of pairs that contain a or b, so a step rescans the table
// and recomputes those 4 (I - 1) entries instead of all 2 I (I - 1) / 2.
// Gains are exact integers, so the chosen interchange is the same as with a
// full recomputation.
// G: the gain type.  int when every gain fits (4 max|c| < 2^31; gains are
// differences of two pairs of costs), which halves the gain table and lets
// seven candidates' blocks share an SM, so a round of 1,024 runs in one wave.
template <typename G>
__global__ void __launch_bounds__(kA4Threads, sizeof(G) == 4 ? 7 : 1)
k_a4_sample(const int32_t* __restrict__ J0, const int32_t* __restrict__ K0,
            const long long* __restrict__ cost, int64_t v0, int I, int L, int s0, int len,
            uint64_t seed, int inst, const GfDState* __restrict__ st, int kw,
            uint32_t* __restrict__ X) {
  __shared__ int32_t J[64], Kk[64], fi[64], fj[64], fk[64];
  __shared__ uint32_t ufy[128];                  // Fisher-Yates draws
  __shared__ long long cold[64];                 // cost of the triple at each i
  __shared__ G gain[2 * kA4MaxPairs];            // [pair][type]
  __shared__ uint8_t pa[kA4MaxPairs], pb[kA4MaxPairs];
  __shared__ G wbest[kA4Threads / 32];
  __shared__ int wcode[kA4Threads / 32];
  const int sidx = blockIdx.x;
  if (sidx >= len) return;
  const int tid = threadIdx.x;
  const uint32_t s = (uint32_t)(s0 + sidx);
  const uint32_t round = st->round_id;
  const long long* c = cost + v0;
  auto C3 = [&](int i, int j, int k) { return __ldg(c + ((int64_t)i * I + j) * I + k); };
  const int np = I * (I - 1) / 2;
  // draws t = 0 .. 2I-3 cover the j shuffle (t < F-1) and the k shuffle
  for (int t = tid; t < 2 * I - 2; t += kA4Threads) {
    const uint4 u4 = gf::philox_call(seed, 6u, (uint32_t)inst, round, s, (uint64_t)t >> 2);
    ufy[t] = gf::lane_of(u4, (uint32_t)(t & 3));
  }
  for (int a = tid; a < I; a += kA4Threads)
    for (int b = a + 1, q = pair_index(a, a + 1, I); b < I; ++b, ++q) {
      pa[q] = (uint8_t)a;
      pb[q] = (uint8_t)b;
    }
  __syncthreads();
  if (tid == 0) {
    // (c) completion of the partial assignment
    int F = 0, Fj = 0, Fk = 0;
    unsigned long long uj = 0ull, uk = 0ull;
    for (int a = 0; a < I; ++a) {
      J[a] = J0[a];
      Kk[a] = K0[a];
      if (J0[a] < 0) fi[F++] = a;
      else { uj |= 1ull << J0[a]; uk |= 1ull << K0[a]; }
    }
    for (int a = 0; a < I; ++a) {
      if (!((uj >> a) & 1ull)) fj[Fj++] = a;
      if (!((uk >> a) & 1ull)) fk[Fk++] = a;
    }
    int t = 0;
    for (int q = F - 1; q >= 1; --q, ++t) {
      const int r = (int)(((unsigned long long)ufy[t] * (unsigned long long)(q + 1)) >> 32);
      const int tmp = fj[q]; fj[q] = fj[r]; fj[r] = tmp;
    }
    for (int q = F - 1; q >= 1; --q, ++t) {
      const int r = (int)(((unsigned long long)ufy[t] * (unsigned long long)(q + 1)) >> 32);
      const int tmp = fk[q]; fk[q] = fk[r]; fk[r] = tmp;
    }
    for (int e = 0; e < F; ++e) { J[fi[e]] = fj[e]; Kk[fi[e]] = fk[e]; }
  }
  __syncthreads();
  for (int a = tid; a < I; a += kA4Threads) cold[a] = C3(a, J[a], Kk[a]);
  __syncthreads();
  auto pair_gains = [&](int q, int a, int b) {
    const long long old = cold[a] + cold[b];
    gain[2 * q] = (G)(C3(a, J[b], Kk[a]) + C3(b, J[a], Kk[b]) - old);       // exchange j
    gain[2 * q + 1] = (G)(C3(a, J[a], Kk[b]) + C3(b, J[b], Kk[a]) - old);   // exchange k
  };
  for (int q = tid; q < np; q += kA4Threads) pair_gains(q, pa[q], pb[q]);
  __syncthreads();
  // (d) best-improvement pairwise interchanges.  Two barriers per step:
  // after the scan (every thread then reduces the warp winners itself and
  // reads the chosen triples), and after the gain updates (then thread 0
  // stores the new triples, which nobody reads before the next scan's
  // barrier).
  const int warp = tid >> 5, lane = tid & 31;
  for (int step = 0; step < L; ++step) {
    G best = 0;                                  // only strict improvements count
    int code = 0x7FFFFFFF;
    for (int e = tid; e < 2 * np; e += kA4Threads) {
      const G g = gain[e];
      if (g < best) { best = g; code = e; }      // ascending e: ties keep the first
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const G ob = __shfl_down_sync(0xFFFFFFFFu, best, off);
      const int oc = __shfl_down_sync(0xFFFFFFFFu, code, off);
      if (ob < best || (ob == best && oc < code)) { best = ob; code = oc; }
    }
    if (lane == 0) { wbest[warp] = best; wcode[warp] = code; }
    __syncthreads();
    G bb = 0;
    int bc = 0x7FFFFFFF;
#pragma unroll
    for (int w = 0; w < kA4Threads / 32; ++w)
      if (wbest[w] < bb || (wbest[w] == bb && wcode[w] < bc)) { bb = wbest[w]; bc = wcode[w]; }
    if (bb >= 0) break;                          // no strict improvement (uniform)
    const int q = bc >> 1, a = pa[q], b = pb[q];
    int Ja = J[a], Jb = J[b], Ka = Kk[a], Kb = Kk[b];
    if ((bc & 1) == 0) { const int tmp = Ja; Ja = Jb; Jb = tmp; }
    else { const int tmp = Ka; Ka = Kb; Kb = tmp; }
    // gains of the pairs (a, x) for every x != a, then (b, x), x not in {a, b}
    for (int t = tid; t < 2 * I; t += kA4Threads) {
      const bool first = t < I;
      const int x = first ? t : t - I;
      if (first ? x == a : (x == a || x == b)) continue;
      const int u = first ? a : b;
      const int Ju = first ? Ja : Jb, Ku = first ? Ka : Kb;
      const long long cu = C3(u, Ju, Ku);
      int Jx, Kx;
      long long cx;
      if (x == b) { Jx = Jb; Kx = Kb; cx = C3(b, Jb, Kb); }
      else { Jx = J[x]; Kx = Kk[x]; cx = cold[x]; }
      const int lo = u < x ? u : x, hi = u < x ? x : u;
      const int Jl = u < x ? Ju : Jx, Kl = u < x ? Ku : Kx;
      const int Jh = u < x ? Jx : Ju, Kh = u < x ? Kx : Ku;
      const long long old = cu + cx;
      const int pq = pair_index(lo, hi, I);
      gain[2 * pq] = (G)(C3(lo, Jh, Kl) + C3(hi, Jl, Kh) - old);       // exchange j
      gain[2 * pq + 1] = (G)(C3(lo, Jl, Kh) + C3(hi, Jh, Kl) - old);   // exchange k
    }
    __syncthreads();
    if (tid == 0) {
      J[a] = Ja; J[b] = Jb; Kk[a] = Ka; Kk[b] = Kb;
      cold[a] = C3(a, Ja, Ka);
      cold[b] = C3(b, Jb, Kb);
    }
  }
  __syncthreads();
  for (int a = tid; a < I; a += kA4Threads) {
    const int64_t var = v0 + ((int64_t)a * I + J[a]) * I + Kk[a];
    atomicOr(&X[var * kw + (sidx >> 5)], 1u << (sidx & 31));
  }
}

}  // namespace

// Candidates [s0, s0+len) of instance b drawn by Algorithm 4 from p.
cudaError_t gf_launch_assign_custom(GfCtx* h, int b, const float* p, int s0, int len) {
  const GfInstHost& I = h->ih[b];
  const int n1 = I.axial_I, K = I.a4_gamma * n1, P = n1 * n1;
  int N1 = 1;
  while (N1 < P) N1 <<= 1;
  int N2 = 1;
  while (N2 < n1 * K) N2 <<= 1;
  cudaError_t e;
  if (K > 0) {
    k_a4_slabtop<<<n1, 1024, sizeof(unsigned long long) * N1, h->stream>>>(p, I.var_off, n1, K,
                                                                            h->a4_cand);
    if ((e = cudaFuncSetAttribute(k_a4_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(unsigned long long) * N2))))
      return e;
    k_a4_partial<<<1, 1024, sizeof(unsigned long long) * N2, h->stream>>>(h->a4_cand, n1, K,
                                                                          h->a4_J0, h->a4_K0);
    h->launches += 2;
  } else {
    cudaMemsetAsync(h->a4_J0, 0xFF, sizeof(int32_t) * n1, h->stream);
    cudaMemsetAsync(h->a4_K0, 0xFF, sizeof(int32_t) * n1, h->stream);
  }
  if (I.a4_gain32)
    k_a4_sample<int><<<len, kA4Threads, 0, h->stream>>>(
        h->a4_J0, h->a4_K0, h->cint, I.var_off, n1, I.a4_L, s0, len, h->prm.seed,
        h->prm.inst_base + b, h->dstate, h->kw, h->X);
  else
    k_a4_sample<long long><<<len, kA4Threads, 0, h->stream>>>(
        h->a4_J0, h->a4_K0, h->cint, I.var_off, n1, I.a4_L, s0, len, h->prm.seed,
        h->prm.inst_base + b, h->dstate, h->kw, h->X);
  h->launches++;
  return cudaGetLastError();
}
