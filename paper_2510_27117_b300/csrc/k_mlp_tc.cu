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
// One persistent CTA per SM, tiles of 128 variables, software-pipelined;
// 25 warps in three roles that meet on mbarriers (every wait bounded by a
// time limit):
//   warps 0-15   layer-1 epilogue: warp w serves TMEM lanes 32 (w mod 4) ..
//                + 31 (one variable per lane) and, per K half h of layer 2,
//                hidden units 64 h + 16 (w / 4) .. + 15: D1 -> +b1, relu ->
//                bf16 pieces -> TMEM slot h (tcgen05.st)
//   warps 16-23  layer-2 epilogue: warp 16 + 4 s + q serves lanes 32 q .. +
//                31 and units 64 s .. + 63: D2 -> +b2, relu, w3 dot; the two
//                halves of z meet in shared memory -> z, p (s = 0 warps);
//                features of the tile two ahead -> pieces -> A1 (s = 1 warps)
//   warp 24      MMA issuer (lane 0): layer 1 = 3 MMAs (M=N=128, K=16, one
//                per feature piece against W1, both from shared memory),
//                layer 2 = 2 x 12 MMAs (per K half: 3 pieces x 4 K-steps of
//                16) with A = the h1 pieces in TMEM and B = W2 in shared
//                memory, issued in the order L1(t + 1), L2(t, half 0),
//                L2(t, half 1)
// The h1 pieces stay in TMEM, so shared memory carries only W1, W2 and the
// features: with both operands in shared memory a 128 x 128 x 16 MMA reads
// as many bytes per cycle as shared memory delivers, and the 96 KB of
// pieces per tile would have to be written there as well.  TMEM holds D1,
// D2 and two K-half slots of pieces (448 of 512 columns).  On a wait that
// gives up the kernel records an error (or writes NaN outputs when no error
// word is given), waits for its MMAs and frees TMEM.
#include "internal.cuh"
#include "tc_util.cuh"

namespace {

using namespace gf_tc;

constexpr int kF = 8, kH = 128, TM = 128;
constexpr int kE1Warps = 16, kE2Warps = 8;
constexpr int kE1Units = 64 / (kE1Warps / 4);   // units per layer-1 warp and K half
constexpr int kMmaWarp = kE1Warps + kE2Warps;
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr uint32_t kIdesc = idesc_bf16(128, 128);
// TMEM columns: D1, D2 (FP32, 128 each) and two K-half slots of h1 pieces
// (bf16 pairs, 3 pieces x 32 columns each), the A operand of layer 2
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t kD1 = 0, kD2 = 128, kSlot0 = 256, kSlotCols = 96;
constexpr int oW1 = 0, oB1 = kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH;
// shared-memory layout (offsets from a 1024-byte aligned base)
constexpr int PANEL = 128 * 128;             // 128 rows x 128 bytes (64 bf16 per row)
constexpr int B1_OFF = 0;                    // W1 at K = 0 (K 8-63 zero)
constexpr int B2_OFF = B1_OFF + PANEL;       // W2: 2 panels (K 0-63, 64-127)
constexpr int A1_OFF = B2_OFF + 2 * PANEL;   // 2 feature tiles: pieces at K = 0, 16, 32
constexpr int VEC_OFF = A1_OFF + 2 * PANEL;  // b1, b2, w3 (FP32), b3
constexpr int ZP_OFF = VEC_OFF + 3 * kH * 4 + 16;   // z halves [tile parity][2][128]
constexpr int BAR_OFF = ZP_OFF + 2 * 2 * 128 * 4;
constexpr int kBars = 16;
constexpr int SMEM_BYTES = BAR_OFF + 8 * kBars + 1024;
// mbarriers
constexpr int BA1_FULL = 0;    // [2] features staged in A1[b] (staging warps arrive)
constexpr int BA1_FREE = 2;    // [2] A1[b] read by layer 1 (commit)
constexpr int BD1_FULL = 4;    // layer 1 done: D1 written (commit)
constexpr int BD1_FREE = 5;    // D1 read (layer-1 epilogue warps arrive)
constexpr int BS_FULL = 6;     // [2] slot h written (layer-1 epilogue warps arrive)
constexpr int BS_FREE = 8;     // [2] slot h read by layer 2 (commit)
constexpr int BD2_FULL = 10;   // layer 2 done: D2 written (commit)
constexpr int BD2_FREE = 11;   // D2 read (layer-2 epilogue warps arrive)
constexpr int BDRAIN = 12;     // last commit, waited before TMEM is freed

// Byte offset of element (row r, k) of a K-major 128-byte-swizzled panel
// (k < 64): 8-row atoms of 1024 bytes, 16-byte chunk index XOR (r mod 8).
GF_DEV uint32_t sw_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
}

GF_DEV uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Packed FP32 pairs (Blackwell's two-lane FP32 add/subtract, each lane
// rounded to nearest like __fadd_rn / __fsub_rn).
GF_DEV uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
GF_DEV void f2_unpack(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
GF_DEV uint64_t f2_add(uint64_t x, uint64_t y) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
GF_DEV uint64_t f2_sub(uint64_t x, uint64_t y) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
// the two bf16 of a packed pair as FP32 (low half = first value)
GF_DEV uint64_t bf16x2_to_f2(uint32_t v) {
  return f2_pack(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

// Exact split of two FP32 values into three bf16 pieces each (8 + 8 + 8
// significand bits), packed in pairs: a = hi.lo16 + mid.lo16 + lo.lo16 and
// likewise for b in the upper halves.  Each remainder a - bf16(a) is exact.
GF_DEV void split_pair(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  hi = pack_bf16x2(a, b);
  const uint64_t r1 = f2_sub(f2_pack(a, b), bf16x2_to_f2(hi));
  float a1, b1;
  f2_unpack(r1, a1, b1);
  mid = pack_bf16x2(a1, b1);
  float a2, b2;
  f2_unpack(f2_sub(r1, bf16x2_to_f2(mid)), a2, b2);
  lo = pack_bf16x2(a2, b2);
}

// Pieces of 8 consecutive values (4 pairs).
struct Pieces8 { uint4 hi, mid, lo; };
GF_DEV Pieces8 split8(const float* v) {
  Pieces8 o;
  split_pair(v[0], v[1], o.hi.x, o.mid.x, o.lo.x);
  split_pair(v[2], v[3], o.hi.y, o.mid.y, o.lo.y);
  split_pair(v[4], v[5], o.hi.z, o.mid.z, o.lo.z);
  split_pair(v[6], v[7], o.hi.w, o.mid.w, o.lo.w);
  return o;
}

GF_DEV float clip_sigmoid(float z) {
  const float p = 1.0f / (1.0f + expf(-z));
  // bounds: the sampler's resolution (threshold floor(p 2^24) >= 1)
  return fminf(fmaxf(p, 0x1p-24f), 1.0f - 0x1p-24f);
}

GF_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM loads of 16 columns of this warp's 32 lanes without waiting; the
// registers are valid after tmem_wait16 (which takes them as operands so
// that no use is scheduled before it).
GF_DEV void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
GF_DEV void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
        "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
      :
      : "memory");
}
// orders the use of q after a wait already issued for the same thread
GF_DEV void tmem_order16(uint32_t (&q)[16]) {
  asm volatile(""
      : "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]),
        "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]),
        "+r"(q[13]), "+r"(q[14]), "+r"(q[15])
      :
      : "memory");
}

// relu(d + b1) of 8 G units -> bf16 pieces of G groups of 8.
template <int G>
GF_DEV void h1_pieces_g(const uint32_t* d, const float* b1u, Pieces8 (&pc)[G]) {
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const float4 bA = *reinterpret_cast<const float4*>(b1u + 8 * g);
    const float4 bB = *reinterpret_cast<const float4*>(b1u + 8 * g + 4);
    const float bb[8] = {bA.x, bA.y, bA.z, bA.w, bB.x, bB.y, bB.z, bB.w};
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      f2_unpack(f2_add(f2_pack(__uint_as_float(d[8 * g + q]), __uint_as_float(d[8 * g + q + 1])),
                       f2_pack(bb[q], bb[q + 1])),
                x[q], x[q + 1]);
      x[q] = fmaxf(x[q], 0.0f);
      x[q + 1] = fmaxf(x[q + 1], 0.0f);
    }
    pc[g] = split8(x);
  }
}

// TMEM store of 8 columns of this warp's 32 lanes; completed (and ordered
// before a later thread synchronisation) by tmem_st_wait.
GF_DEV void tmem_st8(uint32_t taddr, const uint4& a, const uint4& b) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
          taddr),
      "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
      : "memory");
}
GF_DEV void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// tcgen05.mma kind::f16 with A in TMEM (rows on lanes, K along columns,
// two bf16 per column) and B from a shared-memory descriptor.
GF_DEV void mma_f16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                           uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum));
}

// Wait for the phase of use u (0, 1, 2, ...) of a barrier: parity u & 1.
// A "free" barrier is waited for use u - 1, which a fresh barrier reports
// complete (parity 1 before its first phase).
GF_DEV bool wait_use(uint32_t bar, int u, uint64_t limit_ns, volatile int* abort_flag) {
  return mbar_wait(bar, (uint32_t)u & 1u, limit_ns, abort_flag);
}
GF_DEV bool wait_free(uint32_t bar, int u, uint64_t limit_ns, volatile int* abort_flag) {
  return mbar_wait(bar, ((uint32_t)u & 1u) ^ 1u, limit_ns, abort_flag);
}

// One arrival per warp, after the warp's shared-memory writes (made visible
// to the tensor cores) or TMEM reads are done.
GF_DEV void warp_arrive(uint32_t bar, int lane) {
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}

// Features of variables v (8 FP32 each; zero past nv) -> pieces -> A1 tile.
GF_DEV void stage_features(uint8_t* A1b, int r, float4 f0, float4 f1) {
  const float f[kF] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
  const Pieces8 pc = split8(f);
  *reinterpret_cast<uint4*>(A1b + sw_off(r, 0)) = pc.hi;
  *reinterpret_cast<uint4*>(A1b + sw_off(r, 16)) = pc.mid;
  *reinterpret_cast<uint4*>(A1b + sw_off(r, 32)) = pc.lo;
  fence_async_smem();
}

__global__ void __launch_bounds__(kThreads, 1)
k_mlp_fwd_tc(const float* __restrict__ W, int64_t nv, const float* __restrict__ feat,
             float* __restrict__ z_out, float* __restrict__ p_out,
             const uint8_t* __restrict__ live, uint64_t limit_ns, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* B1 = base + B1_OFF;
  uint8_t* B2 = base + B2_OFF;
  uint8_t* A1 = base + A1_OFF;
  float* b1s = reinterpret_cast<float*>(base + VEC_OFF);
  float* b2s = b1s + kH;
  float* w3s = b2s + kH;
  float* b3s = w3s + kH;
  float* zpart = reinterpret_cast<float*>(base + ZP_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + BAR_OFF);
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bar = [&](int i) { return smem_u32(bars + i); };

  // ---- stage weights (bf16-rounded) and biases; zero the operand tiles
  for (int e = threadIdx.x; e < 5 * PANEL / 16; e += kThreads)
    reinterpret_cast<uint4*>(base)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int a = threadIdx.x; a < kH; a += kThreads) {           // W1 row a at K 0-7
    const float* src = W + oW1 + a * kF;
    *reinterpret_cast<uint4*>(B1 + sw_off(a, 0)) =
        make_uint4(pack_bf16x2(src[0], src[1]), pack_bf16x2(src[2], src[3]),
                   pack_bf16x2(src[4], src[5]), pack_bf16x2(src[6], src[7]));
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
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(BA1_FULL + b), kE2Warps / 2);
      mbar_init(bar(BA1_FREE + b), 1);
      mbar_init(bar(BS_FULL + b), kE1Warps);
      mbar_init(bar(BS_FREE + b), 1);
    }
    mbar_init(bar(BD1_FULL), 1);
    mbar_init(bar(BD1_FREE), kE1Warps);
    mbar_init(bar(BD2_FULL), 1);
    mbar_init(bar(BD2_FREE), kE2Warps);
    mbar_init(bar(BDRAIN), 1);
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
  // tiles of this CTA: t_j = blockIdx.x + j gridDim.x, j < nj
  const int nj = blockIdx.x < ntiles
                     ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_of = [&](int j) { return (int64_t)blockIdx.x + (int64_t)j * gridDim.x; };

  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      // descriptors and TMEM operand addresses are the same for every tile
      uint64_t a1d[2][3], b2d[2][4];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int p = 0; p < 3; ++p) a1d[b][p] = sw128_desc(smem_u32(A1 + b * PANEL) + 32 * p);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int s = 0; s < 4; ++s) b2d[h][s] = sw128_desc(smem_u32(B2 + h * PANEL) + 32 * s);
      const uint64_t b1d = sw128_desc(smem_u32(B1));
      auto layer1 = [&](int j) {
        const int b = j & 1;
        ok = ok && wait_use(bar(BA1_FULL + b), j >> 1, limit_ns, &abort_flag);
        ok = ok && wait_free(bar(BD1_FREE), j, limit_ns, &abort_flag);
        if (!ok) return;
        tc_fence_after();
#pragma unroll
        for (int p = 0; p < 3; ++p)
          mma_f16(tmem + kD1, b ? a1d[1][p] : a1d[0][p], b1d, kIdesc, p > 0 ? 1u : 0u);
        mma_commit(bar(BD1_FULL));
        mma_commit(bar(BA1_FREE + b));
      };
      auto layer2 = [&](int j, int h) {
        ok = ok && wait_use(bar(BS_FULL + h), j, limit_ns, &abort_flag);
        if (h == 0) ok = ok && wait_free(bar(BD2_FREE), j, limit_ns, &abort_flag);
        if (!ok) return;
        tc_fence_after();
        const uint32_t slot = tmem + kSlot0 + kSlotCols * (uint32_t)h;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int s = 0; s < 4; ++s)
            mma_f16_tmem_a(tmem + kD2, slot + (uint32_t)(32 * p + 8 * s),
                           h ? b2d[1][s] : b2d[0][s], kIdesc, (h | p | s) != 0 ? 1u : 0u);
        mma_commit(bar(BS_FREE + h));
        if (h == 1) mma_commit(bar(BD2_FULL));
      };
      // layer 1 of tile j + 1 goes in as soon as D1 of tile j has been read
      if (nj > 0) layer1(0);
      for (int j = 0; j < nj && ok; ++j) {
        if (j + 1 < nj) layer1(j + 1);
        layer2(j, 0);
        layer2(j, 1);
      }
      // every MMA issued has completed before TMEM is freed
      volatile int drain = 0;
      mma_commit(bar(BDRAIN));
      mbar_wait(bar(BDRAIN), 0u, limit_ns, &drain);
      if (!ok) abort_flag = 1;
    }
    __syncwarp();
  } else if (warp < kE1Warps) {
    // ------------------------------------------------------ layer-1 epilogue
    // per tile: both halves of this warp's D1 columns -> registers (D1 then
    // free for the next tile's layer 1); per half: pieces -> slot h
    constexpr int G = kE1Units / 8;
    static_assert(G == 2, "one 8-column TMEM store per piece");
    const int qq = warp & 3, sub = warp >> 2;
    const int u0 = kE1Units * sub;
    const uint32_t lane_addr = tmem + ((uint32_t)(qq * 32) << 16);
    auto store = [&](int h, const Pieces8 (&pc)[G]) {
      const uint32_t col = lane_addr + kSlot0 + kSlotCols * (uint32_t)h + (uint32_t)(u0 / 2);
      tc_fence_after();
      tmem_st8(col + 0, pc[0].hi, pc[1].hi);
      tmem_st8(col + 32, pc[0].mid, pc[1].mid);
      tmem_st8(col + 64, pc[0].lo, pc[1].lo);
      tmem_st_wait();
      tc_fence_before();
      warp_arrive(bar(BS_FULL + h), lane);
    };
    for (int j = 0; j < nj; ++j) {
      if (!wait_use(bar(BD1_FULL), j, limit_ns, &abort_flag)) break;
      tc_fence_after();
      uint32_t d0[kE1Units], d1[kE1Units];
      tmem_ld16_async(lane_addr + kD1 + (uint32_t)u0, d0);
      tmem_ld16_async(lane_addr + kD1 + 64u + (uint32_t)u0, d1);
      tmem_wait16(d0);
      tmem_order16(d1);
      tc_fence_before();
      warp_arrive(bar(BD1_FREE), lane);       // D1 read
      Pieces8 pc[G];
      h1_pieces_g<G>(d0, b1s + u0, pc);
      if (!wait_free(bar(BS_FREE + 0), j, limit_ns, &abort_flag)) break;
      store(0, pc);
      h1_pieces_g<G>(d1, b1s + 64 + u0, pc);
      if (!wait_free(bar(BS_FREE + 1), j, limit_ns, &abort_flag)) break;
      store(1, pc);
    }
  } else {
    // ------------------------------------ layer-2 epilogue, feature staging
    // per tile j: the staging warps (s = 1) put the features of tile j + 2
    // (loaded an iteration earlier) into A1[b] once layer 1 of tile j has
    // read it; every warp then reads its 64 units of D2 of tile j (D2 then
    // free for the next tile) and sums them; the s = 0 warps add the halves
    // and write z, p.  The 8 warps leave the loop together (a barrier that
    // also ORs their failures), so none is left waiting on it.
    const int qq = warp & 3, hs = (warp - kE1Warps) >> 2;
    const int r = qq * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(qq * 32) << 16);
    auto load_feat = [&](int j, float4& f0, float4& f1) {
      const int64_t v = tile_of(j) * TM + r;
      if (j < nj && v < nv) {
        f0 = __ldg(reinterpret_cast<const float4*>(feat + v * kF));
        f1 = __ldg(reinterpret_cast<const float4*>(feat + v * kF) + 1);
      } else {
        f0 = f1 = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    float4 f0, f1;
    if (hs == 1) {
      for (int j = 0; j < 2 && j < nj; ++j) { // the first two tiles
        load_feat(j, f0, f1);
        stage_features(A1 + j * PANEL, r, f0, f1);
        warp_arrive(bar(BA1_FULL + j), lane);
      }
      load_feat(2, f0, f1);
    }
    for (int j = 0; j < nj; ++j) {
      const int b = j & 1;
      bool ok = true;
      if (hs == 1 && j + 2 < nj) {
        ok = wait_use(bar(BA1_FREE + b), j >> 1, limit_ns, &abort_flag);
        if (ok) {
          stage_features(A1 + b * PANEL, r, f0, f1);
          warp_arrive(bar(BA1_FULL + b), lane);
          load_feat(j + 3, f0, f1);           // in flight until the next stage
        }
      }
      ok = ok && wait_use(bar(BD2_FULL), j, limit_ns, &abort_flag);
      if (ok) {
        tc_fence_after();
        // this warp's half of z, in unit order: s = 0 from b3 over units
        // 0-63, s = 1 from 0 over units 64-127; two rounds of 32 columns
        float acc = hs ? 0.0f : b3s[0];
        const uint32_t dcol = lane_addr + kD2 + (uint32_t)(64 * hs);
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
          uint32_t d0[16], d1[16];
          tmem_ld16_async(dcol + (uint32_t)c, d0);
          tmem_ld16_async(dcol + (uint32_t)(c + 16), d1);
          tmem_wait16(d0);
          tmem_order16(d1);
          if (c == 32) {
            tc_fence_before();
            warp_arrive(bar(BD2_FREE), lane); // D2 read
          }
          const int u = 64 * hs + c;
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 w = *reinterpret_cast<const float4*>(w3s + u + 4 * q4);
            const float4 c2 = *reinterpret_cast<const float4*>(b2s + u + 4 * q4);
            const float wa[4] = {w.x, w.y, w.z, w.w}, ba[4] = {c2.x, c2.y, c2.z, c2.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t dv = q4 < 4 ? d0[4 * q4 + q] : d1[4 * (q4 - 4) + q];
              acc = fmaf(wa[q], fmaxf(__fadd_rn(__uint_as_float(dv), ba[q]), 0.0f), acc);
            }
          }
        }
        zpart[(b * 2 + hs) * 128 + r] = acc;
      }
      if (named_bar_or(1, 32 * kE2Warps, !ok)) {
        if (!err && hs == 0) {
          const int64_t v = tile_of(j) * TM + r;
          if (v < nv) {
            if (z_out) z_out[v] = __int_as_float(0x7FC00000);
            if (p_out) p_out[v] = __int_as_float(0x7FC00000);
          }
        }
        break;
      }
      if (hs == 0) {
        const int64_t v = tile_of(j) * TM + r;
        const float z = __fadd_rn(zpart[(b * 2) * 128 + r], zpart[(b * 2 + 1) * 128 + r]);
        if (v < nv) {
          if (z_out) z_out[v] = z;
          if (p_out) p_out[v] = (live && !live[v]) ? 0.0f : clip_sigmoid(z);
        }
      }
    }
  }
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
  if (abort_flag && threadIdx.x == 0 && err) atomicExch(err, 1);
}

}  // namespace

// Launch of the tensor-core forward (one persistent CTA per SM); err
// (device, may be NULL) receives 1 if a wait on the tensor cores gave up.
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
