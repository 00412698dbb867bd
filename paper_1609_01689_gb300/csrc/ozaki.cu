// FP64-class block inner products G = L^T R and linear combinations Y = A C (Section 4.4: the
// paper keeps these in FP64, footnote 5) on the fifth-generation tensor cores.
//
// Method: the error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012). Each FP64 operand is cut, per scaling group (a
// column of a chunk of rows for the Gram, a row for the linear combination), into seven signed
// base-2^7 digits after aligning the group to its largest exponent:
//     x = 2^E sum_{t=0..6} d_t 2^{-7(t+1)} + r,   d_t in [-127, 127],   |r| < 2^{E-49}.
// Every digit is exactly a bf16 number, every product of two digits is an integer below 2^14, and
// a sum of up to 1,040 such products is an integer below 2^24, which the FP32 accumulators of
// tcgen05.mma (kind::f16, bf16 inputs) hold exactly. So each digit product d_a^T e_b is exact;
// the products with a + b = L (L = 0..6, those with a + b >= 7 weigh below 2^-49 and are dropped)
// are summed in one TMEM accumulator per level while the sum stays exact, then the levels are
// combined and accumulated across chunks in double-float (df.cuh, ~48 bits) on the FP32 pipes.
// Relative error per accumulated term ~2^-47 (truncation 2^-49 per operand, double-float sums),
// the same class as the double-float CUDA-core kernels, at a fraction of their instructions.
//
// tcgen05 usage: operands are written by the threads into shared memory in the canonical K-major
// no-swizzle layout (8 x 16-byte core matrices; LBO = core matrices along K, SBO = 8-row groups),
// one elected thread issues the MMAs (M = 128, N = 16..64, K = 16 per instruction) and commits
// them to an mbarrier, and four warps read the accumulators back with tcgen05.ld. Every wait is
// bounded; a wait that runs out sets lob_oz_fault, and the CTA waits (bounded) for its own MMAs,
// frees its tensor memory and leaves.
#include <stdint.h>

#include "common.cuh"
#include "df.cuh"

__device__ int lob_oz_fault = 0;

namespace {

constexpr int OZ_S = 7;        // digits per operand
constexpr int OZ_LV = 7;       // levels L = a + b kept (0..6)
constexpr int OZ_HALF = 64;    // rows of the contraction staged at once (one operand buffer)
constexpr long long OZ_WAIT = 1ll << 32;  // SM clocks any wait may take

__device__ __forceinline__ uint32_t oz_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void oz_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(oz_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool oz_bar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(oz_smem(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait of the calling thread for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool oz_bar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!oz_bar_test(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// ---- tcgen05 (tensor memory and the fifth-generation MMA), one CTA, no cluster
// Allocate ncols (a power of two, 32..512) columns of tensor memory; the whole warp executes it.
// The address lands in *slot (shared memory).
__device__ __forceinline__ void oz_tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(oz_smem(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void oz_tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void oz_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void oz_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Make this thread's shared-memory stores visible to the tensor cores (the async proxy).
__device__ __forceinline__ void oz_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Shared-memory matrix descriptor: canonical K-major layout without swizzle. lbo = byte distance
// of core matrices adjacent along K, sbo = byte distance of adjacent 8-row groups; bits 46-47 hold
// the descriptor version of this architecture (1); base offset 0; layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28; dense, no negation.
__host__ __device__ constexpr uint32_t oz_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (tensor memory) = A B^T + (acc ? D : 0), issued by one thread.
__device__ __forceinline__ void oz_mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
// The mbarrier gets one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void oz_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(oz_smem(bar))
               : "memory");
}
// Eight consecutive 32-bit columns of this warp's 32 lanes (thread i: lane 32 (warp % 4) + i).
__device__ __forceinline__ void oz_ld8(uint32_t taddr, float v[8]) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}
__device__ __forceinline__ void oz_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// ---- the digit split
// Biased exponent of x (0 for zero and subnormals, which the split treats as zero).
__device__ __forceinline__ int oz_bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// The seven digits of x relative to the group's largest biased exponent emax (|x| < 2^{emax-1022}),
// as bf16 bit patterns: F = floor(|x| 2^{49 - (emax - 1022)}) < 2^49 is cut into 7-bit fields from
// the top, each carrying the sign of x. A digit d < 128 is exact in FP32 (2^23 + d - 2^23) and
// then in bf16 (its top 16 bits).
__device__ __forceinline__ void oz_split(double x, int emax, uint32_t dg[OZ_S]) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m = ex ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
  const int sh = 4 + emax - ex;  // >= 4
  const uint64_t F = sh < 64 ? (m >> sh) : 0ull;
  const uint32_t sign = (uint32_t)(b >> 48) & 0x8000u;
  const uint32_t hi = (uint32_t)(F >> 21), lo = (uint32_t)F & 0x1FFFFFu;  // 28 + 21 bits
#pragma unroll
  for (int t = 0; t < OZ_S; t++) {
    const int top = 42 - 7 * t;  // bit position of the digit's lowest bit in F
    const uint32_t d = top >= 21 ? ((hi >> (top - 21)) & 127u) : (((lo >> top) | (hi << (21 - top))) & 127u);
    const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
    dg[t] = (__float_as_uint(f) >> 16) | sign;
  }
}

// The digits of two elements x0, x1 of the same scaling group (emax as for oz_split), packed as
// the bf16 pairs (x0's digit in the low half) that an operand row stores for two consecutive k:
// w[t] holds digit t of both. Cheaper than two oz_split calls: one 64-bit shift per element, the
// digit fields read at fixed positions of F < 2^49, and one byte permute per pair of digits.
__device__ __forceinline__ uint32_t oz_fields(uint64_t F, int t) {
  const uint32_t fh = (uint32_t)(F >> 32), fl = (uint32_t)F;
  switch (t) {
    case 0: return fh >> 10;                               // bits 42-48
    case 1: return (fh >> 3) & 127u;                       // 35-41
    case 2: return __funnelshift_r(fl, fh, 28) & 127u;     // 28-34
    case 3: return (fl >> 21) & 127u;                      // 21-27
    case 4: return (fl >> 14) & 127u;                      // 14-20
    case 5: return (fl >> 7) & 127u;                       // 7-13
    default: return fl & 127u;                             // 0-6
  }
}
__device__ __forceinline__ uint64_t oz_fixed(double x, int emax, uint32_t& sign) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m = ex ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
  const int sh = 4 + emax - ex;
  sign = (uint32_t)(b >> 32) & 0x80000000u;
  return sh < 64 ? (m >> sh) : 0ull;
}
__device__ __forceinline__ void oz_split2(double x0, double x1, int emax, uint32_t w[OZ_S]) {
  uint32_t s0, s1;
  const uint64_t F0 = oz_fixed(x0, emax, s0), F1 = oz_fixed(x1, emax, s1);
  const uint32_t sg = (s0 >> 16) | s1;  // bf16 sign bits of the pair
#pragma unroll
  for (int t = 0; t < OZ_S; t++) {
    const float f0 = __uint_as_float(0x4B000000u | oz_fields(F0, t)) - 8388608.0f;
    const float f1 = __uint_as_float(0x4B000000u | oz_fields(F1, t)) - 8388608.0f;
    w[t] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632) | sg;
  }
}

// Byte offset of element (row r, k) inside an operand buffer of K = OZ_HALF columns in the
// canonical K-major no-swizzle layout: core matrix (r / 8, k / 8) at (r / 8) * SBO + (k / 8) * 128,
// row r % 8 at 16 (r % 8), element k % 8 at 2 (k % 8); SBO = 16 * OZ_HALF.
constexpr uint32_t OZ_LBO = 128, OZ_SBO = 16 * OZ_HALF;
__device__ __forceinline__ uint32_t oz_off(int r, int k8) { return (uint32_t)(r >> 3) * OZ_SBO + (uint32_t)k8 * 128u + (uint32_t)(r & 7) * 16u; }

// Issue every digit product with a + b <= 6 for one 16-deep step. The B digit slices lie one after
// another (slice b at sB + b * bsz, each nq rows), and so do the level accumulators in tensor memory
// (level L at column L * nq), so one MMA of A slice a against B slices b0 .. b0 + cnt - 1 stacked
// along N writes levels a + b0 .. a + b0 + cnt - 1 in their own accumulators. N = cnt * nq <= 256.
// The first step (acc = 0) of A slice 0 covers every level and clears them.
template <int NQ>
__device__ __forceinline__ void oz_mma_step(uint32_t tmem, uint32_t sA, uint32_t asz, uint32_t sB, uint32_t bsz,
                                            uint32_t sbo, int ks, bool first) {
  constexpr int SPAN = 256 / NQ;  // B slices per MMA
#pragma unroll
  for (int a = 0; a < OZ_S; a++) {
    const int nb = OZ_S - a;  // B slices 0 .. 6 - a
#pragma unroll
    for (int b0 = 0; b0 < nb; b0 += SPAN) {
      const int cnt = nb - b0 < SPAN ? nb - b0 : SPAN;
      const uint64_t ad = oz_desc(sA + a * asz + ks * 256u, OZ_LBO, sbo);
      const uint64_t bd = oz_desc(sB + b0 * bsz + ks * 256u, OZ_LBO, sbo);
      oz_mma(tmem + (uint32_t)((a + b0) * NQ), ad, bd, oz_idesc(128, cnt * NQ), (first && a == 0) ? 0u : 1u);
    }
  }
}

// Double-float helpers on (hi, lo) pairs of FP32 (Knuth's two-sum).
__device__ __forceinline__ void oz_add(float& h, float& l, float x) {
  const float s = h + x, bb = s - h, e = (h - (s - bb)) + (x - bb);
  h = s;
  l += e;
}
// 2^e as an FP32 (0 below the normal range; e <= 127 by construction).
__device__ __forceinline__ float oz_pow2(int e) { return e < -126 ? 0.f : __uint_as_float((uint32_t)(e + 127) << 23); }

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------------
// Gram products G0 = L0^T R and (optionally) G1 = L1^T R over n rows, p, q <= 64, in one pass:
// the digits of L0's columns fill rows 0..63 of the MMA's A operand and those of L1's rows
// 64..127, so one M = 128 product serves both (the solver's G = S^T (H S) and M = S^T S share
// R = S). Persistent CTAs take chunks of 128 rows in turn; per chunk:
//   1. each column's largest exponent over the chunk (one thread per column);
//   2. for each half of 64 rows: the digits of every element into the operand buffers (A: 7 x
//      128 x 64, B: 7 x NQ x 64 bf16), then one thread issues the 28 digit products with
//      a + b <= 6 per 16-deep step into the 7 level accumulators of tensor memory (7 x NQ
//      columns; the first product of a level in the chunk overwrites it) and commits them;
//   3. warps 0-3 read the levels back (thread = accumulator row), combine them and add the
//      chunk's value, scaled by 2^{E_row + E_col - 14}, into double-float sums kept in registers
//      relative to a per-thread reference exponent.
// Per level at most 7 digit products over 128 rows: 7 * 128 * 127^2 < 2^24, exact in FP32.
// The CTA's partial sums go to part[cta][2][64][NQ] (FP64); k_gram_oz_reduce adds them in
// CTA order.
// ---------------------------------------------------------------------------------------------
constexpr int OZ_KC = 2 * OZ_HALF;  // rows per chunk

template <int NQ>
struct OzG {
  static constexpr uint32_t ASZ = 128u * OZ_HALF * 2u;  // one digit slice of A (16 KB)
  static constexpr uint32_t BSZ = (uint32_t)NQ * OZ_HALF * 2u;
  static constexpr uint32_t A0 = 0;
  static constexpr uint32_t B0 = A0 + OZ_S * ASZ;
  static constexpr uint32_t EX = B0 + OZ_S * BSZ;  // int [3][64]: chunk column exponents of L0, L1, R
  static constexpr uint32_t BAR = EX + 3 * 64 * 4;
  static constexpr uint32_t SLOT = BAR + 8;
  static constexpr uint32_t BYTES = SLOT + 8;
  static constexpr uint32_t TCOLS = OZ_LV * NQ <= 128 ? 128u : (OZ_LV * NQ <= 256 ? 256u : 512u);
  static_assert(NQ % 16 == 0 && NQ >= 16 && NQ <= 64, "N of the MMA");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

// Level combination of one accumulator entry: sum_L v_L 2^{-7L} as a double-float. Levels 4-6
// (below 2^-28 of a full-scale level 0) are summed in FP32 first.
__device__ __forceinline__ void oz_levels(const float v[OZ_LV], float& h, float& l) {
  const float t = fmaf(v[6], 0x1p-42f, fmaf(v[5], 0x1p-35f, v[4] * 0x1p-28f));
  h = v[0];
  l = 0.f;
  oz_add(h, l, v[1] * 0x1p-7f);
  oz_add(h, l, v[2] * 0x1p-14f);
  oz_add(h, l, v[3] * 0x1p-21f);
  oz_add(h, l, t);
}

template <int NQ>
__global__ void __launch_bounds__(256, 1)
    k_gram_oz(int64_t n, int p, const double* __restrict__ L0, int ld0, const double* __restrict__ L1, int ld1, int q,
              const double* __restrict__ R, int ldr, double* __restrict__ part) {
  using C = OzG<NQ>;
  extern __shared__ __align__(1024) unsigned char sm[];
  int* ex = reinterpret_cast<int*>(sm + C::EX);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + C::BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::SLOT);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int np1 = L1 ? p : 0;
  const int ncol = p + np1 + q;  // source columns: L0 (p), L1 (np1), R (q)
  const int64_t nchunks = (n + OZ_KC - 1) / OZ_KC;

  // zero the operand buffers (rows that no column fills stay zero), barrier, tensor memory
  for (uint32_t o = tid * 16u; o < C::EX; o += 256u * 16u) *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    oz_bar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) oz_tmem_alloc(slot, C::TCOLS);
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *slot;

  // readout role (warps 0-3): accumulator row t -> output sel = t / 64 (0: G0, 1: G1), row m = t % 64
  const int sel = tid >> 6, m = tid & 63;
  const bool rd = tid < 128 && m < p && (sel == 0 || L1 != nullptr);
  float ah[NQ], al[NQ];
#pragma unroll
  for (int c = 0; c < NQ; c++) { ah[c] = 0.f; al[c] = 0.f; }
  int eref = 0;
  bool started = false;
  uint32_t phase = 0;
  bool fault = false;
  constexpr uint32_t IDESC = oz_idesc(128, NQ);
  const uint32_t sA = oz_smem(sm + C::A0), sB = oz_smem(sm + C::B0);

  for (int64_t ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    const int64_t r0 = ck * OZ_KC;
    const int rows = (int)((n - r0) < OZ_KC ? (n - r0) : OZ_KC);
    // 1. largest biased exponent of each column over the chunk
    if (tid < ncol) {
      const double* src;
      int ld, j;
      if (tid < p) { src = L0; ld = ld0; j = tid; }
      else if (tid < p + np1) { src = L1; ld = ld1; j = tid - p; }
      else { src = R; ld = ldr; j = tid - p - np1; }
      int e = 0;
      for (int i = 0; i < rows; i++) e = max(e, oz_bexp(src[(r0 + i) * ld + j]));
      ex[(tid < p ? 0 : (tid < p + np1 ? 1 : 2)) * 64 + j] = e;
    }
    __syncthreads();
    // 2. two halves of 64 rows: digits into the operand buffers, then the digit products
    for (int h = 0; h < 2; h++) {
      if (h == 1) {  // the first half's products must have read the buffers
        const bool ok = oz_bar_wait(bar, phase & 1, OZ_WAIT);
        if (__syncthreads_or(!ok)) { fault = true; break; }
        phase++;
      }
      for (int w = tid; w < ncol * 8; w += 256) {
        const int gj = w % ncol, k8 = w / ncol;
        const double* src;
        int ld, j, srow, set;
        if (gj < p) { src = L0; ld = ld0; j = gj; srow = gj; set = 0; }
        else if (gj < p + np1) { src = L1; ld = ld1; j = gj - p; srow = 64 + j; set = 1; }
        else { src = R; ld = ldr; j = gj - p - np1; srow = j; set = 2; }
        const int emax = ex[set * 64 + j];
        uint32_t pk[OZ_S][4];
#pragma unroll
        for (int t = 0; t < OZ_S; t++) pk[t][0] = pk[t][1] = pk[t][2] = pk[t][3] = 0u;
#pragma unroll
        for (int r = 0; r < 8; r++) {
          const int i = h * OZ_HALF + k8 * 8 + r;
          const double x = i < rows ? src[(r0 + i) * ld + j] : 0.0;
          uint32_t dg[OZ_S];
          oz_split(x, emax, dg);
#pragma unroll
          for (int t = 0; t < OZ_S; t++) pk[t][r >> 1] |= dg[t] << (16 * (r & 1));
        }
        const uint32_t off = oz_off(srow, k8);
        unsigned char* base = sm + (set == 2 ? C::B0 : C::A0);
        const uint32_t ssz = set == 2 ? C::BSZ : C::ASZ;
#pragma unroll
        for (int t = 0; t < OZ_S; t++)
          *reinterpret_cast<uint4*>(base + t * ssz + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
      }
      oz_fence_proxy();
      __syncthreads();
      if (tid == 0) {
        oz_fence_after();
        for (int L = 0; L < OZ_LV; L++)
          for (int a = 0; a <= L; a++) {
            const int b = L - a;
#pragma unroll
            for (int ks = 0; ks < OZ_HALF / 16; ks++) {
              const uint64_t ad = oz_desc(sA + a * C::ASZ + ks * 256u, OZ_LBO, OZ_SBO);
              const uint64_t bd = oz_desc(sB + b * C::BSZ + ks * 256u, OZ_LBO, OZ_SBO);
              oz_mma(tmem + (uint32_t)(L * NQ), ad, bd, IDESC, (h > 0 || a > 0 || ks > 0) ? 1u : 0u);
            }
          }
        oz_commit(bar);
      }
    }
    if (fault) break;
    {  // the second half's products
      const bool ok = oz_bar_wait(bar, phase & 1, OZ_WAIT);
      if (__syncthreads_or(!ok)) { fault = true; break; }
      phase++;
    }
    oz_fence_after();
    // 3. readout: levels -> chunk value -> double-float sums
    if (tid < 128) {
      const int er = ex[sel * 64 + m];
      int ecmax = 0;
      for (int c = 0; c < q; c++) ecmax = max(ecmax, ex[128 + c]);
      const bool live = rd && er > 0 && ecmax > 0;
      // exponent of a full-scale chunk value: 2^{E_row + E_colmax - 14} times ~2^24
      const int ech = (er - 1022) + (ecmax - 1022) - 14 + 24;
      if (live) {
        if (!started) { eref = ech; started = true; }
        else if (ech > eref) {  // rescale the sums to the larger reference (exact powers of two)
          const float f = oz_pow2(eref - ech);
#pragma unroll
          for (int c = 0; c < NQ; c++) { ah[c] *= f; al[c] *= f; }
          eref = ech;
        }
      }
      const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
      for (int c0 = 0; c0 < NQ; c0 += 8) {
        float v[OZ_LV][8];
#pragma unroll
        for (int L = 0; L < OZ_LV; L++) oz_ld8(tmem + lane_base + (uint32_t)(L * NQ + c0), v[L]);
        oz_wait_ld();
        if (live) {
#pragma unroll
          for (int c = 0; c < 8; c++) {
            const int col = c0 + c;
            if (col >= q) continue;
            float lv[OZ_LV];
#pragma unroll
            for (int L = 0; L < OZ_LV; L++) lv[L] = v[L][c];
            float vh, vl;
            oz_levels(lv, vh, vl);
            const float s = oz_pow2((er - 1022) + (ex[128 + col] - 1022) - 14 - eref);
            oz_add(ah[col], al[col], vh * s);
            al[col] += vl * s;
          }
        }
      }
    }
    oz_fence_before();
    __syncthreads();
  }

  if (fault) {
    if (tid == 0) atomicExch(&lob_oz_fault, 1);
    // let the MMAs already issued finish before the tensor memory is released
    oz_bar_wait(bar, phase & 1, 1ll << 31);
    __syncthreads();
  } else if (tid < 128) {
    double* out = part + ((int64_t)blockIdx.x * 2 + sel) * 64 * NQ + (int64_t)m * NQ;
#pragma unroll
    for (int c = 0; c < NQ; c++) {
      double v = 0.0;
      if (rd && started) v = ldexp((double)ah[c] + (double)al[c], eref);
      out[c] = v;
    }
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    oz_tmem_free(tmem, C::TCOLS);
  }
}

// G_sel[m][l] = sum over CTAs of part[cta][sel][m][l], in CTA order (deterministic).
__global__ void k_gram_oz_reduce(int ncta, int nq, int p, int q, int nsel, const double* __restrict__ part,
                                 double* __restrict__ G0, double* __restrict__ G1) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nsel * p * q) return;
  const int sel = e / (p * q), r = e % (p * q), m = r / q, l = r % q;
  double s = 0.0;
  for (int c = 0; c < ncta; c++) s += part[((int64_t)c * 2 + sel) * 64 * nq + (int64_t)m * nq + l];
  (sel == 0 ? G0 : G1)[m * q + l] = s;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------------
// Y = A C (+ D) for n x p A (p <= 64) and p x q C (q <= 64): one CTA of 128 threads per 128 rows,
// thread t owning row t of the tile (and lane t of the accumulators). Scaling groups are the rows
// of A (the contraction runs along them) and the columns of C. The digits of the tile's rows fill
// the A operand (7 x 128 x KP bf16, KP = p rounded up to 16), those of C the B operand
// (7 x NQ x KP); 28 digit products per 16-deep step go into 7 level accumulators; each thread then
// combines its row's levels, scales by 2^{E_row + E_col - 14} and writes FP64. Per level at most
// 7 products of depth p <= 64: 7 * 64 * 127^2 < 2^24, exact. All reads of A precede the writes of
// Y in the CTA and the CTA owns its rows, so Y may be the same rows of A (an in-place update).
// ---------------------------------------------------------------------------------------------
template <int NQ, int KP>
struct OzL {
  static constexpr uint32_t SBO = 16u * KP;                   // 8-row groups of a K = KP operand
  static constexpr uint32_t ASZ = 128u * KP * 2u;
  static constexpr uint32_t BSZ = (uint32_t)NQ * KP * 2u;
  static constexpr uint32_t A0 = 0;
  static constexpr uint32_t B0 = A0 + OZ_S * ASZ;
  static constexpr uint32_t EC = B0 + OZ_S * BSZ;             // int [64]: column exponents of C
  static constexpr uint32_t BAR = EC + 64 * 4;
  static constexpr uint32_t SLOT = BAR + 8;
  static constexpr uint32_t BYTES = SLOT + 8;
  static constexpr uint32_t TCOLS = OZ_LV * NQ <= 128 ? 128u : (OZ_LV * NQ <= 256 ? 256u : 512u);
  static_assert(KP % 16 == 0 && KP <= 64 && NQ % 16 == 0 && NQ <= 64, "operand shapes");
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

template <int NQ, int KP>
__global__ void __launch_bounds__(128)
    k_lincomb_oz(int64_t n, int p, const double* A, int lda, int q, const double* __restrict__ Cm, double* Y,
                 int ldy, const double* D, int ldd) {
  using Cf = OzL<NQ, KP>;
  extern __shared__ __align__(1024) unsigned char sm[];
  int* ec = reinterpret_cast<int*>(sm + Cf::EC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + Cf::BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + Cf::SLOT);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int64_t row = i0 + tid;
  const bool valid = row < n;

  if (tid == 0) {
    oz_bar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) oz_tmem_alloc(slot, Cf::TCOLS);
  // column exponents of C
  if (tid < q) {
    int e = 0;
    for (int k = 0; k < p; k++) e = max(e, oz_bexp(Cm[k * q + tid]));
    ec[tid] = e;
  }
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *slot;
  // digits of C into the B operand: row l (output column), K = the p rows of C (zero beyond p, q)
  for (int w = tid; w < NQ * (KP / 8); w += 128) {
    const int l = w % NQ, k8 = w / NQ;
    const int emax = l < q ? ec[l] : 0;
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int t = 0; t < OZ_S; t++) pk[t][0] = pk[t][1] = pk[t][2] = pk[t][3] = 0u;
#pragma unroll
    for (int r = 0; r < 8; r++) {
      const int k = k8 * 8 + r;
      const double x = (l < q && k < p) ? Cm[k * q + l] : 0.0;
      uint32_t dg[OZ_S];
      oz_split(x, emax, dg);
#pragma unroll
      for (int t = 0; t < OZ_S; t++) pk[t][r >> 1] |= dg[t] << (16 * (r & 1));
    }
    const uint32_t off = (uint32_t)(l >> 3) * Cf::SBO + (uint32_t)k8 * 128u + (uint32_t)(l & 7) * 16u;
#pragma unroll
    for (int t = 0; t < OZ_S; t++)
      *reinterpret_cast<uint4*>(sm + Cf::B0 + t * Cf::BSZ + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
  }
  // the row of A: exponent, then its digits into the A operand (row tid, K = p, zero beyond)
  double x[KP];
  int er = 0;
#pragma unroll
  for (int k = 0; k < KP; k++) {
    x[k] = (valid && k < p) ? A[row * lda + k] : 0.0;
    er = max(er, oz_bexp(x[k]));
  }
#pragma unroll
  for (int k8 = 0; k8 < KP / 8; k8++) {
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int t = 0; t < OZ_S; t++) pk[t][0] = pk[t][1] = pk[t][2] = pk[t][3] = 0u;
#pragma unroll
    for (int r = 0; r < 8; r++) {
      uint32_t dg[OZ_S];
      oz_split(x[k8 * 8 + r], er, dg);
#pragma unroll
      for (int t = 0; t < OZ_S; t++) pk[t][r >> 1] |= dg[t] << (16 * (r & 1));
    }
    const uint32_t off = (uint32_t)(tid >> 3) * Cf::SBO + (uint32_t)k8 * 128u + (uint32_t)(tid & 7) * 16u;
#pragma unroll
    for (int t = 0; t < OZ_S; t++)
      *reinterpret_cast<uint4*>(sm + Cf::A0 + t * Cf::ASZ + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
  }
  oz_fence_proxy();
  __syncthreads();
  if (tid == 0) {
    oz_fence_after();
    const uint32_t sA = oz_smem(sm + Cf::A0), sB = oz_smem(sm + Cf::B0);
#pragma unroll
    for (int ks = 0; ks < KP / 16; ks++) oz_mma_step<NQ>(tmem, sA, Cf::ASZ, sB, Cf::BSZ, Cf::SBO, ks, ks == 0);
    oz_commit(bar);
  }
  const bool ok = oz_bar_wait(bar, 0, OZ_WAIT);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicExch(&lob_oz_fault, 1);
    oz_bar_wait(bar, 0, 1ll << 31);  // let the issued MMAs finish before releasing tensor memory
  } else {
    oz_fence_after();
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c0 = 0; c0 < NQ; c0 += 8) {
      float v[OZ_LV][8];
#pragma unroll
      for (int L = 0; L < OZ_LV; L++) oz_ld8(tmem + lane_base + (uint32_t)(L * NQ + c0), v[L]);
      oz_wait_ld();
      if (valid) {
#pragma unroll
        for (int c = 0; c < 8; c++) {
          const int col = c0 + c;
          if (col >= q) continue;
          float lv[OZ_LV];
#pragma unroll
          for (int L = 0; L < OZ_LV; L++) lv[L] = v[L][c];
          float vh, vl;
          oz_levels(lv, vh, vl);
          double y = ldexp((double)vh + (double)vl, (er - 1022) + (ec[col] - 1022) - 14);
          if (er == 0 || ec[col] == 0) y = 0.0;
          if (D) y += D[row * ldd + col];
          Y[row * ldy + col] = y;
        }
      }
    }
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    oz_tmem_free(tmem, Cf::TCOLS);
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------------
// Pipelined Gram (v2): G0 = L0^T R and optionally G1 = L1^T R, p, q <= 64, chunks of 64 rows
// (one MMA round per chunk, scaling groups = columns of a chunk; 7 * 64 * 127^2 < 2^24).
// Warp roles in a persistent CTA of 256 threads:
//   producers (warps 4-7): cp.async the chunk's raw FP64 rows into shared memory (zero beyond n),
//     take each column's largest exponent there, wait until the previous chunk's MMAs have read
//     the operand buffers, write the digits, and signal `full`;
//   consumers (warps 0-3): thread 0 waits for `full` and issues the chunk's 112 MMAs (28 digit
//     products x 4 steps of 16) with a commit to `done`; all four warps wait for `done`, read the
//     levels back and add the chunk into their double-float sums, then count the chunk out.
// While the consumers read chunk k back, the producers already load and split chunk k + 1, so the
// HBM stream, the digit split, the MMAs and the readout overlap. When R is L0 itself (the solver's
// M = S^T S beside (H S)^T S) its columns are loaded once and their digits go to both operands.
// Column exponents are double-buffered by chunk parity; the producers wait (a counter) for the
// readout of chunk k - 2 before overwriting its half.
// ---------------------------------------------------------------------------------------------
template <int NQ>
struct OzG2 {
  static constexpr int KC = 64;
  static constexpr uint32_t ASZ = 128u * KC * 2u;
  static constexpr uint32_t BSZ = (uint32_t)NQ * KC * 2u;
  static constexpr uint32_t A0 = 0;
  static constexpr uint32_t B0 = A0 + OZ_S * ASZ;
  static constexpr uint32_t RAW = B0 + OZ_S * BSZ;  // the chunk's raw FP64 rows: [KC][p] L0, [KC][p] L1, [KC][q] R
  static constexpr int RAWC = NQ <= 48 ? 128 : 96;      // bound on the raw columns 2p + q (p + q when R is L0)
  static constexpr uint32_t EX = RAW + KC * RAWC * 8u;  // int [2][3][64]
  static constexpr uint32_t BAR = EX + 2 * 3 * 64 * 4;   // full, done, raw
  static constexpr uint32_t CTL = BAR + 24;              // int: readout count, abort, commits
  static constexpr uint32_t SLOT = CTL + 16;
  static constexpr uint32_t BYTES = SLOT + 16;
  static constexpr uint32_t TCOLS = OZ_LV * NQ <= 128 ? 128u : (OZ_LV * NQ <= 256 ? 256u : 512u);
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void oz_cp8(void* dst, const void* src, bool valid) {
  // 8-byte async copy; zero fill when the row is beyond n
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(oz_smem(dst)), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void oz_cp_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void oz_named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
// Bounded wait that also gives up once the CTA's abort flag is set; false then.
__device__ __forceinline__ bool oz_wait2(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (!oz_bar_test(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > OZ_WAIT) { *abort = 1; return false; }
  }
  return true;
}

template <int NQ>
__global__ void __launch_bounds__(512, 1)
    k_gram_oz2(int64_t n, int p, const double* __restrict__ L0, int ld0, const double* __restrict__ L1, int ld1,
               int q, const double* __restrict__ R, int ldr, double* __restrict__ part, int bulk) {
  using C = OzG2<NQ>;
  constexpr int KC = C::KC, NP = 256;   // rows per chunk, producer threads
  constexpr int NH = NQ / 2;            // columns per consumer warp half
  extern __shared__ __align__(1024) unsigned char sm[];
  int* ex = reinterpret_cast<int*>(sm + C::EX);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::BAR);
  uint64_t* done = full + 1;
  uint64_t* rawb = full + 2;
  volatile int* rcount = reinterpret_cast<volatile int*>(sm + C::CTL);
  volatile int* abort = rcount + 1;
  volatile int* ncommit = rcount + 2;  // commits issued to `done`
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + C::SLOT);
  double* raw = reinterpret_cast<double*>(sm + C::RAW);
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool shared_r = (R == L0 && ldr == ld0 && q == p);
  const int64_t nchunks = (n + KC - 1) / KC;

  for (uint32_t o = tid * 16u; o < C::RAW; o += 512u * 16u) *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    oz_bar_init(full, 1);
    oz_bar_init(done, 1);
    oz_bar_init(rawb, 1);
    *rcount = 0;
    *abort = 0;
    *ncommit = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) oz_tmem_alloc(slot, C::TCOLS);
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *slot;

  if (tid >= 256) {
    // ===================== producers (warps 8-15) =====================
    const int pt = tid - 256;
    // raw blocks, one after another: L0 (p columns), L1 (p, if given), R (q, unless R is L0);
    // setid = the operand role of a block (0: L0, 1: L1, 2: R)
    int nset = 0, wd[3] = {0, 0, 0}, lds[3] = {0, 0, 0}, setid[3] = {0, 0, 0};
    const double* srcs[3] = {nullptr, nullptr, nullptr};
    wd[nset] = p; lds[nset] = ld0; srcs[nset] = L0; setid[nset] = 0; nset++;
    if (L1) { wd[nset] = p; lds[nset] = ld1; srcs[nset] = L1; setid[nset] = 1; nset++; }
    if (!shared_r) { wd[nset] = q; lds[nset] = ldr; srcs[nset] = R; setid[nset] = 2; nset++; }
    uint32_t roff[3] = {0, 0, 0};
    for (int b = 1; b < nset; b++) roff[b] = roff[b - 1] + (uint32_t)KC * wd[b - 1] * 8u;
    int cstart[3] = {0, 0, 0};
    for (int b = 1; b < nset; b++) cstart[b] = cstart[b - 1] + wd[b - 1];
    int k = 0;
    for (int64_t ck = blockIdx.x; ck < nchunks; ck += gridDim.x, k++) {
      const int64_t r0 = ck * KC;
      const int rows = (int)((n - r0) < KC ? (n - r0) : KC);
      // raw rows of the chunk by bulk copies completing on `rawb` (the previous chunk's digits were
      // written from raw before `full`, and every producer passed that barrier)
      if (bulk) {
        uint32_t bytes = 0;
        for (int b = 0; b < nset; b++) bytes += (uint32_t)rows * wd[b] * 8u;
        if (pt == 0)
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(oz_smem(rawb)), "r"(bytes) : "memory");
        oz_named_sync(1, NP);
        for (int b = 0; b < nset; b++) {
          if (lds[b] == wd[b]) {  // contiguous rows: one copy
            if (pt == b) {
              const uint32_t by = (uint32_t)rows * wd[b] * 8u;
              asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                           ::"r"(oz_smem(reinterpret_cast<unsigned char*>(raw) + roff[b])), "l"(srcs[b] + r0 * lds[b]),
                           "r"(by), "r"(oz_smem(rawb)) : "memory");
            }
          } else {
            for (int i = pt; i < rows; i += NP)
              asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                           ::"r"(oz_smem(reinterpret_cast<unsigned char*>(raw) + roff[b] + (uint32_t)i * wd[b] * 8u)),
                           "l"(srcs[b] + (r0 + i) * lds[b]), "r"((uint32_t)wd[b] * 8u), "r"(oz_smem(rawb)) : "memory");
          }
        }
        if (!oz_wait2(rawb, (uint32_t)(k & 1), abort)) {}
      } else {
        for (int b = 0; b < nset; b++)
          for (int i = pt >> 6; i < rows; i += NP >> 6)
            for (int c = pt & 63; c < wd[b]; c += 64)
              oz_cp8(reinterpret_cast<unsigned char*>(raw) + roff[b] + ((uint32_t)i * wd[b] + c) * 8u,
                     srcs[b] + (r0 + i) * lds[b] + c, true);
        oz_cp_wait();
      }
      // the exponents of chunk k reuse the half of chunk k - 2: wait until that one was read back
      if (k >= 2) {
        const long long t0 = clock64();
        while (*rcount < k - 1 && !*abort)
          if (clock64() - t0 > OZ_WAIT) *abort = 1;
      }
      oz_named_sync(1, NP);
      int* exk = ex + (k & 1) * 3 * 64;
      for (int b = 0; b < nset; b++) {
        const int c = pt - cstart[b];
        if (c < 0 || c >= wd[b]) continue;
        const double* blk = reinterpret_cast<const double*>(reinterpret_cast<unsigned char*>(raw) + roff[b]);
        int e = 0;
#pragma unroll 8
        for (int i = 0; i < rows; i++) e = max(e, oz_bexp(blk[i * wd[b] + c]));
        exk[setid[b] * 64 + c] = e;
        if (shared_r && b == 0) exk[128 + c] = e;
      }
      // the previous chunk's MMAs must have read the operand buffers
      if (k >= 1) oz_wait2(done, (uint32_t)((k - 1) & 1), abort);
      oz_named_sync(1, NP);
      if (*abort) break;
      for (int b = 0; b < nset; b++) {
        const int c = pt & 63;
        if (c >= wd[b]) continue;
        const double* blk = reinterpret_cast<const double*>(reinterpret_cast<unsigned char*>(raw) + roff[b]);
        const int set = setid[b];
        const int emax = exk[set * 64 + c];
#pragma unroll
        for (int pass = 0; pass < 2; pass++) {
          const int k8 = (pt >> 6) + 4 * pass;
          uint32_t pk[OZ_S][4];
#pragma unroll
          for (int r = 0; r < 8; r += 2) {
            const int i0 = k8 * 8 + r;
            const double x0 = i0 < rows ? blk[i0 * wd[b] + c] : 0.0;
            const double x1 = i0 + 1 < rows ? blk[(i0 + 1) * wd[b] + c] : 0.0;
            uint32_t wv[OZ_S];
            oz_split2(x0, x1, emax, wv);
#pragma unroll
            for (int t = 0; t < OZ_S; t++) pk[t][r >> 1] = wv[t];
          }
          if (set < 2) {
            const uint32_t off = oz_off(set * 64 + c, k8);
#pragma unroll
            for (int t = 0; t < OZ_S; t++)
              *reinterpret_cast<uint4*>(sm + C::A0 + t * C::ASZ + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
          }
          if (set == 2 || (set == 0 && shared_r)) {
            const uint32_t off = oz_off(c, k8);
#pragma unroll
            for (int t = 0; t < OZ_S; t++)
              *reinterpret_cast<uint4*>(sm + C::B0 + t * C::BSZ + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
          }
        }
      }
      oz_fence_proxy();
      oz_named_sync(1, NP);
      if (pt == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(oz_smem(full)) : "memory");
    }
  } else {
    // ===================== consumers (warps 0-7) =====================
    // warp w reads accumulator lanes 32 (w % 4) .. + 31 and the columns of half w / 4
    const int lt = tid & 127, sel = lt >> 6, m = lt & 63, cb = (warp >> 2) * NH;
    const bool rd = m < p && (sel == 0 || L1 != nullptr);
    float ah[NH], al[NH];
#pragma unroll
    for (int c = 0; c < NH; c++) { ah[c] = 0.f; al[c] = 0.f; }
    int eref = 0;
    bool started = false;
    const uint32_t sA = oz_smem(sm + C::A0), sB = oz_smem(sm + C::B0);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int k = 0;
    for (int64_t ck = blockIdx.x; ck < nchunks; ck += gridDim.x, k++) {
      if (tid == 0) {
        if (oz_wait2(full, (uint32_t)(k & 1), abort)) {
          oz_fence_after();
#pragma unroll
          for (int ks = 0; ks < KC / 16; ks++) oz_mma_step<NQ>(tmem, sA, C::ASZ, sB, C::BSZ, 16u * KC, ks, ks == 0);
          oz_commit(done);
          *ncommit = k + 1;
        }
      }
      oz_wait2(done, (uint32_t)(k & 1), abort);
      oz_named_sync(2, 256);  // a uniform decision: every consumer goes on, or every one leaves
      if (*abort) break;
      oz_fence_after();
      const int* exk = ex + (k & 1) * 3 * 64;
      const int er = exk[sel * 64 + m];
      int ecmax = 0;
      for (int c = 0; c < q; c++) ecmax = max(ecmax, exk[128 + c]);
      const bool live = rd && er > 0 && ecmax > 0;
      const int ech = (er - 1022) + (ecmax - 1022) - 14 + 24;
      if (live) {
        if (!started) { eref = ech; started = true; }
        else if (ech > eref) {
          const float f = oz_pow2(eref - ech);
#pragma unroll
          for (int c = 0; c < NH; c++) { ah[c] *= f; al[c] *= f; }
          eref = ech;
        }
      }
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 8) {
        float v[OZ_LV][8];
#pragma unroll
        for (int L = 0; L < OZ_LV; L++) oz_ld8(tmem + lane_base + (uint32_t)(L * NQ + cb + c0), v[L]);
        oz_wait_ld();
        if (live) {
#pragma unroll
          for (int c = 0; c < 8; c++) {
            const int col = cb + c0 + c;
            if (col >= q) continue;
            float lv[OZ_LV];
#pragma unroll
            for (int L = 0; L < OZ_LV; L++) lv[L] = v[L][c];
            float vh, vl;
            oz_levels(lv, vh, vl);
            const float s = oz_pow2((er - 1022) + (exk[128 + col] - 1022) - 14 - eref);
            oz_add(ah[c0 + c], al[c0 + c], vh * s);
            al[c0 + c] += vl * s;
          }
        }
      }
      oz_fence_before();
      oz_named_sync(2, 256);
      if (tid == 0) { __threadfence_block(); *rcount = k + 1; }
    }
    if (!*abort) {
      double* out = part + ((int64_t)blockIdx.x * 2 + sel) * 64 * NQ + (int64_t)m * NQ + cb;
#pragma unroll
      for (int c = 0; c < NH; c++) out[c] = (rd && started) ? ldexp((double)ah[c] + (double)al[c], eref) : 0.0;
    }
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) atomicExch(&lob_oz_fault, 1);
    // the last batch of MMAs issued must finish before the tensor memory is released
    const int nc = *ncommit;
    if (nc > 0) oz_bar_wait(done, (uint32_t)((nc - 1) & 1), 1ll << 31);
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    oz_tmem_free(tmem, C::TCOLS);
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------------------
// Pipelined linear combination (v2): Y = A C (+ D), p, q <= 64, tiles of 128 rows. Persistent CTAs
// of 16 warps:
//   producers (warps 8-15): the digits of C once (B operand: 7 x NQ x KP, scaling groups the
//     columns of C); per tile, bulk-copy the 128 rows of A into shared memory, take each row's
//     largest exponent, wait until the previous tile's MMAs have read the A operand, write the
//     digits (scaling groups the rows), signal `full`;
//   consumers (warps 0-7): thread 0 issues the tile's digit products (B slices stacked along N) and
//     commits them; all wait, read the levels of their row (thread = tile row, warp half = column
//     half), combine and scale them, add D and store Y.
// The tile's rows of A are all read before any of its rows of Y is written and a CTA owns its
// tiles, so Y may be the same rows of A (an in-place update).
// ---------------------------------------------------------------------------------------------
template <int NQ, int KP>
struct OzL2 {
  static constexpr uint32_t SBO = 16u * KP;
  static constexpr uint32_t ASZ = 128u * KP * 2u;
  static constexpr uint32_t BSZ = (uint32_t)NQ * KP * 2u;
  static constexpr uint32_t A0 = 0;
  static constexpr uint32_t B0 = A0 + OZ_S * ASZ;
  static constexpr uint32_t RAW = B0 + OZ_S * BSZ;        // [128][p | 1] FP64 rows of the tile
  static constexpr uint32_t ER = RAW + 128u * (KP + 1) * 8u;  // int [2][128]: row exponents by tile parity
  static constexpr uint32_t EC = ER + 2 * 128 * 4;         // int [64]: column exponents of C
  static constexpr uint32_t BAR = EC + 64 * 4;             // full, done, raw
  static constexpr uint32_t CTL = BAR + 24;                // readout count, abort, commits
  static constexpr uint32_t SLOT = CTL + 16;
  static constexpr uint32_t BYTES = SLOT + 16;
  static constexpr uint32_t TCOLS = OZ_LV * NQ <= 128 ? 128u : (OZ_LV * NQ <= 256 ? 256u : 512u);
  static_assert(BYTES <= 227 * 1024, "shared memory");
};

// FP64 value of the double-float (h, l) times 2^e: the two parts converted by their bit fields (no
// FP64 conversion instructions), one FP64 addition, and the scaling as an exponent-field add.
// Requires h, l normal or zero and the result in the normal FP64 range.
__device__ __forceinline__ double oz_f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  if ((u & 0x7F800000u) == 0) return 0.0;  // zero; a subnormal low part is far below the result's ulp
  const uint32_t s = u & 0x80000000u, e = (u >> 23) & 0xFF, mt = u & 0x7FFFFFu;
  const uint32_t hi = s | ((e - 127 + 1023) << 20) | (mt >> 3), lo = mt << 29;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double oz_df_to_f64(float h, float l, int e) {
  const double v = oz_f32_to_f64(h) + oz_f32_to_f64(l);
  if (v == 0.0) return 0.0;
  const int hv = __double2hiint(v);
  const int ef = ((hv >> 20) & 0x7FF) + e;
  if (ef <= 0 || ef >= 2047) return ldexp(v, e);  // outside the normal range: the library scaling
  return __hiloint2double(hv + (e << 20), __double2loint(v));
}

template <int NQ, int KP>
__global__ void __launch_bounds__(512, 1)
    k_lincomb_oz2(int64_t n, int p, const double* A, int lda, int q, const double* __restrict__ Cm, double* Y,
                  int ldy, const double* D, int ldd) {
  using Cf = OzL2<NQ, KP>;
  constexpr int NP = 256, NH = NQ / 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  int* er = reinterpret_cast<int*>(sm + Cf::ER);
  int* ec = reinterpret_cast<int*>(sm + Cf::EC);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + Cf::BAR);
  uint64_t* done = full + 1;
  uint64_t* rawb = full + 2;
  volatile int* rcount = reinterpret_cast<volatile int*>(sm + Cf::CTL);
  volatile int* abort = rcount + 1;
  volatile int* ncommit = rcount + 2;
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + Cf::SLOT);
  double* raw = reinterpret_cast<double*>(sm + Cf::RAW);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t ntiles = (n + 127) / 128;
  const int rs = p | 1;

  for (uint32_t o = tid * 16u; o < Cf::RAW; o += 512u * 16u) *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    oz_bar_init(full, 1);
    oz_bar_init(done, 1);
    oz_bar_init(rawb, 1);
    *rcount = 0;
    *abort = 0;
    *ncommit = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) oz_tmem_alloc(slot, Cf::TCOLS);
  oz_fence_before();
  __syncthreads();
  oz_fence_after();
  const uint32_t tmem = *slot;

  if (tid >= 256) {
    // ===================== producers =====================
    const int pt = tid - 256;
    // C once: column exponents, then the digits (B operand row l = output column l, K = rows of C)
    if (pt < q) {
      int e = 0;
      for (int k = 0; k < p; k++) e = max(e, oz_bexp(Cm[k * q + pt]));
      ec[pt] = e;
    }
    oz_named_sync(1, NP);
    for (int w = pt; w < NQ * (KP / 8); w += NP) {
      const int l = w % NQ, k8 = w / NQ;
      const int emax = l < q ? ec[l] : 0;
      uint32_t pk[OZ_S][4];
#pragma unroll
      for (int r = 0; r < 8; r += 2) {
        const int k = k8 * 8 + r;
        const double x0 = (l < q && k < p) ? Cm[k * q + l] : 0.0;
        const double x1 = (l < q && k + 1 < p) ? Cm[(k + 1) * q + l] : 0.0;
        uint32_t wv[OZ_S];
        oz_split2(x0, x1, emax, wv);
#pragma unroll
        for (int t = 0; t < OZ_S; t++) pk[t][r >> 1] = wv[t];
      }
      const uint32_t off = (uint32_t)(l >> 3) * Cf::SBO + (uint32_t)k8 * 128u + (uint32_t)(l & 7) * 16u;
#pragma unroll
      for (int t = 0; t < OZ_S; t++)
        *reinterpret_cast<uint4*>(sm + Cf::B0 + t * Cf::BSZ + off) = make_uint4(pk[t][0], pk[t][1], pk[t][2], pk[t][3]);
    }
    int k = 0;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, k++) {
      const int64_t i0 = tl * 128;
      const int rows = (int)((n - i0) < 128 ? (n - i0) : 128);
      // the tile's rows of A into raw, row stride rs = p | 1 (odd, so that consecutive rows fall in
      // different banks for the row-wise scans below); the previous tile's digits were written from
      // raw before `full`
      for (int i = pt >> 6; i < rows; i += NP >> 6)
        for (int c = pt & 63; c < p; c += 64) oz_cp8(raw + i * rs + c, A + (i0 + i) * lda + c, true);
      oz_cp_wait();
      // row exponents of tile k use the half of tile k - 2: wait until that one was read back
      if (k >= 2) {
        const long long t0 = clock64();
        while (*rcount < k - 1 && !*abort)
          if (clock64() - t0 > OZ_WAIT) *abort = 1;
      }
      oz_named_sync(1, NP);
      int* erk = er + (k & 1) * 128;
      if (pt < 128) {
        int e = 0;
        if (pt < rows)
          for (int c = 0; c < p; c++) e = max(e, oz_bexp(raw[pt * rs + c]));
        erk[pt] = e;
      }
      if (k >= 1) oz_wait2(done, (uint32_t)((k - 1) & 1), abort);  // previous MMAs read the A operand
      oz_named_sync(1, NP);
      if (*abort) break;
      // digits: item = (row t, octet k8); rows beyond the tile are zero
      for (int w = pt; w < 128 * (KP / 8); w += NP) {
        const int t = w & 127, k8 = w >> 7;
        const int emax = erk[t];
        uint32_t pk[OZ_S][4];
#pragma unroll
        for (int r = 0; r < 8; r += 2) {
          const int c = k8 * 8 + r;
          const double x0 = (t < rows && c < p) ? raw[t * rs + c] : 0.0;
          const double x1 = (t < rows && c + 1 < p) ? raw[t * rs + c + 1] : 0.0;
          uint32_t wv[OZ_S];
          oz_split2(x0, x1, emax, wv);
#pragma unroll
          for (int s = 0; s < OZ_S; s++) pk[s][r >> 1] = wv[s];
        }
        const uint32_t off = (uint32_t)(t >> 3) * Cf::SBO + (uint32_t)k8 * 128u + (uint32_t)(t & 7) * 16u;
#pragma unroll
        for (int s = 0; s < OZ_S; s++)
          *reinterpret_cast<uint4*>(sm + Cf::A0 + s * Cf::ASZ + off) = make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
      }
      oz_fence_proxy();
      oz_named_sync(1, NP);
      if (pt == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(oz_smem(full)) : "memory");
    }
  } else {
    // ===================== consumers =====================
    const int t = tid & 127, cb = (warp >> 2) * NH;
    const uint32_t sA = oz_smem(sm + Cf::A0), sB = oz_smem(sm + Cf::B0);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int k = 0;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x, k++) {
      if (tid == 0) {
        if (oz_wait2(full, (uint32_t)(k & 1), abort)) {
          oz_fence_after();
#pragma unroll
          for (int ks = 0; ks < KP / 16; ks++) oz_mma_step<NQ>(tmem, sA, Cf::ASZ, sB, Cf::BSZ, Cf::SBO, ks, ks == 0);
          oz_commit(done);
          *ncommit = k + 1;
        }
      }
      oz_wait2(done, (uint32_t)(k & 1), abort);
      oz_named_sync(2, 256);
      if (*abort) break;
      oz_fence_after();
      const int64_t row = tl * 128 + t;
      const int erow = er[(k & 1) * 128 + t];
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 8) {
        float v[OZ_LV][8];
#pragma unroll
        for (int L = 0; L < OZ_LV; L++) oz_ld8(tmem + lane_base + (uint32_t)(L * NQ + cb + c0), v[L]);
        oz_wait_ld();
        if (row < n) {
#pragma unroll
          for (int c = 0; c < 8; c++) {
            const int col = cb + c0 + c;
            if (col >= q) continue;
            float lv[OZ_LV];
#pragma unroll
            for (int L = 0; L < OZ_LV; L++) lv[L] = v[L][c];
            float vh, vl;
            oz_levels(lv, vh, vl);
            double y = (erow == 0 || ec[col] == 0) ? 0.0
                                                  : oz_df_to_f64(vh, vl, (erow - 1022) + (ec[col] - 1022) - 14);
            if (D) y += D[row * ldd + col];
            Y[row * ldy + col] = y;
          }
        }
      }
      oz_fence_before();
      oz_named_sync(2, 256);
      if (tid == 0) { __threadfence_block(); *rcount = k + 1; }
    }
  }
  __syncthreads();
  if (*abort) {
    if (tid == 0) atomicExch(&lob_oz_fault, 1);
    const int nc = *ncommit;
    if (nc > 0) oz_bar_wait(done, (uint32_t)((nc - 1) & 1), 1ll << 31);
  }
  oz_fence_before();
  __syncthreads();
  if (warp == 0) {
    oz_fence_after();
    oz_tmem_free(tmem, Cf::TCOLS);
  }
}

}  // namespace

// ---- launchers --------------------------------------------------------------------------------

// Doubles of workspace the tensor-core Gram needs (the CTAs' partial sums).
size_t lob_gram_oz_work_doubles() { return (size_t)256 * 2 * 64 * 64; }

bool lob_oz_fits(int p, int q) { return p >= 1 && p <= 64 && q >= 1 && q <= 64; }

// Whether the tensor-core kernels beat the double-float ones for this shape. Their cost is mostly
// a fixed pipeline cost per 64- or 128-row block, the double-float kernels' grows with p q; measured
// at n = 8,000,000 (ms, tensor cores / double-float): Gram 16 x 16 4.9 / 2.2, 16 x 32 5.2 / 5.7,
// 48 x 48 5.6 / 11.3; X C 16 -> 16 2.4 / 1.7, 32 -> 16 2.7 / 2.9, 48 -> 48 3.9 / 12.1.
bool lob_oz_pays(int p, int q) { return lob_oz_fits(p, q) && p * q >= 512; }

// G0 = L0^T R and, with L1, G1 = L1^T R (p x q each, row-major), FP64-class on the tensor cores.
int lob_gram_oz_launch(int64_t n, int p, const double* L0, int ld0, const double* L1, int ld1, int q,
                       const double* R, int ldr, double* G0, double* G1, double* work, cudaStream_t st) {
  if (!lob_oz_fits(p, q) || n < 0) return LOB_ERR_ARG;
  if (n == 0) {
    LOB_CUDA(cudaMemsetAsync(G0, 0, (size_t)p * q * 8, st));
    if (L1) LOB_CUDA(cudaMemsetAsync(G1, 0, (size_t)p * q * 8, st));
    return LOB_OK;
  }
  const int sms = lob_sm_count();
  if (sms < 0) return LOB_ERR_CUDA;
  const int64_t nchunks = (n + OZ_KC - 1) / OZ_KC;
  const int grid = (int)(nchunks < sms ? nchunks : (sms < 256 ? sms : 256));
  const int nq = (q + 15) / 16 * 16;
  const bool shared_r = (R == L0 && ldr == ld0 && q == p);
  const int rawc = p + (L1 ? p : 0) + (shared_r ? 0 : q);
  if (rawc <= (nq <= 48 ? OzG2<48>::RAWC : OzG2<64>::RAWC)) {  // the pipelined kernel (chunks of 64 rows)
    // bulk copies need 16-byte aligned rows and sizes: even widths and leading dimensions, aligned bases
    auto al16 = [](const void* ptr) { return ((uintptr_t)ptr & 15) == 0; };
    const int bulk = (p % 2 == 0 && q % 2 == 0 && ld0 % 2 == 0 && al16(L0) && (!L1 || (ld1 % 2 == 0 && al16(L1))) &&
                      (shared_r || (ldr % 2 == 0 && al16(R)))) ? 1 : 0;
    const int64_t nc2 = (n + OzG2<64>::KC - 1) / OzG2<64>::KC;
    const int grid2 = (int)(nc2 < sms ? nc2 : (sms < 256 ? sms : 256));
    auto go2 = [&](auto kern, uint32_t bytes) -> int {
      LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      (kern<<<grid2, 512, bytes, st>>>(n, p, L0, ld0, L1, ld1, q, R, ldr, work, bulk), LOB_LAUNCHED());
      return LOB_OK;
    };
    if (nq == 16) LOB_TRY(go2(k_gram_oz2<16>, OzG2<16>::BYTES));
    else if (nq == 32) LOB_TRY(go2(k_gram_oz2<32>, OzG2<32>::BYTES));
    else if (nq == 48) LOB_TRY(go2(k_gram_oz2<48>, OzG2<48>::BYTES));
    else LOB_TRY(go2(k_gram_oz2<64>, OzG2<64>::BYTES));
    const int nsel = L1 ? 2 : 1;
    (k_gram_oz_reduce<<<(nsel * p * q + 255) / 256, 256, 0, st>>>(grid2, nq, p, q, nsel, work, G0, G1),
     LOB_LAUNCHED());
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }
  auto go = [&](auto kern, uint32_t bytes) -> int {
    LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    (kern<<<grid, 256, bytes, st>>>(n, p, L0, ld0, L1, ld1, q, R, ldr, work), LOB_LAUNCHED());
    return LOB_OK;
  };
  if (nq == 16) LOB_TRY(go(k_gram_oz<16>, OzG<16>::BYTES));
  else if (nq == 32) LOB_TRY(go(k_gram_oz<32>, OzG<32>::BYTES));
  else if (nq == 48) LOB_TRY(go(k_gram_oz<48>, OzG<48>::BYTES));
  else LOB_TRY(go(k_gram_oz<64>, OzG<64>::BYTES));
  const int nsel = L1 ? 2 : 1;
  (k_gram_oz_reduce<<<(nsel * p * q + 255) / 256, 256, 0, st>>>(grid, nq, p, q, nsel, work, G0, G1), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

// Y = A C (+ D), FP64-class on the tensor cores (p, q <= 64).
int lob_lincomb_oz_launch(int64_t n, int p, const double* A, int lda, int q, const double* C, double* Y, int ldy,
                          cudaStream_t st, const double* D, int ldd) {
  if (!lob_oz_fits(p, q) || n < 0) return LOB_ERR_ARG;
  if (n == 0) return LOB_OK;
  const int nq = (q + 15) / 16 * 16, kp = (p + 15) / 16 * 16;
  {  // the pipelined kernel: persistent CTAs over tiles of 128 rows
    const int sms = lob_sm_count();
    if (sms < 0) return LOB_ERR_CUDA;
    const int64_t nt = (n + 127) / 128;
    const unsigned grid2 = (unsigned)(nt < sms ? nt : sms);
    auto go2 = [&](auto kern, uint32_t bytes) -> int {
      LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      (kern<<<grid2, 512, bytes, st>>>(n, p, A, lda, q, C, Y, ldy, D, ldd), LOB_LAUNCHED());
      LOB_CUDA(cudaGetLastError());
      return LOB_OK;
    };
#define LOB_OZ_L2(NQ_, KP_) \
    if (nq == NQ_ && kp == KP_) return go2(k_lincomb_oz2<NQ_, KP_>, OzL2<NQ_, KP_>::BYTES)
    LOB_OZ_L2(16, 16); LOB_OZ_L2(16, 32); LOB_OZ_L2(16, 48); LOB_OZ_L2(16, 64);
    LOB_OZ_L2(32, 16); LOB_OZ_L2(32, 32); LOB_OZ_L2(32, 48); LOB_OZ_L2(32, 64);
    LOB_OZ_L2(48, 16); LOB_OZ_L2(48, 32); LOB_OZ_L2(48, 48);
    LOB_OZ_L2(64, 16); LOB_OZ_L2(64, 32);
#undef LOB_OZ_L2
  }
  const unsigned grid = (unsigned)((n + 127) / 128);
  // Shared memory is requested so that no more CTAs share an SM than its 512 tensor-memory columns
  // can hold at once (a CTA whose allocation would not fit waits in tcgen05.alloc otherwise).
  auto go = [&](auto kern, uint32_t bytes, uint32_t tcols) -> int {
    const uint32_t per_sm = 512u / tcols, floor_bytes = 233472u / (per_sm + 1u);
    if (bytes < floor_bytes) bytes = floor_bytes;
    LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    (kern<<<grid, 128, bytes, st>>>(n, p, A, lda, q, C, Y, ldy, D, ldd), LOB_LAUNCHED());
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  };
#define LOB_OZ_L(NQ_, KP_) \
  if (nq == NQ_ && kp == KP_) return go(k_lincomb_oz<NQ_, KP_>, OzL<NQ_, KP_>::BYTES, OzL<NQ_, KP_>::TCOLS)
  LOB_OZ_L(16, 16); LOB_OZ_L(16, 32); LOB_OZ_L(16, 48); LOB_OZ_L(16, 64);
  LOB_OZ_L(32, 16); LOB_OZ_L(32, 32); LOB_OZ_L(32, 48); LOB_OZ_L(32, 64);
  LOB_OZ_L(48, 16); LOB_OZ_L(48, 32); LOB_OZ_L(48, 48); LOB_OZ_L(48, 64);
  LOB_OZ_L(64, 16); LOB_OZ_L(64, 32); LOB_OZ_L(64, 48); LOB_OZ_L(64, 64);
#undef LOB_OZ_L
  return LOB_ERR_ARG;
}

// Nonzero once a tensor-core block product gave up on a bounded wait since the last call (then
// cleared), -1 if the read failed; synchronises st.
int lob_oz_fault_take(cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyFromSymbolAsync(&h, lob_oz_fault, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  if (h) {
    const int z = 0;
    if (cudaMemcpyToSymbolAsync(lob_oz_fault, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
  }
  return h;
}


