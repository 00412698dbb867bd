// Symmetric SpMM Y = H X over the upper-triangle tile store (Sections 4.1-4.2).
//
// Every stored tile T_IJ contributes Y_I += T_IJ X_J and, off the diagonal tile, also
// Y_J += T_IJ^T X_I -- the paper's row pass and column pass over the CSB pointer array,
// fused here into a single pass so each tile streams from HBM once. On a diagonal tile the
// entries with r != c are applied both ways and the diagonal once.
//
// Schedule: one CTA per tile row I. X_I (256 rows) stays in shared memory for the whole row;
// the row's tiles are streamed in chunks of up to LOB_PERM_CHUNK entries -- the records, the chunk's
// column-order permutation, the chunk's row and column start pointers (both derived once at
// create time from the canonical store), and X_J for a new tile -- with cp.async, the next
// chunk loading while the current one computes. A lane group of NB/VW lanes (VW elements =
// 16 bytes, one 16-byte slice of a row of X per lane) owns in-tile row a and column a for all
// tiles of the row:
//   row pass    Y_I[a] += sum_c v X_J[c] over row a's entries, summed in registers;
//   column pass Y_J[a] += sum_r v X_I[r] over column a's entries (via the permutation).
// No shared-memory accumulators and no shared-memory atomics (FP32 ones are emulated on this
// GPU). Column partials go to Y with FP64 atomics in L2 after each tile; row partials are
// summed across the row's tiles in registers and written once per tile row, so every sum
// across tiles is done in FP64 (or double-float) and the order of all sums is fixed.
//
// MIXED: FP32 values, X rounded to FP32 (once per call), FP32 products and in-tile sums; the
// row side's tile partials are summed across the tiles of the row in double-float, and all
// cross-tile sums in Y are FP64 (footnote 5 of Section 4.4). FP64: every operation in FP64.
#include "common.cuh"
#include "df.cuh"

// Staged-X scratch of a matrix (grown on demand, owned by the matrix).
int lob_ensure_xs(const lob_matrix* m, size_t need) {
  lob_matrix* mm = const_cast<lob_matrix*>(m);
  if (mm->xs_bytes >= need) return LOB_OK;
  cudaFree(mm->xs);
  mm->xs = nullptr;
  mm->xs_bytes = 0;
  if (cudaMalloc(&mm->xs, need) != cudaSuccess) { cudaGetLastError(); return LOB_ERR_NOMEM; }
  mm->xs_bytes = need;
  return LOB_OK;
}

namespace {

template <bool MIXED>
struct Elt;
template <>
struct Elt<true> {
  using T = float;
  using V = float4;  // 16-byte slice: 4 vector columns
  static constexpr int VW = 4;
};
template <>
struct Elt<false> {
  using T = double;
  using V = double2;
  static constexpr int VW = 2;
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void fma_v(float4& a, float v, const float4& x) {
  a.x = fmaf(v, x.x, a.x); a.y = fmaf(v, x.y, a.y); a.z = fmaf(v, x.z, a.z); a.w = fmaf(v, x.w, a.w);
}
__device__ __forceinline__ void fma_v(double2& a, double v, const double2& x) {
  a.x = fma(v, x.x, a.x); a.y = fma(v, x.y, a.y);
}
__device__ __forceinline__ void zero_v(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void zero_v(double2& a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ void mul_v(float4& a, float v, const float4& x) {
  a.x = v * x.x; a.y = v * x.y; a.z = v * x.z; a.w = v * x.w;
}
__device__ __forceinline__ void mul_v(double2& a, double v, const double2& x) { a.x = v * x.x; a.y = v * x.y; }

// FP64 -> FP32 round-to-nearest-even with integer operations (normal FP32 range; other
// magnitudes take the conversion instruction).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 897 || e > 1149) return __double2float_rn(x);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long r = mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull);  // ties to even at bit 29
  const unsigned bits = (unsigned)(r >> 29) - (896u << 23);
  return __uint_as_float(bits | ((unsigned)(b >> 32) & 0x80000000u));
}

// Columns [c0, c0 + w) of X (n x nb FP64) -> Xs (rows x NB, element type T); zero in padded
// columns and in rows >= n_act.
template <typename T>
__global__ void k_stage_x(int64_t rows, int64_t n_act, int nb, int c0, int w, int NB, const double* __restrict__ X,
                          T* __restrict__ Xs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * NB) return;
  const int64_t i = t / NB;
  const int j = (int)(t % NB);
  const double v = (j < w && i < n_act) ? X[i * nb + c0 + j] : 0.0;
  if constexpr (sizeof(T) == 4)
    Xs[t] = f64_to_f32_rn(v);
  else
    Xs[t] = v;
}

// Launch shape and shared-memory layout (byte offsets) of the SpMM kernel. A lane group of
// G = NB / VW lanes handles one entry at a time; the CTA has NG = THREADS / G groups and group g
// owns the in-tile rows and columns g, g + NG, ... (RPG of each) for every tile of its tile row.
template <bool MIXED, int NB>
struct Cfg {
  using T = typename Elt<MIXED>::T;
  static constexpr int VW = Elt<MIXED>::VW;
  static constexpr int G = NB / VW;
  static constexpr int CH = LOB_PERM_CHUNK;
  static constexpr int PTRS = 2 * (LOB_TILE + 1);  // row starts then column starts, uint16
  static constexpr size_t XV = sizeof(T) * LOB_TILE * NB;
  static constexpr size_t XI = 0;
  static constexpr size_t XJ = XI + XV;               // 2 buffers
  static constexpr size_t RC = XJ + 2 * XV;           // 2 x CH uint32
  static constexpr size_t VV = RC + 2 * 4 * CH;       // 2 x CH values
  static constexpr size_t PM = VV + 2 * sizeof(T) * CH;    // 2 x (CH + 8) uint16
  static constexpr size_t PT = PM + 2 * 2 * (CH + 8);      // 2 x PTRS uint16
  static constexpr size_t BYTES = PT + 2 * 2 * PTRS;
  // one CTA per SM: 1,024 threads, one in-tile row and column per lane group at NB = 16 (a
  // variant with two 512-thread CTAs per SM and 2,048-entry chunks measured 15% slower)
  static constexpr int MINB = 1;
  static constexpr int THREADS = (LOB_TILE * G) < 1024 ? (LOB_TILE * G) : 1024;
  static constexpr int NG = THREADS / G;
  static constexpr int RPG = LOB_TILE / NG;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void atomic_out(double* y, float v) { if (v != 0.f) atomicAdd(y, f32_to_f64(v)); }
__device__ __forceinline__ void atomic_out(double* y, double v) { if (v != 0.0) atomicAdd(y, v); }

// One CTA per tile row I (see the file comment). Group g, for each owned in-tile index a:
//   row pass    acc_t[a] += v X_J[c] over the entries of row a (chunk order (r, c)), FP32 in MIXED;
//               at tile end acc_t is added to the row accumulator (double-float in MIXED);
//   column pass acc_c[a] += v X_I[r] over the entries of column a (order (c, r)); at tile end
//               it goes to Y_J with FP64 atomics, or, on the diagonal tile, into the row
//               accumulator (row a and column a have the same owner).
// Nothing is accumulated in shared memory and no shared-memory atomics are used.
template <bool MIXED, int NB>
__global__ void __launch_bounds__(Cfg<MIXED, NB>::THREADS, Cfg<MIXED, NB>::MINB)
    k_spmm4(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol, const int64_t* __restrict__ tptr,
            const int32_t* __restrict__ tchunk, const uint32_t* __restrict__ rc,
            const typename Elt<MIXED>::T* __restrict__ vals, const uint16_t* __restrict__ cperm,
            const uint16_t* __restrict__ cptrs, const typename Elt<MIXED>::T* __restrict__ Xs,
            double* __restrict__ Y, int ldy, int c0, int w, int64_t n_act, const lob_spmm_job* __restrict__ jobs,
            int njobs) {
  using C = Cfg<MIXED, NB>;
  using T = typename C::T;
  using V = typename Elt<MIXED>::V;
  constexpr int VW = C::VW, G = C::G, NG = C::NG, RPG = C::RPG, CH = C::CH, THREADS = C::THREADS;
  constexpr int XN = LOB_TILE * NB;
  constexpr int EPT = 16 / (int)sizeof(T);  // elements per 16-byte copy
  extern __shared__ __align__(16) unsigned char sm[];
  T* XI = reinterpret_cast<T*>(sm + C::XI);
  T* XJb = reinterpret_cast<T*>(sm + C::XJ);
  uint32_t* RCb = reinterpret_cast<uint32_t*>(sm + C::RC);
  T* VVb = reinterpret_cast<T*>(sm + C::VV);
  uint16_t* PMb = reinterpret_cast<uint16_t*>(sm + C::PM);
  uint16_t* PTb = reinterpret_cast<uint16_t*>(sm + C::PT);

  int64_t I = blockIdx.x;
  if (jobs) {  // batched launch: find this CTA's matrix and tile row
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].cta_begin <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const lob_spmm_job& jb = jobs[lo];
    rowptr = jb.rowptr; tcol = jb.tcol; tptr = jb.tptr; tchunk = jb.tchunk; rc = jb.rc;
    vals = reinterpret_cast<const T*>(jb.vals); cperm = jb.cperm; cptrs = jb.cptrs;
    Xs = reinterpret_cast<const T*>(jb.Xs); Y = jb.Y; ldy = jb.ldy; c0 = jb.c0; w = jb.w; n_act = jb.n_act;
    I = (int64_t)blockIdx.x - jb.cta_begin;
  }
  const int64_t row0 = I * LOB_TILE;
  const int tid = threadIdx.x;
  const int g = tid / G, gl = tid % G;
  const int64_t t0 = rowptr[I];
  int64_t t1 = rowptr[I + 1];
  while (t1 > t0 && (int64_t)tcol[t1 - 1] * LOB_TILE >= n_act) t1--;  // tiles outside the active block

  for (int e = tid * EPT; e < XN; e += THREADS * EPT) cp_async16(&XI[e], &Xs[row0 * NB + e]);
  cp_async_commit();

  auto issue = [&](int64_t t, int64_t k, int buf, int xbuf) {
    const int64_t J = tcol[t];
    if (k == 0 && J != I) {
      T* XJ = XJb + xbuf * XN;
      const T* src = Xs + J * LOB_TILE * NB;
      for (int e = tid * EPT; e < XN; e += THREADS * EPT) cp_async16(&XJ[e], &src[e]);
    }
    const int64_t base = tptr[t] + k * CH;
    const int64_t rem = tptr[t + 1] - base;
    const int cnt = (int)(rem < CH ? rem : CH);
    uint32_t* RCs = RCb + buf * CH;
    T* VVs = VVb + buf * CH;
    for (int i = tid; i < cnt; i += THREADS) {
      cp_async4(&RCs[i], &rc[base + i]);
      if (MIXED) cp_async4(&VVs[i], &vals[base + i]); else cp_async8(&VVs[i], &vals[base + i]);
    }
    uint32_t* PM32 = reinterpret_cast<uint32_t*>(PMb + buf * (CH + 8));
    const int64_t wb = base & ~(int64_t)1;
    const int nwords = (int)((base + cnt - wb + 1) / 2);
    const uint32_t* src32 = reinterpret_cast<const uint32_t*>(cperm + wb);
    for (int i = tid; i < nwords; i += THREADS) cp_async4(&PM32[i], &src32[i]);
    uint32_t* PT32 = reinterpret_cast<uint32_t*>(PTb + buf * C::PTRS);
    const uint32_t* srcp = reinterpret_cast<const uint32_t*>(cptrs + (int64_t)(tchunk[t] + k) * C::PTRS);
    for (int i = tid; i < C::PTRS / 2; i += THREADS) cp_async4(&PT32[i], &srcp[i]);
    cp_async_commit();
  };

  // accumulators of the owned rows/columns
  V acc_t[RPG], acc_c[RPG];
  float rh[RPG][VW], rl[RPG][VW];  // MIXED: row accumulator (double-float)
  double rd[RPG][VW];              // FP64: row accumulator
#pragma unroll
  for (int a = 0; a < RPG; a++) {
    zero_v(acc_t[a]); zero_v(acc_c[a]);
#pragma unroll
    for (int q = 0; q < VW; q++) { rh[a][q] = 0.f; rl[a][q] = 0.f; rd[a][q] = 0.0; }
  }

  int64_t t = t0, k = 0;
  int tl = 0, buf = 0;
  if (t < t1) issue(t, 0, 0, 0);
  while (t < t1) {
    const int64_t J = tcol[t];
    const bool diag = (J == I);
    const bool last = (tptr[t] + (k + 1) * CH >= tptr[t + 1]);
    int64_t tn = t, kn = k + 1;
    int tln = tl;
    if (last) { tn = t + 1; kn = 0; tln = tl + 1; }
    if (tn < t1) { issue(tn, kn, buf ^ 1, tln & 1); cp_async_wait_1(); } else { cp_async_wait_all(); }
    __syncthreads();
    const uint32_t* RCs = RCb + buf * CH;
    const T* VVs = VVb + buf * CH;
    const uint16_t* PM = PMb + buf * (CH + 8) + (int)((tptr[t] + k * CH) & 1);
    const uint16_t* PR = PTb + buf * C::PTRS;
    const uint16_t* PC = PR + (LOB_TILE + 1);
    const T* xj = diag ? XI : XJb + (tl & 1) * XN;
#pragma unroll
    for (int a = 0; a < RPG; a++) {
      const int idx = g + a * NG;
      // row pass
      {
        const int s = PR[idx], e = PR[idx + 1];
        V acc = acc_t[a];
#pragma unroll 4
        for (int i = s; i < e; i++) {
          const int c = (int)(RCs[i] & 0xFFFFu);
          const V x = *reinterpret_cast<const V*>(&xj[c * NB + gl * VW]);
          fma_v(acc, VVs[i], x);
        }
        acc_t[a] = acc;
      }
      // column pass
      {
        const int s = PC[idx], e = PC[idx + 1];
        V acc = acc_c[a];
#pragma unroll 4
        for (int i = s; i < e; i++) {
          const int q = PM[i] & (CH - 1);  // a chunk-local index (mask keeps a stray value inside the chunk)
          const int r = (int)(RCs[q] >> 16);
          if (diag && r == idx) continue;  // the diagonal entry is applied once (row pass)
          const V xi = *reinterpret_cast<const V*>(&XI[r * NB + gl * VW]);
          fma_v(acc, VVs[q], xi);
        }
        acc_c[a] = acc;
      }
    }
    if (last) {
#pragma unroll
      for (int a = 0; a < RPG; a++) {
        const int idx = g + a * NG;
        const T* ta = reinterpret_cast<const T*>(&acc_t[a]);
        const T* ca = reinterpret_cast<const T*>(&acc_c[a]);
#pragma unroll
        for (int q = 0; q < VW; q++) {
          if (MIXED) {
            df_add(rh[a][q], rl[a][q], (float)ta[q], 0.f);
            if (diag) df_add(rh[a][q], rl[a][q], (float)ca[q], 0.f);
          } else {
            rd[a][q] += (double)ta[q];
            if (diag) rd[a][q] += (double)ca[q];
          }
          const int kk = gl * VW + q;
          const int64_t gr = J * LOB_TILE + idx;
          if (!diag && kk < w && gr < n_act) atomic_out(&Y[gr * ldy + c0 + kk], ca[q]);
        }
        zero_v(acc_t[a]);
        zero_v(acc_c[a]);
      }
    }
    __syncthreads();  // this buffer is refilled two chunks from now
    t = tn; k = kn; tl = tln; buf ^= 1;
  }
  cp_async_wait_all();
#pragma unroll
  for (int a = 0; a < RPG; a++) {
    const int64_t gr = row0 + g + a * NG;
#pragma unroll
    for (int q = 0; q < VW; q++) {
      const int kk = gl * VW + q;
      if (kk >= w || gr >= n_act) continue;
      if (MIXED) {
        if (rh[a][q] != 0.f) atomicAdd(&Y[gr * ldy + c0 + kk], f32_to_f64(rh[a][q]));
        if (rl[a][q] != 0.f) atomicAdd(&Y[gr * ldy + c0 + kk], f32_to_f64(rl[a][q]));
      } else {
        if (rd[a][q] != 0.0) atomicAdd(&Y[gr * ldy + c0 + kk], rd[a][q]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Ring-pipelined variant of the FP32-value product (MIXED, NB = 16): same ownership and
// arithmetic as k_spmm4, without its two CTA-wide barriers per chunk.
//
// Each CTA is persistent and takes a contiguous range of tile rows holding about 1/grid of the
// stored entries. The chunks of that range pass through a ring of D shared-memory stages. A
// stage is filled by bulk async copies ((record, value) pairs, permutation, chunk pointers, X_J)
// that complete on the stage's mbarrier; a warp waits on that barrier, works the chunk, and
// counts itself out of the stage with a shared-memory counter. The warp that counts out last
// refills the stage with the chunk D places further on. So warps drift apart by up to D chunks
// instead of meeting at every chunk: the work of a lane group differs from chunk to chunk (the
// row and column counts of a tile are uneven) and the slack absorbs most of it. X_I has two
// slots, refilled the same way by the last warp to finish a tile row.
//
// Every wait is bounded by the launch's `limit` (SM clocks; about 2^32 by default, settable per
// matrix at create). A wait that runs out sets bit 0 of the matrix's status word and the CTA's
// abort flag; every warp then leaves at its next wait (or right away if it is waiting), no new copy
// is issued, and the last warp of the CTA to leave waits -- with its own bound -- for every copy
// the CTA issued to land before the CTA ends, so no bulk copy is still writing shared memory that
// the next CTA on the SM may own. The same last-warp drain runs on the normal exit, where every
// issued copy has already been consumed.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bulk global -> shared copy completing on bar; addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// Shared-memory control words of a ring kernel's abort protocol.
struct RingCtl {
  int abort;        // set once any warp of the CTA gave up on a wait
  int left;         // warps that have left the main loop
  int issued[8];    // fills issued per ring stage (at most 6 stages) and X_I slot (2)
};

// Wait, with the whole warp, for the completion of the phase with the given parity. Every lane
// waits (each acquires the copied data); the outcome is warp-uniform. False if the wait ran out
// (the status word and the CTA's abort flag are then set) or another warp already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit, RingCtl* ctl,
                                          int* status) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    if (__all_sync(0xffffffffu, mbar_test(a, parity))) return true;
    const bool give_up = clock64() - t0 > limit || *(volatile int*)&ctl->abort != 0;
    if (__any_sync(0xffffffffu, give_up)) {
      if ((threadIdx.x & 31) == 0 && atomicExch(&ctl->abort, 1) == 0) atomicOr(status, 1);
      return false;
    }
  }
}

// Leave the ring: the last warp of the CTA waits (bounded; the copies were issued and complete in
// microseconds unless the memory system failed) for the latest fill of every stage and slot it
// ever issued. nslots = ring stages + X_I slots, bars[i] their mbarriers (stages first).
__device__ __forceinline__ void ring_leave(RingCtl* ctl, uint64_t* bars, int nslots, int nwarps) {
  __syncwarp();
  int last = 0;
  if ((threadIdx.x & 31) == 0) {
    __threadfence_block();
    last = atomicAdd(&ctl->left, 1) == nwarps - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence_block();
  for (int i = 0; i < nslots; i++) {
    const int k = *(volatile int*)&ctl->issued[i];
    if (k == 0) continue;
    const uint32_t a = smem_u32(&bars[i]);
    const long long t0 = clock64();
    while (!__all_sync(0xffffffffu, mbar_test(a, (uint32_t)((k - 1) & 1))))
      if (__any_sync(0xffffffffu, clock64() - t0 > (1ll << 31))) break;
  }
}

// The chunk walk of one CTA: tile rows [I, Ie), in each the tiles left after trimming to the
// active rows, in each tile its chunks.
struct RingCur {
  int64_t I, Ie, t, t1;
  int32_t k, nk;
};

template <int NB>
struct CfgR {
  static constexpr int VW = 4;  // FP32 vector columns per lane (one 16-byte slice)
  static constexpr int G = NB / VW;
  static constexpr int THREADS = LOB_TILE * G;  // one lane group per in-tile row and column
  static constexpr int NW = THREADS / 32;
  static constexpr int D = 3;  // ring stages
  static constexpr int CH = LOB_PERM_CHUNK;
  static constexpr int PTRS = 2 * (LOB_TILE + 1);
  static constexpr size_t XV = sizeof(float) * LOB_TILE * NB;
  // one stage: (record, value) pairs (16-byte aligned window around the chunk), permutation,
  // chunk pointers, X_J
  static constexpr size_t S_RV = 0;
  static constexpr size_t S_PM = S_RV + 8 * (CH + 8);
  static constexpr size_t S_PT = S_PM + 2 * (CH + 16);
  static constexpr size_t S_XJ = (S_PT + 2 * PTRS + 32 + 15) / 16 * 16;
  static constexpr size_t STAGE = S_XJ + XV;
  static constexpr size_t XI = 0;              // two X_I slots
  static constexpr size_t ST = XI + 2 * XV;    // D stages
  static constexpr size_t BAR = ST + D * STAGE;  // full[D], xfull[2] (8 B each)
  static constexpr size_t RNG = BAR + 8 * (D + 2);  // this CTA's tile rows [Ib, Ie)
  static constexpr size_t CUR = RNG + 16;           // the refill cursor
  static constexpr size_t CNT = CUR + 48;           // stage and X_I counters
  static constexpr size_t CTL = (CNT + 4 * (D + 2) + 7) / 8 * 8;  // abort protocol (RingCtl)
  static constexpr size_t BYTES = CTL + sizeof(RingCtl);
  static_assert(VW * G == NB && THREADS <= 1024 && THREADS % 32 == 0, "launch shape");
  static_assert(sizeof(RingCur) <= 48, "cursor slot");
  static_assert(S_PM % 16 == 0 && S_PT % 16 == 0 && STAGE % 16 == 0 && ST % 16 == 0,
                "bulk copy destinations must be 16-byte aligned");
};

__device__ __forceinline__ int64_t ring_trim(const int64_t* rowptr, const int32_t* tcol, int64_t n_act, int64_t I,
                                             int64_t* t0) {
  *t0 = rowptr[I];
  int64_t t1 = rowptr[I + 1];
  while (t1 > *t0 && (int64_t)tcol[t1 - 1] * LOB_TILE >= n_act) t1--;
  return t1;
}

// Move c to the first chunk at or after its position (k == nk means "past this tile").
// Returns false at the end of the range.
__device__ __forceinline__ bool ring_settle(RingCur& c, const int64_t* rowptr, const int32_t* tcol,
                                           const int32_t* tchunk, int64_t n_act) {
  while (c.k >= c.nk) {
    c.t++;
    c.k = 0;
    while (c.t >= c.t1) {
      c.I++;
      if (c.I >= c.Ie) return false;
      int64_t t0;
      c.t1 = ring_trim(rowptr, tcol, n_act, c.I, &t0);
      c.t = t0;
    }
    c.nk = tchunk[c.t + 1] - tchunk[c.t];
  }
  return true;
}

// Issue the copies of chunk (t, k) of tile row I into a stage.
template <int NB>
__device__ __forceinline__ void ring_issue(unsigned char* stage, uint64_t* bar, int64_t I, int64_t t, int k,
                                           const int32_t* tcol, const int64_t* tptr, const int32_t* tchunk,
                                           const uint2* rv, const uint16_t* cperm, const uint16_t* cptrs,
                                           const float* Xs) {
  using C = CfgR<NB>;
  const int64_t J = tcol[t];
  const int64_t base = tptr[t] + (int64_t)k * C::CH;
  const int64_t rem = tptr[t + 1] - base;
  const int64_t cnt = rem < C::CH ? rem : C::CH;
  const int64_t a0 = base & ~(int64_t)1, e1 = (base + cnt + 1) & ~(int64_t)1;      // 8-byte pairs
  const int64_t p0 = base & ~(int64_t)7, p1 = (base + cnt + 7) & ~(int64_t)7;      // 2-byte array
  const int64_t bo = (int64_t)(tchunk[t] + k) * (C::PTRS * 2);                     // chunk pointers, bytes
  const int64_t q0 = bo & ~(int64_t)15, q1 = (bo + C::PTRS * 2 + 15) & ~(int64_t)15;
  const uint32_t brv = (uint32_t)((e1 - a0) * 8), bpm = (uint32_t)((p1 - p0) * 2), bpt = (uint32_t)(q1 - q0);
  const uint32_t bxj = (J != I) ? (uint32_t)C::XV : 0u;
  mbar_expect_tx(bar, brv + bpm + bpt + bxj);
  bulk_g2s(stage + C::S_RV, rv + a0, brv, bar);
  bulk_g2s(stage + C::S_PM, cperm + p0, bpm, bar);
  bulk_g2s(stage + C::S_PT, reinterpret_cast<const unsigned char*>(cptrs) + q0, bpt, bar);
  if (bxj) bulk_g2s(stage + C::S_XJ, Xs + J * LOB_TILE * NB, bxj, bar);
}

template <int NB>
__global__ void __launch_bounds__(CfgR<NB>::THREADS, 1)
    k_spmm_ring(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol,
                const int64_t* __restrict__ tptr, const int32_t* __restrict__ tchunk,
                const uint2* __restrict__ rv, const uint16_t* __restrict__ cperm,
                const uint16_t* __restrict__ cptrs, const float* __restrict__ Xs, double* __restrict__ Y, int ldy,
                int c0, int w, int64_t n_act, int64_t ntr, int* __restrict__ status, long long limit, int poison) {
  using C = CfgR<NB>;
  constexpr int VW = C::VW, G = C::G, NW = C::NW, D = C::D, CH = C::CH;
  constexpr int XN = LOB_TILE * NB;
  extern __shared__ __align__(16) unsigned char sm[];
  float* XIb = reinterpret_cast<float*>(sm + C::XI);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::BAR);
  uint64_t* xfull = full + D;
  int* cnt = reinterpret_cast<int*>(sm + C::CNT);
  int* xcnt = cnt + D;
  int64_t* range = reinterpret_cast<int64_t*>(sm + C::RNG);
  RingCur* cur = reinterpret_cast<RingCur*>(sm + C::CUR);
  RingCtl* ctl = reinterpret_cast<RingCtl*>(sm + C::CTL);
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = tid / G, gl = tid % G;
  static_assert(D + 2 <= 8, "RingCtl slots");

  if (tid == 0) {
    ctl->abort = 0;
    ctl->left = 0;
    for (int i = 0; i < 8; i++) ctl->issued[i] = 0;
    // this CTA's tile rows: entries before row I are tptr[rowptr[I]]; split them evenly
    const int64_t E = tptr[rowptr[ntr]];
    auto first_row = [&](int64_t b) -> int64_t {
      if (b >= (int64_t)gridDim.x) return ntr;
      const int64_t target = E * b / (int64_t)gridDim.x;
      int64_t lo = 0, hi = ntr;  // first I with tptr[rowptr[I]] >= target
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tptr[rowptr[mid]] >= target) hi = mid; else lo = mid + 1;
      }
      return lo;
    };
    range[0] = first_row(blockIdx.x);
    range[1] = first_row((int64_t)blockIdx.x + 1);
    for (int s = 0; s < D; s++) { mbar_init(&full[s], 1); cnt[s] = 0; }
    for (int s = 0; s < 2; s++) { mbar_init(&xfull[s], 1); xcnt[s] = 0; }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const int64_t Ib = range[0], Ie = range[1];
  if (tid == 0 && Ib < Ie) {
    for (int s = 0; s < 2 && Ib + s < Ie; s++) {
      ctl->issued[D + s]++;
      mbar_expect_tx(&xfull[s], (uint32_t)C::XV);
      bulk_g2s(XIb + s * XN, Xs + (Ib + s) * LOB_TILE * NB, (uint32_t)C::XV, &xfull[s]);
    }
    RingCur c;
    c.I = Ib; c.Ie = Ie;
    int64_t t0;
    c.t1 = ring_trim(rowptr, tcol, n_act, Ib, &t0);
    c.t = t0 - 1; c.k = 0; c.nk = 0;  // settle moves to the first chunk
    bool more = ring_settle(c, rowptr, tcol, tchunk, n_act);
    for (int s = 0; s < D && more; s++) {
      if (poison && s == 0) {  // test mode: stage 0 expects bytes that nothing sends (nothing in flight)
        mbar_expect_tx(&full[0], 16u);
      } else {
        ctl->issued[s]++;
        ring_issue<NB>(sm + C::ST + s * C::STAGE, &full[s], c.I, c.t, c.k, tcol, tptr, tchunk, rv, cperm, cptrs, Xs);
      }
      c.k++;
      more = ring_settle(c, rowptr, tcol, tchunk, n_act);
    }
    if (!more) c.I = Ie;
    *cur = c;
  }
  __syncthreads();

  int64_t ch = 0;  // chunks this CTA has worked so far
  for (int64_t I = Ib; I < Ie; I++) {
    const int64_t ri = I - Ib;
    const int xs = (int)(ri & 1);
    if (!mbar_wait(&xfull[xs], (uint32_t)((ri >> 1) & 1), limit, ctl, status)) goto leave;
    const float* XI = XIb + xs * XN;
    int64_t t0;
    const int64_t t1 = ring_trim(rowptr, tcol, n_act, I, &t0);
    float rh[VW], rl[VW];
#pragma unroll
    for (int q = 0; q < VW; q++) { rh[q] = 0.f; rl[q] = 0.f; }
    for (int64_t t = t0; t < t1; t++) {
      const int64_t J = tcol[t];
      const bool diag = (J == I);
      const int nk = tchunk[t + 1] - tchunk[t];
      float4 acc_t = make_float4(0.f, 0.f, 0.f, 0.f), acc_c = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int k = 0; k < nk; k++) {
        const int s = (int)(ch % D);
        if (!mbar_wait(&full[s], (uint32_t)((ch / D) & 1), limit, ctl, status)) goto leave;
        unsigned char* stage = sm + C::ST + s * C::STAGE;
        const int64_t base = tptr[t] + (int64_t)k * CH;
        const uint2* RV = reinterpret_cast<const uint2*>(stage + C::S_RV) + (base & 1);
        const uint16_t* PM = reinterpret_cast<const uint16_t*>(stage + C::S_PM) + (base & 7);
        const int64_t bo = (int64_t)(tchunk[t] + k) * (C::PTRS * 2);
        const uint16_t* PR = reinterpret_cast<const uint16_t*>(stage + C::S_PT + (bo & 15));
        const uint16_t* PC = PR + (LOB_TILE + 1);
        const float* xj = diag ? XI : reinterpret_cast<const float*>(stage + C::S_XJ);
        {  // row pass
          const int s0 = PR[g], e0 = PR[g + 1];
          float4 acc = acc_t;
#pragma unroll 3  // 4 spills at the 64-register limit of 1,024 threads
          for (int i = s0; i < e0; i++) {
            const uint2 e = RV[i];
            const int c = (int)(e.x & 0xFFFFu);
            const float4 x = *reinterpret_cast<const float4*>(&xj[c * NB + gl * VW]);
            fma_v(acc, __uint_as_float(e.y), x);
          }
          acc_t = acc;
        }
        {  // column pass
          const int s0 = PC[g], e0 = PC[g + 1];
          float4 acc = acc_c;
#pragma unroll 4
          for (int i = s0; i < e0; i++) {
            const uint2 e = RV[PM[i] & (CH - 1)];
            const int r = (int)(e.x >> 16);
            if (diag && r == g) continue;  // the diagonal entry is applied once (row pass)
            const float4 xi = *reinterpret_cast<const float4*>(&XI[r * NB + gl * VW]);
            fma_v(acc, __uint_as_float(e.y), xi);
          }
          acc_c = acc;
        }
        // count this warp out of the stage; the last one refills it with the chunk D places on
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          const int old = atomicAdd(&cnt[s], 1);
          if (old == NW * (int)(ch / D + 1) - 1) {
            __threadfence_block();
            RingCur c = *cur;
            if (c.I < c.Ie && *(volatile int*)&ctl->abort == 0) {
              asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
              ctl->issued[s]++;
              ring_issue<NB>(stage, &full[s], c.I, c.t, c.k, tcol, tptr, tchunk, rv, cperm, cptrs, Xs);
              c.k++;
              if (!ring_settle(c, rowptr, tcol, tchunk, n_act)) c.I = c.Ie;
              *cur = c;
            }
            __threadfence_block();
          }
        }
        ch++;
      }
      // tile end: column partials to Y_J (FP64 atomics), row partials into the row accumulator
      const float* ta = reinterpret_cast<const float*>(&acc_t);
      const float* ca = reinterpret_cast<const float*>(&acc_c);
#pragma unroll
      for (int q = 0; q < VW; q++) {
        df_add(rh[q], rl[q], ta[q], 0.f);
        if (diag) df_add(rh[q], rl[q], ca[q], 0.f);
        const int kk = gl * VW + q;
        const int64_t gr = J * LOB_TILE + g;
        if (!diag && kk < w && gr < n_act) atomic_out(&Y[gr * ldy + c0 + kk], ca[q]);
      }
    }
    // tile row end: row sums to Y_I
    const int64_t gr = I * LOB_TILE + g;
#pragma unroll
    for (int q = 0; q < VW; q++) {
      const int kk = gl * VW + q;
      if (kk >= w || gr >= n_act) continue;
      if (rh[q] != 0.f) atomicAdd(&Y[gr * ldy + c0 + kk], f32_to_f64(rh[q]));
      if (rl[q] != 0.f) atomicAdd(&Y[gr * ldy + c0 + kk], f32_to_f64(rl[q]));
    }
    // count this warp out of the X_I slot; the last one loads the row two places on into it
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      const int old = atomicAdd(&xcnt[xs], 1);
      if (old == NW * (int)((ri >> 1) + 1) - 1 && I + 2 < Ie && *(volatile int*)&ctl->abort == 0) {
        __threadfence_block();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        ctl->issued[D + xs]++;
        mbar_expect_tx(&xfull[xs], (uint32_t)C::XV);
        bulk_g2s(XIb + xs * XN, Xs + (I + 2) * LOB_TILE * NB, (uint32_t)C::XV, &xfull[xs]);
      }
    }
  }
leave:
  ring_leave(ctl, full, D + 2, NW);
}

// FP64-class variant (LOB_SPMM_DF64): values as (hi, lo) FP32 pairs (hi = the FP32 value,
// lo = the rounded remainder, ~48 significant bits together), X staged as (hi, lo) pairs, every
// product and sum in double-float (df.cuh) on the FP32 pipes. Same schedule as k_spmm4: lane
// group g owns in-tile rows/columns g, g + NG, ...; each lane holds VW = 2 vector columns.
template <int NB>
struct CfgDF {
  static constexpr int VW = 2;  // vector columns per lane (four measured slower: register-limited at 1,024 threads)
  static constexpr int G = NB / VW;
  static constexpr int THREADS = (LOB_TILE * G) < 1024 ? (LOB_TILE * G) : 1024;
  static constexpr int NG = THREADS / G;
  static constexpr int RPG = LOB_TILE / NG;
  static constexpr int CH = LOB_PERM_CHUNK;
  static constexpr int PTRS = 2 * (LOB_TILE + 1);
  static constexpr size_t XV = sizeof(float2) * LOB_TILE * NB;
  static constexpr size_t XI = 0;
  static constexpr size_t XJ = XI + XV;
  static constexpr size_t RC = XJ + 2 * XV;
  static constexpr size_t VH = RC + 2 * 4 * CH;
  static constexpr size_t VL = VH + 2 * 4 * CH;
  static constexpr size_t PM = VL + 2 * 4 * CH;
  static constexpr size_t PT = PM + 2 * 2 * (CH + 8);
  static constexpr size_t BYTES = PT + 2 * 2 * PTRS;
};

__global__ void k_stage_x_df(int64_t rows, int64_t n_act, int nb, int c0, int w, int NB, const double* __restrict__ X,
                             float2* __restrict__ Xs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * NB) return;
  const int64_t i = t / NB;
  const int j = (int)(t % NB);
  const double v = (j < w && i < n_act) ? X[i * nb + c0 + j] : 0.0;
  Xs[t] = df_split(v);
}

__device__ __forceinline__ void stage_put(float* p, double v) { *p = f64_to_f32_rn(v); }
__device__ __forceinline__ void stage_put(double* p, double v) { *p = v; }
__device__ __forceinline__ void stage_put(float2* p, double v) { *p = df_split(v); }

// Staging for a batched class: every job's X into its matrix's staged copy (NB columns, rows
// padded to whole tiles, zero beyond n_act and w) and its Y zeroed, in one launch.
template <typename T, int NB>
__global__ void k_stage_batch(const lob_spmm_job* __restrict__ jobs, int njobs) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].stage_begin <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const lob_spmm_job& j = jobs[lo];
  const int64_t t = ((int64_t)blockIdx.x - j.stage_begin) * blockDim.x + threadIdx.x;
  if (t < j.rows_pad * NB) {
    const int64_t i = t / NB;
    const int c = (int)(t % NB);
    const double v = (c < j.w && i < j.n_act) ? j.Xsrc[i * j.w + c] : 0.0;
    stage_put(reinterpret_cast<T*>(const_cast<void*>(j.Xs)) + t, v);
  }
  if (t < j.n_rows * j.w) j.Y[t] = 0.0;
}

template <int NB>
__global__ void __launch_bounds__(CfgDF<NB>::THREADS, 1)
    k_spmm4df(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol, const int64_t* __restrict__ tptr,
              const int32_t* __restrict__ tchunk, const uint32_t* __restrict__ rc, const float* __restrict__ vhi,
              const float* __restrict__ vlo, const uint16_t* __restrict__ cperm, const uint16_t* __restrict__ cptrs,
              const float2* __restrict__ Xs, double* __restrict__ Y, int ldy, int c0, int w, int64_t n_act,
              const lob_spmm_job* __restrict__ jobs, int njobs) {
  using C = CfgDF<NB>;
  constexpr int VW = C::VW, G = C::G, NG = C::NG, RPG = C::RPG, CH = C::CH, THREADS = C::THREADS;
  constexpr int XN = LOB_TILE * NB;
  extern __shared__ __align__(16) unsigned char sm[];
  float2* XI = reinterpret_cast<float2*>(sm + C::XI);
  float2* XJb = reinterpret_cast<float2*>(sm + C::XJ);
  uint32_t* RCb = reinterpret_cast<uint32_t*>(sm + C::RC);
  float* VHb = reinterpret_cast<float*>(sm + C::VH);
  float* VLb = reinterpret_cast<float*>(sm + C::VL);
  uint16_t* PMb = reinterpret_cast<uint16_t*>(sm + C::PM);
  uint16_t* PTb = reinterpret_cast<uint16_t*>(sm + C::PT);

  int64_t I = blockIdx.x;
  if (jobs) {  // batched launch: find this CTA's matrix and tile row
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].cta_begin <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const lob_spmm_job& jb = jobs[lo];
    rowptr = jb.rowptr; tcol = jb.tcol; tptr = jb.tptr; tchunk = jb.tchunk; rc = jb.rc;
    vhi = reinterpret_cast<const float*>(jb.vals); vlo = reinterpret_cast<const float*>(jb.vlo);
    cperm = jb.cperm; cptrs = jb.cptrs;
    Xs = reinterpret_cast<const float2*>(jb.Xs); Y = jb.Y; ldy = jb.ldy; c0 = jb.c0; w = jb.w; n_act = jb.n_act;
    I = (int64_t)blockIdx.x - jb.cta_begin;
  }
  const int64_t row0 = I * LOB_TILE;
  const int tid = threadIdx.x;
  const int g = tid / G, gl = tid % G;
  const int64_t t0 = rowptr[I];
  int64_t t1 = rowptr[I + 1];
  while (t1 > t0 && (int64_t)tcol[t1 - 1] * LOB_TILE >= n_act) t1--;

  for (int e = tid * 2; e < XN; e += THREADS * 2) cp_async16(&XI[e], &Xs[row0 * NB + e]);
  cp_async_commit();

  auto issue = [&](int64_t t, int64_t k, int buf, int xbuf) {
    const int64_t J = tcol[t];
    if (k == 0 && J != I) {
      float2* XJ = XJb + xbuf * XN;
      const float2* src = Xs + J * LOB_TILE * NB;
      for (int e = tid * 2; e < XN; e += THREADS * 2) cp_async16(&XJ[e], &src[e]);
    }
    const int64_t base = tptr[t] + k * CH;
    const int64_t rem = tptr[t + 1] - base;
    const int cnt = (int)(rem < CH ? rem : CH);
    for (int i = tid; i < cnt; i += THREADS) {
      cp_async4(&RCb[buf * CH + i], &rc[base + i]);
      cp_async4(&VHb[buf * CH + i], &vhi[base + i]);
      cp_async4(&VLb[buf * CH + i], &vlo[base + i]);
    }
    uint32_t* PM32 = reinterpret_cast<uint32_t*>(PMb + buf * (CH + 8));
    const int64_t wb = base & ~(int64_t)1;
    const int nwords = (int)((base + cnt - wb + 1) / 2);
    const uint32_t* src32 = reinterpret_cast<const uint32_t*>(cperm + wb);
    for (int i = tid; i < nwords; i += THREADS) cp_async4(&PM32[i], &src32[i]);
    uint32_t* PT32 = reinterpret_cast<uint32_t*>(PTb + buf * C::PTRS);
    const uint32_t* srcp = reinterpret_cast<const uint32_t*>(cptrs + (int64_t)(tchunk[t] + k) * C::PTRS);
    for (int i = tid; i < C::PTRS / 2; i += THREADS) cp_async4(&PT32[i], &srcp[i]);
    cp_async_commit();
  };

  // per owned index a and lane column q: tile row partial, column partial, row accumulator (all df)
  float th[RPG][VW], tlo[RPG][VW], chh[RPG][VW], clo[RPG][VW], rh[RPG][VW], rl[RPG][VW];
#pragma unroll
  for (int a = 0; a < RPG; a++)
#pragma unroll
    for (int q = 0; q < VW; q++) { th[a][q] = tlo[a][q] = chh[a][q] = clo[a][q] = rh[a][q] = rl[a][q] = 0.f; }

  int64_t t = t0, k = 0;
  int tl = 0, buf = 0;
  if (t < t1) issue(t, 0, 0, 0);
  while (t < t1) {
    const int64_t J = tcol[t];
    const bool diag = (J == I);
    const bool last = (tptr[t] + (k + 1) * CH >= tptr[t + 1]);
    int64_t tn = t, kn = k + 1;
    int tln = tl;
    if (last) { tn = t + 1; kn = 0; tln = tl + 1; }
    if (tn < t1) { issue(tn, kn, buf ^ 1, tln & 1); cp_async_wait_1(); } else { cp_async_wait_all(); }
    __syncthreads();
    const uint32_t* RCs = RCb + buf * CH;
    const float* VH = VHb + buf * CH;
    const float* VL = VLb + buf * CH;
    const uint16_t* PM = PMb + buf * (CH + 8) + (int)((tptr[t] + k * CH) & 1);
    const uint16_t* PR = PTb + buf * C::PTRS;
    const uint16_t* PC = PR + (LOB_TILE + 1);
    const float2* xj = diag ? XI : XJb + (tl & 1) * XN;
#pragma unroll
    for (int a = 0; a < RPG; a++) {
      const int idx = g + a * NG;
      {
        const int s = PR[idx], e = PR[idx + 1];
        for (int i = s; i < e; i++) {
          const int c = (int)(RCs[i] & 0xFFFFu);
          const float vh = VH[i], vl = VL[i];
#pragma unroll
          for (int h = 0; h < VW; h += 2) {
            const float4 x = *reinterpret_cast<const float4*>(&xj[c * NB + gl * VW + h]);  // (h0, l0, h1, l1)
            df_mac(th[a][h], tlo[a][h], vh, vl, x.x, x.y);
            df_mac(th[a][h + 1], tlo[a][h + 1], vh, vl, x.z, x.w);
          }
        }
      }
      {
        const int s = PC[idx], e = PC[idx + 1];
        for (int i = s; i < e; i++) {
          const int q = PM[i] & (CH - 1);
          const int r = (int)(RCs[q] >> 16);
          if (diag && r == idx) continue;
          const float vh = VH[q], vl = VL[q];
#pragma unroll
          for (int h = 0; h < VW; h += 2) {
            const float4 x = *reinterpret_cast<const float4*>(&XI[r * NB + gl * VW + h]);
            df_mac(chh[a][h], clo[a][h], vh, vl, x.x, x.y);
            df_mac(chh[a][h + 1], clo[a][h + 1], vh, vl, x.z, x.w);
          }
        }
      }
    }
    if (last) {
#pragma unroll
      for (int a = 0; a < RPG; a++) {
        const int idx = g + a * NG;
#pragma unroll
        for (int q = 0; q < VW; q++) {
          df_renorm(th[a][q], tlo[a][q]);
          df_renorm(chh[a][q], clo[a][q]);
          df_add(rh[a][q], rl[a][q], th[a][q], tlo[a][q]);
          if (diag) {
            df_add(rh[a][q], rl[a][q], chh[a][q], clo[a][q]);
          } else {
            const int kk = gl * VW + q;
            const int64_t gr = J * LOB_TILE + idx;
            if (kk < w && gr < n_act) {
              atomic_out(&Y[gr * ldy + c0 + kk], chh[a][q]);
              atomic_out(&Y[gr * ldy + c0 + kk], clo[a][q]);
            }
          }
          th[a][q] = tlo[a][q] = chh[a][q] = clo[a][q] = 0.f;
        }
      }
    }
    __syncthreads();
    t = tn; k = kn; tl = tln; buf ^= 1;
  }
  cp_async_wait_all();
#pragma unroll
  for (int a = 0; a < RPG; a++) {
    const int64_t gr = row0 + g + a * NG;
#pragma unroll
    for (int q = 0; q < VW; q++) {
      const int kk = gl * VW + q;
      if (kk >= w || gr >= n_act) continue;
      df_renorm(rh[a][q], rl[a][q]);
      atomic_out(&Y[gr * ldy + c0 + kk], rh[a][q]);
      atomic_out(&Y[gr * ldy + c0 + kk], rl[a][q]);
    }
  }
}

// Ring-pipelined FP64-class (double-float) product at NB = 16: the schedule of k_spmm_ring with
// the ownership and arithmetic of k_spmm4df (lane group of NB/2 lanes, two vector columns a
// lane, two owned rows and columns a group). Its X tiles are (hi, lo) pairs, twice the FP32
// size, so the ring has two stages and X_I one slot: the warps meet once per tile row, when
// the last of them loads the next X_I.
template <int NB>
struct CfgRD {
  static constexpr int VW = 2;
  static constexpr int G = NB / VW;
  static constexpr int THREADS = 1024;
  static constexpr int NG = THREADS / G;
  static constexpr int RPG = LOB_TILE / NG;
  static constexpr int NW = THREADS / 32;
  static constexpr int D = 2;
  static constexpr int CH = LOB_PERM_CHUNK;
  static constexpr int PTRS = 2 * (LOB_TILE + 1);
  static constexpr size_t XV = sizeof(float2) * LOB_TILE * NB;
  static constexpr size_t S_RV = 0;  // (record, high part) pairs
  static constexpr size_t S_VL = S_RV + 8 * (CH + 8);
  static constexpr size_t S_PM = S_VL + 4 * (CH + 8);
  static constexpr size_t S_PT = S_PM + 2 * (CH + 16);
  static constexpr size_t S_XJ = (S_PT + 2 * PTRS + 32 + 15) / 16 * 16;
  static constexpr size_t STAGE = S_XJ + XV;
  static constexpr size_t XI = 0;  // one X_I slot
  static constexpr size_t ST = XI + XV;
  static constexpr size_t BAR = ST + D * STAGE;  // full[D], xfull
  static constexpr size_t RNG = BAR + 8 * (D + 1);
  static constexpr size_t CUR = RNG + 16;
  static constexpr size_t CNT = CUR + 48;
  static constexpr size_t CTL = (CNT + 4 * (D + 1) + 7) / 8 * 8;  // abort protocol (RingCtl)
  static constexpr size_t BYTES = CTL + sizeof(RingCtl);
  static_assert(VW * G == NB && NG * RPG == LOB_TILE && THREADS % G == 0, "launch shape");
  static_assert(sizeof(RingCur) <= 48, "cursor slot");
  static_assert(S_VL % 16 == 0 && S_PM % 16 == 0 && S_PT % 16 == 0 && STAGE % 16 == 0 &&
                    ST % 16 == 0,
                "bulk copy destinations must be 16-byte aligned");
};

template <int NB>
__device__ __forceinline__ void ring_issue_df(unsigned char* stage, uint64_t* bar, int64_t I, int64_t t, int k,
                                              const int32_t* tcol, const int64_t* tptr, const int32_t* tchunk,
                                              const uint2* rv, const float* vlo, const uint16_t* cperm,
                                              const uint16_t* cptrs, const float2* Xs) {
  using C = CfgRD<NB>;
  const int64_t J = tcol[t];
  const int64_t base = tptr[t] + (int64_t)k * C::CH;
  const int64_t rem = tptr[t + 1] - base;
  const int64_t cnt = rem < C::CH ? rem : C::CH;
  const int64_t r0 = base & ~(int64_t)1, r1 = (base + cnt + 1) & ~(int64_t)1;      // 8-byte pairs
  const int64_t a0 = base & ~(int64_t)3, e1 = (base + cnt + 3) & ~(int64_t)3;      // 4-byte low parts
  const int64_t p0 = base & ~(int64_t)7, p1 = (base + cnt + 7) & ~(int64_t)7;
  const int64_t bo = (int64_t)(tchunk[t] + k) * (C::PTRS * 2);
  const int64_t q0 = bo & ~(int64_t)15, q1 = (bo + C::PTRS * 2 + 15) & ~(int64_t)15;
  const uint32_t brv = (uint32_t)((r1 - r0) * 8), bvl = (uint32_t)((e1 - a0) * 4);
  const uint32_t bpm = (uint32_t)((p1 - p0) * 2), bpt = (uint32_t)(q1 - q0);
  const uint32_t bxj = (J != I) ? (uint32_t)C::XV : 0u;
  mbar_expect_tx(bar, brv + bvl + bpm + bpt + bxj);
  bulk_g2s(stage + C::S_RV, rv + r0, brv, bar);
  bulk_g2s(stage + C::S_VL, vlo + a0, bvl, bar);
  bulk_g2s(stage + C::S_PM, cperm + p0, bpm, bar);
  bulk_g2s(stage + C::S_PT, reinterpret_cast<const unsigned char*>(cptrs) + q0, bpt, bar);
  if (bxj) bulk_g2s(stage + C::S_XJ, Xs + J * LOB_TILE * NB, bxj, bar);
}

template <int NB>
__global__ void __launch_bounds__(CfgRD<NB>::THREADS, 1)
    k_spmm_ring_df(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol,
                   const int64_t* __restrict__ tptr, const int32_t* __restrict__ tchunk,
                   const uint2* __restrict__ rv, const float* __restrict__ vlo,
                   const uint16_t* __restrict__ cperm, const uint16_t* __restrict__ cptrs,
                   const float2* __restrict__ Xs, double* __restrict__ Y, int ldy, int c0, int w, int64_t n_act,
                   int64_t ntr, int* __restrict__ status, long long limit, int poison) {
  using C = CfgRD<NB>;
  constexpr int VW = C::VW, G = C::G, NG = C::NG, RPG = C::RPG, NW = C::NW, D = C::D, CH = C::CH;
  extern __shared__ __align__(16) unsigned char sm[];
  float2* XI = reinterpret_cast<float2*>(sm + C::XI);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::BAR);
  uint64_t* xfull = full + D;
  int* cnt = reinterpret_cast<int*>(sm + C::CNT);
  int* xcnt = cnt + D;
  int64_t* range = reinterpret_cast<int64_t*>(sm + C::RNG);
  RingCur* cur = reinterpret_cast<RingCur*>(sm + C::CUR);
  RingCtl* ctl = reinterpret_cast<RingCtl*>(sm + C::CTL);
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = tid / G, gl = tid % G;
  static_assert(D + 1 <= 8, "RingCtl slots");

  if (tid == 0) {
    ctl->abort = 0;
    ctl->left = 0;
    for (int i = 0; i < 8; i++) ctl->issued[i] = 0;
    const int64_t E = tptr[rowptr[ntr]];
    auto first_row = [&](int64_t b) -> int64_t {
      if (b >= (int64_t)gridDim.x) return ntr;
      const int64_t target = E * b / (int64_t)gridDim.x;
      int64_t lo = 0, hi = ntr;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tptr[rowptr[mid]] >= target) hi = mid; else lo = mid + 1;
      }
      return lo;
    };
    range[0] = first_row(blockIdx.x);
    range[1] = first_row((int64_t)blockIdx.x + 1);
    for (int s = 0; s < D; s++) { mbar_init(&full[s], 1); cnt[s] = 0; }
    mbar_init(xfull, 1);
    *xcnt = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const int64_t Ib = range[0], Ie = range[1];
  if (tid == 0 && Ib < Ie) {
    ctl->issued[D]++;
    mbar_expect_tx(xfull, (uint32_t)C::XV);
    bulk_g2s(XI, Xs + Ib * LOB_TILE * NB, (uint32_t)C::XV, xfull);
    RingCur c;
    c.I = Ib; c.Ie = Ie;
    int64_t t0;
    c.t1 = ring_trim(rowptr, tcol, n_act, Ib, &t0);
    c.t = t0 - 1; c.k = 0; c.nk = 0;
    bool more = ring_settle(c, rowptr, tcol, tchunk, n_act);
    for (int s = 0; s < D && more; s++) {
      if (poison && s == 0) {  // test mode: stage 0 expects bytes that nothing sends (nothing in flight)
        mbar_expect_tx(&full[0], 16u);
      } else {
        ctl->issued[s]++;
        ring_issue_df<NB>(sm + C::ST + s * C::STAGE, &full[s], c.I, c.t, c.k, tcol, tptr, tchunk, rv, vlo, cperm,
                          cptrs, Xs);
      }
      c.k++;
      more = ring_settle(c, rowptr, tcol, tchunk, n_act);
    }
    if (!more) c.I = Ie;
    *cur = c;
  }
  __syncthreads();

  int64_t ch = 0;
  for (int64_t I = Ib; I < Ie; I++) {
    const int64_t ri = I - Ib;
    if (!mbar_wait(xfull, (uint32_t)(ri & 1), limit, ctl, status)) goto leave;
    int64_t t0;
    const int64_t t1 = ring_trim(rowptr, tcol, n_act, I, &t0);
    float rh[RPG][VW], rl[RPG][VW];
#pragma unroll
    for (int a = 0; a < RPG; a++)
#pragma unroll
      for (int q = 0; q < VW; q++) { rh[a][q] = 0.f; rl[a][q] = 0.f; }
    for (int64_t t = t0; t < t1; t++) {
      const int64_t J = tcol[t];
      const bool diag = (J == I);
      const int nk = tchunk[t + 1] - tchunk[t];
      float th[RPG][VW], tlo[RPG][VW], chh[RPG][VW], clo[RPG][VW];
#pragma unroll
      for (int a = 0; a < RPG; a++)
#pragma unroll
        for (int q = 0; q < VW; q++) { th[a][q] = tlo[a][q] = chh[a][q] = clo[a][q] = 0.f; }
      for (int k = 0; k < nk; k++) {
        const int s = (int)(ch % D);
        if (!mbar_wait(&full[s], (uint32_t)((ch / D) & 1), limit, ctl, status)) goto leave;
        unsigned char* stage = sm + C::ST + s * C::STAGE;
        const int64_t base = tptr[t] + (int64_t)k * CH;
        const uint2* RV = reinterpret_cast<const uint2*>(stage + C::S_RV) + (base & 1);
        const float* VL = reinterpret_cast<const float*>(stage + C::S_VL) + (base & 3);
        const uint16_t* PM = reinterpret_cast<const uint16_t*>(stage + C::S_PM) + (base & 7);
        const int64_t bo = (int64_t)(tchunk[t] + k) * (C::PTRS * 2);
        const uint16_t* PR = reinterpret_cast<const uint16_t*>(stage + C::S_PT + (bo & 15));
        const uint16_t* PC = PR + (LOB_TILE + 1);
        const float2* xj = diag ? XI : reinterpret_cast<const float2*>(stage + C::S_XJ);
#pragma unroll
        for (int a = 0; a < RPG; a++) {
          const int idx = g + a * NG;
          {
            const int s0 = PR[idx], e0 = PR[idx + 1];
            for (int i = s0; i < e0; i++) {
              const uint2 e = RV[i];
              const int c = (int)(e.x & 0xFFFFu);
              const float vh = __uint_as_float(e.y), vl = VL[i];
#pragma unroll
              for (int h = 0; h < VW; h += 2) {
                const float4 x = *reinterpret_cast<const float4*>(&xj[c * NB + gl * VW + h]);  // (h0, l0, h1, l1)
                df_mac(th[a][h], tlo[a][h], vh, vl, x.x, x.y);
                df_mac(th[a][h + 1], tlo[a][h + 1], vh, vl, x.z, x.w);
              }
            }
          }
          {
            const int s0 = PC[idx], e0 = PC[idx + 1];
            for (int i = s0; i < e0; i++) {
              const int q = PM[i] & (CH - 1);
              const uint2 e = RV[q];
              const int r = (int)(e.x >> 16);
              if (diag && r == idx) continue;
              const float vh = __uint_as_float(e.y), vl = VL[q];
#pragma unroll
              for (int h = 0; h < VW; h += 2) {
                const float4 x = *reinterpret_cast<const float4*>(&XI[r * NB + gl * VW + h]);
                df_mac(chh[a][h], clo[a][h], vh, vl, x.x, x.y);
                df_mac(chh[a][h + 1], clo[a][h + 1], vh, vl, x.z, x.w);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          const int old = atomicAdd(&cnt[s], 1);
          if (old == NW * (int)(ch / D + 1) - 1) {
            __threadfence_block();
            RingCur c = *cur;
            if (c.I < c.Ie && *(volatile int*)&ctl->abort == 0) {
              asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
              ctl->issued[s]++;
              ring_issue_df<NB>(stage, &full[s], c.I, c.t, c.k, tcol, tptr, tchunk, rv, vlo, cperm, cptrs, Xs);
              c.k++;
              if (!ring_settle(c, rowptr, tcol, tchunk, n_act)) c.I = c.Ie;
              *cur = c;
            }
            __threadfence_block();
          }
        }
        ch++;
      }
#pragma unroll
      for (int a = 0; a < RPG; a++) {
        const int idx = g + a * NG;
#pragma unroll
        for (int q = 0; q < VW; q++) {
          df_renorm(th[a][q], tlo[a][q]);
          df_renorm(chh[a][q], clo[a][q]);
          df_add(rh[a][q], rl[a][q], th[a][q], tlo[a][q]);
          if (diag) {
            df_add(rh[a][q], rl[a][q], chh[a][q], clo[a][q]);
          } else {
            const int kk = gl * VW + q;
            const int64_t gr = J * LOB_TILE + idx;
            if (kk < w && gr < n_act) {
              atomic_out(&Y[gr * ldy + c0 + kk], chh[a][q]);
              atomic_out(&Y[gr * ldy + c0 + kk], clo[a][q]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < RPG; a++) {
      const int64_t gr = I * LOB_TILE + g + a * NG;
#pragma unroll
      for (int q = 0; q < VW; q++) {
        const int kk = gl * VW + q;
        if (kk >= w || gr >= n_act) continue;
        df_renorm(rh[a][q], rl[a][q]);
        atomic_out(&Y[gr * ldy + c0 + kk], rh[a][q]);
        atomic_out(&Y[gr * ldy + c0 + kk], rl[a][q]);
      }
    }
    // count this warp out of X_I; the last one loads the next row's
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      const int old = atomicAdd(xcnt, 1);
      if (old == NW * (int)(ri + 1) - 1 && I + 1 < Ie && *(volatile int*)&ctl->abort == 0) {
        __threadfence_block();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        ctl->issued[D]++;
        mbar_expect_tx(xfull, (uint32_t)C::XV);
        bulk_g2s(XI, Xs + (I + 1) * LOB_TILE * NB, (uint32_t)C::XV, xfull);
      }
    }
  }
leave:
  ring_leave(ctl, full, D + 1, NW);
}


template <int NB>
int launch_df(const lob_matrix* m, const double* X, double* Y, int nb, int64_t n_act, cudaStream_t st) {
  using C = CfgDF<NB>;
  static_assert(C::BYTES <= 227 * 1024, "shared memory budget");
  const lob_tiles& TS = m->T;
  const int64_t nt_act = (n_act + LOB_TILE - 1) / LOB_TILE;
  if (nt_act == 0) return LOB_OK;
  const int64_t rows_pad = TS.nt * LOB_TILE;
  LOB_TRY(lob_ensure_xs(m, (size_t)rows_pad * NB * sizeof(float2)));
  float2* Xs = reinterpret_cast<float2*>(m->xs);
  auto kern = k_spmm4df<NB>;
  int64_t grid = nt_act;
  if constexpr (NB == 16) {
    if (!TS.rv) return LOB_ERR_ARG;
    static_assert(CfgRD<NB>::BYTES <= 227 * 1024, "shared memory budget");
    const int sms = lob_sm_count();
    if (sms < 0) return LOB_ERR_CUDA;
    grid = nt_act < sms ? nt_act : sms;
    LOB_CUDA(cudaFuncSetAttribute(k_spmm_ring_df<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)CfgRD<NB>::BYTES));
  } else {
    LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
  }
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int w = (nb - c0) < NB ? (nb - c0) : NB;
    (k_stage_x_df<<<(unsigned)((rows_pad * NB + 255) / 256), 256, 0, st>>>(rows_pad, n_act, nb, c0, w, NB, X, Xs),
     LOB_LAUNCHED());
    if constexpr (NB == 16) {
      (k_spmm_ring_df<NB><<<(unsigned)grid, CfgRD<NB>::THREADS, CfgRD<NB>::BYTES, st>>>(
           TS.rowptr, TS.tcol, TS.tptr, TS.tchunk, TS.rv, TS.v32lo, TS.cperm, TS.cptrs, Xs, Y, nb, c0, w, n_act,
           nt_act, m->status, m->wait_limit, m->wait_poison),
       LOB_LAUNCHED());
    } else {
      (kern<<<(unsigned)nt_act, C::THREADS, C::BYTES, st>>>(TS.rowptr, TS.tcol, TS.tptr, TS.tchunk, TS.rc, TS.v32,
                                                             TS.v32lo, TS.cperm, TS.cptrs, Xs, Y, nb, c0, w, n_act,
                                                             nullptr, 0),
       LOB_LAUNCHED());
    }
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

template <bool MIXED, int NB>
int launch(const lob_matrix* m, const double* X, double* Y, int nb, int64_t n_act, cudaStream_t st) {
  using C = Cfg<MIXED, NB>;
  using T = typename Elt<MIXED>::T;
  static_assert(C::BYTES <= 227 * 1024, "shared memory budget");
  const lob_tiles& TS = m->T;
  const int64_t nt_act = (n_act + LOB_TILE - 1) / LOB_TILE;
  if (nt_act == 0) return LOB_OK;
  // staged X: rows padded to whole tiles, NB columns (scratch owned by the matrix)
  const int64_t rows_pad = TS.nt * LOB_TILE;
  LOB_TRY(lob_ensure_xs(m, (size_t)rows_pad * NB * sizeof(T)));
  T* Xs = reinterpret_cast<T*>(m->xs);
  auto kern = k_spmm4<MIXED, NB>;
  LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int w = (nb - c0) < NB ? (nb - c0) : NB;
    (k_stage_x<T><<<(unsigned)((rows_pad * NB + 255) / 256), 256, 0, st>>>(rows_pad, n_act, nb, c0, w, NB, X, Xs),
     LOB_LAUNCHED());
    (kern<<<(unsigned)nt_act, C::THREADS, C::BYTES, st>>>(
         TS.rowptr, TS.tcol, TS.tptr, TS.tchunk, TS.rc,
         MIXED ? (const T*)(const void*)TS.v32 : (const T*)(const void*)TS.v64, TS.cperm, TS.cptrs, Xs, Y, nb, c0, w,
         n_act, nullptr, 0),
     LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

// FP32-value product at NB = 16 through the ring kernel: one persistent CTA per SM (fewer when
// the matrix has fewer tile rows).
int launch_ring16(const lob_matrix* m, const double* X, double* Y, int nb, int64_t n_act, cudaStream_t st) {
  constexpr int NB = 16;
  using C = CfgR<NB>;
  static_assert(C::BYTES <= 227 * 1024, "shared memory budget");
  const lob_tiles& TS = m->T;
  if (!TS.rv) return LOB_ERR_ARG;
  const int64_t nt_act = (n_act + LOB_TILE - 1) / LOB_TILE;
  if (nt_act == 0) return LOB_OK;
  const int64_t rows_pad = TS.nt * LOB_TILE;
  LOB_TRY(lob_ensure_xs(m, (size_t)rows_pad * NB * sizeof(float)));
  float* Xs = reinterpret_cast<float*>(m->xs);
  const int sms = lob_sm_count();
  if (sms < 0) return LOB_ERR_CUDA;
  const int64_t grid = nt_act < sms ? nt_act : sms;
  LOB_CUDA(cudaFuncSetAttribute(k_spmm_ring<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
  for (int c0 = 0; c0 < nb; c0 += NB) {
    const int w = (nb - c0) < NB ? (nb - c0) : NB;
    (k_stage_x<float><<<(unsigned)((rows_pad * NB + 255) / 256), 256, 0, st>>>(rows_pad, n_act, nb, c0, w, NB, X, Xs),
     LOB_LAUNCHED());
    (k_spmm_ring<NB><<<(unsigned)grid, C::THREADS, C::BYTES, st>>>(TS.rowptr, TS.tcol, TS.tptr, TS.tchunk,
                                                                  TS.rvp ? TS.rvp : TS.rv,
                                                                  TS.rvp ? TS.cpermp : TS.cperm, TS.cptrs, Xs, Y, nb,
                                                                  c0, w, n_act,
                                                                  nt_act, m->status, m->wait_limit, m->wait_poison),
     LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

template <int MODE, int NB>
int batch_class(const lob_matrix* const* ms, const double* const* X, double* const* Y, const int* ncol,
                const int64_t* nact, const std::vector<int>& idx, lob_spmm_job* jobs_host, lob_spmm_job* jobs_dev, cudaStream_t st) {
  int njob = 0;
  int64_t ctas = 0, sctas = 0;
  for (int j : idx) {
    const lob_matrix* m = ms[j];
    const lob_tiles& TS = m->T;
    const int64_t na = nact ? nact[j] : TS.n;
    const int64_t nt_act = (na + LOB_TILE - 1) / LOB_TILE;
    if (nt_act == 0) continue;
    const int64_t rows_pad = TS.nt * LOB_TILE;
    const size_t esz = MODE == LOB_SPMM_MIXED ? 4 : 8;
    LOB_TRY(lob_ensure_xs(m, (size_t)rows_pad * NB * esz));
    lob_spmm_job jb;
    jb.rowptr = TS.rowptr; jb.tcol = TS.tcol; jb.tptr = TS.tptr; jb.tchunk = TS.tchunk; jb.rc = TS.rc;
    jb.vals = MODE == LOB_SPMM_FP64 ? (const void*)TS.v64 : (const void*)TS.v32;
    jb.vlo = TS.v32lo; jb.cperm = TS.cperm; jb.cptrs = TS.cptrs; jb.Xs = m->xs; jb.Y = Y[j];
    jb.ldy = ncol[j]; jb.c0 = 0; jb.w = ncol[j]; jb.pad = 0; jb.n_act = na; jb.cta_begin = ctas;
    jb.Xsrc = X[j]; jb.n_rows = TS.n; jb.rows_pad = rows_pad; jb.stage_begin = sctas;
    jobs_host[njob++] = jb;
    ctas += nt_act;
    const int64_t work = std::max<int64_t>(rows_pad * NB, TS.n * ncol[j]);
    sctas += (work + 255) / 256;
  }
  if (njob == 0) return LOB_OK;
  LOB_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, njob * sizeof(lob_spmm_job), cudaMemcpyHostToDevice, st));
  if (MODE == LOB_SPMM_DF64) (k_stage_batch<float2, NB><<<(unsigned)sctas, 256, 0, st>>>(jobs_dev, njob), LOB_LAUNCHED());
  else if (MODE == LOB_SPMM_MIXED) (k_stage_batch<float, NB><<<(unsigned)sctas, 256, 0, st>>>(jobs_dev, njob), LOB_LAUNCHED());
  else (k_stage_batch<double, NB><<<(unsigned)sctas, 256, 0, st>>>(jobs_dev, njob), LOB_LAUNCHED());
  if (MODE == LOB_SPMM_DF64) {
    using C = CfgDF<NB>;
    LOB_CUDA(cudaFuncSetAttribute(k_spmm4df<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
    (k_spmm4df<NB><<<(unsigned)ctas, C::THREADS, C::BYTES, st>>>(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                 nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0,
                                                                 jobs_dev, njob), LOB_LAUNCHED());
  } else {
    constexpr bool MX = MODE == LOB_SPMM_MIXED;
    using C = Cfg<MX, NB>;
    LOB_CUDA(cudaFuncSetAttribute(k_spmm4<MX, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
    (k_spmm4<MX, NB><<<(unsigned)ctas, C::THREADS, C::BYTES, st>>>(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                   nullptr, nullptr, nullptr, nullptr, 0, 0, 0, 0,
                                                                   jobs_dev, njob), LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

}  // namespace

// SMs of the current device (-1 if the query fails).
int lob_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return sms;
}

int lob_spmm_batch_launch(const lob_matrix* const* ms, const double* const* X, double* const* Y, const int* ncol,
                          const int* mode, const int64_t* nact, int njobs, lob_spmm_job* jobs_host,
                          lob_spmm_job* jobs_dev, cudaStream_t st, int* n_kernels) {
  if (n_kernels) *n_kernels = 0;
  // classes by (arithmetic, vector width); each class is one launch
  std::vector<int> cls[3][4];
  for (int j = 0; j < njobs; j++) {
    if (ncol[j] < 1 || ncol[j] > 16) return LOB_ERR_ARG;
    const int md = mode[j];
    if (md < 0 || md > 2) return LOB_ERR_ARG;
    if (nact && (nact[j] < 0 || nact[j] > ms[j]->T.n)) return LOB_ERR_ARG;
    if ((md == LOB_SPMM_MIXED && !ms[j]->T.v32) || (md == LOB_SPMM_FP64 && !ms[j]->T.v64) ||
        (md == LOB_SPMM_DF64 && !ms[j]->T.v32lo))
      return LOB_ERR_ARG;
    for (int i = 0; i < j; i++)
      if (ms[i] == ms[j]) return LOB_ERR_ARG;  // one staged-X scratch per matrix
    const int w = ncol[j];
    const int c = md == LOB_SPMM_MIXED ? (w <= 4 ? 1 : (w <= 8 ? 2 : 3)) : (w <= 2 ? 0 : (w <= 4 ? 1 : (w <= 8 ? 2 : 3)));
    cls[md][c].push_back(j);
  }
  // offsets into the caller's job buffer per class (each class uses a disjoint slice)
  int off = 0;
  auto run = [&](int md, int c) -> int {
    const std::vector<int>& v = cls[md][c];
    if (v.empty()) return LOB_OK;
    lob_spmm_job* jd = jobs_dev + off;
    lob_spmm_job* jh = jobs_host + off;
    off += (int)v.size();
    if (n_kernels) (*n_kernels)++;
    if (md == LOB_SPMM_MIXED) {
      if (c == 1) return batch_class<LOB_SPMM_MIXED, 4>(ms, X, Y, ncol, nact, v, jh, jd, st);
      if (c == 2) return batch_class<LOB_SPMM_MIXED, 8>(ms, X, Y, ncol, nact, v, jh, jd, st);
      return batch_class<LOB_SPMM_MIXED, 16>(ms, X, Y, ncol, nact, v, jh, jd, st);
    }
    if (md == LOB_SPMM_DF64) {
      if (c == 0) return batch_class<LOB_SPMM_DF64, 2>(ms, X, Y, ncol, nact, v, jh, jd, st);
      if (c == 1) return batch_class<LOB_SPMM_DF64, 4>(ms, X, Y, ncol, nact, v, jh, jd, st);
      if (c == 2) return batch_class<LOB_SPMM_DF64, 8>(ms, X, Y, ncol, nact, v, jh, jd, st);
      return batch_class<LOB_SPMM_DF64, 16>(ms, X, Y, ncol, nact, v, jh, jd, st);
    }
    if (c == 0) return batch_class<LOB_SPMM_FP64, 2>(ms, X, Y, ncol, nact, v, jh, jd, st);
    if (c == 1) return batch_class<LOB_SPMM_FP64, 4>(ms, X, Y, ncol, nact, v, jh, jd, st);
    if (c == 2) return batch_class<LOB_SPMM_FP64, 8>(ms, X, Y, ncol, nact, v, jh, jd, st);
    return batch_class<LOB_SPMM_FP64, 16>(ms, X, Y, ncol, nact, v, jh, jd, st);
  };
  for (int md = 0; md < 3; md++)
    for (int c = 0; c < 4; c++) LOB_TRY(run(md, c));
  return LOB_OK;
}

int lob_matrix_fault_take(const lob_matrix* m, cudaStream_t st) {
  int h = 0;
  if (cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  if (h && cudaMemsetAsync(m->status, 0, sizeof(int), st) != cudaSuccess) return -1;
  return h;
}

int lob_spmm_launch(const lob_matrix* m, int mode, const double* X, double* Y, int nb, int64_t n_act,
                    cudaStream_t st) {
  if (nb < 1 || nb > 64 || n_act < 0 || n_act > m->T.n) return LOB_ERR_ARG;
  if (mode == LOB_SPMM_MIXED && !m->T.v32) return LOB_ERR_ARG;
  if (mode == LOB_SPMM_FP64 && !m->T.v64) return LOB_ERR_ARG;
  if (mode == LOB_SPMM_DF64 && !m->T.v32lo) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_MIXED && mode != LOB_SPMM_FP64 && mode != LOB_SPMM_DF64) return LOB_ERR_ARG;
  LOB_CUDA(cudaMemsetAsync(Y, 0, (size_t)m->T.n * nb * sizeof(double), st));
  if (mode == LOB_SPMM_DF64) {
    if (nb <= 2) return launch_df<2>(m, X, Y, nb, n_act, st);
    if (nb <= 4) return launch_df<4>(m, X, Y, nb, n_act, st);
    if (nb <= 8) return launch_df<8>(m, X, Y, nb, n_act, st);
    return launch_df<16>(m, X, Y, nb, n_act, st);
  }
  if (mode == LOB_SPMM_MIXED) {
    if (nb <= 4) return launch<true, 4>(m, X, Y, nb, n_act, st);
    if (nb <= 8) return launch<true, 8>(m, X, Y, nb, n_act, st);
    return launch_ring16(m, X, Y, nb, n_act, st);
  }
  if (nb <= 2) return launch<false, 2>(m, X, Y, nb, n_act, st);
  if (nb <= 4) return launch<false, 4>(m, X, Y, nb, n_act, st);
  if (nb <= 8) return launch<false, 8>(m, X, Y, nb, n_act, st);
  return launch<false, 16>(m, X, Y, nb, n_act, st);
}
