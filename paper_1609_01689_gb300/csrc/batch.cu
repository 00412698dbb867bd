// Batched small instances: many independent symmetric matrices (n up to 65,535, typically a few
// thousand rows) solved by LOBPCG (Algorithm 1) in ONE persistent kernel launch, captured in a
// CUDA graph. The serving and batching row's small-instance workload: the per-solve launch chain
// of the single-solve driver would be launch- and host-bound at this size.
//
// Schedule: a persistent grid of per_sm CTAs per SM. A CTA takes the next instance from an
// atomic ticket and runs that instance's whole solve on its own -- SpMM, Gram matrices, linear
// combinations, the Cholesky-QR and Rayleigh-Ritz solves (eq. 9, FP64, rr.cuh) -- then takes
// the next. Instances are ticketed largest first, so the slowest ones do not end the schedule
// alone. No CTA waits on another: the ticket is the only shared state.
//
// Storage of an instance's matrix: both triangles (the symmetric product needs no scatter on one
// CTA), as SELL slices of `tile` rows (8, 16 or 32): slice s holds width_s = its longest row's
// entries column by column (entry j of slice row i at base_s + j * tile + i, padded with zero
// values), so the lanes of a warp read consecutive addresses. Column indices are 16-bit
// instance-local; values FP32 and FP64.
//
// Arithmetic (the mixed precision of Section 4.3 and the precision study of the workloads):
// phase 1 computes in FP32 -- FP32 values and X in the SpMM, FP32 products in the Gram matrices
// (summed in FP32 over a thread's rows of a 32-row chunk, in double-float beyond), FP32 linear
// combinations -- until the first k relative residuals reach the phase target or stall; phase 2
// restarts from those vectors in double-float (values as the FP32 value plus its rounded
// remainder, ~48-bit products and sums) and runs to tol. The Cholesky factors and the
// Rayleigh-Ritz eigenproblems are FP64 in both phases. Vectors are stored in FP64 throughout.
// LOB_MODE_FP64 runs one phase in native FP64.
//
// Autotuner: tile height, threads per CTA and instances resident per SM are chosen by timing the
// whole schedule on a sample of the batch for every candidate (lob_batch_solve, first call).
#include <algorithm>
#include <chrono>
#include <cub/cub.cuh>
#include <thread>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "df.cuh"
#include "rr.cuh"

namespace {

constexpr int BNB = 8;             // widest block (nb) of the batched solver
constexpr int BM = 3 * BNB;        // widest Rayleigh-Ritz order (3 nb)
constexpr int BMAXT = 512;         // threads per CTA, at most
constexpr int BSTALL = 12;         // phase-1 iterations without halving of the worst residual
constexpr int BGSC = 9 * BMAXT;    // doubles of a CTA's Gram partial sums (row groups x p x q <= 9 threads)
constexpr int BRC = 32;            // rows of a Gram chunk staged in shared memory

// Per instance (device).
struct BInst {
  int32_t n, nsl;       // rows, SELL slices
  int64_t sl0;          // first slice (index into the batch's slice offsets)
  int64_t row0;         // first row in the batch (X output)
  double normH;         // ||H||_inf
};

// Everything the kernel reads (passed by value).
struct BDev {
  const BInst* inst;
  const int32_t* order;      // ticket -> instance (largest first)
  int32_t count;
  const int64_t* soff;       // [total slices + 1] first entry of each slice
  const uint16_t* col;       // [entries] instance-local column
  const float* v32;
  const float* v32lo;        // FP64 value minus its FP32 rounding, rounded to FP32
  const double* v64;
  double* work;              // per CTA: S, HS (n_max x 3 nb each, row-major), Xs (n_max x 8 pairs of FP32)
  int64_t wstride;           // doubles per CTA slot
  int32_t* ticket;
  double* lambda;            // [count][k]
  int32_t* status;           // [count]
  int32_t* iters;            // [count][2]: iterations, of which phase 2
  double* X;                 // [rows][nb] or null
  int32_t k, nb, mode, max_iter;
  double tol, tol1;          // final and phase-1 relative residual targets
  uint64_t seed;
};

__device__ __forceinline__ uint64_t b_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// uniform in [-1, 1) from (seed, instance, row, column): splitmix64 finaliser of a counter
__device__ __forceinline__ double b_rand(uint64_t seed, int inst, int r, int j) {
  const uint64_t z = b_mix(seed * 0x9E3779B97F4A7C15ull + ((uint64_t)(uint32_t)inst << 32) +
                           (uint64_t)(uint32_t)r * 8u + (uint64_t)(uint32_t)j);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Arithmetic of a phase. Vectors are stored in FP64; a phase loads them into its element type T,
// computes in T and stores back:
//   float  -- the FP32 phase;
//   B2     -- the FP64-class phase: double-float (hi + lo, two FP32 numbers, ~48 significant
//             bits) on the FP32 pipes, the FP64 pipe of this GPU being a small fraction of them;
//   double -- native FP64 (LOB_MODE_FP64).
struct B2 {
  float h, l;
  __device__ __forceinline__ B2() {}
  __device__ __forceinline__ explicit B2(int) : h(0.f), l(0.f) {}
  __device__ __forceinline__ B2(float a, float b) : h(a), l(b) {}
};
__device__ __forceinline__ B2 operator*(B2 a, B2 b) {
  const d2 r = d2_mul(d2{a.h, a.l}, d2{b.h, b.l});
  return B2(r.hi, r.lo);
}
__device__ __forceinline__ B2 operator+(B2 a, B2 b) {
  const d2 r = d2_add(d2{a.h, a.l}, d2{b.h, b.l});
  return B2(r.hi, r.lo);
}
__device__ __forceinline__ B2 operator-(B2 a, B2 b) { return a + B2(-b.h, -b.l); }
__device__ __forceinline__ B2& operator+=(B2& a, B2 b) { a = a + b; return a; }
__device__ __forceinline__ B2& operator-=(B2& a, B2 b) { a = a - b; return a; }

// Conversions between the FP64 storage and the phases' element types, branch-free (integer
// operations and selects only, so a thread's loads are not serialised behind data-dependent
// branches), flushing magnitudes below 2^-126 (FP32) or 2^-74 (the low part) to zero; the vectors
// are normalised, so nothing that small matters to a product. FP64 values above 2^128 do not occur.
__device__ __forceinline__ float b_f32(double x) {  // rounded toward zero
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FF);
  const unsigned f = (hi & 0x80000000u) | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  return __uint_as_float(e < 897 ? (hi & 0x80000000u) : f);
}
__device__ __forceinline__ double b_f64(float x) {  // exact for normal numbers
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long v = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  const unsigned long long z = (unsigned long long)(u & 0x80000000u) << 32;
  return __longlong_as_double((long long)(e == 0u ? z : v));
}
__device__ __forceinline__ B2 b_split(double x) {  // hi = x truncated to 24 bits, lo = the rest rounded
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = b_f32(x);
  const unsigned m = (unsigned)(b & 0x1FFFFFFFull);  // low 29 bits of the significand
  const float mh = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 6)), 8388608.0f);   // exact
  const float ml = __fsub_rn(__uint_as_float(0x4B000000u | (m & 63u)), 8388608.0f);  // exact
  const float mf = __fmaf_rn(mh, 64.0f, ml);
  const int es = e < 949 ? 949 : e;  // scale 2^(e - 1075) >= 2^-126
  const float lo = __fmul_rn(mf, __uint_as_float((unsigned)(es - 948) << 23));
  return B2(hi, __uint_as_float(e < 949 ? 0u : (__float_as_uint(lo) | sign)));
}

template <typename T> struct BAr;
template <> struct BAr<float> {
  static __device__ __forceinline__ float ld(double x) { return b_f32(x); }
  static __device__ __forceinline__ double st(float x) { return b_f64(x); }
  static __device__ __forceinline__ float f32(float x) { return x; }
};
template <> struct BAr<B2> {
  static __device__ __forceinline__ B2 ld(double x) { return b_split(x); }
  static __device__ __forceinline__ double st(B2 x) { df_renorm(x.h, x.l); return df_join_int(x.h, x.l); }
  static __device__ __forceinline__ float f32(B2 x) { return x.h; }
};
template <> struct BAr<double> {
  static __device__ __forceinline__ double ld(double x) { return x; }
  static __device__ __forceinline__ double st(double x) { return x; }
  static __device__ __forceinline__ float f32(double x) { return (float)x; }
};
// Gram accumulator: double-float sums (of FP32 chunk sums of FP32 products in the FP32 phase);
// double-float products and sums; FP64.
template <typename T> struct BAcc;
template <> struct BAcc<float> {
  float h = 0.f, l = 0.f;
  // a += x (TwoSum on the high part, the error kept in the low part)
  __device__ __forceinline__ void add_sum(float x) {
    const float s = h + x, bb = s - h;
    l += (h - (s - bb)) + (x - bb);
    h = s;
  }
  __device__ __forceinline__ void add(float a, float b) { add_sum(a * b); }
  __device__ __forceinline__ double get() const { return b_f64(h) + b_f64(l); }
};
template <> struct BAcc<B2> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(B2 a, B2 b) { df_mac(h, l, a.h, a.l, b.h, b.l); }
  __device__ __forceinline__ double get() const {
    float a = h, b = l;
    df_renorm(a, b);
    return b_f64(a) + b_f64(b);
  }
};
template <> struct BAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double get() const { return v; }
};

// Shared state of a CTA (static shared memory).
struct BShared {
  double G[BM * BM], Mg[BM * BM], C[BM * BM];
  double cf[BM * BM];        // coefficients converted to the phase's element type
  double theta[BM];
  double red[2][32][BNB];    // per-warp column sums (residual norms)
  double relres[BNB];
  int32_t idx[BM];           // active basis columns (soft locking)
  int32_t na;
  int32_t info;
  int32_t inst;
};

// The q x p coefficient matrix Cm (FP64, shared) in the element type T, converted once per call
// into sh.cf (FP64 needs no copy).
template <typename T>
__device__ __forceinline__ const T* b_coef(const double* Cm, int count, BShared& sh) {
  if constexpr (std::is_same<T, double>::value) return reinterpret_cast<const T*>(Cm);
  T* cf = reinterpret_cast<T*>(sh.cf);
  for (int e = threadIdx.x; e < count; e += blockDim.x) cf[e] = BAr<T>::ld(Cm[e]);
  __syncthreads();
  return cf;
}

// Layout of an instance's vectors: column-major blocks, element (r, j) of an n-row block B at
// B[j n + r], so the threads of a warp, taking consecutive rows, touch consecutive addresses.

// G (p x q, row-major, FP64, shared) = A^T B for the n x p block A and the n x q block B. Rows pass
// through shared memory (`stage`) in chunks of BRC, converted to the phase's element type once and
// loaded with consecutive threads on consecutive rows; each thread owns a 3 x 3 block of G over
// every rg-th row of a chunk, and the rg partial sums (FP64, `scratch`) are added in group order.
template <typename T>
__device__ void b_gram(int n, const double* A, int p, const double* B, int q, double* out, double* scratch,
                       unsigned char* stage) {
  using R = BAr<T>;
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool same = A == B && p == q;
  T* ta = reinterpret_cast<T*>(stage);  // [BRC][p]
  T* tb = same ? ta : ta + BRC * p;     // [BRC][q]
  const int bp = (p + 2) / 3, bq = (q + 2) / 3, nblk = bp * bq;
  int rg = nt / nblk;
  if (rg * p * q > BGSC) rg = BGSC / (p * q);
  if (rg < 1) rg = 1;
  const int g = tid / nblk, b = tid % nblk;
  const int a0 = (b / bq) * 3, b0 = (b % bq) * 3;
  const int na = g < rg ? min(3, p - a0) : 0, nq = g < rg ? min(3, q - b0) : 0;
  BAcc<T> acc[3][3];
  for (int r0 = 0; r0 < n; r0 += BRC) {
    const int rows = min(BRC, n - r0);
    for (int e = tid; e < BRC * p; e += nt) {
      const int j = e / BRC, i = e % BRC;
      ta[i * p + j] = i < rows ? R::ld(A[(int64_t)j * n + r0 + i]) : T(0);
    }
    if (!same)
      for (int e = tid; e < BRC * q; e += nt) {
        const int j = e / BRC, i = e % BRC;
        tb[i * q + j] = i < rows ? R::ld(B[(int64_t)j * n + r0 + i]) : T(0);
      }
    __syncthreads();
    if constexpr (std::is_same<T, float>::value) {
      // FP32 phase: a thread's products over its rows of the chunk (at most BRC) summed in FP32,
      // each chunk sum then added in double-float
      if (g < rg) {
        float cs[3][3];
#pragma unroll
        for (int u = 0; u < 3; u++)
#pragma unroll
          for (int v = 0; v < 3; v++) cs[u][v] = 0.f;
        for (int i = g; i < rows; i += rg) {
          float x[3], y[3];
#pragma unroll
          for (int u = 0; u < 3; u++) {
            x[u] = u < na ? ta[i * p + a0 + u] : 0.f;
            y[u] = u < nq ? tb[i * q + b0 + u] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 3; u++)
#pragma unroll
            for (int v = 0; v < 3; v++) cs[u][v] = fmaf(x[u], y[v], cs[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 3; u++)
#pragma unroll
          for (int v = 0; v < 3; v++) acc[u][v].add_sum(cs[u][v]);
      }
    } else {
      if (g < rg) {
        for (int i = g; i < rows; i += rg) {
          T x[3], y[3];
#pragma unroll
          for (int u = 0; u < 3; u++) {
            x[u] = u < na ? ta[i * p + a0 + u] : T(0);
            y[u] = u < nq ? tb[i * q + b0 + u] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 3; u++)
#pragma unroll
            for (int v = 0; v < 3; v++) acc[u][v].add(x[u], y[v]);
        }
      }
    }
    __syncthreads();
  }
  if (g < rg) {
#pragma unroll
    for (int u = 0; u < 3; u++)
#pragma unroll
      for (int v = 0; v < 3; v++)
        if (u < na && v < nq) scratch[g * p * q + (a0 + u) * q + b0 + v] = acc[u][v].get();
  }
  __syncthreads();
  for (int e = tid; e < p * q; e += nt) {
    double s = 0.0;
    for (int gg = 0; gg < rg; gg++) s += scratch[gg * p * q + e];
    out[e] = s;
  }
  __syncthreads();
}

// In place, row by row: the q columns of Y (and of HY when given) <- Y Cm, Cm q x q (shared,
// row-major FP64).
template <typename T>
__device__ void b_rotate(int n, double* Y, int q, const double* Cm, double* HY, BShared& sh) {
  using R = BAr<T>;
  const T* cf = b_coef<T>(Cm, q * q, sh);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    for (int pass = 0; pass < (HY ? 2 : 1); pass++) {
      double* y = pass ? HY : Y;
      T x[BNB];
#pragma unroll
      for (int a = 0; a < BNB; a++) x[a] = a < q ? R::ld(y[(int64_t)a * n + r]) : T(0);
#pragma unroll
      for (int b = 0; b < BNB; b++) {
        if (b >= q) continue;
        T s = T(0);
#pragma unroll
        for (int a = 0; a < BNB; a++)
          if (a < q) s += x[a] * cf[a * q + b];
        y[(int64_t)b * n + r] = R::st(s);
      }
    }
  }
  __syncthreads();
}

// Columns [c0, c0 + nb) of S <- themselves - S[:, 0:q] Z (Z = S[:, 0:q]^T S[:, c0:c0+nb], q x nb,
// shared), row by row; the same on HS when given (H applied to both sides of the projection).
template <typename T>
__device__ void b_project(int n, double* S, double* HS, int q, int c0, int nb, const double* Z, BShared& sh) {
  using R = BAr<T>;
  const T* cf = b_coef<T>(Z, q * nb, sh);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    for (int pass = 0; pass < (HS ? 2 : 1); pass++) {
      double* y = pass ? HS : S;
      double raw[2 * BNB], dst[BNB];
#pragma unroll
      for (int a = 0; a < 2 * BNB; a++) raw[a] = a < q ? y[(int64_t)a * n + r] : 0.0;
#pragma unroll
      for (int b = 0; b < BNB; b++) dst[b] = b < nb ? y[(int64_t)(c0 + b) * n + r] : 0.0;
      T acc[BNB];
#pragma unroll
      for (int b = 0; b < BNB; b++) acc[b] = R::ld(dst[b]);
#pragma unroll
      for (int a = 0; a < 2 * BNB; a++) {
        if (a >= q) continue;
        const T xa = R::ld(raw[a]);
#pragma unroll
        for (int b = 0; b < BNB; b++)
          if (b < nb) acc[b] -= xa * cf[a * nb + b];
      }
#pragma unroll
      for (int b = 0; b < BNB; b++)
        if (b < nb) y[(int64_t)(c0 + b) * n + r] = R::st(acc[b]);
    }
  }
  __syncthreads();
}

// The LOBPCG update (eq. 7) from the Rayleigh-Ritz coefficients C (m x m, shared): with
// C = [Cx; C2] split after row nb (first nb columns),
//   P <- S[:, nb:m] C2, X <- X Cx + P, and the same on HS; P goes to columns [2 nb, 3 nb).
// A thread streams over the m entries of its row (loads issued together, one value live at a
// time) into 2 nb accumulators.
template <typename T>
__device__ void b_update(int n, double* S, double* HS, int nb, int m, const double* C, BShared& sh) {
  using R = BAr<T>;
  const T* cf = b_coef<T>(C, m * m, sh);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    for (int pass = 0; pass < 2; pass++) {
      double* y = pass ? HS : S;
      double raw[BM];
#pragma unroll
      for (int a = 0; a < BM; a++) raw[a] = a < m ? y[(int64_t)a * n + r] : 0.0;
      T xv[BNB], pv[BNB];
#pragma unroll
      for (int j = 0; j < BNB; j++) { xv[j] = T(0); pv[j] = T(0); }
#pragma unroll
      for (int a = 0; a < BM; a++) {
        if (a >= m) continue;
        const T sa = R::ld(raw[a]);
#pragma unroll
        for (int j = 0; j < BNB; j++) {
          if (j >= nb) continue;
          if (a < nb) xv[j] += sa * cf[a * m + j];
          else pv[j] += sa * cf[a * m + j];
        }
      }
#pragma unroll
      for (int j = 0; j < BNB; j++) {
        if (j >= nb) continue;
        y[(int64_t)j * n + r] = R::st(xv[j] + pv[j]);
        y[(int64_t)(2 * nb + j) * n + r] = R::st(pv[j]);
      }
    }
  }
  __syncthreads();
}

// W <- HX - X diag(theta) into columns [nb, 2 nb); relres_j = ||w_j|| / (||H|| ||x_j||) into sh.relres.
template <typename T>
__device__ void b_residual(int n, double* S, const double* HS, int nb, double normH, BShared& sh) {
  using R = BAr<T>;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  float rr[BNB], xx[BNB];
  T th[BNB];
#pragma unroll
  for (int j = 0; j < BNB; j++) {
    rr[j] = 0.f;
    xx[j] = 0.f;
    th[j] = j < nb ? R::ld(sh.theta[j]) : T(0);
  }
  for (int r = tid; r < n; r += nt) {
#pragma unroll
    for (int j = 0; j < BNB; j++) {
      if (j >= nb) continue;
      const T x = R::ld(S[(int64_t)j * n + r]);
      const T w = R::ld(HS[(int64_t)j * n + r]) - th[j] * x;
      S[(int64_t)(nb + j) * n + r] = R::st(w);
      const float wf = R::f32(w), xf = R::f32(x);
      rr[j] += wf * wf;
      xx[j] += xf * xf;
    }
  }
#pragma unroll
  for (int j = 0; j < BNB; j++) {
    for (int o = 16; o > 0; o >>= 1) {
      rr[j] += __shfl_down_sync(0xFFFFFFFFu, rr[j], o);
      xx[j] += __shfl_down_sync(0xFFFFFFFFu, xx[j], o);
    }
    if (lane == 0) { sh.red[0][warp][j] = rr[j]; sh.red[1][warp][j] = xx[j]; }
  }
  __syncthreads();
  if (tid < nb) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nt / 32; w++) { a += sh.red[0][w][tid]; b += sh.red[1][w][tid]; }
    sh.relres[tid] = sqrt(a) / (normH * sqrt(b));
  }
  __syncthreads();
}

// HY = H X for one instance (X, HY: n x nb blocks): SELL slices of TS rows, a lane per slice row,
// 32 / TS slices per warp. X is first staged row-major into Xs in the phase's arithmetic: FP32
// (n x 8), double-float (n x (8 hi, 8 lo)) or FP64 (n x 8), so an entry's X row is one contiguous
// gather. Values: FP32, double-float (the FP32 value and the FP32-rounded remainder), FP64.
template <typename T, int TS>
__device__ void b_spmm(const BDev& d, const BInst& in, const double* X, double* HY, int nb, float* Xs) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int n = in.n;
  constexpr bool F32 = std::is_same<T, float>::value, DF = std::is_same<T, B2>::value;
  double* Xd = reinterpret_cast<double*>(Xs);
  for (int e = tid; e < n * BNB; e += nt) {
    const int j = e / n, r = e % n;  // consecutive threads: consecutive rows of one column
    const double x = j < nb ? X[(int64_t)j * n + r] : 0.0;
    if constexpr (F32) {
      Xs[r * BNB + j] = b_f32(x);
    } else if constexpr (DF) {
      const B2 f = b_split(x);
      Xs[r * 2 * BNB + j] = f.h;
      Xs[r * 2 * BNB + BNB + j] = f.l;
    } else {
      Xd[r * BNB + j] = x;
    }
  }
  __syncthreads();
  constexpr int SPW = 32 / TS;
  for (int sg = warp; sg * SPW < in.nsl; sg += nw) {
    const int s = sg * SPW + lane / TS, i = lane % TS;
    if (s >= in.nsl) continue;
    const int64_t base = d.soff[in.sl0 + s];
    const int w = (int)((d.soff[in.sl0 + s + 1] - base) / TS);
    const int r = s * TS + i;
    if constexpr (F32) {
      float acc[BNB];
#pragma unroll
      for (int j = 0; j < BNB; j++) acc[j] = 0.f;
      for (int t = 0; t < w; t++) {
        const int64_t e = base + (int64_t)t * TS + i;
        const int c = d.col[e];
        const float v = __ldg(d.v32 + e);
        const float4 x0 = *reinterpret_cast<const float4*>(Xs + c * BNB);  // written by this CTA: no __ldg
        const float4 x1 = *reinterpret_cast<const float4*>(Xs + c * BNB + 4);
        acc[0] = fmaf(v, x0.x, acc[0]); acc[1] = fmaf(v, x0.y, acc[1]);
        acc[2] = fmaf(v, x0.z, acc[2]); acc[3] = fmaf(v, x0.w, acc[3]);
        acc[4] = fmaf(v, x1.x, acc[4]); acc[5] = fmaf(v, x1.y, acc[5]);
        acc[6] = fmaf(v, x1.z, acc[6]); acc[7] = fmaf(v, x1.w, acc[7]);
      }
      if (r < n) {
#pragma unroll
        for (int j = 0; j < BNB; j++)
          if (j < nb) HY[(int64_t)j * n + r] = b_f64(acc[j]);
      }
    } else if constexpr (DF) {
      float ah[BNB], al[BNB];
#pragma unroll
      for (int j = 0; j < BNB; j++) { ah[j] = 0.f; al[j] = 0.f; }
      for (int t = 0; t < w; t++) {
        const int64_t e = base + (int64_t)t * TS + i;
        const int c = d.col[e];
        const float vh = __ldg(d.v32 + e), vl = __ldg(d.v32lo + e);
        const float* xr = Xs + c * 2 * BNB;
#pragma unroll
        for (int q = 0; q < BNB; q += 4) {
          const float4 xh = *reinterpret_cast<const float4*>(xr + q);
          const float4 xl = *reinterpret_cast<const float4*>(xr + BNB + q);
          df_mac(ah[q], al[q], vh, vl, xh.x, xl.x);
          df_mac(ah[q + 1], al[q + 1], vh, vl, xh.y, xl.y);
          df_mac(ah[q + 2], al[q + 2], vh, vl, xh.z, xl.z);
          df_mac(ah[q + 3], al[q + 3], vh, vl, xh.w, xl.w);
        }
      }
      if (r < n) {
#pragma unroll
        for (int j = 0; j < BNB; j++)
          if (j < nb) HY[(int64_t)j * n + r] = BAr<B2>::st(B2(ah[j], al[j]));
      }
    } else {
      double acc[BNB];
#pragma unroll
      for (int j = 0; j < BNB; j++) acc[j] = 0.0;
      for (int t = 0; t < w; t++) {
        const int64_t e = base + (int64_t)t * TS + i;
        const int c = d.col[e];
        const double v = __ldg(d.v64 + e);
        const double2* xr = reinterpret_cast<const double2*>(Xd + c * BNB);
#pragma unroll
        for (int q = 0; q < BNB / 2; q++) {
          const double2 x2 = xr[q];
          acc[2 * q] = fma(v, x2.x, acc[2 * q]);
          acc[2 * q + 1] = fma(v, x2.y, acc[2 * q + 1]);
        }
      }
      if (r < n) {
#pragma unroll
        for (int j = 0; j < BNB; j++)
          if (j < nb) HY[(int64_t)j * n + r] = acc[j];
      }
    }
  }
  __syncthreads();
}

}  // namespace

namespace {

// dynamic shared memory of a CTA: the Rayleigh-Ritz matrices of order 3 nb <= BM (rr_body<true>),
// also the scratch of the Gram partial sums
__host__ __device__ constexpr size_t rr_dsm_bytes() { return 5ull * 8 * BM * (BM + 1); }

// One Rayleigh-Ritz (chol = 0) or Cholesky-QR (chol = 1) solve of order m on the CTA, FP64, with
// the matrices in the dynamic shared memory; one copy of the code for every call site.
__device__ __noinline__ void b_rr(int m, const double* G, const double* Mg, double* theta, double* C, int32_t* info,
                                  int chol, unsigned char* dsm) {
  rr_body<true>(m, G, Mg, theta, C, info, nullptr, chol, dsm);
  __syncthreads();
}

enum { B_OK = 0, B_NOCONV = 1, B_BREAKDOWN = 2 };

// The Cholesky-QR of the active columns (bit j of act) of columns [c0, c0 + nb) of S (and HS when
// withH); the inactive columns are set to zero. With G the Gram matrix of the active columns and
// D = diag(G)^(-1/2), the equilibrated D G D = L L^T, C = D L^{-T}, then B <- B C. The scaling
// removes the spread of the column norms (columns near convergence are orders of magnitude shorter
// than the others) from the condition number the Cholesky factorisation sees. Returns the
// Cholesky status (0 = done; a zero active column, or no active column, counts as a failure).
template <typename T>
__device__ int b_cholqr(int n, double* S, double* HS, int c0, int nb, unsigned act, bool withH, BShared& sh,
                        unsigned char* dsm, double* scr) {
  b_gram<T>(n, S + (int64_t)c0 * n, nb, S + (int64_t)c0 * n, nb, sh.G, scr, dsm);
  if (threadIdx.x == 0) {
    int a = 0;
    for (int j = 0; j < nb; j++)
      if ((act >> j) & 1u) sh.idx[a++] = j;
    sh.na = a;
  }
  if (threadIdx.x < nb) {
    const double d = sh.G[threadIdx.x * nb + threadIdx.x];
    sh.theta[threadIdx.x] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  const int na = sh.na;
  for (int e = threadIdx.x; e < na * na; e += blockDim.x) {
    const int i = sh.idx[e / na], j = sh.idx[e % na];
    sh.Mg[e] = sh.G[i * nb + j] * sh.theta[i] * sh.theta[j];
  }
  int zero = na == 0;
  for (int a = 0; a < na; a++) zero |= sh.theta[sh.idx[a]] == 0.0;
  __syncthreads();
  if (zero) return 1;
  b_rr(na, sh.Mg, sh.Mg, sh.red[0][0], sh.G, &sh.info, 1, dsm);
  const int info = sh.info;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) sh.C[e] = 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < na * na; e += blockDim.x) {
    const int i = sh.idx[e / na], j = sh.idx[e % na];
    sh.C[i * nb + j] = sh.G[e] * sh.theta[i];
  }
  __syncthreads();
  if (info) return info;
  b_rotate<T>(n, S + (int64_t)c0 * n, nb, sh.C, withH ? HS + (int64_t)c0 * n : nullptr, sh);
  return 0;
}

// One phase of LOBPCG on one instance (T = float: the FP32 phase; double: FP64). Starts from the
// X in columns [0, nb) of S (any basis: it is orthonormalised and rotated to Ritz vectors first).
// Returns B_OK (the first k relative residuals reached target), B_NOCONV (iteration budget spent
// or, in the FP32 phase, stalled) or B_BREAKDOWN; *it counts the iterations.
template <typename T, int TS>
__device__ int b_phase(const BDev& d, const BInst& in, int inst, double* S, double* HS, float* Xs, double target,
                       int max_it, int* it, BShared& sh, unsigned char* dsm, double* scr) {
  const int n = in.n, nb = d.nb, k = d.k;
  // step 1: orthonormalise X, H X, Rayleigh-Ritz on X alone
  const unsigned all = (1u << nb) - 1u;
  if (b_cholqr<T>(n, S, HS, 0, nb, all, false, sh, dsm, scr)) return B_BREAKDOWN;
  b_spmm<T, TS>(d, in, S, HS, nb, Xs);
  b_gram<T>(n, S, nb, HS, nb, sh.G, scr, dsm);
  b_gram<T>(n, S, nb, S, nb, sh.Mg, scr, dsm);
  b_rr(nb, sh.G, sh.Mg, sh.theta, sh.C, &sh.info, 0, dsm);
  if (sh.info) return B_BREAKDOWN;
  b_rotate<T>(n, S, nb, sh.C, HS, sh);
  bool haveP = false, wretry = false;
  double best = 1e300;
  int best_it = 0;
  for (*it = 0;;) {
    b_residual<T>(n, S, HS, nb, in.normH, sh);
    double worst = 0.0;
    bool conv = true;
    for (int j = 0; j < k; j++) {
      if (!(sh.relres[j] <= target)) conv = false;
      worst = fmax(worst, sh.relres[j]);
    }
    if (conv) return B_OK;
    if (*it >= max_it) return B_NOCONV;
    if (worst < 0.5 * best) { best = worst; best_it = *it; }
    if (sizeof(T) == 4 && *it - best_it >= BSTALL) return B_NOCONV;
    // soft locking: a column whose residual is at the phase target keeps its X column in the
    // basis but drops its W and P columns (past the arithmetic's floor they would be rounding
    // noise, normalised to unit length, and H W, H P would no longer match them)
    unsigned act = 0u;
    for (int j = 0; j < nb; j++)
      if (!(sh.relres[j] <= target)) act |= 1u << j;
    // W <- W - X (X^T W) and Cholesky-QR of W, twice (CholQR2); a W whose Gram matrix is not
    // positive definite is replaced by random directions once
    for (int pass = 0; pass < 2;) {
      b_gram<T>(n, S, nb, S + (int64_t)nb * n, nb, sh.G, scr, dsm);
      b_project<T>(n, S, nullptr, nb, nb, nb, sh.G, sh);
      if (!b_cholqr<T>(n, S, HS, nb, nb, act, false, sh, dsm, scr)) { pass++; continue; }
      if (wretry) return B_BREAKDOWN;
      wretry = true;
      pass = 0;
      for (int e = threadIdx.x; e < n * nb; e += blockDim.x)
        S[(int64_t)(nb + e / n) * n + e % n] = b_rand(d.seed ^ 0xB10Cull, inst, e % n, nb + e / n + 97 * *it);
      __syncthreads();
    }
    wretry = false;
    b_spmm<T, TS>(d, in, S + (int64_t)nb * n, HS + (int64_t)nb * n, nb, Xs);
    // P <- P - [X W] ([X W]^T P) with H P alike, then Cholesky-QR of P's active columns with H P;
    // a P whose Gram matrix is not positive definite is dropped for this iteration
    bool pok = false;
    if (haveP) {
      b_gram<T>(n, S, 2 * nb, S + (int64_t)2 * nb * n, nb, sh.G, scr, dsm);
      b_project<T>(n, S, HS, 2 * nb, 2 * nb, nb, sh.G, sh);
      pok = !b_cholqr<T>(n, S, HS, 2 * nb, nb, act, true, sh, dsm, scr);
    }
    // Rayleigh-Ritz (eq. 9) on X and the active columns of W and P, the Gram matrices taken over
    // all of [X W P] and compacted; with P dropped if the compacted Gram matrix is not positive
    // definite
    for (;;) {
      const int m = pok ? 3 * nb : 2 * nb;
      b_gram<T>(n, S, m, HS, m, sh.G, scr, dsm);
      b_gram<T>(n, S, m, S, m, sh.Mg, scr, dsm);
      if (threadIdx.x == 0) {
        int a = 0;
        for (int j = 0; j < m; j++)
          if (j < nb || ((act >> (j % nb)) & 1u)) sh.idx[a++] = j;
        sh.na = a;
      }
      __syncthreads();
      const int mc = sh.na;
      for (int e = threadIdx.x; e < mc * mc; e += blockDim.x) {
        const int i = sh.idx[e / mc], j = sh.idx[e % mc];
        sh.cf[e] = sh.G[i * m + j];
        sh.C[e] = sh.Mg[i * m + j];
      }
      __syncthreads();
      b_rr(mc, sh.cf, sh.C, sh.theta, sh.G, &sh.info, 0, dsm);
      if (!sh.info) {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) sh.Mg[e] = 0.0;
        __syncthreads();
        for (int e = threadIdx.x; e < mc * nb; e += blockDim.x) sh.Mg[sh.idx[e / nb] * m + e % nb] = sh.G[(e / nb) * mc + e % nb];
        __syncthreads();
        b_update<T>(n, S, HS, nb, m, sh.Mg, sh);
        break;
      }
      if (!pok) return B_BREAKDOWN;
      pok = false;
      __syncthreads();
    }
    haveP = true;
    (*it)++;
  }
}

template <int TS>
__global__ void __launch_bounds__(BMAXT) k_batch_lobpcg(BDev d) {
  __shared__ BShared sh;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int tid = threadIdx.x;
  double* S = d.work + (int64_t)blockIdx.x * d.wstride;
  double* scr = S + d.wstride - BGSC;  // Gram partial sums
  for (;;) {
    if (tid == 0) {
      const int t = atomicAdd(d.ticket, 1);
      sh.inst = t < d.count ? d.order[t] : -1;
    }
    __syncthreads();
    const int inst = sh.inst;
    __syncthreads();
    if (inst < 0) break;
    const BInst in = d.inst[inst];
    const int n = in.n, nb = d.nb, ld = 3 * nb;
    double* HS = S + (int64_t)n * ld;
    float* Xs = reinterpret_cast<float*>(HS + (int64_t)n * ld);
    for (int e = tid; e < n * ld; e += blockDim.x) {
      const int j = e / n, r = e % n;
      S[e] = j < nb ? b_rand(d.seed, inst, r, j) : 0.0;
    }
    __syncthreads();
    int it1 = 0, it2 = 0, rc;
    if (d.mode == LOB_MODE_MIXED) {
      rc = b_phase<float, TS>(d, in, inst, S, HS, Xs, d.tol1, d.max_iter, &it1, sh, dsm, scr);
      if (rc != B_BREAKDOWN && !(rc == B_OK && d.tol1 <= d.tol))
        rc = b_phase<B2, TS>(d, in, inst, S, HS, Xs, d.tol, d.max_iter > it1 ? d.max_iter - it1 : 1, &it2, sh, dsm,
                             scr);
    } else {
      rc = b_phase<double, TS>(d, in, inst, S, HS, Xs, d.tol, d.max_iter, &it2, sh, dsm, scr);
    }
    if (tid < d.k) d.lambda[(int64_t)inst * d.k + tid] = sh.theta[tid];
    if (tid == 0) {
      d.status[inst] = rc == B_OK ? LOB_OK : (rc == B_NOCONV ? LOB_ERR_NOCONV : LOB_ERR_BREAKDOWN);
      d.iters[2 * inst] = it1 + it2;
      d.iters[2 * inst + 1] = it2;
    }
    if (d.X) {
      // unit 2-norm columns (the Rayleigh-Ritz vectors are S-orthonormal up to rounding)
      for (int e = tid; e < n * nb; e += blockDim.x)
        d.X[(in.row0 + e % n) * nb + e / n] = S[e];
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Building the SELL store on the device from the instances' upper-triangle COO.
// ---------------------------------------------------------------------------------------------
namespace {

// instance of global entry e: last i with eoff[i] <= e
__device__ __forceinline__ int b_inst_of(const int64_t* eoff, int count, int64_t e) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (eoff[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One instance's COO (int64 indices, FP64 values) into the batch's arrays (int32 local indices);
// bad entries (row > col, outside [0, n)) set *bad.
__global__ void k_b_gather(int64_t nnz, int64_t n, const int64_t* __restrict__ r, const int64_t* __restrict__ c,
                           const double* __restrict__ v, int32_t* __restrict__ ro, int32_t* __restrict__ co,
                           double* __restrict__ vo, int* __restrict__ bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t a = r[e], b = c[e];
  if (a < 0 || b >= n || a > b) { atomicOr(bad, 1); ro[e] = 0; co[e] = 0; vo[e] = 0.0; return; }
  ro[e] = (int32_t)a; co[e] = (int32_t)b; vo[e] = v[e];
}

// row lengths of both triangles and the row sums of |h_ij| (||H||_inf)
__global__ void k_b_count(int64_t ne, const int64_t* __restrict__ eoff, int count, const BInst* __restrict__ inst,
                          const int32_t* __restrict__ ro, const int32_t* __restrict__ co, const double* __restrict__ vo,
                          int32_t* __restrict__ rowlen, double* __restrict__ rowabs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int i = b_inst_of(eoff, count, e);
  const int64_t g0 = inst[i].row0;
  const int a = ro[e], b = co[e];
  const double av = fabs(vo[e]);
  atomicAdd(&rowlen[g0 + a], 1);
  atomicAdd(&rowabs[g0 + a], av);
  if (a != b) {
    atomicAdd(&rowlen[g0 + b], 1);
    atomicAdd(&rowabs[g0 + b], av);
  }
}

// ||H||_inf of each instance (one CTA per instance)
__global__ void k_b_norm(BInst* inst, const double* __restrict__ rowabs) {
  __shared__ double red[32];
  const BInst in = inst[blockIdx.x];
  double m = 0.0;
  for (int r = threadIdx.x; r < in.n; r += blockDim.x) m = fmax(m, rowabs[in.row0 + r]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmax(m, red[w]);
    inst[blockIdx.x].normH = m > 0.0 ? m : 1.0;
  }
}

// entries of each slice: its longest row times the tile height (slice s of instance i is global
// slice inst[i].sl0 + s); slices are enumerated through sl_inst (the instance of each slice)
__global__ void k_b_slice_size(int64_t nslices, const int32_t* __restrict__ sl_inst, const BInst* __restrict__ inst,
                               const int32_t* __restrict__ rowlen, int ts, int64_t* __restrict__ ssize) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  const BInst in = inst[sl_inst[s]];
  const int64_t r0 = (s - in.sl0) * ts;
  int w = 0;
  for (int i = 0; i < ts && r0 + i < in.n; i++) w = max(w, rowlen[in.row0 + r0 + i]);
  ssize[s] = (int64_t)w * ts;
}

// padding: every slot of a slice gets its own row as column (in range) and value zero
__global__ void k_b_pad(int64_t nslices, const int32_t* __restrict__ sl_inst, const BInst* __restrict__ inst,
                        const int64_t* __restrict__ soff, int ts, uint16_t* __restrict__ col, float* __restrict__ v32,
                        double* __restrict__ v64) {
  const int64_t s = blockIdx.x;
  if (s >= nslices) return;
  const BInst in = inst[sl_inst[s]];
  const int64_t base = soff[s], cnt = soff[s + 1] - base;
  const int64_t r0 = (s - in.sl0) * ts;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int64_t r = r0 + e % ts;
    col[base + e] = (uint16_t)(r < in.n ? r : in.n - 1);
    v32[base + e] = 0.f;
    v64[base + e] = 0.0;
  }
}

// scatter both triangles into their rows' slots (slot order fixed later by k_b_sort)
__global__ void k_b_fill(int64_t ne, const int64_t* __restrict__ eoff, int count, const BInst* __restrict__ inst,
                         const int32_t* __restrict__ ro, const int32_t* __restrict__ co, const double* __restrict__ vo,
                         const int64_t* __restrict__ soff, int ts, int32_t* __restrict__ fill,
                         uint16_t* __restrict__ col, float* __restrict__ v32, double* __restrict__ v64) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const BInst in = inst[b_inst_of(eoff, count, e)];
  const int a = ro[e], b = co[e];
  const double v = vo[e];
  for (int side = 0; side < (a != b ? 2 : 1); side++) {
    const int r = side ? b : a, c = side ? a : b;
    const int pos = atomicAdd(&fill[in.row0 + r], 1);
    const int64_t slot = soff[in.sl0 + r / ts] + (int64_t)pos * ts + r % ts;
    col[slot] = (uint16_t)c;
    v64[slot] = v;
    v32[slot] = __double2float_rn(v);
  }
}

// each row's entries in ascending column order (deterministic sums); a repeated column sets *bad
__global__ void k_b_sort(int64_t nrows, const int32_t* __restrict__ row_inst, const BInst* __restrict__ inst,
                         const int32_t* __restrict__ rowlen, const int64_t* __restrict__ soff, int ts,
                         uint16_t* __restrict__ col, float* __restrict__ v32, double* __restrict__ v64,
                         int* __restrict__ bad) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nrows) return;
  const BInst in = inst[row_inst[g]];
  const int r = (int)(g - in.row0), len = rowlen[g];
  const int64_t base = soff[in.sl0 + r / ts] + r % ts;
  for (int i = 1; i < len; i++) {
    const uint16_t c = col[base + (int64_t)i * ts];
    const float a = v32[base + (int64_t)i * ts];
    const double b = v64[base + (int64_t)i * ts];
    int j = i - 1;
    while (j >= 0 && col[base + (int64_t)j * ts] > c) {
      col[base + (int64_t)(j + 1) * ts] = col[base + (int64_t)j * ts];
      v32[base + (int64_t)(j + 1) * ts] = v32[base + (int64_t)j * ts];
      v64[base + (int64_t)(j + 1) * ts] = v64[base + (int64_t)j * ts];
      j--;
    }
    col[base + (int64_t)(j + 1) * ts] = c;
    v32[base + (int64_t)(j + 1) * ts] = a;
    v64[base + (int64_t)(j + 1) * ts] = b;
  }
  for (int i = 1; i < len; i++)
    if (col[base + (int64_t)i * ts] == col[base + (int64_t)(i - 1) * ts]) atomicOr(bad, 1);
}

// the low parts of the double-float values: v64 - v32 rounded to FP32 (zero in the padding)
__global__ void k_b_lo(int64_t ne, const float* __restrict__ v32, const double* __restrict__ v64,
                       float* __restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) lo[e] = __double2float_rn(v64[e] - (double)v32[e]);
}

template <typename X>
struct DMem {  // device array owned by the batch
  X* p = nullptr;
  size_t n = 0;
  DMem() = default;
  DMem(const DMem&) = delete;
  DMem& operator=(const DMem&) = delete;
  ~DMem() { if (p) cudaFree(p); }
  int alloc(size_t cnt) {
    if (p) { cudaFree(p); p = nullptr; }
    n = cnt;
    if (cudaMalloc((void**)&p, (cnt ? cnt : 1) * sizeof(X)) != cudaSuccess) { cudaGetLastError(); p = nullptr; return LOB_ERR_NOMEM; }
    return LOB_OK;
  }
};

// SELL store of the batch for one tile height
struct BSell {
  int ts = 0;
  int64_t nslices = 0, entries = 0;
  DMem<int64_t> soff;
  DMem<uint16_t> col;
  DMem<float> v32, v32lo;
  DMem<double> v64;
  DMem<BInst> inst;       // with this store's slice offsets
};

}  // namespace

struct lob_batch {
  int32_t count = 0;
  int64_t rows = 0, ne = 0;
  int32_t n_max = 0;
  std::vector<BInst> h_inst;      // n, row0 (slices filled per store)
  std::vector<int32_t> h_order;   // largest first
  DMem<int32_t> ro, co, row_inst, rowlen, order;
  DMem<double> vo, rowabs;
  DMem<int64_t> eoff;
  BSell sell[3];                  // tile heights 8, 16, 32 (built on demand)
  DMem<double> work;              // schedule workspace (grown on demand)
  DMem<int32_t> ticket;
  // autotuned schedule, kept for later calls with the same (k, nb, mode)
  int tuned_k = -1, tuned_nb = -1, tuned_mode = -1;
  int tuned_ts = 0, tuned_threads = 0, tuned_per_sm = 0;
  int sms = 0;
  int device = 0;
};

namespace {

int ts_slot(int ts) { return ts == 8 ? 0 : (ts == 16 ? 1 : (ts == 32 ? 2 : -1)); }

int build_sell(lob_batch* b, int ts, cudaStream_t st) {
  BSell& S = b->sell[ts_slot(ts)];
  if (S.ts == ts) return LOB_OK;
  std::vector<BInst> hi = b->h_inst;
  std::vector<int32_t> sl_inst;
  int64_t ns = 0;
  for (int i = 0; i < b->count; i++) {
    hi[i].nsl = (hi[i].n + ts - 1) / ts;
    hi[i].sl0 = ns;
    ns += hi[i].nsl;
    for (int s = 0; s < hi[i].nsl; s++) sl_inst.push_back(i);
  }
  DMem<int32_t> d_sl;
  DMem<int64_t> ssize;
  LOB_TRY(S.inst.alloc(b->count));
  LOB_TRY(d_sl.alloc(ns));
  LOB_TRY(ssize.alloc(ns + 1));
  LOB_TRY(S.soff.alloc(ns + 1));
  LOB_CUDA(cudaMemcpyAsync(S.inst.p, hi.data(), sizeof(BInst) * b->count, cudaMemcpyHostToDevice, st));
  LOB_CUDA(cudaMemcpyAsync(d_sl.p, sl_inst.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
  // ||H||_inf into the store's instance table
  (k_b_norm<<<b->count, 256, 0, st>>>(S.inst.p, b->rowabs.p), LOB_LAUNCHED());
  (k_b_slice_size<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, d_sl.p, S.inst.p, b->rowlen.p, ts, ssize.p),
   LOB_LAUNCHED());
  LOB_CUDA(cudaMemsetAsync(ssize.p + ns, 0, sizeof(int64_t), st));
  size_t tmp = 0;
  LOB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, ssize.p, S.soff.p, (int)(ns + 1), st));
  DMem<unsigned char> tbuf;
  LOB_TRY(tbuf.alloc(tmp));
  LOB_CUDA(cub::DeviceScan::ExclusiveSum(tbuf.p, tmp, ssize.p, S.soff.p, (int)(ns + 1), st));
  int64_t entries = 0;
  LOB_CUDA(cudaMemcpyAsync(&entries, S.soff.p + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaStreamSynchronize(st));
  LOB_TRY(S.col.alloc(entries + 8));
  LOB_TRY(S.v32.alloc(entries + 8));
  LOB_TRY(S.v32lo.alloc(entries + 8));
  LOB_TRY(S.v64.alloc(entries + 8));
  (k_b_pad<<<(unsigned)ns, 128, 0, st>>>(ns, d_sl.p, S.inst.p, S.soff.p, ts, S.col.p, S.v32.p, S.v64.p), LOB_LAUNCHED());
  DMem<int32_t> fill, bad;
  LOB_TRY(fill.alloc(b->rows));
  LOB_TRY(bad.alloc(1));
  LOB_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int32_t) * b->rows, st));
  LOB_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), st));
  if (b->ne > 0)
    (k_b_fill<<<(unsigned)((b->ne + 255) / 256), 256, 0, st>>>(b->ne, b->eoff.p, b->count, S.inst.p, b->ro.p, b->co.p,
                                                                b->vo.p, S.soff.p, ts, fill.p, S.col.p, S.v32.p,
                                                                S.v64.p),
     LOB_LAUNCHED());
  (k_b_sort<<<(unsigned)((b->rows + 127) / 128), 128, 0, st>>>(b->rows, b->row_inst.p, S.inst.p, b->rowlen.p, S.soff.p,
                                                               ts, S.col.p, S.v32.p, S.v64.p, bad.p),
   LOB_LAUNCHED());
  if (entries > 0)
    (k_b_lo<<<(unsigned)((entries + 255) / 256), 256, 0, st>>>(entries, S.v32.p, S.v64.p, S.v32lo.p), LOB_LAUNCHED());
  int hbad = 0;
  LOB_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaStreamSynchronize(st));
  if (hbad) return LOB_ERR_ARG;  // a repeated entry
  S.ts = ts;
  S.nslices = ns;
  S.entries = entries;
  return LOB_OK;
}

int64_t b_wstride(int n_max, int nb) {
  // S and HS (n_max x 3 nb FP64 each), Xs (n_max x 8 pairs of FP32) and the Gram partial sums, in
  // doubles, 32-byte aligned
  const int64_t d = 2ll * n_max * 3 * nb + (int64_t)n_max * BNB + BGSC;
  return (d + 3) & ~3ll;
}

struct BRun {
  int ts, threads, per_sm;
};

// One run of the schedule over the tickets [0, count) of `order` (a graph: ticket reset, kernel).
int b_run(lob_batch* b, const BRun& r, const int32_t* order, int count, int k, int nb, int mode, double tol,
          double tol1, int max_iter, uint64_t seed, double* lambda, int32_t* status, int32_t* iters, double* X,
          cudaStream_t st, double* ms) {
  const BSell& S = b->sell[ts_slot(r.ts)];
  const int grid = r.per_sm * b->sms;
  const int64_t ws = b_wstride(b->n_max, nb);
  DMem<double>& work = b->work;
  DMem<int32_t>& ticket = b->ticket;
  if (work.n < (size_t)ws * grid) LOB_TRY(work.alloc((size_t)ws * grid));
  if (!ticket.p) LOB_TRY(ticket.alloc(1));
  BDev d;
  d.inst = S.inst.p; d.order = order; d.count = count;
  d.soff = S.soff.p; d.col = S.col.p; d.v32 = S.v32.p; d.v32lo = S.v32lo.p; d.v64 = S.v64.p;
  d.work = work.p; d.wstride = ws; d.ticket = ticket.p;
  d.lambda = lambda; d.status = status; d.iters = iters; d.X = X;
  d.k = k; d.nb = nb; d.mode = mode; d.max_iter = max_iter; d.tol = tol; d.tol1 = tol1; d.seed = seed;
  const size_t dsm = rr_dsm_bytes();
  cudaStream_t cs = st;
  bool own = false;
  if (cs == nullptr || cs == cudaStreamLegacy) {  // capture needs a stream of its own
    LOB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    own = true;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LOB_OK;
  auto fail = [&](int code) { rc = code; };
  do {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { fail(LOB_ERR_CUDA); break; }
    cudaMemsetAsync(ticket.p, 0, sizeof(int32_t), cs);
    switch (r.ts) {
      case 8: k_batch_lobpcg<8><<<grid, r.threads, dsm, cs>>>(d); break;
      case 16: k_batch_lobpcg<16><<<grid, r.threads, dsm, cs>>>(d); break;
      default: k_batch_lobpcg<32><<<grid, r.threads, dsm, cs>>>(d); break;
    }
    LOB_LAUNCHED();
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) { fail(LOB_ERR_CUDA); break; }
    if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) { fail(LOB_ERR_CUDA); break; }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, cs);
    if (cudaGraphLaunch(ge, cs) != cudaSuccess) { fail(LOB_ERR_CUDA); break; }
    cudaEventRecord(e1, cs);
    if (cudaStreamSynchronize(cs) != cudaSuccess) { fail(LOB_ERR_CUDA); break; }
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    *ms = f;
  } while (0);
  if (rc != LOB_OK) cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (own) cudaStreamDestroy(cs);
  return rc;
}

int b_set_attrs() {
  const int dsm = (int)rr_dsm_bytes();
  LOB_CUDA(cudaFuncSetAttribute(k_batch_lobpcg<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
  LOB_CUDA(cudaFuncSetAttribute(k_batch_lobpcg<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
  LOB_CUDA(cudaFuncSetAttribute(k_batch_lobpcg<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
  return LOB_OK;
}

int b_max_resident(int ts, int threads) {
  int nbk = 0;
  const size_t dsm = rr_dsm_bytes();
  cudaError_t e = ts == 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_batch_lobpcg<8>, threads, dsm)
                : ts == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_batch_lobpcg<16>, threads, dsm)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, k_batch_lobpcg<32>, threads, dsm);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return nbk;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" int lob_batch_create(int32_t count, const lob_coo* H, void* stream, lob_batch** out) {
  if (!out || !H || count < 1) return LOB_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; i++) {
    const lob_coo& h = H[i];
    if (h.n < 1 || h.n > 65535 || h.nnz < 1 || !h.row || !h.col || !h.val) return LOB_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  lob_batch* b = new lob_batch();
  auto fail = [&](int rc) { delete b; return rc; };
  b->count = count;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return fail(LOB_ERR_CUDA);
  b->h_inst.resize(count);
  std::vector<int64_t> eoff(count + 1, 0);
  for (int i = 0; i < count; i++) {
    BInst& in = b->h_inst[i];
    in.n = (int32_t)H[i].n;
    in.row0 = b->rows;
    in.nsl = 0;
    in.sl0 = 0;
    in.normH = 1.0;
    b->rows += H[i].n;
    b->n_max = std::max<int32_t>(b->n_max, in.n);
    eoff[i + 1] = eoff[i] + H[i].nnz;
  }
  b->ne = eoff[count];
  int rc;
  if ((rc = b->ro.alloc(b->ne)) || (rc = b->co.alloc(b->ne)) || (rc = b->vo.alloc(b->ne)) ||
      (rc = b->eoff.alloc(count + 1)) || (rc = b->rowlen.alloc(b->rows)) || (rc = b->rowabs.alloc(b->rows)) ||
      (rc = b->row_inst.alloc(b->rows)) || (rc = b->order.alloc(count)))
    return fail(rc);
  DMem<int> bad;
  DMem<BInst> dinst;
  if ((rc = bad.alloc(1)) || (rc = dinst.alloc(count))) return fail(rc);
  if (cudaMemsetAsync(bad.p, 0, sizeof(int), st) != cudaSuccess) return fail(LOB_ERR_CUDA);
  // gather every instance's COO into the batch arrays (host inputs through one staging copy)
  int64_t host_ne = 0;
  for (int i = 0; i < count; i++)
    if (!H[i].on_device) host_ne += H[i].nnz;
  DMem<int64_t> hr, hc;
  DMem<double> hv;
  if (host_ne) {
    if ((rc = hr.alloc(host_ne)) || (rc = hc.alloc(host_ne)) || (rc = hv.alloc(host_ne))) return fail(rc);
  }
  int64_t hpos = 0;
  for (int i = 0; i < count; i++) {
    const lob_coo& h = H[i];
    const int64_t* r = h.row;
    const int64_t* c = h.col;
    const double* v = h.val;
    if (!h.on_device) {
      if (cudaMemcpyAsync(hr.p + hpos, h.row, sizeof(int64_t) * h.nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(hc.p + hpos, h.col, sizeof(int64_t) * h.nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(hv.p + hpos, h.val, sizeof(double) * h.nnz, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(LOB_ERR_CUDA);
      r = hr.p + hpos;
      c = hc.p + hpos;
      v = hv.p + hpos;
      hpos += h.nnz;
    }
    k_b_gather<<<(unsigned)((h.nnz + 255) / 256), 256, 0, st>>>(h.nnz, h.n, r, c, v, b->ro.p + eoff[i],
                                                                 b->co.p + eoff[i], b->vo.p + eoff[i], bad.p);
    LOB_LAUNCHED();
  }
  std::vector<int32_t> row_inst(b->rows);
  for (int i = 0; i < count; i++)
    for (int r = 0; r < b->h_inst[i].n; r++) row_inst[b->h_inst[i].row0 + r] = i;
  // largest instances first (ties: lower index first), so the last tickets are the short solves
  b->h_order.resize(count);
  for (int i = 0; i < count; i++) b->h_order[i] = i;
  std::stable_sort(b->h_order.begin(), b->h_order.end(),
                   [&](int x, int y) { return b->h_inst[x].n > b->h_inst[y].n; });
  if (cudaMemcpyAsync(b->eoff.p, eoff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(b->row_inst.p, row_inst.data(), sizeof(int32_t) * b->rows, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(b->order.p, b->h_order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync(dinst.p, b->h_inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice, st) ||
      cudaMemsetAsync(b->rowlen.p, 0, sizeof(int32_t) * b->rows, st) ||
      cudaMemsetAsync(b->rowabs.p, 0, sizeof(double) * b->rows, st))
    return fail(LOB_ERR_CUDA);
  if (b->ne > 0) {
    k_b_count<<<(unsigned)((b->ne + 255) / 256), 256, 0, st>>>(b->ne, b->eoff.p, count, dinst.p, b->ro.p, b->co.p,
                                                              b->vo.p, b->rowlen.p, b->rowabs.p);
    LOB_LAUNCHED();
  }
  int hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LOB_ERR_CUDA);
  if (hbad) return fail(LOB_ERR_ARG);
  if ((rc = b_set_attrs())) return fail(rc);
  // the default slice height's store now: repeated entries are found while it is built
  if ((rc = build_sell(b, 16, st))) return fail(rc);
  *out = b;
  return LOB_OK;
}

extern "C" int lob_batch_destroy(lob_batch* b) {
  if (b) {
    int dev = 0;
    const int own = b->device;
    cudaGetDevice(&dev);
    if (dev != own) cudaSetDevice(own);
    cudaDeviceSynchronize();
    delete b;
    if (dev != own) cudaSetDevice(dev);
  }
  return LOB_OK;
}

namespace {

// the autotuner's candidate schedules (tile height, threads per CTA, CTAs per SM)
const BRun kCandidates[] = {{8, 128, 4},  {8, 256, 2},  {8, 256, 4},  {8, 512, 1},  {8, 512, 2},
                            {16, 128, 4}, {16, 256, 2}, {16, 256, 4}, {16, 512, 1}, {16, 512, 2},
                            {32, 128, 4}, {32, 256, 2}, {32, 256, 4}, {32, 512, 1}, {32, 512, 2}};

}  // namespace

extern "C" int lob_batch_solve(lob_batch* b, const lob_batch_opts* o, double* lambda, int32_t* status, int32_t* iters,
                               double* X, lob_batch_stats* stt) {
  if (!b || !o || !lambda || !status) return LOB_ERR_ARG;
  const int k = o->k, nb = o->nb, mode = o->mode;
  if (nb < 1 || nb > BNB || k < 1 || k > nb || (mode != LOB_MODE_FP64 && mode != LOB_MODE_MIXED)) return LOB_ERR_ARG;
  if (!(o->tol > 0.0) || o->max_iter < 0 || o->mixed_tol < 0.0) return LOB_ERR_ARG;
  if (o->tile && ts_slot(o->tile) < 0) return LOB_ERR_ARG;
  if (o->threads && (o->threads < 64 || o->threads > BMAXT || o->threads % 32)) return LOB_ERR_ARG;
  if (o->per_sm < 0 || o->tune_iter < 0) return LOB_ERR_ARG;
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)o->stream;
  const int max_iter = o->max_iter ? o->max_iter : 500;
  const double tol1 = o->mixed_tol > 0.0 ? o->mixed_tol : std::max(o->tol, 1e-6);
  lob_batch_stats s{};
  // iteration counters for the tuning runs and when the caller passes none
  DMem<int32_t> it_scratch;
  int32_t* it_out = iters;
  if (!it_out) {
    LOB_TRY(it_scratch.alloc(2ull * b->count));
    it_out = it_scratch.p;
  }
  BRun run{o->tile, o->threads, o->per_sm};
  const bool need_tune = !run.ts || !run.threads || !run.per_sm;
  const bool have_tuned = b->tuned_k == k && b->tuned_nb == nb && b->tuned_mode == mode && b->tuned_ts;
  if (need_tune && have_tuned) {
    if (!run.ts) run.ts = b->tuned_ts;
    if (!run.threads) run.threads = b->tuned_threads;
    if (!run.per_sm) run.per_sm = b->tuned_per_sm;
  } else if (need_tune) {
    // time every candidate that matches the fixed fields, on all instances for a few iterations
    const auto t0 = std::chrono::steady_clock::now();
    const int tune_iter = o->tune_iter ? o->tune_iter : 4;
    double best = 1e300;
    BRun pick{0, 0, 0};
    for (const BRun& c0 : kCandidates) {
      BRun c = c0;
      if ((run.ts && c.ts != run.ts) || (run.threads && c.threads != run.threads)) continue;
      if (run.per_sm) c.per_sm = run.per_sm;
      const int fit = b_max_resident(c.ts, c.threads);
      if (fit < 1) continue;
      c.per_sm = std::min(c.per_sm, fit);
      LOB_TRY(build_sell(b, c.ts, st));
      double ms = 0.0;
      LOB_TRY(b_run(b, c, b->order.p, b->count, k, nb, mode, o->tol, tol1, tune_iter, o->seed, lambda, status,
                    it_out, nullptr, st, &ms));
      s.candidates++;
      if (ms < best) { best = ms; pick = c; }
    }
    if (!pick.ts) return LOB_ERR_ARG;  // nothing fits
    run = pick;
    if (!o->tile && !o->threads && !o->per_sm) {
      b->tuned_k = k; b->tuned_nb = nb; b->tuned_mode = mode;
      b->tuned_ts = pick.ts; b->tuned_threads = pick.threads; b->tuned_per_sm = pick.per_sm;
    }
    s.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  const int fit = b_max_resident(run.ts, run.threads);
  if (fit < 1) return LOB_ERR_ARG;
  run.per_sm = std::min(run.per_sm, fit);
  LOB_TRY(build_sell(b, run.ts, st));
  double ms = 0.0;
  LOB_TRY(b_run(b, run, b->order.p, b->count, k, nb, mode, o->tol, tol1, max_iter, o->seed, lambda, status, it_out,
                X, st, &ms));
  s.tile = run.ts;
  s.threads = run.threads;
  s.per_sm = run.per_sm;
  s.kernel_ms = ms;
  s.rows = b->rows;
  s.entries = b->sell[ts_slot(run.ts)].entries;
  s.work_bytes = (int64_t)b->work.n * 8;
  s.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (stt) *stt = s;
  return LOB_OK;
}
