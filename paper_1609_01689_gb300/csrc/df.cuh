// Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers,
// giving about 48 significant bits on the FP32 pipes. The FP64 pipe of this GPU runs at
// 1/70 of the FP32 rate, so the FP64-class block products (Section 4.4, footnote 5) use
// this representation; their error bounds are stated where they are used.
//
// Building blocks (error-free transformations):
//   TwoSum(a, b) = (s, t) with s = fl(a + b) and a + b = s + t exactly (Knuth);
//   TwoProd(a, b) = (p, e) with p = fl(a * b) and a * b = p + e exactly, e = fma(a, b, -p).
// The intrinsics __fadd_rn / __fmul_rn / __fsub_rn are never contracted or reassociated.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// x = hi + lo with hi = x truncated to 24 significant bits (exact in FP32) and lo = the
// remainder rounded to FP32, so |x - (hi + lo)| <= 2^-48 |x|. Integer and FP32 operations
// only, for 2^-74 <= |x| < 2^128; other magnitudes (including 0) take the conversion path.
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 949 || e > 1150) {
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    return make_float2(hi, lo);
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  const unsigned m = (unsigned)(b & 0x1FFFFFFFull);  // low 29 bits of the significand
  const float mh = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 6)), 8388608.0f);   // exact
  const float ml = __fsub_rn(__uint_as_float(0x4B000000u | (m & 63u)), 8388608.0f);  // exact
  const float mf = __fmaf_rn(mh, 64.0f, ml);  // m, correctly rounded to 24 bits
  const float lo = __fmul_rn(mf, __uint_as_float((unsigned)(e - 948) << 23));  // * 2^(e-1075), exact
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// hi + lo rounded to FP64.
__device__ __forceinline__ double df_join(float hi, float lo) { return (double)hi + (double)lo; }

// Renormalise so that |lo| <= ulp(hi)/2 (Fast2Sum; valid because |lo| is small against hi
// or hi == 0).
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// a += x * y with x = (xh, xl), y = (yh, yl). The hi-hi product is exact (TwoProd), the
// cross products are added to the low part (their own rounding is ~2^-48 relative), the
// lo*lo term (~2^-48) is dropped, and the addition into a.hi is error-free (TwoSum) with its
// error kept in a.lo. a.lo is not renormalised here; call df_renorm at the end.
__device__ __forceinline__ void df_mac(float& ahi, float& alo, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -p);
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  const float s = __fadd_rn(ahi, p);
  const float bb = __fsub_rn(s, ahi);
  const float t = __fadd_rn(__fsub_rn(ahi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  ahi = s;
  alo = __fadd_rn(alo, __fadd_rn(t, e));
}

// a += b for two df numbers (TwoSum on the high parts, low parts summed).
__device__ __forceinline__ void df_add(float& ahi, float& alo, float bh, float bl) {
  const float s = __fadd_rn(ahi, bh);
  const float bb = __fsub_rn(s, ahi);
  const float t = __fadd_rn(__fsub_rn(ahi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  ahi = s;
  alo = __fadd_rn(alo, __fadd_rn(t, bl));
}

// x rounded toward zero to FP32 using integer operations in the normal range (2^-126 <= |x|
// < 2^128); other magnitudes use the conversion instruction.
__device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 897 || e > 1150) return __double2float_rz(x);
  return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                         (unsigned)((b >> 29) & 0x7FFFFFu));
}

// Exact widening of an FP32 value to FP64 with integer operations (normal numbers and zero);
// subnormal, infinite and NaN inputs use the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
    return (double)f;
  }
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// hi + lo rounded to FP64 using integer operations only (no FP64 instructions): both parts
// are put on a common fixed-point scale where hi fills the top 24 of 54 bits, added as
// integers, and the sum is normalised and rounded to 53 bits (ties to even). Parts of lo below
// 2^-29 ulp(hi) are rounded away first, so the result is within one FP64 ulp of hi + lo.
// Normal FP32 inputs; zero, subnormal, infinite or NaN parts use the FP64 path.
__device__ __forceinline__ double df_join_int(float hi, float lo) {
  const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = (int)((uh >> 23) & 0xFF), el = (int)((ul >> 23) & 0xFF);
  if (eh == 0 || eh == 0xFF || el == 0xFF || (el == 0 && (ul & 0x7FFFFFFFu) != 0)) return (double)hi + (double)lo;
  long long mh = (long long)((uh & 0x7FFFFFu) | 0x800000u);
  if (uh >> 31) mh = -mh;
  long long s = mh << 29;  // hi as an integer at scale 2^(eh - 127 - 23 - 29)
  if (el != 0) {
    long long ml = (long long)((ul & 0x7FFFFFu) | 0x800000u);
    if (ul >> 31) ml = -ml;
    const int d = eh - el;  // lo is 2^-d times hi's scale
    if (d < 24) return (double)hi + (double)lo;  // not a renormalised pair
    if (d <= 29) s += ml << (29 - d);
    else if (d < 29 + 26) {
      const int sh = d - 29;  // round ml / 2^sh to nearest (ties away; below FP64 resolution)
      const long long half = 1ll << (sh - 1);
      s += (ml >= 0) ? ((ml + half) >> sh) : -((-ml + half) >> sh);
    }
  }
  if (s == 0) return 0.0;
  const unsigned long long sign = s < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = (unsigned long long)(s < 0 ? -s : s);
  const int lz = __clzll((long long)m);  // m < 2^55
  // normalise to 53 significant bits with round-to-nearest-even
  const int shift = (64 - lz) - 53;      // >= -? (m has at least 25 bits when nonzero hi)
  long long e2 = (long long)eh - 127 - 23 - 29 + (64 - lz - 1);  // unbiased exponent of the result
  if (shift > 0) {
    const unsigned long long rem = m & ((1ull << shift) - 1), halfway = 1ull << (shift - 1);
    m >>= shift;
    if (rem > halfway || (rem == halfway && (m & 1ull))) {
      m++;
      if (m == (1ull << 53)) { m >>= 1; e2++; }
    }
  } else if (shift < 0) {
    m <<= -shift;
  }
  if (e2 < -1022 || e2 > 1023) return (double)hi + (double)lo;
  const unsigned long long bits = sign | ((unsigned long long)(e2 + 1023) << 52) | (m & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// ---- double-float values as a pair type, for small dense kernels ----
struct d2 {
  float hi, lo;
};
__device__ __forceinline__ d2 d2_from(double x) { const float2 f = df_split(x); return d2{f.x, f.y}; }
__device__ __forceinline__ double d2_to(d2 a) { df_renorm(a.hi, a.lo); return df_join_int(a.hi, a.lo); }
__device__ __forceinline__ double d2_hi64(d2 a) { return f32_to_f64(a.hi); }  // leading part only
__device__ __forceinline__ d2 d2_norm(d2 a) { df_renorm(a.hi, a.lo); return a; }
// a * b (TwoProd on the high parts, cross terms into the low part)
__device__ __forceinline__ d2 d2_mul(d2 a, d2 b) {
  d2 r{0.f, 0.f};
  df_mac(r.hi, r.lo, a.hi, a.lo, b.hi, b.lo);
  return d2_norm(r);
}
__device__ __forceinline__ d2 d2_add(d2 a, d2 b) {
  df_add(a.hi, a.lo, b.hi, b.lo);
  return d2_norm(a);
}
__device__ __forceinline__ d2 d2_neg(d2 a) { return d2{-a.hi, -a.lo}; }
// c x - s y and s x + c y (one plane rotation of the pair (x, y))
__device__ __forceinline__ void d2_rot(d2& x, d2& y, d2 c, d2 s) {
  d2 u{0.f, 0.f}, v{0.f, 0.f};
  df_mac(u.hi, u.lo, c.hi, c.lo, x.hi, x.lo);
  df_mac(u.hi, u.lo, -s.hi, -s.lo, y.hi, y.lo);
  df_mac(v.hi, v.lo, s.hi, s.lo, x.hi, x.lo);
  df_mac(v.hi, v.lo, c.hi, c.lo, y.hi, y.lo);
  x = d2_norm(u);
  y = d2_norm(v);
}
// 1/sqrt(x) for x > 0 in double-float: FP32 estimate refined by one Newton step done in
// double-float (y1 = y0 + y0 (1 - x y0^2) / 2; relative error ~ (3/2) e0^2 ~ 2^-43).
__device__ __forceinline__ d2 d2_rsqrt(d2 x) {
  const float y0 = rsqrtf(x.hi);
  const d2 y2 = d2_mul(d2{y0, 0.f}, d2{y0, 0.f});
  const d2 r = d2_add(d2{1.f, 0.f}, d2_neg(d2_mul(x, y2)));
  const d2 corr = d2_mul(d2{0.5f * y0, 0.f}, r);
  return d2_add(d2{y0, 0.f}, corr);
}

// One CTA of 256 threads, rows [256 blk, 256 blk + 256) of the residual R = HX - X diag(theta)
// (Algorithm 1, step 4): R written (FP64), and the CTA's column sums of (r / ||H||)^2 and x^2
// (step 5) into part[blk][0 .. 2 nb). Thread t takes column t mod NBP (NBP = nb rounded up to a
// power of two) and every (256 / NBP)-th row, so a warp reads whole 8-byte-column rows
// (coalesced). Squares are summed in FP32 -- the norms decide convergence at relative accuracy
// ~1e-6, which is plenty -- in a fixed order (registers, lanes, warps), and each CTA's sum is
// stored as FP64. sred: 8 x 64 floats. nb <= 32.
__device__ __forceinline__ void lob_residual_rows(int64_t n, int nb, const double* __restrict__ X, int ldx,
                                                  const double* __restrict__ HX, int ldh,
                                                  const double* __restrict__ theta, double inv_norm,
                                                  double* __restrict__ R, double* __restrict__ part, int64_t blk,
                                                  float* sred) {
  const int tid = threadIdx.x;
  int NBP = 1;
  while (NBP < nb) NBP <<= 1;
  const int c = tid % NBP, r0 = tid / NBP, rstep = 256 / NBP;
  const float sc = (float)inv_norm;
  float rr = 0.f, xx = 0.f;
  if (c < nb) {
    const double th = theta[c];
    for (int i = r0; i < 256; i += rstep) {
      const int64_t r = blk * 256 + i;
      if (r >= n) break;
      const double x = X[r * ldx + c];
      const double v = HX[r * ldh + c] - x * th;
      R[r * nb + c] = v;
      const float vs = f64_to_f32_rz(v) * sc, xf = f64_to_f32_rz(x);
      rr = fmaf(vs, vs, rr);
      xx = fmaf(xf, xf, xx);
    }
  }
  for (int o = NBP; o < 32; o <<= 1) {
    rr += __shfl_xor_sync(0xFFFFFFFFu, rr, o);
    xx += __shfl_xor_sync(0xFFFFFFFFu, xx, o);
  }
  const int warp = tid / 32, lane = tid % 32;
  if (lane < NBP) {
    sred[warp * 64 + lane] = rr;
    sred[warp * 64 + 32 + lane] = xx;
  }
  __syncthreads();
  if (tid < nb) {
    double s = 0.0, t = 0.0;
    for (int w = 0; w < 8; w++) {
      s += (double)sred[w * 64 + tid];
      t += (double)sred[w * 64 + 32 + tid];
    }
    part[blk * 2 * nb + tid] = s;
    part[blk * 2 * nb + nb + tid] = t;
  }
}
