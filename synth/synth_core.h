/* Seeded synthetic Hamiltonian generator: the per-entry definition shared by the
 * host (C) and device (CUDA) generators so both produce the same matrix bit for bit.
 *
 * This module holds input generation only. None of the eigensolver's arithmetic
 * lives here. Both the CPU oracle and the CUDA path consume its output.
 *
 * The matrix imitates the structure the paper describes for nuclear CI Hamiltonians.
 * The paper orders basis states by total oscillator quanta (Section 2.1, eq. 3). States
 * interact only within a bounded difference of single-particle content (Section 2.2),
 * which gives a graded diagonal and block-banded coupling between neighbouring
 * truncation levels. The paper's matrices themselves are not available. The recipe:
 *   levels q = 0..Q, level sizes proportional to 2.2^q (largest-remainder rounding);
 *   diagonal  h_ii = 10*q_i + U(-1,1);
 *   each row draws m = ceil(f*nu) partners in levels q-2..q+2, centred on the row's
 *   relative position inside its level, within a half-width w (band); f = 0.6 unless the
 *   layout sets it (draw_pct), chosen so the symmetric union holds about nu per full row;
 *   off-diagonal value 0.3*(sum of 12 uniforms - 6)  (Irwin-Hall, mean 0, var 0.09),
 *   a function of the unordered pair so that the symmetric union is consistent.
 * All arithmetic that decides a structure is integer. The values use exact integer
 * sums, one power-of-two scaling and one rounding multiply, so host and device agree.
 */
#ifndef SYNTH_CORE_H
#define SYNTH_CORE_H
#include <stdint.h>

#ifdef __CUDACC__
#define SYN_HD __host__ __device__ __forceinline__
#else
#define SYN_HD static inline
#endif

#define SYN_MAX_LEVELS 32

/* splitmix64 finaliser (Steele, Lea, Flood 2014; public-domain reference by Vigna). */
SYN_HD uint64_t syn_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Counter-based hash of (seed, stream tag, a, b, c). */
SYN_HD uint64_t syn_hash(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c) {
  uint64_t h = syn_mix(seed ^ (tag * 0xD1B54A32D192ED03ull));
  h = syn_mix(h ^ a);
  h = syn_mix(h ^ (b * 0x9E3779B97F4A7C15ull));
  return syn_mix(h ^ (c * 0xC2B2AE3D27D4EB4Full));
}

enum { SYN_TAG_LEVEL = 1, SYN_TAG_OFFSET = 2, SYN_TAG_VALUE = 3, SYN_TAG_DIAG = 4 };

typedef struct {
  int64_t n;
  int32_t Q;          /* levels 0..Q */
  int32_t nu;         /* target nonzeros per full row (both triangles) */
  int32_t w_min;      /* band half-width floor */
  int32_t w_div;      /* if > 0, half-width = max(w_min, ceil(c_q / w_div)) */
  int32_t draw_pct;   /* draws per row in percent of nu; 0 = 60 */
  int32_t reserved;
  uint64_t seed;
  int64_t start[SYN_MAX_LEVELS + 1]; /* level q occupies rows [start[q], start[q+1]) */
} syn_layout;

SYN_HD int syn_level_of(const syn_layout* L, int64_t i) {
  int q = 0;
  while (q < L->Q && i >= L->start[q + 1]) q++;
  return q;
}

SYN_HD int64_t syn_halfwidth(const syn_layout* L, int q) {
  int64_t c = L->start[q + 1] - L->start[q];
  int64_t w = L->w_min;
  if (L->w_div > 0) {
    int64_t w2 = (c + L->w_div - 1) / L->w_div;
    if (w2 > w) w = w2;
  }
  return w;
}

/* ceil(f*nu) draws per row, f = draw_pct / 100 (default 0.6): the symmetric union with
 * duplicates merged then holds about nu entries per full row. Half as many draws would leave it
 * ~15% short at nu = 200; with more draws per band slot (larger nu) more of them coincide, and the
 * layout raises f to keep the row count at nu. */
SYN_HD int64_t syn_draws(const syn_layout* L) {
  const int64_t pct = L->draw_pct > 0 ? L->draw_pct : 60;
  return (pct * (int64_t)L->nu + 99) / 100;
}

/* floor(v / 2^32) for signed v, without relying on arithmetic right shift. */
SYN_HD int64_t syn_floor_div_2p32(int64_t v) {
  if (v >= 0) return v >> 32;
  return -(int64_t)(((uint64_t)(-v) + 0xFFFFFFFFull) >> 32);
}

/* Partner column for draw d of row i, or -1 if the draw lands on the diagonal. */
SYN_HD int64_t syn_partner(const syn_layout* L, int64_t i, int64_t d) {
  int q = syn_level_of(L, i);
  int lo = q - 2 < 0 ? 0 : q - 2;
  int hi = q + 2 > L->Q ? L->Q : q + 2;
  uint64_t h1 = syn_hash(L->seed, SYN_TAG_LEVEL, (uint64_t)i, (uint64_t)d, 0);
  int qp = lo + (int)(h1 % (uint64_t)(hi - lo + 1));
  int64_t sq = L->start[q], cq = L->start[q + 1] - sq;
  int64_t sp = L->start[qp], cp = L->start[qp + 1] - sp;
  if (cp <= 0 || cq <= 0) return -1;
  /* centre = floor((i - s_q + 1/2) / c_q * c_p), computed exactly in integers */
  int64_t centre = ((2 * (i - sq) + 1) * cp) / (2 * cq);
  uint64_t U = syn_hash(L->seed, SYN_TAG_OFFSET, (uint64_t)i, (uint64_t)d, 0) >> 32;
  int64_t w = syn_halfwidth(L, qp);
  int64_t off = syn_floor_div_2p32(((int64_t)(2 * U) - (int64_t)4294967296ll) * w); /* in [-w, w-1] */
  int64_t j = sp + centre + off;
  if (j < sp) j = sp;
  if (j > sp + cp - 1) j = sp + cp - 1;
  if (j == i) return -1;
  return j;
}

/* Off-diagonal value of the unordered pair (i, j), i < j. */
SYN_HD double syn_offdiag(uint64_t seed, int64_t i, int64_t j) {
  int64_t s = 0;
  for (int t = 0; t < 12; t++) s += (int64_t)(syn_hash(seed, SYN_TAG_VALUE, (uint64_t)i, (uint64_t)j, (uint64_t)t) >> 32);
  double centred = (double)(s - 6ll * 4294967296ll) * 2.3283064365386962890625e-10; /* exact */
  return 0.3 * centred;
}

/* Diagonal value 10*q + U(-1,1). */
SYN_HD double syn_diag(const syn_layout* L, int64_t i) {
  int q = syn_level_of(L, i);
  uint64_t U = syn_hash(L->seed, SYN_TAG_DIAG, (uint64_t)i, 0, 0) >> 32;
  double u = (double)((int64_t)(2 * U) - 4294967296ll) * 2.3283064365386962890625e-10; /* exact, in [-1,1) */
  return 10.0 * (double)q + u;
}

#endif
