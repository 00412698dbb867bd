/* Host generator of the seeded synthetic Hamiltonian (upper triangle incl. diagonal, COO).
 * Entry definitions live in synth_core.h; this file lays out the levels, enumerates the
 * draws, sorts and de-duplicates the (min, max) pairs and attaches values. */
#include <stdlib.h>
#include <string.h>
#include "synth_core.h"
#include "synth.h"

int syn_layout_init(syn_layout* L, int64_t n, int32_t Q, int32_t nu, int32_t w_min, int32_t w_div, uint64_t seed) {
  if (!L || n < 1 || Q < 0 || Q >= SYN_MAX_LEVELS || nu < 0 || w_min < 1 || w_div < 0) return -1;
  memset(L, 0, sizeof(*L));
  L->n = n; L->Q = Q; L->nu = nu; L->w_min = w_min; L->w_div = w_div; L->seed = seed;
  double w[SYN_MAX_LEVELS], tot = 0.0, f[SYN_MAX_LEVELS];
  int64_t c[SYN_MAX_LEVELS], used = 0;
  w[0] = 1.0;
  for (int q = 1; q <= Q; q++) w[q] = w[q - 1] * 2.2;
  for (int q = 0; q <= Q; q++) tot += w[q];
  for (int q = 0; q <= Q; q++) {
    double x = (double)n * w[q] / tot;
    c[q] = (int64_t)x;
    f[q] = x - (double)c[q];
    used += c[q];
  }
  /* largest remainder; ties go to the lower level */
  for (int64_t r = n - used; r > 0; r--) {
    int best = -1;
    for (int q = 0; q <= Q; q++)
      if (best < 0 || f[q] > f[best]) best = q;
    c[best]++;
    f[best] = -1.0;
  }
  L->start[0] = 0;
  for (int q = 0; q <= Q; q++) L->start[q + 1] = L->start[q] + c[q];
  return 0;
}

int64_t syn_draws_per_row(const syn_layout* L) { return syn_draws(L); }

int64_t syn_candidate_cap(const syn_layout* L) { return L->n * (syn_draws_per_row(L) + 1); }

static void radix_sort_u64(uint64_t* a, uint64_t* tmp, int64_t m, int bits) {
  int64_t cnt[256];
  uint64_t *src = a, *dst = tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    memset(cnt, 0, sizeof(cnt));
    for (int64_t k = 0; k < m; k++) cnt[(src[k] >> shift) & 255]++;
    int64_t s = 0;
    for (int b = 0; b < 256; b++) { int64_t t = cnt[b]; cnt[b] = s; s += t; }
    for (int64_t k = 0; k < m; k++) dst[cnt[(src[k] >> shift) & 255]++] = src[k];
    uint64_t* t = src; src = dst; dst = t;
  }
  if (src != a) memcpy(a, src, (size_t)m * sizeof(uint64_t));
}

int64_t syn_generate_host(const syn_layout* L, int64_t* rows, int64_t* cols, double* vals, int64_t cap) {
  int64_t n = L->n, m = syn_draws_per_row(L);
  if (cap < syn_candidate_cap(L)) return -1;
  /* The candidate keys and the sort's scratch live in the caller's rows and cols arrays (both
   * cap entries of 8 bytes), so a large matrix needs no second copy of its size. */
  uint64_t* keys = (uint64_t*)rows;
  uint64_t* tmp = (uint64_t*)cols;
  int64_t k = 0;
  for (int64_t i = 0; i < n; i++) {
    keys[k++] = ((uint64_t)i << 32) | (uint64_t)i;
    for (int64_t d = 0; d < m; d++) {
      int64_t j = syn_partner(L, i, d);
      if (j < 0) continue;
      int64_t a = i < j ? i : j, b = i < j ? j : i;
      keys[k++] = ((uint64_t)a << 32) | (uint64_t)b;
    }
  }
  int bits = 0;
  while (bits < 64 && ((((uint64_t)(n - 1) << 32) | (uint64_t)(n - 1)) >> bits) != 0) bits += 8;
  radix_sort_u64(keys, tmp, k, bits);
  /* unique keys -> (row, col, value); entry nnz is written after key t >= nnz has been read */
  int64_t nnz = 0;
  uint64_t prev = 0;
  for (int64_t t = 0; t < k; t++) {
    const uint64_t key = keys[t];
    if (t > 0 && key == prev) continue;
    prev = key;
    int64_t i = (int64_t)(key >> 32), j = (int64_t)(key & 0xFFFFFFFFull);
    rows[nnz] = i; cols[nnz] = j;
    vals[nnz] = (i == j) ? syn_diag(L, i) : syn_offdiag(L->seed, i, j);
    nnz++;
  }
  return nnz;
}
