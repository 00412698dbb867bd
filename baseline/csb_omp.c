/*
 * Threaded CPU CSB SpMM, organised the way Section 4.4 describes the paper's own CPU kernel.
 * It is a timing baseline for the GPU product; it is not the oracle and not a product path.
 *
 * Storage (Sections 2.2 and 4.2): the upper triangle in fixed b x b tiles, each nonzero tile
 * addressed from a 2D pointer structure. Here that is the tile list by (tile row, tile column)
 * with row pointers, plus a column index: for each tile column J, the tiles (I, J), I < J,
 * in order of I. Inside a tile, an entry is (r, c) as two uint16 offsets and an FP32 value.
 * H is held in single precision, as footnote 5 of Section 4.4 says the paper's code does.
 *
 * Product Y = H X for X, Y n x nb row-major FP64:
 *   row pass     threads take tile rows I (OpenMP dynamic schedule); Y_I = sum_J T_IJ X_J;
 *   column pass  threads take tile columns J (dynamic schedule); Y_J += sum_{I<J} T_IJ^T X_I,
 *                plus the mirror of the diagonal tile's entries above its diagonal.
 * Each pass writes disjoint row blocks of Y per thread, so there are no races and no atomics.
 * X is rounded to FP32 once per call. In the row pass the products and the sums inside a tile
 * are FP32 and each tile's partial sums are added into Y in FP64; the column pass sums a whole
 * tile column in FP32 before adding it into Y.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t n, nnz, nt, ntiles;
  int b;
  int64_t* rowptr;   /* [nt+1] first tile of each tile row */
  int64_t* colptr;   /* [nt+1] first slot of each tile column in colidx */
  int64_t* colidx;   /* tile ids of the off-diagonal tiles, by tile column, then tile row */
  int32_t* tcol;     /* [ntiles] */
  int32_t* trow;     /* [ntiles] */
  int64_t* tptr;     /* [ntiles+1] first entry of each tile */
  uint16_t* er;      /* [nnz] in-tile row */
  uint16_t* ec;      /* [nnz] in-tile column */
  float* ev;         /* [nnz] FP32 value */
  float* xs;         /* scratch: X rounded to FP32 (n x nb_cap) */
  int nb_cap;
} csb_matrix;

typedef struct {
  int64_t key;
  int64_t idx;
} keyidx;

static int cmp_key(const void* a, const void* b) {
  const int64_t x = ((const keyidx*)a)->key, y = ((const keyidx*)b)->key;
  return (x > y) - (x < y);
}

void csb_free(csb_matrix* m) {
  if (!m) return;
  free(m->rowptr); free(m->colptr); free(m->colidx); free(m->tcol); free(m->trow); free(m->tptr);
  free(m->er); free(m->ec); free(m->ev); free(m->xs);
  free(m);
}

/* Build from the upper triangle (row <= col) as COO. Returns NULL on bad input or no memory. */
csb_matrix* csb_build(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val, int b) {
  if (n < 1 || nnz < 1 || b < 1 || b > 65536) return NULL;
  csb_matrix* m = (csb_matrix*)calloc(1, sizeof(csb_matrix));
  if (!m) return NULL;
  m->n = n; m->nnz = nnz; m->b = b;
  m->nt = (n + b - 1) / b;
  keyidx* k = (keyidx*)malloc(sizeof(keyidx) * nnz);
  if (!k) { csb_free(m); return NULL; }
  const int64_t nt = m->nt;
  for (int64_t e = 0; e < nnz; e++) {
    if (row[e] < 0 || col[e] >= n || row[e] > col[e]) { free(k); csb_free(m); return NULL; }
    const int64_t I = row[e] / b, J = col[e] / b;
    k[e].key = ((I * nt + J) * b + row[e] % b) * b + col[e] % b;
    k[e].idx = e;
  }
  qsort(k, (size_t)nnz, sizeof(keyidx), cmp_key);
  int64_t ntiles = 0;
  for (int64_t e = 0; e < nnz; e++)
    if (e == 0 || k[e].key / ((int64_t)b * b) != k[e - 1].key / ((int64_t)b * b)) ntiles++;
  m->ntiles = ntiles;
  m->rowptr = (int64_t*)calloc((size_t)nt + 1, 8);
  m->colptr = (int64_t*)calloc((size_t)nt + 1, 8);
  m->colidx = (int64_t*)malloc(8 * (size_t)ntiles);
  m->tcol = (int32_t*)malloc(4 * (size_t)ntiles);
  m->trow = (int32_t*)malloc(4 * (size_t)ntiles);
  m->tptr = (int64_t*)malloc(8 * ((size_t)ntiles + 1));
  m->er = (uint16_t*)malloc(2 * (size_t)nnz);
  m->ec = (uint16_t*)malloc(2 * (size_t)nnz);
  m->ev = (float*)malloc(4 * (size_t)nnz);
  if (!m->rowptr || !m->colptr || !m->colidx || !m->tcol || !m->trow || !m->tptr || !m->er || !m->ec || !m->ev) {
    free(k); csb_free(m); return NULL;
  }
  int64_t t = -1;
  for (int64_t e = 0; e < nnz; e++) {
    const int64_t tk = k[e].key / ((int64_t)b * b);
    if (e > 0 && k[e].key == k[e - 1].key) { free(k); csb_free(m); return NULL; } /* duplicate */
    if (e == 0 || tk != k[e - 1].key / ((int64_t)b * b)) {
      t++;
      m->trow[t] = (int32_t)(tk / nt);
      m->tcol[t] = (int32_t)(tk % nt);
      m->tptr[t] = e;
      m->rowptr[m->trow[t] + 1]++;
    }
    const int64_t s = k[e].idx;
    m->er[e] = (uint16_t)(row[s] % b);
    m->ec[e] = (uint16_t)(col[s] % b);
    m->ev[e] = (float)val[s];
  }
  m->tptr[ntiles] = nnz;
  free(k);
  for (int64_t I = 0; I < nt; I++) m->rowptr[I + 1] += m->rowptr[I];
  /* column index of the off-diagonal tiles: counting sort by tile column, stable in tile row */
  for (int64_t q = 0; q < ntiles; q++)
    if (m->trow[q] != m->tcol[q]) m->colptr[m->tcol[q] + 1]++;
  for (int64_t J = 0; J < nt; J++) m->colptr[J + 1] += m->colptr[J];
  int64_t* fill = (int64_t*)malloc(8 * ((size_t)nt + 1));
  if (!fill) { csb_free(m); return NULL; }
  memcpy(fill, m->colptr, 8 * ((size_t)nt + 1));
  for (int64_t q = 0; q < ntiles; q++)
    if (m->trow[q] != m->tcol[q]) m->colidx[fill[m->tcol[q]]++] = q;
  free(fill);
  return m;
}

int64_t csb_ntiles(const csb_matrix* m) { return m->ntiles; }

/* Y = H X. X, Y: n x nb row-major FP64 (host). nthreads <= 0: the OpenMP default. Returns 0,
 * or -1 on bad arguments or no memory. */
int csb_spmm(csb_matrix* m, const double* X, double* Y, int nb, int nthreads) {
  if (!m || !X || !Y || nb < 1 || nb > 64) return -1;
  const int64_t n = m->n, nt = m->nt;
  const int b = m->b;
  if (m->nb_cap < nb) {
    free(m->xs);
    m->xs = (float*)malloc(sizeof(float) * (size_t)n * nb);
    if (!m->xs) { m->nb_cap = 0; return -1; }
    m->nb_cap = nb;
  }
  float* xs = m->xs;
  int fail = 0;  /* a thread could not get its scratch tile */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n * nb; i++) xs[i] = (float)X[i];

  /* row pass: Y_I = sum_J T_IJ X_J */
#pragma omp parallel
  {
    float* acc = (float*)malloc(sizeof(float) * (size_t)b * nb);
    if (!acc) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t I = 0; I < nt; I++) {
      if (!acc) continue;
      const int64_t r0 = I * b;
      const int64_t rows = (n - r0) < b ? (n - r0) : b;
      double* y = Y + r0 * nb;
      for (int64_t i = 0; i < rows * nb; i++) y[i] = 0.0;
      for (int64_t t = m->rowptr[I]; t < m->rowptr[I + 1]; t++) {
        const float* xj = xs + (int64_t)m->tcol[t] * b * nb;
        memset(acc, 0, sizeof(float) * (size_t)rows * nb);
        for (int64_t e = m->tptr[t]; e < m->tptr[t + 1]; e++) {
          const float v = m->ev[e];
          float* a = acc + (int64_t)m->er[e] * nb;
          const float* x = xj + (int64_t)m->ec[e] * nb;
          for (int q = 0; q < nb; q++) a[q] += v * x[q];
        }
        for (int64_t i = 0; i < rows * nb; i++) y[i] += (double)acc[i];
      }
    }
    free(acc);
  }

  /* column pass: Y_J += sum_{I<J} T_IJ^T X_I, then the mirror of the diagonal tile's entries
   * above its diagonal (the row pass applied the stored entries only) */
#pragma omp parallel
  {
    float* acc = (float*)malloc(sizeof(float) * (size_t)b * nb);
    if (!acc) {
#pragma omp atomic write
      fail = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t J = 0; J < nt; J++) {
      if (!acc) continue;
      const int64_t c0 = J * b;
      const int64_t cols = (n - c0) < b ? (n - c0) : b;
      memset(acc, 0, sizeof(float) * (size_t)cols * nb);
      for (int64_t s = m->colptr[J]; s < m->colptr[J + 1]; s++) {
        const int64_t t = m->colidx[s];
        const float* xi = xs + (int64_t)m->trow[t] * b * nb;
        for (int64_t e = m->tptr[t]; e < m->tptr[t + 1]; e++) {
          const float v = m->ev[e];
          float* a = acc + (int64_t)m->ec[e] * nb;
          const float* x = xi + (int64_t)m->er[e] * nb;
          for (int q = 0; q < nb; q++) a[q] += v * x[q];
        }
      }
      const int64_t t = m->rowptr[J];
      if (t < m->rowptr[J + 1] && m->tcol[t] == J) {  /* the diagonal tile is first in its row */
        const float* xi = xs + c0 * nb;
        for (int64_t e = m->tptr[t]; e < m->tptr[t + 1]; e++) {
          if (m->er[e] == m->ec[e]) continue;
          const float v = m->ev[e];
          float* a = acc + (int64_t)m->ec[e] * nb;
          const float* x = xi + (int64_t)m->er[e] * nb;
          for (int q = 0; q < nb; q++) a[q] += v * x[q];
        }
      }
      double* y = Y + c0 * nb;
      for (int64_t i = 0; i < cols * nb; i++) y[i] += (double)acc[i];
    }
    free(acc);
  }
  return fail ? -1 : 0;
}

int csb_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
