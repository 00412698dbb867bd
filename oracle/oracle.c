/* ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct FP64 CPU reference for what the GPU path computes. Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it; the library never does.
 * It shares no code with the CUDA path (neither includes nor links the other).
 *
 * What the method computes (Section 3.1, eq. 6 and the output of Algorithm 1): the k smallest
 * eigenpairs of a symmetric H of which only one triangle is stored (Section 4.1). Because the
 * LOBPCG iteration converges to that plain definition, the oracle computes the definition
 * directly, by two independent dense methods and a Lanczos method for large n:
 *   orc_spmm          Y = H X from the stored triangle (Section 4.1: U_i = H_ij W_j, U_j = H_ij^T W_i)
 *   orc_dense         dense expansion of the stored triangle
 *   orc_syev          Householder tridiagonalisation + implicit-shift QL (the QL algorithm of
 *                     Bowdler, Martin, Reinsch and Wilkinson, 1968; all eigenpairs)
 *   orc_tridiag_eig   the QL part alone, for a symmetric tridiagonal matrix
 *   orc_jacobi        the cyclic-by-row Jacobi method (Jacobi 1846; Forsythe and Henrici 1960),
 *                     a second, independent dense method
 *   orc_spmm_csr, orc_lanczos_csr  the same on the triangle in CSR form with 32-bit columns
 *                     (for matrices of ~1e9 entries, whose 64-bit COO would not fit beside the
 *                     Lanczos basis in host memory)
 *   orc_lanczos       Lanczos with full reorthogonalisation (the legacy solver, Section 3 and
 *                     the footnote to Table 3), Ritz-residual stopping test every 10 steps
 *   orc_tiles         CSB-style tile store: tiles by (tile row, tile col), COO inside each tile
 *                     with the two in-tile offsets packed in one word (Section 4.2)
 *   orc_gram          block inner product X^T Y (Section 4.4)
 *   orc_lincomb       linear combination Y = X G (Section 4.4, eq. 7)
 *   orc_block_precond block-diagonal shifted solve (H~_[i] - mu_j I) W_[i] = R_[i] (eq. 11)
 *   orc_block_krylov  the same systems solved approximately by a few FOM or minimal-residual
 *                     iterations from a zero start (Sections 3.2, 4.3), or by |H~_[i] - mu_j I|^{-1}
 *   orc_rayleigh_ritz generalised projected problem (Y^T H Y) G = (Y^T Y) G Theta (eq. 9)
 *   orc_norm_inf      ||H||_inf, the norm used in the relative residual (Section 3.3.1)
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- sparse basics */

/* Y = H X, H given by its upper triangle (row <= col) incl. diagonal; X, Y are n x nb row-major.
 * Each stored off-diagonal entry is applied as h_ij and as h_ji (Section 4.1). */
void orc_spmm(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val, int64_t nb,
              const double* X, double* Y) {
  memset(Y, 0, (size_t)(n * nb) * sizeof(double));
  for (int64_t t = 0; t < nnz; t++) {
    int64_t i = row[t], j = col[t];
    double v = val[t];
    for (int64_t c = 0; c < nb; c++) Y[i * nb + c] += v * X[j * nb + c];
    if (i != j)
      for (int64_t c = 0; c < nb; c++) Y[j * nb + c] += v * X[i * nb + c];
  }
}

/* The same product with the stored triangle in CSR form (rows in order, each row's columns in
 * order, 32-bit column indices): rowptr[n+1], col[rowptr[n]], val[rowptr[n]]. Visits the entries
 * in the order of a COO sorted by (row, col), so it matches orc_spmm on such a COO exactly. It
 * exists for matrices whose 64-bit COO would not fit beside the Lanczos basis in host memory. */
void orc_spmm_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int64_t nb,
                  const double* X, double* Y) {
  memset(Y, 0, (size_t)(n * nb) * sizeof(double));
  for (int64_t i = 0; i < n; i++)
    for (int64_t t = rowptr[i]; t < rowptr[i + 1]; t++) {
      const int64_t j = col[t];
      const double v = val[t];
      for (int64_t c = 0; c < nb; c++) Y[i * nb + c] += v * X[j * nb + c];
      if (i != j)
        for (int64_t c = 0; c < nb; c++) Y[j * nb + c] += v * X[i * nb + c];
    }
}

/* Dense n x n (row-major) expansion of the stored triangle. */
void orc_dense(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val, double* A) {
  memset(A, 0, (size_t)(n * n) * sizeof(double));
  for (int64_t t = 0; t < nnz; t++) {
    A[row[t] * n + col[t]] = val[t];
    A[col[t] * n + row[t]] = val[t];
  }
}

/* max_i sum_j |h_ij| over the full symmetric matrix. */
double orc_norm_inf(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val) {
  double* s = (double*)calloc((size_t)n, sizeof(double));
  for (int64_t t = 0; t < nnz; t++) {
    s[row[t]] += fabs(val[t]);
    if (row[t] != col[t]) s[col[t]] += fabs(val[t]);
  }
  double m = 0.0;
  for (int64_t i = 0; i < n; i++) m = s[i] > m ? s[i] : m;
  free(s);
  return m;
}

/* ---------------------------------------------------------------- dense eigensolvers */

/* Sort eigenvalues ascending (stable by index) and permute the eigenvector columns of Z. */
static void sort_eig(int64_t n, double* w, double* Z, int64_t ldz, int64_t nrows) {
  for (int64_t a = 1; a < n; a++) {
    int64_t b = a;
    while (b > 0 && w[b - 1] > w[b]) {
      double t = w[b]; w[b] = w[b - 1]; w[b - 1] = t;
      if (Z)
        for (int64_t r = 0; r < nrows; r++) {
          double u = Z[r * ldz + b]; Z[r * ldz + b] = Z[r * ldz + b - 1]; Z[r * ldz + b - 1] = u;
        }
      b--;
    }
  }
}

/* Implicit-shift QL (Bowdler, Martin, Reinsch and Wilkinson, "The QR and QL algorithms for
 * symmetric matrices", Numer. Math. 11, 1968) on the symmetric tridiagonal matrix with diagonal
 * d[0..m-1] and off-diagonal e[0..m-2]. Each sweep chases a bulge from the bottom of the unreduced block
 * upward with Givens rotations, shifted by the eigenvalue of the leading 2x2 closer to d[l].
 * The rotations are applied to the ROWS of Zt (m rows of length nrows, leading dimension ldz):
 * start from the identity to get T's eigenvectors, or from Q^T (Householder basis) to get those
 * of the original matrix. On return d holds the eigenvalues ascending and row t of Zt the
 * eigenvector of d[t]. Returns 0, or -1 if an eigenvalue needed more than 60 sweeps. */
static int ql_rows(int64_t m, double* d, const double* e_in, double* Zt, int64_t ldz, int64_t nrows) {
  double* e = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int64_t i = 0; i + 1 < m; i++) e[i] = e_in[i];
  int status = 0;
  for (int64_t l = 0; l < m; l++) {
    int iter = 0;
    for (;;) {
      int64_t mm;
      for (mm = l; mm + 1 < m; mm++)
        if (fabs(e[mm]) <= DBL_EPSILON * (fabs(d[mm]) + fabs(d[mm + 1]))) break;
      if (mm == l) break;
      if (iter++ == 60) { status = -1; break; }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + (g >= 0.0 ? fabs(r) : -fabs(r)));
      double s = 1.0, c = 1.0, p = 0.0;
      int deflated = 0;
      for (int64_t i = mm - 1; i >= l; i--) {
        double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) { d[i + 1] -= p; e[mm] = 0.0; deflated = 1; break; }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        double* zi = Zt + i * ldz;
        double* zi1 = Zt + (i + 1) * ldz;
        for (int64_t k = 0; k < nrows; k++) {
          double a0 = zi[k], a1 = zi1[k];
          zi1[k] = s * a0 + c * a1;
          zi[k] = c * a0 - s * a1;
        }
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
    if (status) break;
  }
  free(e);
  /* ascending order, stable by index; permute rows of Zt alongside */
  double* tmp = (double*)malloc((size_t)(nrows > 0 ? nrows : 1) * sizeof(double));
  for (int64_t a = 1; a < m; a++) {
    int64_t b = a;
    while (b > 0 && d[b - 1] > d[b]) {
      double t = d[b]; d[b] = d[b - 1]; d[b - 1] = t;
      memcpy(tmp, Zt + b * ldz, (size_t)nrows * sizeof(double));
      memcpy(Zt + b * ldz, Zt + (b - 1) * ldz, (size_t)nrows * sizeof(double));
      memcpy(Zt + (b - 1) * ldz, tmp, (size_t)nrows * sizeof(double));
      b--;
    }
  }
  free(tmp);
  return status;
}

/* Eigenpairs of the symmetric tridiagonal (d, e) of order m by ql_rows. Z (m x m, row-major)
 * receives the eigenvectors as columns; d the eigenvalues ascending. Returns 0 or -1. */
int orc_tridiag_eig(int64_t m, double* d, const double* e_in, double* Z, int64_t ldz, int64_t nrows) {
  (void)nrows;
  double* Zt = (double*)calloc((size_t)(m * m > 0 ? m * m : 1), sizeof(double));
  for (int64_t i = 0; i < m; i++) Zt[i * m + i] = 1.0;
  int st = ql_rows(m, d, e_in, Zt, m, m);
  for (int64_t i = 0; i < m; i++)
    for (int64_t j = 0; j < m; j++) Z[i * ldz + j] = Zt[j * m + i];
  free(Zt);
  return st;
}

/* All eigenpairs of the dense symmetric n x n A (row-major). On return w holds the eigenvalues
 * ascending and A the eigenvectors as columns (A[i*n + j] = component i of vector j).
 * Householder reflections H_k = I - beta v v^T reduce A to tridiagonal T = Q^T A Q; then QL on T
 * with Z = Q gives the eigenvectors of A. Returns 0 or -1 (QL did not converge). */
int orc_syev(int64_t n, double* A, double* w) {
  double* Q = (double*)calloc((size_t)(n * n), sizeof(double));
  double* v = (double*)malloc((size_t)n * sizeof(double));
  double* p = (double*)malloc((size_t)n * sizeof(double));
  double* e = (double*)calloc((size_t)(n > 1 ? n : 1), sizeof(double));
  double* tq = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (int64_t i = 0; i < n; i++) Q[i * n + i] = 1.0;
  for (int64_t k = 0; k + 2 < n; k++) {
    int64_t m = n - k - 1; /* length of the column below the diagonal */
    double x0 = A[(k + 1) * n + k], sigma = 0.0;
    for (int64_t i = 1; i < m; i++) sigma += A[(k + 1 + i) * n + k] * A[(k + 1 + i) * n + k];
    if (sigma == 0.0) continue; /* already tridiagonal in this column */
    double alpha = sqrt(x0 * x0 + sigma);
    if (x0 > 0.0) alpha = -alpha;
    v[0] = x0 - alpha;
    for (int64_t i = 1; i < m; i++) v[i] = A[(k + 1 + i) * n + k];
    double vnorm2 = v[0] * v[0] + sigma;
    double beta = 2.0 / vnorm2;
    /* trailing block B = A[k+1:, k+1:] <- H B H = B - v w^T - w v^T with
     * p = beta B v, K = beta/2 v^T p, w = p - K v */
    double K = 0.0;
    for (int64_t i = 0; i < m; i++) {
      double s = 0.0;
      for (int64_t j = 0; j < m; j++) s += A[(k + 1 + i) * n + (k + 1 + j)] * v[j];
      p[i] = beta * s;
    }
    for (int64_t i = 0; i < m; i++) K += v[i] * p[i];
    K *= 0.5 * beta;
    for (int64_t i = 0; i < m; i++) p[i] -= K * v[i];
    for (int64_t i = 0; i < m; i++)
      for (int64_t j = 0; j < m; j++) A[(k + 1 + i) * n + (k + 1 + j)] -= v[i] * p[j] + p[i] * v[j];
    A[(k + 1) * n + k] = alpha;
    A[k * n + k + 1] = alpha;
    for (int64_t i = 1; i < m; i++) { A[(k + 1 + i) * n + k] = 0.0; A[k * n + k + 1 + i] = 0.0; }
    /* Q <- Q H, kept transposed: rows k+1.. of Qt <- (I - beta v v^T) rows k+1.. */
    for (int64_t c = 0; c < n; c++) tq[c] = 0.0;
    for (int64_t j = 0; j < m; j++) {
      const double* qr = Q + (k + 1 + j) * n;
      for (int64_t c = 0; c < n; c++) tq[c] += v[j] * qr[c];
    }
    for (int64_t j = 0; j < m; j++) {
      double* qr = Q + (k + 1 + j) * n;
      double f = beta * v[j];
      for (int64_t c = 0; c < n; c++) qr[c] -= f * tq[c];
    }
  }
  for (int64_t i = 0; i < n; i++) w[i] = A[i * n + i];
  for (int64_t i = 0; i + 1 < n; i++) e[i] = A[(i + 1) * n + i];
  int st = ql_rows(n, w, e, Q, n, n); /* Q holds Q^T: rows are basis vectors */
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++) A[i * n + j] = Q[j * n + i];
  free(Q); free(v); free(p); free(e); free(tq);
  return st;
}

/* The cyclic-by-row Jacobi method (Forsythe and Henrici, Trans. AMS 94, 1960): rotations J(p,q,theta) zero a_pq one pair at a time, A <- J^T A J, until
 * the off-diagonal Frobenius norm is below 1e-15 of the whole (or max_sweeps). A (row-major) is
 * destroyed; w gets the eigenvalues ascending and V (n x n) the eigenvectors as columns.
 * Returns the number of sweeps used, or -1 if not converged. */
int orc_jacobi(int64_t n, double* A, double* w, double* V, int max_sweeps) {
  for (int64_t i = 0; i < n * n; i++) V[i] = 0.0;
  for (int64_t i = 0; i < n; i++) V[i * n + i] = 1.0;
  double fro = 0.0;
  for (int64_t i = 0; i < n * n; i++) fro += A[i] * A[i];
  int sweep;
  for (sweep = 0; sweep < max_sweeps; sweep++) {
    double off = 0.0;
    for (int64_t p = 0; p < n; p++)
      for (int64_t q = p + 1; q < n; q++) off += 2.0 * A[p * n + q] * A[p * n + q];
    if (off <= 1e-30 * fro) break;
    for (int64_t p = 0; p < n; p++)
      for (int64_t q = p + 1; q < n; q++) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int64_t k = 0; k < n; k++) { /* columns p, q */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; k++) { /* rows p, q */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int64_t k = 0; k < n; k++) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int64_t i = 0; i < n; i++) w[i] = A[i * n + i];
  sort_eig(n, w, V, n, n);
  return sweep < max_sweeps ? sweep : -1;
}

/* ---------------------------------------------------------------- Lanczos (legacy solver) */

static double orc_unif(uint64_t seed, uint64_t i) {
  uint64_t z = seed * 0xD1B54A32D192ED03ull + i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* Lanczos with full reorthogonalisation (classical Gram-Schmidt applied twice every step),
 * started from a seeded uniform vector. Every 10 steps the tridiagonal T_m is diagonalised
 * (orc_tridiag_eig) and the run stops once the Ritz residual estimates beta_m |s_{m,j}| are at
 * most tol * normH for the k smallest Ritz values. lam gets those Ritz values and X (n x k,
 * row-major) the Ritz vectors. Returns 0 when converged, 1 if max_steps was reached,
 * -1 on QL failure, -2 on allocation failure. *steps gets the number of Lanczos steps. */
/* The matrix a Lanczos run multiplies by: the stored triangle as COO or as CSR. */
typedef struct {
  int64_t n, nnz;
  const int64_t *row, *col, *rowptr;
  const int32_t* col32;
  const double* val;
} orc_op;

static void op_apply(const orc_op* A, const double* x, double* y) {
  if (A->rowptr) orc_spmm_csr(A->n, A->rowptr, A->col32, A->val, 1, x, y);
  else orc_spmm(A->n, A->nnz, A->row, A->col, A->val, 1, x, y);
}

static int lanczos_run(const orc_op* A, int64_t k, double tol, double normH, int64_t max_steps, uint64_t seed,
                       double* lam, double* X, int64_t* steps);

int orc_lanczos(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val, int64_t k,
                double tol, double normH, int64_t max_steps, uint64_t seed, double* lam, double* X, int64_t* steps) {
  const orc_op A = {n, nnz, row, col, NULL, NULL, val};
  return lanczos_run(&A, k, tol, normH, max_steps, seed, lam, X, steps);
}

/* orc_lanczos on the CSR form of the stored triangle (see orc_spmm_csr). */
int orc_lanczos_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int64_t k, double tol,
                    double normH, int64_t max_steps, uint64_t seed, double* lam, double* X, int64_t* steps) {
  const orc_op A = {n, rowptr[n], NULL, NULL, rowptr, col, val};
  return lanczos_run(&A, k, tol, normH, max_steps, seed, lam, X, steps);
}

static int lanczos_run(const orc_op* A, int64_t k, double tol, double normH, int64_t max_steps, uint64_t seed,
                       double* lam, double* X, int64_t* steps) {
  const int64_t n = A->n;
  if (max_steps > n) max_steps = n;
  double* Qv = (double*)malloc((size_t)(n * max_steps) * sizeof(double)); /* vector j at Qv + j*n */
  double* w = (double*)malloc((size_t)n * sizeof(double));
  double* alpha = (double*)malloc((size_t)max_steps * sizeof(double));
  double* beta = (double*)malloc((size_t)max_steps * sizeof(double));
  double* dd = (double*)malloc((size_t)max_steps * sizeof(double));
  double* S = (double*)malloc((size_t)(max_steps * max_steps) * sizeof(double));
  double* coef = (double*)malloc((size_t)max_steps * sizeof(double));
  if (!Qv || !w || !alpha || !beta || !dd || !S || !coef) {
    free(Qv); free(w); free(alpha); free(beta); free(dd); free(S); free(coef);
    return -2;
  }
  double nrm = 0.0;
  for (int64_t i = 0; i < n; i++) { Qv[i] = orc_unif(seed, (uint64_t)i); nrm += Qv[i] * Qv[i]; }
  nrm = sqrt(nrm);
  for (int64_t i = 0; i < n; i++) Qv[i] /= nrm;
  int status = 1;
  int64_t m = 0;
  for (int64_t j = 0; j < max_steps; j++) {
    double* qj = Qv + j * n;
    op_apply(A, qj, w);
    double a = 0.0;
    for (int64_t i = 0; i < n; i++) a += qj[i] * w[i];
    alpha[j] = a;
    for (int64_t i = 0; i < n; i++) w[i] -= a * qj[i];
    if (j > 0)
      for (int64_t i = 0; i < n; i++) w[i] -= beta[j - 1] * Qv[(j - 1) * n + i];
    for (int pass = 0; pass < 2; pass++) {
      for (int64_t t = 0; t <= j; t++) {
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) s += Qv[t * n + i] * w[i];
        coef[t] = s;
      }
      for (int64_t t = 0; t <= j; t++)
        for (int64_t i = 0; i < n; i++) w[i] -= coef[t] * Qv[t * n + i];
    }
    double b = 0.0;
    for (int64_t i = 0; i < n; i++) b += w[i] * w[i];
    b = sqrt(b);
    beta[j] = b;
    m = j + 1;
    int last = (m == max_steps) || (b <= 1e-14 * normH);
    if (m % 10 == 0 || last) {
      for (int64_t i = 0; i < m; i++) dd[i] = alpha[i];
      for (int64_t i = 0; i < m * m; i++) S[i] = 0.0;
      for (int64_t i = 0; i < m; i++) S[i * m + i] = 1.0;
      if (orc_tridiag_eig(m, dd, beta, S, m, m) != 0) { status = -1; break; }
      int conv = (m >= k);
      for (int64_t t = 0; t < k && t < m && conv; t++)
        if (b * fabs(S[(m - 1) * m + t]) > tol * normH) conv = 0;
      if (conv || last) {
        status = conv ? 0 : 1;
        int64_t kk = k < m ? k : m;
        for (int64_t t = 0; t < kk; t++) lam[t] = dd[t];
        for (int64_t i = 0; i < n; i++)
          for (int64_t t = 0; t < kk; t++) {
            double s = 0.0;
            for (int64_t r = 0; r < m; r++) s += Qv[r * n + i] * S[r * m + t];
            X[i * k + t] = s;
          }
        break;
      }
    }
    double* qn = Qv + (j + 1) * n;
    for (int64_t i = 0; i < n; i++) qn[i] = w[i] / b;
  }
  *steps = m;
  free(Qv); free(w); free(alpha); free(beta); free(dd); free(S); free(coef);
  return status;
}

/* ---------------------------------------------------------------- tile store (CSB) */

typedef struct { int64_t tr, tc, r, c, src; } orc_ent;

static int cmp_ent(const void* a, const void* b) {
  const orc_ent* x = (const orc_ent*)a;
  const orc_ent* y = (const orc_ent*)b;
  if (x->tr != y->tr) return x->tr < y->tr ? -1 : 1;
  if (x->tc != y->tc) return x->tc < y->tc ? -1 : 1;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

/* CSB-style store with fixed b x b tiles (Sections 2.2 and 4.2): nonzero tiles ordered by
 * (tile row, tile col); inside a tile, entries in (r, c) order with rc = (r << 16) | c.
 * tile_rowptr (nt+1): first tile of each tile row; tile_col (ntiles); tile_ptr (ntiles+1): first
 * entry of each tile; v64 / v32: values in FP64 and rounded to FP32. Input: upper triangle
 * (row <= col) COO in any order. Returns the number of tiles, or -1 for an entry out of range,
 * -2 for an entry below the diagonal, -3 for a duplicate, -4 for a bad tile size. */
int64_t orc_tiles(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val, int64_t b,
                  int64_t* tile_rowptr, int32_t* tile_col, int64_t* tile_ptr, uint32_t* rc, double* v64,
                  float* v32) {
  if (b < 1 || b > 65536) return -4;
  orc_ent* E = (orc_ent*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(orc_ent));
  for (int64_t t = 0; t < nnz; t++) {
    int64_t i = row[t], j = col[t];
    if (i < 0 || j < 0 || i >= n || j >= n) { free(E); return -1; }
    if (i > j) { free(E); return -2; }
    E[t].tr = i / b; E[t].tc = j / b; E[t].r = i % b; E[t].c = j % b; E[t].src = t;
  }
  qsort(E, (size_t)nnz, sizeof(orc_ent), cmp_ent);
  for (int64_t t = 1; t < nnz; t++)
    if (cmp_ent(&E[t - 1], &E[t]) == 0) { free(E); return -3; }
  int64_t nt = (n + b - 1) / b, ntiles = 0;
  for (int64_t t = 0; t <= nt; t++) tile_rowptr[t] = 0;
  for (int64_t t = 0; t < nnz; t++) {
    if (t == 0 || E[t].tr != E[t - 1].tr || E[t].tc != E[t - 1].tc) {
      tile_col[ntiles] = (int32_t)E[t].tc;
      tile_ptr[ntiles] = t;
      tile_rowptr[E[t].tr + 1]++;
      ntiles++;
    }
    rc[t] = (uint32_t)((E[t].r << 16) | E[t].c);
    v64[t] = val[E[t].src];
    v32[t] = (float)val[E[t].src];
  }
  tile_ptr[ntiles] = nnz;
  for (int64_t t = 0; t < nt; t++) tile_rowptr[t + 1] += tile_rowptr[t];
  free(E);
  return ntiles;
}

/* ---------------------------------------------------------------- dense block kernels */

/* G = A^T B with A n x p and B n x q row-major; G is p x q row-major (Section 4.4). */
void orc_gram(int64_t n, int64_t p, const double* A, int64_t q, const double* B, double* G) {
  for (int64_t a = 0; a < p; a++)
    for (int64_t c = 0; c < q; c++) {
      double s = 0.0;
      for (int64_t r = 0; r < n; r++) s += A[r * p + a] * B[r * q + c];
      G[a * q + c] = s;
    }
}

/* Y = A C with A n x p, C p x q, Y n x q, all row-major (Section 4.4, eq. 7). */
void orc_lincomb(int64_t n, int64_t p, const double* A, int64_t q, const double* C, double* Y) {
  for (int64_t r = 0; r < n; r++)
    for (int64_t c = 0; c < q; c++) {
      double s = 0.0;
      for (int64_t a = 0; a < p; a++) s += A[r * p + a] * C[a * q + c];
      Y[r * q + c] = s;
    }
}

/* Solve the dense m x m system M x = rhs by Gaussian elimination with partial pivoting
 * (M and rhs destroyed). Returns 0, or -1 if a pivot is exactly zero. */
static int gauss_solve(int64_t m, double* M, double* rhs) {
  for (int64_t k = 0; k < m; k++) {
    int64_t piv = k;
    for (int64_t i = k + 1; i < m; i++)
      if (fabs(M[i * m + k]) > fabs(M[piv * m + k])) piv = i;
    if (M[piv * m + k] == 0.0) return -1;
    if (piv != k) {
      for (int64_t j = 0; j < m; j++) { double t = M[k * m + j]; M[k * m + j] = M[piv * m + j]; M[piv * m + j] = t; }
      double t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
    }
    for (int64_t i = k + 1; i < m; i++) {
      double f = M[i * m + k] / M[k * m + k];
      for (int64_t j = k; j < m; j++) M[i * m + j] -= f * M[k * m + j];
      rhs[i] -= f * rhs[k];
    }
  }
  for (int64_t k = m - 1; k >= 0; k--) {
    double s = rhs[k];
    for (int64_t j = k + 1; j < m; j++) s -= M[k * m + j] * rhs[j];
    rhs[k] = s / M[k * m + k];
  }
  return 0;
}

/* Block-diagonal preconditioner apply of eq. 11: for every diagonal block [bounds[i], bounds[i+1])
 * of the full symmetric H and every column j, solve (H~_[i] - mu_j I) w = r. R, W are n x nb
 * row-major; bounds has nblk+1 entries from 0 to n. Returns 0, or -1 for an exactly singular
 * block system. */
int orc_block_precond(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                      int64_t nblk, const int64_t* bounds, int64_t nb, const double* mu, const double* R,
                      double* W) {
  int64_t maxb = 0;
  for (int64_t i = 0; i < nblk; i++) maxb = bounds[i + 1] - bounds[i] > maxb ? bounds[i + 1] - bounds[i] : maxb;
  double* blk = (double*)malloc((size_t)(maxb * maxb > 0 ? maxb * maxb : 1) * sizeof(double) * (size_t)nblk);
  double* M = (double*)malloc((size_t)(maxb * maxb > 0 ? maxb * maxb : 1) * sizeof(double));
  double* rhs = (double*)malloc((size_t)(maxb > 0 ? maxb : 1) * sizeof(double));
  int64_t* owner = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < nblk; i++)
    for (int64_t r = bounds[i]; r < bounds[i + 1]; r++) owner[r] = i;
  memset(blk, 0, (size_t)(maxb * maxb) * sizeof(double) * (size_t)nblk);
  for (int64_t t = 0; t < nnz; t++) {
    int64_t i = row[t], j = col[t];
    int64_t bi = owner[i];
    if (owner[j] != bi) continue;
    int64_t o = bounds[bi];
    blk[bi * maxb * maxb + (i - o) * maxb + (j - o)] = val[t];
    blk[bi * maxb * maxb + (j - o) * maxb + (i - o)] = val[t];
  }
  int st = 0;
  for (int64_t bi = 0; bi < nblk && !st; bi++) {
    int64_t o = bounds[bi], m = bounds[bi + 1] - o;
    for (int64_t c = 0; c < nb && !st; c++) {
      for (int64_t a = 0; a < m; a++) {
        for (int64_t b2 = 0; b2 < m; b2++) M[a * m + b2] = blk[bi * maxb * maxb + a * maxb + b2];
        M[a * m + a] -= mu[c];
        rhs[a] = R[(o + a) * nb + c];
      }
      if (gauss_solve(m, M, rhs) != 0) st = -1;
      for (int64_t a = 0; a < m; a++) W[(o + a) * nb + c] = rhs[a];
    }
  }
  free(blk); free(M); free(rhs); free(owner);
  return st;
}

/* One shifted block system A w = r (A = H~_[i] - mu I, m x m dense, row-major) solved by a
 * Krylov method from a zero start (the paper's FOM or GMRES with two or three iterations,
 * Sections 3.2 and 4.3). Lanczos with full reorthogonalisation builds V = [v_1 .. v_s],
 * v_1 = r / beta, and the tridiagonal T = V^T A V (diagonal alpha, off-diagonal b); b_s couples
 * v_s to the next vector. The process stops early when b_i <= 1e-12 (|alpha_i| + b_{i-1})
 * (an invariant subspace: the iterate is then exact).
 *   method 0, FOM: w = V y with T y = beta e_1 (Galerkin condition V^T (r - A w) = 0). A pivot
 *     of the unpivoted elimination of T below 1e-4 max_i (|alpha_i| + b_i) counts as a FOM
 *     breakdown, and the minimal-residual iterate is returned instead.
 *   method 2, minimal residual: w = V y minimising || beta e_1 - Tbar y ||, Tbar = [T; b_s e_s^T]
 *     ((s+1) x s), through the normal equations Tbar^T Tbar y = beta Tbar^T e_1. */
static void krylov_block(int64_t m, const double* A, const double* r, int method, int steps, double* w) {
  double* Vbuf = (double*)malloc((size_t)(4 * m + m) * sizeof(double));
  double* V[4] = {Vbuf, Vbuf + m, Vbuf + 2 * m, Vbuf + 3 * m};
  double* u = Vbuf + 4 * m;
  double al[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
  for (int64_t a = 0; a < m; a++) w[a] = 0.0;
  double beta = 0.0;
  for (int64_t a = 0; a < m; a++) beta += r[a] * r[a];
  beta = sqrt(beta);
  if (beta == 0.0) { free(Vbuf); return; }
  for (int64_t a = 0; a < m; a++) V[0][a] = r[a] / beta;
  int s = 0;
  for (int i = 0; i < steps; i++) {
    for (int64_t a = 0; a < m; a++) {
      double t = 0.0;
      for (int64_t c = 0; c < m; c++) t += A[a * m + c] * V[i][c];
      u[a] = t;
    }
    al[i] = 0.0;
    for (int64_t a = 0; a < m; a++) al[i] += V[i][a] * u[a];
    for (int t = 0; t <= i; t++) {
      double h = 0.0;
      for (int64_t a = 0; a < m; a++) h += V[t][a] * u[a];
      for (int64_t a = 0; a < m; a++) u[a] -= h * V[t][a];
    }
    double nu = 0.0;
    for (int64_t a = 0; a < m; a++) nu += u[a] * u[a];
    b[i] = sqrt(nu);
    s = i + 1;
    const double scale = fabs(al[i]) + (i > 0 ? b[i - 1] : 0.0);
    if (!(b[i] > 1e-12 * scale)) { b[i] = 0.0; break; }
    if (i + 1 == steps) break;
    for (int64_t a = 0; a < m; a++) V[i + 1][a] = u[a] / b[i];
  }
  double y[4] = {0, 0, 0, 0};
  double tmax = 0.0;
  for (int i = 0; i < s; i++) tmax = fmax(tmax, fabs(al[i]) + b[i]);
  int fom_ok = 0;
  if (method == 0) {
    double dg[4], rhs[4] = {beta, 0, 0, 0};
    fom_ok = 1;
    for (int i = 0; i < s; i++) {
      dg[i] = al[i];
      if (i > 0) {
        const double l = b[i - 1] / dg[i - 1];
        dg[i] -= l * b[i - 1];
        rhs[i] -= l * rhs[i - 1];
      }
      if (!(fabs(dg[i]) > 1e-4 * tmax)) fom_ok = 0;
    }
    if (fom_ok)
      for (int i = s - 1; i >= 0; i--) y[i] = (rhs[i] - (i + 1 < s ? b[i] * y[i + 1] : 0.0)) / dg[i];
  }
  if (!fom_ok) {
    /* Tbar ((s+1) x s): Tbar[i][i] = al[i], Tbar[i+1][i] = b[i], Tbar[i][i+1] = b[i] */
    double Tb[5][4], N[16], g[4];
    memset(Tb, 0, sizeof(Tb));
    for (int i = 0; i < s; i++) {
      Tb[i][i] = al[i];
      Tb[i + 1][i] = b[i];
      if (i + 1 < s) Tb[i][i + 1] = b[i];
    }
    for (int i = 0; i < s; i++) {
      for (int j = 0; j < s; j++) {
        double t = 0.0;
        for (int k = 0; k <= s; k++) t += Tb[k][i] * Tb[k][j];
        N[i * s + j] = t;
      }
      g[i] = beta * Tb[0][i];
    }
    if (gauss_solve(s, N, g) == 0)
      for (int i = 0; i < s; i++) y[i] = g[i];
  }
  for (int i = 0; i < s; i++)
    for (int64_t a = 0; a < m; a++) w[a] += y[i] * V[i][a];
  free(Vbuf);
}

/* Approximate solves of eq. 11 on the diagonal blocks given by bounds (block sizes <= 256, so the
 * blocks may be whole diagonal tiles, as in Section 4.3):
 * method 0 FOM / 2 minimal residual with `steps` (1..3) Krylov iterations (krylov_block), or
 * method 3: w = |H~_[i] - mu_j I|^{-1} r through the block's eigendecomposition (orc_syev),
 * shifted eigenvalues of magnitude below `guard` replaced by +-guard. Returns 0, or -2 if a
 * block eigendecomposition failed. */
int orc_block_krylov(int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                     int64_t nblk, const int64_t* bounds, int64_t nb, const double* mu, const double* R,
                     int method, int steps, double guard, double* W) {
  int64_t* owner = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < nblk; i++)
    for (int64_t r = bounds[i]; r < bounds[i + 1]; r++) owner[r] = i;
  int64_t mmax = 1;
  for (int64_t i = 0; i < nblk; i++)
    if (bounds[i + 1] - bounds[i] > mmax) mmax = bounds[i + 1] - bounds[i];
  double* blk = (double*)malloc((size_t)(mmax * mmax) * sizeof(double));
  double* A = (double*)malloc((size_t)(mmax * mmax) * sizeof(double));
  double* Z = (double*)malloc((size_t)(mmax * mmax) * sizeof(double));
  double* lam = (double*)malloc((size_t)mmax * sizeof(double));
  double* r = (double*)malloc((size_t)mmax * sizeof(double));
  double* w = (double*)malloc((size_t)mmax * sizeof(double));
  int st = 0;
  for (int64_t bi = 0; bi < nblk && !st; bi++) {
    const int64_t o = bounds[bi], m = bounds[bi + 1] - o;
    memset(blk, 0, (size_t)(m * m) * sizeof(double));
    for (int64_t t = 0; t < nnz; t++) {
      const int64_t i = row[t], j = col[t];
      if (owner[i] != bi || owner[j] != bi) continue;
      blk[(i - o) * m + (j - o)] = val[t];
      blk[(j - o) * m + (i - o)] = val[t];
    }
    if (method == 3) {
      memcpy(Z, blk, (size_t)(m * m) * sizeof(double));
      if (orc_syev(m, Z, lam) != 0) { st = -2; break; }
    }
    for (int64_t c = 0; c < nb; c++) {
      for (int64_t a = 0; a < m; a++) r[a] = R[(o + a) * nb + c];
      if (method == 3) {
        for (int64_t k = 0; k < m; k++) {
          double ck = 0.0;
          for (int64_t a = 0; a < m; a++) ck += Z[a * m + k] * r[a];
          double d = fabs(lam[k] - mu[c]);
          if (d < guard) d = guard;
          w[k] = ck / d;
        }
        for (int64_t a = 0; a < m; a++) {
          double t = 0.0;
          for (int64_t k = 0; k < m; k++) t += Z[a * m + k] * w[k];
          W[(o + a) * nb + c] = t;
        }
      } else {
        for (int64_t a = 0; a < m; a++) {
          for (int64_t b2 = 0; b2 < m; b2++) A[a * m + b2] = blk[a * m + b2];
          A[a * m + a] -= mu[c];
        }
        krylov_block(m, A, r, method, steps, w);
        for (int64_t a = 0; a < m; a++) W[(o + a) * nb + c] = w[a];
      }
    }
  }
  free(owner); free(blk); free(A); free(Z); free(lam); free(r); free(w);
  return st;
}

/* Rayleigh-Ritz of eq. 9: given the projected m x m matrices G = Y^T H Y and M = Y^T Y, solve
 * G c = theta M c. M = L L^T (Cholesky), then the standard problem L^{-1} G L^{-T} z = theta z by
 * orc_syev, and c = L^{-T} z. theta (m) ascending; C (m x m row-major) has the M-orthonormal
 * eigenvectors as columns. Returns 0, -1 if M is not positive definite, -2 if QL failed. */
int orc_rayleigh_ritz(int64_t m, const double* G, const double* M, double* theta, double* C) {
  double* L = (double*)calloc((size_t)(m * m), sizeof(double));
  double* A = (double*)malloc((size_t)(m * m) * sizeof(double));
  for (int64_t j = 0; j < m; j++) {
    double s = M[j * m + j];
    for (int64_t t = 0; t < j; t++) s -= L[j * m + t] * L[j * m + t];
    if (!(s > 0.0)) { free(L); free(A); return -1; }
    L[j * m + j] = sqrt(s);
    for (int64_t i = j + 1; i < m; i++) {
      double u = M[i * m + j];
      for (int64_t t = 0; t < j; t++) u -= L[i * m + t] * L[j * m + t];
      L[i * m + j] = u / L[j * m + j];
    }
  }
  /* A = L^{-1} G L^{-T}: first B = L^{-1} G (forward substitution per column), then A = (L^{-1} B^T)^T */
  double* B = (double*)malloc((size_t)(m * m) * sizeof(double));
  for (int64_t c = 0; c < m; c++)
    for (int64_t i = 0; i < m; i++) {
      double s = 0.5 * (G[i * m + c] + G[c * m + i]);
      for (int64_t t = 0; t < i; t++) s -= L[i * m + t] * B[t * m + c];
      B[i * m + c] = s / L[i * m + i];
    }
  for (int64_t r = 0; r < m; r++) /* row r of A = L^{-1} applied to row r of B, as a column */
    for (int64_t i = 0; i < m; i++) {
      double s = B[r * m + i];
      for (int64_t t = 0; t < i; t++) s -= L[i * m + t] * A[r * m + t];
      A[r * m + i] = s / L[i * m + i];
    }
  for (int64_t i = 0; i < m; i++)
    for (int64_t j = i + 1; j < m; j++) {
      double s = 0.5 * (A[i * m + j] + A[j * m + i]);
      A[i * m + j] = s; A[j * m + i] = s;
    }
  int st = orc_syev(m, A, theta);
  /* C = L^{-T} Z: back substitution per column */
  for (int64_t c = 0; c < m; c++)
    for (int64_t i = m - 1; i >= 0; i--) {
      double s = A[i * m + c];
      for (int64_t t = i + 1; t < m; t++) s -= L[t * m + i] * C[t * m + c];
      C[i * m + c] = s / L[i * m + i];
    }
  free(L); free(A); free(B);
  return st ? -2 : 0;
}
