// Rayleigh-Ritz step of LOBPCG (eq. 9, Algorithm 1 steps 7-8): the generalised symmetric
// eigenproblem G c = theta M c of order m = 3 nb, in FP64 on one CTA.
//
//   1. M = L L^T (Cholesky; a non-positive pivot j reports info = j + 1),
//   2. A = L^{-1} G L^{-T} (two triangular solves),
//   3. A = V diag(theta) V^T by cyclic Jacobi with the round-robin ("tournament") order, so
//      the m/2 rotations of a round act on disjoint index pairs and run in parallel,
//   4. sort ascending, C = L^{-T} V.
// The matrices live in a global workspace of 3 m^2 doubles (L1-resident for m <= 96).
#include "common.cuh"
#include "df.cuh"

namespace {

constexpr int RR_THREADS = 512;

__device__ __forceinline__ int rr_player(int pos, int round, int mp) {
  // circle method: position 0 holds player 0; the others rotate by one each round
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (mp - 1);
}

__global__ void __launch_bounds__(RR_THREADS) k_rayleigh_ritz(int m, const double* __restrict__ G,
                                                              const double* __restrict__ Mi, double* __restrict__ theta,
                                                              double* __restrict__ C, int32_t* __restrict__ info,
                                                              double* __restrict__ work) {
  double* A = work;          // m x m
  double* L = work + m * m;  // m x m, lower Cholesky factor
  double* V = L + m * m;     // m x m, eigenvectors
  __shared__ double cs_c[96], cs_s[96];
  __shared__ int pr_p[96], pr_q[96];
  __shared__ double red[RR_THREADS / 32];
  __shared__ int s_fail;
  __shared__ double s_off, s_fro;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m;

  // symmetric copies from the upper triangles
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    const int a = i < j ? i : j, b = i < j ? j : i;
    A[e] = G[a * m + b];
    L[e] = Mi[a * m + b];
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();

  // 1. right-looking Cholesky in place on L (lower part)
  for (int j = 0; j < m; j++) {
    if (tid == 0) {
      const double d = L[j * m + j];
      if (!(d > 0.0)) s_fail = j + 1;
      else L[j * m + j] = sqrt(d);
    }
    __syncthreads();
    if (s_fail) break;
    const double ljj = L[j * m + j];
    for (int i = j + 1 + tid; i < m; i += nt) L[i * m + j] /= ljj;
    __syncthreads();
    const int rem = m - j - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) L[i * m + k] -= L[i * m + j] * L[k * m + j];
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) *info = s_fail;
    return;
  }
  // 2a. A <- L^{-1} A: forward substitution, one column per thread
  for (int c = tid; c < m; c += nt)
    for (int i = 0; i < m; i++) {
      double s = A[i * m + c];
      for (int t = 0; t < i; t++) s -= L[i * m + t] * A[t * m + c];
      A[i * m + c] = s / L[i * m + i];
    }
  __syncthreads();
  // 2b. A <- A L^{-T}: forward substitution on each row
  for (int r = tid; r < m; r += nt)
    for (int i = 0; i < m; i++) {
      double s = A[r * m + i];
      for (int t = 0; t < i; t++) s -= L[i * m + t] * A[r * m + t];
      A[r * m + i] = s / L[i * m + i];
    }
  __syncthreads();
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    if (i < j) {
      const double s = 0.5 * (A[i * m + j] + A[j * m + i]);
      A[i * m + j] = s;
      A[j * m + i] = s;
    }
  }
  __syncthreads();

  // 3. parallel cyclic Jacobi
  const int mp = m + (m & 1);  // players incl. a dummy when m is odd
  const int npairs = mp / 2;
  for (int sweep = 0; sweep < 40; sweep++) {
    // convergence: off-diagonal Frobenius norm vs the whole
    double off = 0.0, fro = 0.0;
    for (int e = tid; e < mm; e += nt) {
      const double x = A[e];
      fro += x * x;
      if (e / m != e % m) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) { off += __shfl_down_sync(0xFFFFFFFFu, off, o); fro += __shfl_down_sync(0xFFFFFFFFu, fro, o); }
    if (tid % 32 == 0) red[tid / 32] = off;
    __syncthreads();
    if (tid == 0) { double s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_off = s; }
    __syncthreads();
    if (tid % 32 == 0) red[tid / 32] = fro;
    __syncthreads();
    if (tid == 0) { double s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_fro = s; }
    __syncthreads();
    if (s_off <= 1e-30 * s_fro || s_off == 0.0) break;
    for (int round = 0; round < mp - 1; round++) {
      for (int k = tid; k < npairs; k += nt) {
        int p = rr_player(k, round, mp), q = rr_player(mp - 1 - k, round, mp);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p * m + q];
          if (apq != 0.0) {
            const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pr_p[k] = p; pr_q[k] = q; cs_c[k] = c; cs_s[k] = s;
      }
      __syncthreads();
      // rows p, q of A
      for (int e = tid; e < npairs * m; e += nt) {
        const int k = e / m, col = e % m;
        const int p = pr_p[k], q = pr_q[k];
        if (q >= m || cs_s[k] == 0.0) continue;
        const double c = cs_c[k], s = cs_s[k];
        const double ap = A[p * m + col], aq = A[q * m + col];
        A[p * m + col] = c * ap - s * aq;
        A[q * m + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and of V
      for (int e = tid; e < npairs * m; e += nt) {
        const int k = e / m, row = e % m;
        const int p = pr_p[k], q = pr_q[k];
        if (q >= m || cs_s[k] == 0.0) continue;
        const double c = cs_c[k], s = cs_s[k];
        const double ap = A[row * m + p], aq = A[row * m + q];
        A[row * m + p] = c * ap - s * aq;
        A[row * m + q] = s * ap + c * aq;
        const double vp = V[row * m + p], vq = V[row * m + q];
        V[row * m + p] = c * vp - s * vq;
        V[row * m + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // 4. rank sort (ties by index), C = L^{-T} V in the sorted order
  for (int j = tid; j < m; j += nt) {
    const double wj = A[j * m + j];
    int rank = 0;
    for (int i = 0; i < m; i++) {
      const double wi = A[i * m + i];
      rank += (wi < wj) || (wi == wj && i < j);
    }
    theta[rank] = wj;
    for (int i = m - 1; i >= 0; i--) {
      double s = V[i * m + j];
      for (int t = i + 1; t < m; t++) s -= L[t * m + i] * C[t * m + rank];
      C[i * m + rank] = s / L[i * m + i];
    }
  }
  if (tid == 0) *info = 0;
}

// The same Rayleigh-Ritz step in double-float (df.cuh): every element operation of the
// Cholesky factorisation, the triangular solves and the Jacobi rotations runs on the FP32
// pipes with ~48-bit significands; only scalar work per pivot or per rotation (square roots,
// reciprocals, rotation angles, convergence sums) is done in FP64. The workspace holds the
// three m x m matrices as (hi, lo) pairs.
__global__ void __launch_bounds__(RR_THREADS) k_rayleigh_ritz_df(int m, const double* __restrict__ G,
                                                                 const double* __restrict__ Mi,
                                                                 double* __restrict__ theta, double* __restrict__ C,
                                                                 int32_t* __restrict__ info, double* __restrict__ work) {
  d2* A = reinterpret_cast<d2*>(work);
  d2* L = A + m * m;
  d2* V = L + m * m;
  __shared__ d2 cs_c[96], cs_s[96];
  __shared__ int pr_p[96], pr_q[96];
  __shared__ d2 inv[192];
  __shared__ double red[RR_THREADS / 32];
  __shared__ int s_fail;
  __shared__ double s_off, s_fro;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m;
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    const int a = i < j ? i : j, b = i < j ? j : i;
    A[e] = d2_from(G[a * m + b]);
    L[e] = d2_from(Mi[a * m + b]);
    V[e] = d2{(i == j) ? 1.f : 0.f, 0.f};
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // 1. Cholesky (right-looking); inv[j] = 1 / L_jj
  for (int j = 0; j < m; j++) {
    if (tid == 0) {
      const double d = d2_to(L[j * m + j]);
      if (!(d > 0.0)) s_fail = j + 1;
      else {
        const double sq = sqrt(d);
        L[j * m + j] = d2_from(sq);
        inv[j] = d2_from(1.0 / sq);
      }
    }
    __syncthreads();
    if (s_fail) break;
    const d2 ij = inv[j];
    for (int i = j + 1 + tid; i < m; i += nt) L[i * m + j] = d2_mul(L[i * m + j], ij);
    __syncthreads();
    const int rem = m - j - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) {
        d2 x = L[i * m + k];
        const d2 a = L[i * m + j], b = L[k * m + j];
        df_mac(x.hi, x.lo, -a.hi, -a.lo, b.hi, b.lo);
        L[i * m + k] = d2_norm(x);
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) *info = s_fail;
    return;
  }
  // 2a. A <- L^{-1} A (columns), 2b. A <- A L^{-T} (rows)
  for (int c = tid; c < m; c += nt)
    for (int i = 0; i < m; i++) {
      d2 s = A[i * m + c];
      for (int t = 0; t < i; t++) { const d2 l = L[i * m + t], a = A[t * m + c]; df_mac(s.hi, s.lo, -l.hi, -l.lo, a.hi, a.lo); }
      A[i * m + c] = d2_mul(d2_norm(s), inv[i]);
    }
  __syncthreads();
  for (int r = tid; r < m; r += nt)
    for (int i = 0; i < m; i++) {
      d2 s = A[r * m + i];
      for (int t = 0; t < i; t++) { const d2 l = L[i * m + t], a = A[r * m + t]; df_mac(s.hi, s.lo, -l.hi, -l.lo, a.hi, a.lo); }
      A[r * m + i] = d2_mul(d2_norm(s), inv[i]);
    }
  __syncthreads();
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    if (i < j) {
      d2 s = d2_add(A[i * m + j], A[j * m + i]);
      s.hi *= 0.5f; s.lo *= 0.5f;  // exact
      A[i * m + j] = s;
      A[j * m + i] = s;
    }
  }
  __syncthreads();
  // 3. parallel cyclic Jacobi, rotations computed in FP64 and applied in double-float
  const int mp = m + (m & 1), npairs = mp / 2;
  for (int sweep = 0; sweep < 40; sweep++) {
    double off = 0.0, fro = 0.0;
    for (int e = tid; e < mm; e += nt) {
      const double x = d2_hi64(A[e]);
      fro += x * x;
      if (e / m != e % m) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) { off += __shfl_down_sync(0xFFFFFFFFu, off, o); fro += __shfl_down_sync(0xFFFFFFFFu, fro, o); }
    if (tid % 32 == 0) red[tid / 32] = off;
    __syncthreads();
    if (tid == 0) { double s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_off = s; }
    __syncthreads();
    if (tid % 32 == 0) red[tid / 32] = fro;
    __syncthreads();
    if (tid == 0) { double s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_fro = s; }
    __syncthreads();
    if (s_off <= 1e-30 * s_fro || s_off == 0.0) break;
    for (int round = 0; round < mp - 1; round++) {
      for (int k = tid; k < npairs; k += nt) {
        int p = rr_player(k, round, mp), q = rr_player(mp - 1 - k, round, mp);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = d2_to(A[p * m + q]);
          if (apq != 0.0) {
            const double tau = (d2_to(A[q * m + q]) - d2_to(A[p * m + p])) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pr_p[k] = p; pr_q[k] = q; cs_c[k] = d2_from(c); cs_s[k] = d2_from(s);
      }
      __syncthreads();
      for (int e = tid; e < npairs * m; e += nt) {
        const int k = e / m, col = e % m;
        const int p = pr_p[k], q = pr_q[k];
        if (q >= m || cs_s[k].hi == 0.f) continue;
        d2_rot(A[p * m + col], A[q * m + col], cs_c[k], cs_s[k]);
      }
      __syncthreads();
      for (int e = tid; e < npairs * m; e += nt) {
        const int k = e / m, row = e % m;
        const int p = pr_p[k], q = pr_q[k];
        if (q >= m || cs_s[k].hi == 0.f) continue;
        d2_rot(A[row * m + p], A[row * m + q], cs_c[k], cs_s[k]);
        d2_rot(V[row * m + p], V[row * m + q], cs_c[k], cs_s[k]);
      }
      __syncthreads();
    }
  }
  // 4. rank sort, C = L^{-T} V
  for (int j = tid; j < m; j += nt) {
    const double wj = d2_to(A[j * m + j]);
    int rank = 0;
    for (int i = 0; i < m; i++) {
      const double wi = d2_to(A[i * m + i]);
      rank += (wi < wj) || (wi == wj && i < j);
    }
    theta[rank] = wj;
    // back substitution in double-float; column `rank` of C kept in V's column j
    for (int i = m - 1; i >= 0; i--) {
      d2 s = V[i * m + j];
      for (int t = i + 1; t < m; t++) {
        const d2 l = L[t * m + i], x = V[t * m + j];
        df_mac(s.hi, s.lo, -l.hi, -l.lo, x.hi, x.lo);
      }
      V[i * m + j] = d2_mul(d2_norm(s), inv[i]);
    }
    for (int i = 0; i < m; i++) C[i * m + rank] = d2_to(V[i * m + j]);
  }
  if (tid == 0) *info = 0;
}

}  // namespace

int lob_rr_launch_df(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                     cudaStream_t st) {
  if (m < 1 || m > 192) return LOB_ERR_ARG;
  (k_rayleigh_ritz_df<<<1, RR_THREADS, 0, st>>>(m, G, M, theta, C, info, work), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

size_t lob_rr_work_doubles(int m) { return 3ull * m * m; }

int lob_rr_launch(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                  cudaStream_t st) {
  if (m < 1 || m > 192) return LOB_ERR_ARG;
  (k_rayleigh_ritz<<<1, RR_THREADS, 0, st>>>(m, G, M, theta, C, info, work), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}
