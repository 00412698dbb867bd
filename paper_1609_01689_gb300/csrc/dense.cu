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

}  // namespace

size_t lob_rr_work_doubles(int m) { return 3ull * m * m; }

int lob_rr_launch(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                  cudaStream_t st) {
  if (m < 1 || m > 192) return LOB_ERR_ARG;
  (k_rayleigh_ritz<<<1, RR_THREADS, 0, st>>>(m, G, M, theta, C, info, work), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}
