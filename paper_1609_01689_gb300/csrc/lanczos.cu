// Lanczos baseline on the GPU: the legacy single-vector solver that the paper compares LOBPCG
// against (Section 1, Section 5.2 and Table 3). One FP64 SpMV per step through the same tile
// store, full reorthogonalisation (classical Gram-Schmidt, twice) against every previous
// Lanczos vector, and every `check` steps the k smallest eigenpairs of the tridiagonal T_j
// (bisection and inverse iteration on the host) with the Ritz residual estimate
// beta_j |s_{j,i}| <= tol ||H|| as the stopping test -- the same relative residual that LOBPCG's
// convergence test uses.
//
// Device state: V (n x max_steps, one contiguous vector per step), w, and the recurrence scalars
// (alpha, beta, dot products) -- none of them leave the device between checks.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "common.cuh"

namespace {

constexpr int BS = 256;
constexpr int DCOLS = 8;  // vectors per CTA in the dot-product kernel
inline unsigned nblk(int64_t n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

// seeded uniform(-1, 1) start vector (splitmix64 of (seed, i))
__global__ void k_start(int64_t n, uint64_t seed, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed * 0xD1B54A32D192ED03ull + (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// part[chunk][c] = sum over the chunk's rows of V[c][r] * w[r], c < ncol (V column c at V + c*n)
__global__ void __launch_bounds__(BS) k_dots(int64_t n, int64_t rpc, int ncol, const double* __restrict__ V,
                                             const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[BS / 32][DCOLS];
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = r0 + rpc < n ? r0 + rpc : n;
  const int c0 = blockIdx.y * DCOLS;
  double acc[DCOLS];
#pragma unroll
  for (int c = 0; c < DCOLS; c++) acc[c] = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += BS) {
    const double x = w[r];
#pragma unroll
    for (int c = 0; c < DCOLS; c++)
      if (c0 + c < ncol) acc[c] = fma(V[(int64_t)(c0 + c) * n + r], x, acc[c]);
  }
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
#pragma unroll
  for (int c = 0; c < DCOLS; c++) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[wid][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < DCOLS && c0 + (int)threadIdx.x < ncol) {
    double v = 0.0;
    for (int q = 0; q < BS / 32; q++) v += red[q][threadIdx.x];
    part[(int64_t)blockIdx.x * ncol + c0 + threadIdx.x] = v;
  }
}

// h[c] = sum over chunks of part[chunk][c] (fixed order), one warp per c; add_to: h accumulates
// into acc[c] as well (the reorthogonalisation coefficients corrected into alpha / beta).
__global__ void k_dots_reduce(int nchunks, int ncol, const double* __restrict__ part, double* __restrict__ h) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (c >= ncol) return;
  double s = 0.0;
  for (int q = lane; q < nchunks; q += 32) s += part[(int64_t)q * ncol + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) h[c] = s;
}

// w[r] -= sum_c V[c][r] h[c]
__global__ void k_subtract(int64_t n, int ncol, const double* __restrict__ V, const double* __restrict__ h,
                           double* __restrict__ w) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = w[r];
  for (int c = 0; c < ncol; c++) s = fma(-V[(int64_t)c * n + r], h[c], s);
  w[r] = s;
}

// alpha_j = first-pass coefficient of v_j plus the two reorthogonalisation corrections;
// beta_j = ||w|| (from its dot with itself), and v_{j+1} = w / beta_j.
__global__ void k_coeffs(int j, const double* __restrict__ h1, const double* __restrict__ h2,
                         const double* __restrict__ ww, double* __restrict__ alpha, double* __restrict__ beta) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  alpha[j] = h1[j] + h2[j];
  beta[j] = sqrt(ww[0]);
}

__global__ void k_scale(int64_t n, const double* __restrict__ w, const double* __restrict__ beta, int j,
                        double* __restrict__ vnext) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double b = beta[j];
  vnext[r] = b > 0.0 ? w[r] / b : 0.0;
}

// X[r][i] = sum_c V[c][r] S[c][i] (S m x k row-major), i < k <= 16
__global__ void k_ritz(int64_t n, int m, int k, const double* __restrict__ V, const double* __restrict__ S,
                       double* __restrict__ X) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double acc[16];
  for (int i = 0; i < 16; i++) acc[i] = 0.0;
  for (int c = 0; c < m; c++) {
    const double v = V[(int64_t)c * n + r];
    for (int i = 0; i < k; i++) acc[i] = fma(v, S[c * k + i], acc[i]);
  }
  for (int i = 0; i < k; i++) X[r * k + i] = acc[i];
}

// The k smallest eigenpairs of the symmetric tridiagonal T (diagonal a[0..m), off-diagonal
// b[0..m-1), b[i] coupling i and i+1), from first principles:
//  - eigenvalues by bisection on the Sturm count: the number of eigenvalues below x equals the
//    number of negative pivots of the LDL^T factorisation of T - x I (Sylvester's law of
//    inertia), pivots q_0 = a_0 - x, q_i = a_i - x - b_{i-1}^2 / q_{i-1};
//  - eigenvectors by inverse iteration: a few solves (T - lambda I) y = y_prev with Gaussian
//    elimination (partial pivoting) of the tridiagonal, then normalisation; vectors of close
//    eigenvalues are orthogonalised against the earlier ones.
static int sturm_below(int m, const double* a, const double* b, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; i++) {
    const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    q = (a[i] - x) - (i > 0 ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;  // treat an exact zero pivot as a tiny negative one
    if (q < 0.0) cnt++;
  }
  return cnt;
}

static void tridiag_smallest(int m, const double* a, const double* b, int k, double* lam) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; i++) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  const double span = fmax(hi - lo, 1e-300);
  for (int j = 0; j < k; j++) {  // j-th smallest: the x with exactly j eigenvalues below
    double l = j > 0 ? lam[j - 1] : lo, h = hi;
    for (int it = 0; it < 200 && h - l > 4e-16 * span; it++) {
      const double mid = 0.5 * (l + h);
      if (sturm_below(m, a, b, mid) > j) h = mid; else l = mid;
    }
    lam[j] = 0.5 * (l + h);
  }
}

// Solve (T - s I) y = rhs in place (rhs -> y) by Gaussian elimination with partial pivoting on
// the tridiagonal (one extra super-diagonal appears); tiny pivots are replaced by eps ||T||.
static void tridiag_shift_solve(int m, const double* a, const double* b, double s, double tnorm, double* y) {
  std::vector<double> dg(m), up(m, 0.0), up2(m, 0.0), lo(m, 0.0);
  for (int i = 0; i < m; i++) { dg[i] = a[i] - s; if (i + 1 < m) up[i] = b[i]; if (i > 0) lo[i] = b[i - 1]; }
  const double tiny = 1e-14 * tnorm;
  for (int i = 0; i + 1 < m; i++) {
    // rows i and i+1 (row i+1 has lo[i+1] in column i)
    if (fabs(lo[i + 1]) > fabs(dg[i])) {  // swap rows i and i+1
      std::swap(dg[i], lo[i + 1]);
      std::swap(up[i], dg[i + 1]);
      std::swap(up2[i], up[i + 1]);
      std::swap(y[i], y[i + 1]);
    }
    if (fabs(dg[i]) < tiny) dg[i] = tiny;
    const double f = lo[i + 1] / dg[i];
    dg[i + 1] -= f * up[i];
    up[i + 1] -= f * up2[i];
    y[i + 1] -= f * y[i];
    lo[i + 1] = 0.0;
  }
  if (fabs(dg[m - 1]) < tiny) dg[m - 1] = tiny;
  for (int i = m - 1; i >= 0; i--) {
    double t = y[i];
    if (i + 1 < m) t -= up[i] * y[i + 1];
    if (i + 2 < m) t -= up2[i] * y[i + 2];
    y[i] = t / dg[i];
  }
}

// Columns i < k of Z (m x k row-major): unit eigenvectors of T for lam[i].
static void tridiag_vectors(int m, const double* a, const double* b, int k, const double* lam, double* Z) {
  double tnorm = 0.0;
  for (int i = 0; i < m; i++)
    tnorm = fmax(tnorm, fabs(a[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0));
  std::vector<double> y(m);
  for (int j = 0; j < k; j++) {
    for (int i = 0; i < m; i++) y[i] = 1.0 + 1e-3 * ((i * 7 + j * 13) % 17);  // generic start
    for (int it = 0; it < 3; it++) {
      tridiag_shift_solve(m, a, b, lam[j], tnorm, y.data());
      for (int p = 0; p < j; p++)  // orthogonalise against earlier vectors of close eigenvalues
        if (fabs(lam[p] - lam[j]) < 1e-6 * tnorm) {
          double dot = 0.0;
          for (int i = 0; i < m; i++) dot += Z[(size_t)i * k + p] * y[i];
          for (int i = 0; i < m; i++) y[i] -= dot * Z[(size_t)i * k + p];
        }
      double nrm = 0.0;
      for (int i = 0; i < m; i++) nrm += y[i] * y[i];
      nrm = sqrt(nrm);
      for (int i = 0; i < m; i++) y[i] /= nrm;
    }
    for (int i = 0; i < m; i++) Z[(size_t)i * k + j] = y[i];
  }
}

struct DBuf {
  double* p = nullptr;
  ~DBuf() { if (p) cudaFree(p); }
  int alloc(size_t n) {
    if (cudaMalloc((void**)&p, (n ? n : 1) * sizeof(double)) != cudaSuccess) { cudaGetLastError(); p = nullptr; return LOB_ERR_NOMEM; }
    return LOB_OK;
  }
};

}  // namespace

extern "C" int lob_lanczos(lob_matrix* H, int32_t k, double tol, int32_t max_steps, int32_t check, uint64_t seed,
                           double* lambda, double* X, lob_lanczos_stats* stats, void* stream) {
  if (!H || !lambda || k < 1 || k > 16 || !(tol > 0.0) || max_steps < k + 1 || !H->T.v64) return LOB_ERR_ARG;
  const int64_t n = H->T.n;
  if (max_steps > n) max_steps = (int32_t)n;
  if (check < 1) check = 10;
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  const double normH = H->norm_inf;
  // row chunks of the dot products: about 4 CTAs per SM for the widest basis
  const int nch = (int)std::min<int64_t>(608, (n + 1023) / 1024);
  const int64_t rpc = (n + nch - 1) / nch;
  DBuf V, w, part, h1, h2, alpha, beta, ww, S;
  LOB_TRY(V.alloc((size_t)n * max_steps));
  LOB_TRY(w.alloc(n));
  LOB_TRY(part.alloc((size_t)nch * max_steps));
  LOB_TRY(h1.alloc(max_steps)); LOB_TRY(h2.alloc(max_steps));
  LOB_TRY(alpha.alloc(max_steps)); LOB_TRY(beta.alloc(max_steps)); LOB_TRY(ww.alloc(1));
  if (stats) memset(stats, 0, sizeof(*stats));
  // v_0 = random / ||random||
  (k_start<<<nblk(n), BS, 0, st>>>(n, seed, w.p), LOB_LAUNCHED());
  auto dots = [&](int ncol, const double* Vp, const double* x, double* h) -> int {
    dim3 grid(nch, (ncol + DCOLS - 1) / DCOLS);
    (k_dots<<<grid, BS, 0, st>>>(n, rpc, ncol, Vp, x, part.p), LOB_LAUNCHED());
    (k_dots_reduce<<<nblk((int64_t)ncol * 32), BS, 0, st>>>(nch, ncol, part.p, h), LOB_LAUNCHED());
    return LOB_OK;
  };
  LOB_TRY(dots(1, w.p, w.p, ww.p));
  (k_coeffs<<<1, 32, 0, st>>>(0, ww.p, ww.p, ww.p, h2.p, beta.p), LOB_LAUNCHED());  // beta[0] = ||w|| (h2 scratch)
  (k_scale<<<nblk(n), BS, 0, st>>>(n, w.p, beta.p, 0, V.p), LOB_LAUNCHED());
  std::vector<double> ha(max_steps), hb(max_steps);
  int steps = 0, status = LOB_ERR_NOCONV;
  double spmv_ms = 0.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int j = 0; j < max_steps; j++) {
    double* vj = V.p + (int64_t)j * n;
    cudaEventRecord(e0, st);
    LOB_TRY(lob_spmm_launch(H, LOB_SPMM_FP64, vj, w.p, 1, n, st));
    cudaEventRecord(e1, st);
    // w <- w - V_{0..j} h, twice (the first pass gives alpha_j and beta_{j-1} as its last two
    // coefficients; the full pass removes every earlier direction)
    LOB_TRY(dots(j + 1, V.p, w.p, h1.p));
    (k_subtract<<<nblk(n), BS, 0, st>>>(n, j + 1, V.p, h1.p, w.p), LOB_LAUNCHED());
    LOB_TRY(dots(j + 1, V.p, w.p, h2.p));
    (k_subtract<<<nblk(n), BS, 0, st>>>(n, j + 1, V.p, h2.p, w.p), LOB_LAUNCHED());
    LOB_TRY(dots(1, w.p, w.p, ww.p));
    (k_coeffs<<<1, 32, 0, st>>>(j, h1.p, h2.p, ww.p, alpha.p, beta.p + 1), LOB_LAUNCHED());
    if (j + 1 < max_steps)
      (k_scale<<<nblk(n), BS, 0, st>>>(n, w.p, beta.p + 1, j, V.p + (int64_t)(j + 1) * n), LOB_LAUNCHED());
    steps = j + 1;
    if (steps < k || (steps % check != 0 && steps != max_steps)) continue;
    // Ritz values of T_steps and the last components of its eigenvectors
    LOB_CUDA(cudaMemcpyAsync(ha.data(), alpha.p, steps * 8, cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaMemcpyAsync(hb.data(), beta.p + 1, steps * 8, cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) spmv_ms = ms;  // the latest SpMV
    // k smallest Ritz values and their residual estimates beta_steps |s_{last,i}|
    std::vector<double> th(k), Zk((size_t)steps * k);
    tridiag_smallest(steps, ha.data(), hb.data(), k, th.data());
    tridiag_vectors(steps, ha.data(), hb.data(), k, th.data(), Zk.data());
    const double bl = hb[steps - 1];
    bool conv = true;
    for (int i = 0; i < k; i++)
      if (!(fabs(bl * Zk[(size_t)(steps - 1) * k + i]) <= tol * normH)) conv = false;
    if (conv) { status = LOB_OK; break; }
  }
  // final Ritz pairs: X = V S with S the k smallest eigenvectors of T_steps
  LOB_CUDA(cudaMemcpyAsync(ha.data(), alpha.p, steps * 8, cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaMemcpyAsync(hb.data(), beta.p + 1, steps * 8, cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaStreamSynchronize(st));
  const int kk = k < steps ? k : steps;
  std::vector<double> th(kk), Sk((size_t)steps * kk);
  tridiag_smallest(steps, ha.data(), hb.data(), kk, th.data());
  for (int i = 0; i < kk; i++) lambda[i] = th[i];
  if (X) {
    tridiag_vectors(steps, ha.data(), hb.data(), kk, th.data(), Sk.data());
    LOB_TRY(S.alloc(Sk.size()));
    LOB_CUDA(cudaMemcpyAsync(S.p, Sk.data(), Sk.size() * 8, cudaMemcpyHostToDevice, st));
    (k_ritz<<<nblk(n), BS, 0, st>>>(n, steps, kk, V.p, S.p, X), LOB_LAUNCHED());
    LOB_CUDA(cudaStreamSynchronize(st));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    stats->steps = steps;
    stats->spmv_ms = spmv_ms;  // device time of one SpMV (the last one timed)
    stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->device_bytes = (double)n * max_steps * 8.0;
  }
  return status;
}
