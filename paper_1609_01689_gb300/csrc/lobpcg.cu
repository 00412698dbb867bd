// LOBPCG driver (Section 3.1, Algorithm 1) with the block-diagonal preconditioner
// (Section 3.2, eq. 11), the robustness rules of Section 4.3, and the initial guess of
// Section 3.3.1 (eq. 12). All vectors stay on the device; the host orchestrates launches and
// reads back nb residual norms per iteration for the convergence test (step 5).
//
// Per iteration i (S = [X W P], HS = H S, m = nb + 2 na columns):
//   R = H X - X Theta                         (step 4)
//   W = T^{-1} R on the active columns        (step 6; T = I while the rules forbid it)
//   W <- W - X (X^T W), then W <- W L^{-T} with W^T W = L L^T (Cholesky-QR)   (step 7)
//   H W by one SpMM; P <- P L_P^{-T}, H P likewise (Cholesky-QR of P)
//   G = S^T H S, M = S^T S; G C = M C Theta  (eq. 9, steps 7-8)
//   X <- S C_x, H X <- H S C_x, P <- [W P] C_wp, H P <- [H W H P] C_wp   (eq. 7, steps 9-10)
// The search direction is P = W G_2 + P G_3 (eq. 7), which spans the same space as the
// orthogonalised X^(i+1) - X^(i) of step 10, and lets H P be updated with the same
// coefficients, so each iteration needs exactly one SpMM. Columns whose residual already
// meets the tolerance are kept in X but leave W and P ("soft locking").
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "common.cuh"
#include "df.cuh"

namespace {

constexpr int BS = 256;
inline unsigned nblk(int64_t n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

// Seeded uniform(-1, 1) entries (splitmix64 of (seed, i, j)) in rows < n_act, zero below.
__global__ void k_random(int64_t n, int64_t n_act, int nb, int ld, int col0, int ncol, uint64_t seed,
                         double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ncol) return;
  const int64_t i = t / ncol;
  const int j = col0 + (int)(t % ncol);
  double v = 0.0;
  if (i < n_act) {
    uint64_t z = seed * 0xD1B54A32D192ED03ull + (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)j * 0xC2B2AE3D27D4EB4Full;
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  out[i * ld + j] = v;
  (void)nb;
}

// dst[:, i] = src[:, map ? map[i] : i] for i < ncol, rows < n.
__global__ void k_copy_cols(int64_t n, int ncol, const double* __restrict__ src, int lds, const int* __restrict__ map,
                            double* __restrict__ dst, int ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ncol) return;
  const int64_t r = t / ncol;
  const int i = (int)(t % ncol);
  dst[r * ldd + i] = src[r * lds + (map ? map[i] : i)];
}

// R = HX - X diag(theta); per-CTA partial column sums of r^2 and x^2 into part[blk][2*nb].
__global__ void k_residual(int64_t n, int nb, const double* __restrict__ X, int ldx, const double* __restrict__ HX,
                           int ldh, const double* __restrict__ theta, double* __restrict__ R, double* __restrict__ part) {
  extern __shared__ double sred[];  // [BS/32][2*nb]
  const int tid = threadIdx.x;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + tid;
  const int lane = tid % 32, warp = tid / 32;
  for (int j = 0; j < nb; j++) {
    double rr = 0.0, xx = 0.0;
    if (r < n) {
      const double x = X[r * ldx + j];
      const double v = HX[r * ldh + j] - x * theta[j];
      R[r * nb + j] = v;
      rr = v * v;
      xx = x * x;
    }
    for (int o = 16; o > 0; o >>= 1) { rr += __shfl_down_sync(0xFFFFFFFFu, rr, o); xx += __shfl_down_sync(0xFFFFFFFFu, xx, o); }
    if (lane == 0) { sred[warp * 2 * nb + j] = rr; sred[warp * 2 * nb + nb + j] = xx; }
  }
  __syncthreads();
  for (int j = tid; j < 2 * nb; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)blockDim.x / 32; w++) s += sred[w * 2 * nb + j];
    part[(int64_t)blockIdx.x * 2 * nb + j] = s;
  }
}

// relres_j = sqrt(sum r^2) / (normH sqrt(sum x^2)), fixed-order reduction over the partials.
__global__ void k_relres(int nparts, int nb, const double* __restrict__ part, double normH, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= nb) return;
  double rr = 0.0, xx = 0.0;
  for (int b = 0; b < nparts; b++) { rr += part[(int64_t)b * 2 * nb + j]; xx += part[(int64_t)b * 2 * nb + nb + j]; }
  out[j] = sqrt(rr) / (normH * sqrt(xx > 0.0 ? xx : 1.0));
}

// Shifts mu_j for the preconditioner. mode 0: mu_j = theta_j. mode 1 (Section 4.3 rules 3-4):
// nearly converged columns (relres < 1e-2) get mu_i = theta_i - 2 ||r_i|| / ||x_i||; from the
// first column that is far from converged on, all get the previous column's shift.
__global__ void k_shifts(int nb, int mode, const double* __restrict__ theta, const double* __restrict__ relres,
                         double normH, double* __restrict__ mu) {
  if (threadIdx.x != 0) return;
  for (int j = 0; j < nb; j++) mu[j] = theta[j];
  if (mode != 1) return;
  for (int j = 0; j < nb; j++) {
    if (relres[j] < 1e-2) {
      mu[j] = theta[j] - 2.0 * relres[j] * normH;
    } else if (j > 0) {
      for (int t = j; t < nb; t++) mu[t] = mu[j - 1];
      break;
    }
  }
}

// C2 = [-Z; I] (rows: nb rows of -Z then na rows of the identity), for W - X Z as [X W] C2.
__global__ void k_proj_coef(int nb, int na, const double* __restrict__ Z, double* __restrict__ C2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (nb + na) * na) return;
  const int r = t / na, c = t % na;
  C2[t] = r < nb ? -Z[r * na + c] : (r - nb == c ? 1.0 : 0.0);
}

// Phase timing with CUDA events on the solver's stream. Event pairs are recorded without
// synchronising and resolved in bulk whenever the solver synchronises anyway (the per-iteration
// convergence readback), so timing adds no host-device round trips.
struct PhaseClock {
  struct Pair { cudaEvent_t a, b; double* acc; };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (pool.empty()) { cudaEvent_t e; cudaEventCreate(&e); return e; }
    cudaEvent_t e = pool.back(); pool.pop_back(); return e;
  }
  void resolve() {  // call after the stream has been synchronised
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.acc) *p.acc += ms;
      pool.push_back(p.a); pool.push_back(p.b);
    }
    pending.clear();
  }
  ~PhaseClock() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};
thread_local PhaseClock* g_clock = nullptr;

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  double* acc;
  Timer(cudaStream_t s, double* accum) : st(s), acc(accum) {
    if (acc && g_clock) { a = g_clock->get(); cudaEventRecord(a, st); }
  }
  ~Timer() {
    if (a) {
      b = g_clock->get();
      cudaEventRecord(b, st);
      g_clock->pending.push_back({a, b, acc});
    }
  }
};

struct DBuf {
  double* p = nullptr;
  ~DBuf() { if (p) cudaFree(p); }
  int alloc(size_t n) {
    if (cudaMalloc((void**)&p, (n ? n : 1) * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return LOB_ERR_NOMEM; }
    return LOB_OK;
  }
};

enum { PH_SPMM, PH_GRAM, PH_RR, PH_UPDATE, PH_PRECOND, PH_RESID, PH_ORTH, PH_GUESS };

struct Solver {
  const lob_matrix* M;
  int64_t n, n_act;
  int nb, k, spmm_mode, blas_mode;
  cudaStream_t st;
  double normH;
  lob_stats* stats;
  bool timing;
  int ldS;
  DBuf S, HS, P, HP, R, W, Tn, THn, Tp, THp, G, Mm, Cc, Cx, theta, thw, work, rrwork, part, relres_d, mu, C2, Z;
  DBuf info_d;
  int* map_d = nullptr;
  std::vector<double> relres_h;
  int npart;

  ~Solver() { if (map_d) cudaFree(map_d); }

  int alloc() {
    ldS = 3 * nb;
    const size_t nS = (size_t)n * ldS, nv = (size_t)n * nb, m = ldS;
    LOB_TRY(S.alloc(nS)); LOB_TRY(HS.alloc(nS));
    LOB_TRY(P.alloc(nv)); LOB_TRY(HP.alloc(nv)); LOB_TRY(R.alloc(nv)); LOB_TRY(W.alloc(nv));
    LOB_TRY(Tn.alloc(nv)); LOB_TRY(THn.alloc(nv)); LOB_TRY(Tp.alloc(nv)); LOB_TRY(THp.alloc(nv));
    LOB_TRY(G.alloc(m * m)); LOB_TRY(Mm.alloc(m * m)); LOB_TRY(Cc.alloc(m * m)); LOB_TRY(Cx.alloc(m * m)); LOB_TRY(theta.alloc(m)); LOB_TRY(thw.alloc(m));
    LOB_TRY(work.alloc(lob_gram_work_doubles(n, 1, 1) * m * m));  // bound over every (p, q) <= m
    LOB_TRY(rrwork.alloc(lob_rr_work_doubles((int)m)));
    npart = (int)nblk(n);
    LOB_TRY(part.alloc((size_t)npart * 2 * m));
    LOB_TRY(relres_d.alloc(nb)); LOB_TRY(mu.alloc(nb)); LOB_TRY(C2.alloc(m * m)); LOB_TRY(Z.alloc(m * m));
    LOB_TRY(info_d.alloc(1));
    if (cudaMalloc((void**)&map_d, 64 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return LOB_ERR_NOMEM; }
    relres_h.assign(nb, 0.0);
    return LOB_OK;
  }

  double* ph(int i) { return (timing && stats) ? &stats->phase_ms[i] : nullptr; }

  // projected eigenproblem in the solver's block arithmetic (native FP64 or double-float)
  int rr(int m, const double* Gp, const double* Mp, double* th, double* Cp, int chol_only = 0) {
    if (blas_mode == LOB_SPMM_MIXED)
      return lob_rr_launch_df(m, Gp, Mp, th, Cp, (int32_t*)info_d.p, rrwork.p, st, chol_only);
    return lob_rr_launch(m, Gp, Mp, th, Cp, (int32_t*)info_d.p, rrwork.p, st, chol_only);
  }

  int spmm(const double* X, int ldx, double* Y, int ldy, int ncol) {
    // the SpMM kernel wants contiguous n x ncol blocks: stage through Tp / THp when strided
    const double* src = X;
    double* dst = Y;
    if (ldx != ncol) {
      (k_copy_cols<<<nblk(n * ncol), BS, 0, st>>>(n, ncol, X, ldx, nullptr, Tp.p, ncol), LOB_LAUNCHED());
      src = Tp.p;
    }
    if (ldy != ncol) dst = THp.p;
    {
      Timer t(st, ph(PH_SPMM));  // the SpMM launch itself (zeroing of Y and the kernel)
      Timer tm(st, (timing && stats) ? &stats->spmm_ms_mode[spmm_mode] : nullptr);
      LOB_TRY(lob_spmm_launch(M, spmm_mode, src, dst, ncol, n_act, st));
    }
    if (ldy != ncol) (k_copy_cols<<<nblk(n * ncol), BS, 0, st>>>(n, ncol, THp.p, ncol, nullptr, Y, ldy), LOB_LAUNCHED());
    if (stats) {
      stats->spmm_calls++;
      const double vb = spmm_mode == LOB_SPMM_MIXED ? 4.0 : 8.0;  // FP32 or FP64 (split pair) values
      const double bytes = (double)M->T.nnz * (vb + 4.0) + (double)M->T.ntiles * 12.0 + (double)n * ncol * 16.0;
      stats->spmm_bytes += bytes;
      stats->spmm_bytes_mode[spmm_mode] += bytes;
      stats->spmm_calls_mode[spmm_mode]++;
    }
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  // Rayleigh-Ritz on the first m columns of S / HS. Returns info (0 ok).
  int rayleigh_ritz(int m, int* info) {
    {
      Timer t(st, ph(PH_GRAM));
      LOB_TRY(lob_gram_launch_ws(n_act, m, S.p, ldS, m, HS.p, ldS, G.p, blas_mode, work.p, st));
      LOB_TRY(lob_gram_launch_ws(n_act, m, S.p, ldS, m, S.p, ldS, Mm.p, blas_mode, work.p, st));
    }
    Timer t(st, ph(PH_RR));
    LOB_TRY(rr(m, G.p, Mm.p, theta.p, Cc.p));
    int hinfo = 0;
    LOB_CUDA(cudaMemcpyAsync(&hinfo, info_d.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaStreamSynchronize(st));
    *info = hinfo;
    return LOB_OK;
  }

  // Cholesky-QR of ncol columns at S[:, col0] (and the same transform on HS if withH):
  // B <- B L^{-T} with B^T B = L L^T. Uses the RR kernel with G = M (then C = L^{-T}).
  int cholqr(int col0, int ncol, bool withH, int* info) {
    Timer t(st, ph(PH_ORTH));
    const double* B = S.p + col0;
    LOB_TRY(lob_gram_launch_ws(n_act, ncol, B, ldS, ncol, B, ldS, Mm.p, blas_mode, work.p, st));
    LOB_TRY(rr(ncol, Mm.p, Mm.p, thw.p, Cc.p, 1));
    int hinfo = 0;
    LOB_CUDA(cudaMemcpyAsync(&hinfo, info_d.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaStreamSynchronize(st));
    *info = hinfo;
    if (hinfo) return LOB_OK;
    LOB_TRY(lob_lincomb_launch(n_act, ncol, B, ldS, ncol, Cc.p, Tn.p, ncol, blas_mode, st));
    (k_copy_cols<<<nblk(n_act * ncol), BS, 0, st>>>(n_act, ncol, Tn.p, ncol, nullptr, S.p + col0, ldS), LOB_LAUNCHED());
    if (withH) {
      LOB_TRY(lob_lincomb_launch(n_act, ncol, HS.p + col0, ldS, ncol, Cc.p, Tn.p, ncol, blas_mode, st));
      (k_copy_cols<<<nblk(n_act * ncol), BS, 0, st>>>(n_act, ncol, Tn.p, ncol, nullptr, HS.p + col0, ldS), LOB_LAUNCHED());
    }
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  int residual() {
    Timer t(st, ph(PH_RESID));
    const size_t smem = (BS / 32) * 2 * nb * sizeof(double);
    (k_residual<<<nblk(n_act), BS, smem, st>>>(n_act, nb, S.p, ldS, HS.p, ldS, theta.p, R.p, part.p), LOB_LAUNCHED());
    (k_relres<<<1, 64, 0, st>>>((int)nblk(n_act), nb, part.p, normH, relres_d.p), LOB_LAUNCHED());
    LOB_CUDA(cudaMemcpyAsync(relres_h.data(), relres_d.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaStreamSynchronize(st));
    if (g_clock) g_clock->resolve();
    return LOB_OK;
  }

  // X <- S C[:, :nb], HX <- HS C[:, :nb]; P <- S[:, nb:m] C[nb:m, :nb], HP likewise.
  int update(int m) {
    Timer t(st, ph(PH_UPDATE));
    // first nb columns of the m x m (leading dimension m) Ritz coefficients -> compact m x nb
    (k_copy_cols<<<nblk((int64_t)m * nb), BS, 0, st>>>(m, nb, Cc.p, m, nullptr, Cx.p, nb), LOB_LAUNCHED());
    LOB_TRY(lob_lincomb_launch(n_act, m, S.p, ldS, nb, Cx.p, Tn.p, nb, blas_mode, st));
    LOB_TRY(lob_lincomb_launch(n_act, m, HS.p, ldS, nb, Cx.p, THn.p, nb, blas_mode, st));
    if (m > nb) {
      // C rows nb..m-1 (a row-major m x m matrix: rows start at Cc + nb*m, leading dimension m)
      // -> compact (m-nb) x nb coefficient block in C2
      (k_copy_cols<<<nblk((int64_t)(m - nb) * nb), BS, 0, st>>>(m - nb, nb, Cc.p + (size_t)nb * m, m, nullptr, C2.p, nb), LOB_LAUNCHED());
      LOB_TRY(lob_lincomb_launch(n_act, m - nb, S.p + nb, ldS, nb, C2.p, P.p, nb, blas_mode, st));
      LOB_TRY(lob_lincomb_launch(n_act, m - nb, HS.p + nb, ldS, nb, C2.p, HP.p, nb, blas_mode, st));
    }
    (k_copy_cols<<<nblk(n_act * nb), BS, 0, st>>>(n_act, nb, Tn.p, nb, nullptr, S.p, ldS), LOB_LAUNCHED());
    (k_copy_cols<<<nblk(n_act * nb), BS, 0, st>>>(n_act, nb, THn.p, nb, nullptr, HS.p, ldS), LOB_LAUNCHED());
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  // One full solve from X currently in S[:, :nb] (rows < n_act). Returns LOB_OK,
  // LOB_ERR_NOCONV or an error.
  int run(double tol, int max_iter, bool use_precond, int shift_mode, int* iters_out, int* restarts_out) {
    int info = 0;
    // step 1: Rayleigh-Ritz on X alone (also orthonormalises it)
    LOB_TRY(spmm(S.p, ldS, HS.p, ldS, nb));
    LOB_TRY(rayleigh_ritz(nb, &info));
    if (info) {  // X0 rank-deficient: orthonormalise a randomised copy
      (k_random<<<nblk(n * nb), BS, 0, st>>>(n, n_act, nb, ldS, 0, nb, 0x5EEDull, S.p), LOB_LAUNCHED());
      LOB_TRY(spmm(S.p, ldS, HS.p, ldS, nb));
      LOB_TRY(rayleigh_ritz(nb, &info));
      if (info) return LOB_ERR_BREAKDOWN;
    }
    LOB_TRY(update(nb));
    bool haveP = false;
    int restarts = 0, it = 0;
    std::vector<int> act;
    int status = LOB_ERR_NOCONV;
    for (it = 1; it <= max_iter; it++) {
      LOB_TRY(residual());
      act.clear();
      bool conv = true;
      for (int j = 0; j < nb; j++) {
        if (j < k && !(relres_h[j] <= tol)) conv = false;
        if (!(relres_h[j] <= tol)) act.push_back(j);
      }
      if (conv) { status = LOB_OK; break; }
      const int na = (int)act.size();
      // W = T^{-1} R (step 6) with the rules of Section 4.3
      {
        Timer t(st, ph(PH_PRECOND));
        const bool pc = use_precond && M->P.bp > 0 && it > 3 && relres_h[0] <= 1e-1;
        if (pc) {
          (k_shifts<<<1, 32, 0, st>>>(nb, shift_mode, theta.p, relres_d.p, normH, mu.p), LOB_LAUNCHED());
          LOB_TRY(lob_precond_launch(M, mu.p, R.p, W.p, nb, n_act, st));
        }
        LOB_CUDA(cudaMemcpyAsync(map_d, act.data(), na * sizeof(int), cudaMemcpyHostToDevice, st));
        (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, pc ? W.p : R.p, nb, map_d, S.p + nb, ldS), LOB_LAUNCHED());
      }
      // W <- W - X (X^T W), then Cholesky-QR (step 7)
      {
        Timer t(st, ph(PH_ORTH));
        LOB_TRY(lob_gram_launch_ws(n_act, nb, S.p, ldS, na, S.p + nb, ldS, Z.p, blas_mode, work.p, st));
        (k_proj_coef<<<nblk((nb + na) * na), BS, 0, st>>>(nb, na, Z.p, C2.p), LOB_LAUNCHED());
        LOB_TRY(lob_lincomb_launch(n_act, nb + na, S.p, ldS, na, C2.p, Tn.p, na, blas_mode, st));
        (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, Tn.p, na, nullptr, S.p + nb, ldS), LOB_LAUNCHED());
      }
      LOB_TRY(cholqr(nb, na, false, &info));
      if (info) {
        // W lost rank: replace it by seeded random directions projected as above
        (k_random<<<nblk(n * na), BS, 0, st>>>(n, n_act, nb, ldS, nb, na, 0xB10Cull + it, S.p), LOB_LAUNCHED());
        LOB_TRY(cholqr(nb, na, false, &info));
        if (info) { status = LOB_ERR_BREAKDOWN; break; }
      }
      LOB_TRY(spmm(S.p + nb, ldS, HS.p + nb, ldS, na));
      int m = nb + na;
      if (haveP) {
        (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, P.p, nb, map_d, S.p + m, ldS), LOB_LAUNCHED());
        (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, HP.p, nb, map_d, HS.p + m, ldS), LOB_LAUNCHED());
        LOB_TRY(cholqr(m, na, true, &info));
        if (!info) m += na;
        else restarts++;
      }
      LOB_TRY(rayleigh_ritz(m, &info));
      if (info && m > nb + na) {  // drop P and retry (restart)
        restarts++;
        m = nb + na;
        LOB_TRY(rayleigh_ritz(m, &info));
      }
      if (info) { status = LOB_ERR_BREAKDOWN; break; }
      LOB_TRY(update(m));
      haveP = true;
    }
    if (it > max_iter) it = max_iter;
    *iters_out = it;
    *restarts_out = restarts;
    return status;
  }
};

}  // namespace

static int initial_guess(lob_matrix* m, int nb, const lob_solve_opts* o, double* Xout, cudaStream_t st) {
  // eq. 12: eigenvectors of the leading n_small x n_small block (the smaller configuration
  // space), zero-padded. The small problem is solved by this same LOBPCG from seeded random
  // vectors (the paper's multi-level use, Section 3.3.1), or directly when it is tiny.
  const int64_t n = m->T.n, ns = o->n_small;
  lob_solve_opts so = *o;
  so.n_small = 0;
  so.precond = o->precond;
  so.max_iter = 2000;
  so.refine_iter = 0;
  so.mixed_tol = 0.0;
  so.verbose = 0;
  std::vector<double> lam(nb);
  if (ns <= 3 * nb) {
    // dense: G = H11 (by SpMM of identity columns), M = I, Rayleigh-Ritz gives all eigenpairs
    const int nsi = (int)ns;
    DBuf E, HE, Gd, Md, th, Cd, wk, inf;
    LOB_TRY(E.alloc((size_t)n * nsi)); LOB_TRY(HE.alloc((size_t)n * nsi));
    LOB_TRY(Gd.alloc((size_t)nsi * nsi)); LOB_TRY(Md.alloc((size_t)nsi * nsi)); LOB_TRY(th.alloc(nsi));
    LOB_TRY(Cd.alloc((size_t)nsi * nsi)); LOB_TRY(wk.alloc(lob_rr_work_doubles(nsi))); LOB_TRY(inf.alloc(1));
    std::vector<double> eye((size_t)nsi * nsi, 0.0);
    for (int i = 0; i < nsi; i++) eye[(size_t)i * nsi + i] = 1.0;
    LOB_CUDA(cudaMemsetAsync(E.p, 0, (size_t)n * nsi * 8, st));
    LOB_CUDA(cudaMemcpyAsync(E.p, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, st));
    LOB_CUDA(cudaMemcpyAsync(Md.p, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice, st));
    for (int c0 = 0; c0 < nsi; c0 += 64) {
      const int w = nsi - c0 < 64 ? nsi - c0 : 64;
      DBuf Ec, HEc;
      LOB_TRY(Ec.alloc((size_t)n * w)); LOB_TRY(HEc.alloc((size_t)n * w));
      (k_copy_cols<<<nblk(n * w), BS, 0, st>>>(n, w, E.p + c0, nsi, nullptr, Ec.p, w), LOB_LAUNCHED());
      LOB_TRY(lob_spmm_launch(m, LOB_SPMM_FP64, Ec.p, HEc.p, w, ns, st));
      (k_copy_cols<<<nblk(ns * w), BS, 0, st>>>(ns, w, HEc.p, w, nullptr, Gd.p + c0, nsi), LOB_LAUNCHED());
      LOB_CUDA(cudaStreamSynchronize(st));
    }
    LOB_TRY(lob_rr_launch(nsi, Gd.p, Md.p, th.p, Cd.p, (int32_t*)inf.p, wk.p, st));
    // X = [C[:, :min(nb, ns)] ; 0], remaining columns seeded random (in the first ns rows)
    (k_random<<<nblk(n * nb), BS, 0, st>>>(n, ns, nb, nb, 0, nb, o->seed ^ 0x1A5Eull, Xout), LOB_LAUNCHED());
    const int nc = nsi < nb ? nsi : nb;
    (k_copy_cols<<<nblk(ns * nc), BS, 0, st>>>(ns, nc, Cd.p, nsi, nullptr, Xout, nb), LOB_LAUNCHED());
    LOB_CUDA(cudaStreamSynchronize(st));
    return LOB_OK;
  }
  LOB_CUDA(cudaMemsetAsync(Xout, 0, (size_t)n * nb * 8, st));
  // The guess only needs the accuracy of eq. 12 itself (its residual is set by the coupling
  // ||H_21||), so the smaller problem is solved to a moderate tolerance.
  int rc = lob_solve_impl(m, nb, nb, 1e-4, nullptr, &so, lam.data(), Xout, nullptr, ns);
  if (rc != LOB_OK && rc != LOB_ERR_NOCONV) return rc;
  return LOB_OK;
}

int lob_solve_impl(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0,
                              const lob_solve_opts* o, double* lambda, double* X, lob_stats* st, int64_t n_act) {
  lob_solve_opts dflt;
  memset(&dflt, 0, sizeof(dflt));
  if (!o) o = &dflt;
  if (!m || !lambda || !X || k < 1 || nb < k || nb > 32 || !(tol > 0.0)) return LOB_ERR_ARG;
  if (n_act < 3 * nb) return LOB_ERR_ARG;
  if (o->mode != LOB_MODE_FP64 && o->mode != LOB_MODE_MIXED) return LOB_ERR_ARG;
  if (o->mode == LOB_MODE_MIXED && (!m->T.v32 || !m->T.v64)) return LOB_ERR_ARG;
  if (o->mode == LOB_MODE_FP64 && !m->T.v64) return LOB_ERR_ARG;
  if (o->precond && m->P.bp < 1) return LOB_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)o->stream;
  const auto t0 = std::chrono::steady_clock::now();
  if (st) memset(st, 0, sizeof(*st));

  Solver S;
  S.M = m; S.n = m->T.n; S.n_act = n_act; S.nb = nb; S.k = k; S.st = stream;
  S.normH = o->norm_H > 0.0 ? o->norm_H : m->norm_inf;
  S.stats = st; S.timing = st != nullptr;
  // block products: native FP64 in the plain solver, FP64-class double-float in MIXED
  S.blas_mode = o->mode == LOB_MODE_MIXED ? LOB_SPMM_MIXED : LOB_SPMM_FP64;
  LOB_TRY(S.alloc());
  PhaseClock clock;
  PhaseClock* prev_clock = g_clock;
  if (st) g_clock = &clock;
  struct ClockReset { PhaseClock* p; ~ClockReset() { g_clock = p; } } clock_reset{prev_clock};

  // X0 into S[:, :nb]
  {
    Timer t(stream, st ? &st->phase_ms[PH_GUESS] : nullptr);
    if (X0) {
      (k_copy_cols<<<nblk(S.n * nb), BS, 0, stream>>>(S.n, nb, X0, nb, nullptr, S.S.p, S.ldS), LOB_LAUNCHED());
    } else if (o->n_small > 0 && o->n_small < n_act) {
      LOB_TRY(initial_guess(m, nb, o, S.W.p, stream));
      (k_copy_cols<<<nblk(S.n * nb), BS, 0, stream>>>(S.n, nb, S.W.p, nb, nullptr, S.S.p, S.ldS), LOB_LAUNCHED());
    } else {
      (k_random<<<nblk(S.n * nb), BS, 0, stream>>>(S.n, n_act, nb, S.ldS, 0, nb, o->seed, S.S.p), LOB_LAUNCHED());
    }
    LOB_CUDA(cudaGetLastError());
  }
  const int max_iter = o->max_iter > 0 ? o->max_iter : 500;
  int iters = 0, restarts = 0, status;
  if (o->mode == LOB_MODE_MIXED) {
    // phase 1: FP32-value SpMM down to the FP32 floor; phase 2: FP64 refinement from there
    const double tol1 = o->mixed_tol > 0.0 ? o->mixed_tol : (tol > 1e-6 ? tol : 1e-6);
    S.spmm_mode = LOB_SPMM_MIXED;
    status = S.run(tol1, max_iter, o->precond != 0, o->precond_shift, &iters, &restarts);
    if (status != LOB_OK && status != LOB_ERR_NOCONV) return status;
    int it2 = 0, rs2 = 0;
    S.spmm_mode = m->T.v32lo ? LOB_SPMM_DF64 : LOB_SPMM_FP64;  // FP64-class refinement products
    const int max2 = o->refine_iter > 0 ? o->refine_iter : 50;
    status = S.run(tol, max2, o->precond != 0, o->precond_shift, &it2, &rs2);
    if (st) st->refine_iterations = it2;
    iters += it2;
    restarts += rs2;
  } else {
    S.spmm_mode = LOB_SPMM_FP64;
    status = S.run(tol, max_iter, o->precond != 0, o->precond_shift, &iters, &restarts);
  }
  if (status != LOB_OK && status != LOB_ERR_NOCONV) return status;
  // outputs: X = S[:, :nb], lambda = theta[:k], final residuals
  LOB_TRY(S.residual());
  (k_copy_cols<<<nblk(S.n * nb), BS, 0, stream>>>(S.n, nb, S.S.p, S.ldS, nullptr, X, nb), LOB_LAUNCHED());
  if (n_act < S.n) LOB_CUDA(cudaMemsetAsync(X + n_act * nb, 0, (size_t)(S.n - n_act) * nb * 8, stream));
  LOB_CUDA(cudaMemcpyAsync(lambda, S.theta.p, k * sizeof(double), cudaMemcpyDeviceToHost, stream));
  LOB_CUDA(cudaStreamSynchronize(stream));
  if (st) clock.resolve();
  if (st) {
    st->iterations = iters;
    st->restarts = restarts;
    for (int j = 0; j < nb && j < 64; j++) st->residual[j] = S.relres_h[j];
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}
