// Lockstep engine: many LOBPCG solves (Algorithm 1, Section 3.1) advanced together, one iteration
// per round, every kernel of the iteration launched once for all solves through job tables.
//
// A round for the set of active solves:
//   A  decide (host, from the residual norms read back in the previous round); block-diagonal
//      preconditioner (eq. 11, Section 4.3) for the solves that use it this round; gather W;
//      W <- W - X (X^T W); Gram matrices of W and P for Cholesky-QR; Cholesky factors.
//   B  Cholesky-QR updates of W and P; SpMM on W (or on X for a solve that (re)starts: the
//      Rayleigh-Ritz step on X alone of Algorithm 1, step 1); G = S^T H S and M = S^T S; the
//      projected eigenproblem (eq. 9). A and B are enqueued together; the factorisation and
//      Rayleigh-Ritz statuses come back in one readback.                                  [sync]
//   C  update X, H X, P, H P (eq. 7); residuals and their norms (steps 4-5).              [sync]
// The host cost of a round is a fixed number of launches and two host synchronisations whatever
// the number of solves (a third only when some factorisation failed); the per-
// solve control (convergence, active columns, the rules of Section 4.3, the mixed-precision
// phases, the stagnation safeguard) is the same as the single-solve task's. A solve whose
// Cholesky-QR of W breaks down restarts from its current X in the next round; a solve whose
// Cholesky-QR of P or Rayleigh-Ritz with P fails repeats Rayleigh-Ritz without P in the same
// round.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "common.cuh"
#include "df.cuh"

namespace {

constexpr int BS = 256;
constexpr int NBMAX = 16;
inline unsigned nblk(int64_t n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

__device__ __forceinline__ int find_job(const lob_bjob* __restrict__ jobs, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].cta_begin <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Y[r * ldy + i] = A[r * lda + (map ? map[i] : i)], r < n, i < p; ceil(n p / 256) CTAs.
__global__ void k_copy_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  const int64_t t = ((int64_t)blockIdx.x - j.cta_begin) * BS + threadIdx.x;
  if (t >= j.n * j.p) return;
  const int64_t r = t / j.p;
  const int i = (int)(t % j.p);
  const int* map = reinterpret_cast<const int*>(j.P0);
  j.Y[r * j.ldy + i] = j.A[r * j.lda + (map ? map[i] : i)];
}

// C2 = [-Z; I] for W - X Z as [X W] C2: Z = A (x0 x x1), Y = C2; one CTA per job.
__global__ void k_proj_batch(const lob_bjob* __restrict__ jobs) {
  const lob_bjob& j = jobs[blockIdx.x];
  const int nb = j.x0, na = j.x1;
  for (int t = threadIdx.x; t < (nb + na) * na; t += blockDim.x) {
    const int r = t / na, c = t % na;
    j.Y[t] = r < nb ? -j.A[r * na + c] : (r - nb == c ? 1.0 : 0.0);
  }
}

// R = HX - X diag(theta) and per-CTA column sums of r^2 and x^2: X = A (lda), HX = B (ldb),
// theta = C, R = Y (x0 columns), partials W0; ceil(n / 256) CTAs.
// job fields: A = X (lda), B = H X (ldb), C = theta, Y = R, W0 = partials, n, x0 = nb, s0 = 1 / normH
__global__ void __launch_bounds__(BS) k_resid_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  __shared__ float sred[8 * 64];
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  lob_residual_rows(j.n, j.x0, j.A, j.lda, j.B, j.ldb, j.C, j.s0, j.Y, j.W0, (int64_t)blockIdx.x - j.cta_begin, sred);
}

// Column norms from the residual partials (already scaled by 1 / normH, so s0 = 1 here)
__global__ void __launch_bounds__(BS) k_relres_batch(const lob_bjob* __restrict__ jobs) {
  __shared__ double sr[BS], sx[BS];
  const lob_bjob& j = jobs[blockIdx.x];
  const int tid = threadIdx.x, nb = j.x0;
  for (int c = 0; c < nb; c++) {
    double rr = 0.0, xx = 0.0;
    for (int b = tid; b < j.x1; b += BS) { rr += j.W0[(int64_t)b * 2 * nb + c]; xx += j.W0[(int64_t)b * 2 * nb + nb + c]; }
    sr[tid] = rr;
    sx[tid] = xx;
    __syncthreads();
    for (int o = BS / 2; o > 0; o >>= 1) {
      if (tid < o) { sr[tid] += sr[tid + o]; sx[tid] += sx[tid + o]; }
      __syncthreads();
    }
    if (tid == 0) j.Y[c] = sqrt(sr[0]) / (j.s0 * sqrt(sx[0] > 0.0 ? sx[0] : 1.0));
    __syncthreads();
  }
}

// Preconditioner shifts (Section 4.3): theta = C, relres = D, mu = Y, x0 (nb), x1 (rule), s0 (normH).
__global__ void k_shifts_batch(const lob_bjob* __restrict__ jobs) {
  const lob_bjob& j = jobs[blockIdx.x];
  if (threadIdx.x != 0) return;
  const int nb = j.x0;
  for (int c = 0; c < nb; c++) j.Y[c] = j.C[c];
  if (j.x1 != 1) return;
  for (int c = 0; c < nb; c++) {
    if (j.D[c] < 1e-2) {
      j.Y[c] = j.C[c] - 2.0 * j.D[c] * j.s0;
    } else if (c > 0) {
      for (int t = c; t < nb; t++) j.Y[t] = j.Y[c - 1];
      break;
    }
  }
}

// Seeded uniform(-1, 1) entries in rows < x2 (zero below), columns x0 .. x0 + x1 of Y (ldy),
// rows < n; seed from x3; ceil(n x1 / 256) CTAs.
__global__ void k_random_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  const int64_t t = ((int64_t)blockIdx.x - j.cta_begin) * BS + threadIdx.x;
  if (t >= j.n * j.x1) return;
  const int64_t i = t / j.x1;
  const int c = j.x0 + (int)(t % j.x1);
  double v = 0.0;
  if (i < j.x2) {
    uint64_t z = (uint64_t)(uint32_t)j.x3 * 0xD1B54A32D192ED03ull + (uint64_t)i * 0x9E3779B97F4A7C15ull +
                 (uint64_t)c * 0xC2B2AE3D27D4EB4Full + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  j.Y[i * j.ldy + c] = v;
}

}  // namespace

// ------------------------------------------------------------------------------------------------

struct lob_ltask {
  // problem
  lob_matrix* M = nullptr;
  int64_t n = 0, n_act = 0;
  int nb = 0, k = 0, ldS = 0;
  double tol = 0.0, normH = 0.0;
  lob_solve_opts o{};
  double* Xout = nullptr;
  int slot = 0;  // index into the engine's readback arrays
  // device state (one allocation)
  void* mem = nullptr;
  double *S, *HS, *P, *HP, *R, *W, *Tp, *THp, *G, *Mm, *Cc, *Cx, *C2, *Z, *MmP, *CcP, *theta, *thw, *thP, *mu,
      *part, *gw, *rrw;
  int* map;
  int nparts = 0;
  size_t gw_half = 0;  // doubles in each half of the Gram partial buffer
  // control
  int blas = LOB_SPMM_FP64;
  int rrb = LOB_SPMM_FP64;  // arithmetic of the small dense solves (Cholesky-QR factors, Rayleigh-Ritz)
  int phase = 0;        // MIXED: 0 = FP32-value products, 1 = FP64-class refinement
  bool start = true;    // the next round computes H X and the Rayleigh-Ritz step on X alone
  bool active = false;  // iterating (has residual norms)
  int it = 0, iters_total = 0, restarts = 0, refine_its = 0, na = 0, m = 0;
  bool haveP = false, pok = false, pc_on = false, wfail = false, rrfail = false;
  double run_tol = 0.0;
  int run_max = 0, max_iter = 0;
  double best_res = 1e300;
  int best_it = 0;
  bool pc_dropped = false;
  int precond_dropped = 0;
  int status = LOB_OK;
  bool finished = false;
  int hmap[NBMAX];
  // the eq. 12 guess: a child solve on the leading block; the parent waits for it
  lob_ltask* child = nullptr;
  lob_ltask* parent = nullptr;
  bool waiting = false;
  int64_t user = 0;  // caller's tag
  std::chrono::steady_clock::time_point t0;
};

namespace {

size_t task_doubles(int64_t n, int nb, int* nch) {
  const int mm = 3 * nb;
  *nch = lob_gram_chunks(n, 16, 16);  // the most chunks any Gram of this solve uses (one 16 x 16 tile)
  size_t d = 2 * (size_t)n * mm + 6 * (size_t)n * nb;
  d += 8 * (size_t)mm * mm + 5 * (size_t)mm + 64;
  d += (size_t)nblk(n) * 2 * nb + 2 * (size_t)(*nch) * mm * mm + lob_rr_work_doubles(mm);
  return d;
}

}  // namespace

struct lob_engine {
  cudaStream_t st = nullptr;
  int cap = 0;  // readback slots
  std::vector<int> free_slots;
  // readback arrays: relres [cap][NBMAX], theta [cap][3 NBMAX], info [cap][4]
  double *d_relres = nullptr, *h_relres = nullptr, *d_theta = nullptr, *h_theta = nullptr;
  int32_t *d_info = nullptr, *h_info = nullptr;
  // job tables (pinned host, device), bump-allocated per round
  lob_bjob *jh = nullptr, *jd = nullptr;
  size_t jcap = 0, joff = 0;
  lob_spmm_job *sh = nullptr, *sd = nullptr;
  int scap = 0;
  std::vector<lob_ltask*> tasks;  // admitted (active, waiting, or starting)
  long long rounds = 0, spmm_launches = 0, spmm_products = 0;
  double host_ms = 0.0, wait_ms = 0.0;  // time in rounds outside / inside stream synchronisation

  lob_bjob* take(size_t k, lob_bjob** dev) {
    if (joff + k > jcap) return nullptr;
    lob_bjob* h = jh + joff;
    *dev = jd + joff;
    joff += k;
    memset(h, 0, k * sizeof(lob_bjob));
    return h;
  }
};

namespace {

// launch helpers over a host job vector (fills cta_begin by the given count per job)
template <class F>
int launch_rows(lob_engine* E, std::vector<lob_bjob>& v, F ctas_of,
                void (*kern)(const lob_bjob*, int), size_t smem = 0) {
  if (v.empty()) return LOB_OK;
  lob_bjob* dev = nullptr;
  lob_bjob* h = E->take(v.size(), &dev);
  if (!h) return LOB_ERR_NOMEM;
  int64_t c = 0;
  for (size_t i = 0; i < v.size(); i++) {
    v[i].cta_begin = c;
    c += ctas_of(v[i]);
    h[i] = v[i];
  }
  if (c == 0) return LOB_OK;
  LOB_CUDA(cudaMemcpyAsync(dev, h, v.size() * sizeof(lob_bjob), cudaMemcpyHostToDevice, E->st));
  (kern<<<(unsigned)c, BS, smem, E->st>>>(dev, (int)v.size()), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

int launch_per_job(lob_engine* E, std::vector<lob_bjob>& v, void (*kern)(const lob_bjob*)) {
  if (v.empty()) return LOB_OK;
  lob_bjob* dev = nullptr;
  lob_bjob* h = E->take(v.size(), &dev);
  if (!h) return LOB_ERR_NOMEM;
  for (size_t i = 0; i < v.size(); i++) { v[i].cta_begin = (int64_t)i; h[i] = v[i]; }
  LOB_CUDA(cudaMemcpyAsync(dev, h, v.size() * sizeof(lob_bjob), cudaMemcpyHostToDevice, E->st));
  (kern<<<(unsigned)v.size(), BS, 0, E->st>>>(dev), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

int copy_batch(lob_engine* E, std::vector<lob_bjob>& v) {
  return launch_rows(E, v, [](const lob_bjob& j) { return (j.n * j.p + BS - 1) / BS; }, k_copy_batch);
}

lob_bjob cp_job(int64_t n, int ncol, const double* src, int lds, const int* map, double* dst, int ldd) {
  lob_bjob j{};
  j.n = n; j.p = ncol; j.A = src; j.lda = lds; j.P0 = map; j.Y = dst; j.ldy = ldd;
  return j;
}

lob_bjob gram_job(const lob_ltask* t, const double* A, int p, const double* B, int q, double* out, double* partials,
                  int sym) {
  lob_bjob j{};
  j.x2 = t->blas;
  j.A = A; j.lda = t->ldS; j.p = p; j.B = B; j.ldb = t->ldS; j.q = q; j.n = t->n_act; j.W0 = partials;
  // in a batch the solves fill the GPU together: about 1,024 rows per chunk (at most the
  // single-solve chunk count, which sizes the partial buffers)
  j.x0 = (int)std::max<int64_t>(1, std::min<int64_t>(lob_gram_chunks(t->n_act, p, q), (t->n_act + 1023) / 1024));
  j.x1 = sym; j.Y = out;
  return j;
}

// The block products of a batch run in each solve's own arithmetic (x2: LOB_SPMM_FP64 or
// LOB_SPMM_MIXED, i.e. double-float): one launch per arithmetic present.
// Gram jobs also split by size: products with at most 1,024 2 x 2 output blocks (counting only the
// upper triangle when symmetric) use the block kernel (class 0); larger ones a tile of edge 16,
// 32 or 48.
inline int tile_class(const lob_bjob& j) {
  const int bp = (j.p + 1) / 2, bq = (j.q + 1) / 2;
  if ((j.x1 ? bp * (bp + 1) / 2 : bp * bq) <= 1024) return 0;
  const int e = std::max(j.p, j.q);
  return e <= 16 ? 1 : (e <= 32 ? 2 : 3);
}

// Classes: (arithmetic, tile class, fused); fused jobs (x3 == 2: G and M of one solve in one pass)
// are all of tile class 0.
int gram_batch(lob_engine* E, std::vector<lob_bjob>& v, int) {
  for (int blas : {LOB_SPMM_FP64, LOB_SPMM_MIXED})
    for (int u = 0; u <= 3; u++)
      for (int fused = 0; fused <= (u == 0 ? 1 : 0); fused++) {
        auto in_class = [&](const lob_bjob& j) { return j.x2 == blas && tile_class(j) == u && (j.x3 == 2) == (fused == 1); };
        size_t cnt = 0;
        for (const lob_bjob& j : v) cnt += in_class(j);
        if (!cnt) continue;
        lob_bjob *d1 = nullptr, *d2 = nullptr;
        lob_bjob* h1 = E->take(cnt, &d1);
        lob_bjob* h2 = E->take(fused ? 2 * cnt : cnt, &d2);
        if (!h1 || !h2) return LOB_ERR_NOMEM;
        int i = 0;
        for (const lob_bjob& j : v)
          if (in_class(j)) h1[i++] = j;
        LOB_TRY(lob_gram_batch_launch(h1, d1, (int)cnt, u == 0 ? 48 : 16 * u, blas, h2, d2, E->st, u == 0, fused));
      }
  return LOB_OK;
}

// G = S^T H S into G and M = S^T S into M: one fused job when the solve's 2 x 2 blocks fit one
// row-group pass (m <= 30), else two jobs
void push_gm(std::vector<lob_bjob>& v, const lob_ltask* t) {
  const int bp = (t->m + 1) / 2;
  if (bp * (bp + 1) / 2 <= 128) {
    lob_bjob j = gram_job(t, t->S, t->m, t->HS, t->m, t->G, t->gw, 1);
    j.W1 = t->gw + t->gw_half;
    j.D = t->Mm;
    j.x3 = 2;
    v.push_back(j);
  } else {
    v.push_back(gram_job(t, t->S, t->m, t->HS, t->m, t->G, t->gw, 1));
    v.push_back(gram_job(t, t->S, t->m, t->S, t->m, t->Mm, t->gw + t->gw_half, 1));
  }
}

inline int width_class(const lob_bjob& j) { return j.q <= 1 ? 1 : (j.q <= 2 ? 2 : (j.q <= 4 ? 4 : (j.q <= 8 ? 8 : 16))); }

int lincomb_batch(lob_engine* E, std::vector<lob_bjob>& v, int) {
  for (int blas : {LOB_SPMM_FP64, LOB_SPMM_MIXED})
    for (int w : {1, 2, 4, 8, 16}) {
      size_t cnt = 0;
      for (const lob_bjob& j : v) cnt += j.x2 == blas && width_class(j) == w;
      if (!cnt) continue;
      lob_bjob* d = nullptr;
      lob_bjob* h = E->take(cnt, &d);
      if (!h) return LOB_ERR_NOMEM;
      int pmax = 1, i = 0;
      for (const lob_bjob& j : v)
        if (j.x2 == blas && width_class(j) == w) { h[i++] = j; pmax = std::max(pmax, j.p); }
      LOB_TRY(lob_lincomb_batch_launch(h, d, (int)cnt, pmax, w, blas, E->st));
    }
  return LOB_OK;
}

lob_bjob lc_job(const lob_ltask* t, int64_t n, const double* A, int lda, int p, const double* C, int q, double* Y,
                int ldy, const double* D = nullptr, int ldd = 0) {
  lob_bjob j{};
  j.n = n; j.A = A; j.lda = lda; j.p = p; j.C = C; j.q = q; j.Y = Y; j.ldy = ldy; j.D = D; j.ldd = ldd;
  j.x2 = t->blas;
  return j;
}

int rr_batch(lob_engine* E, std::vector<lob_bjob>& v, int) {
  for (int blas : {LOB_SPMM_FP64, LOB_SPMM_MIXED}) {
    size_t cnt = 0;
    for (const lob_bjob& j : v) cnt += j.x2 == blas;
    if (!cnt) continue;
    lob_bjob* d = nullptr;
    lob_bjob* h = E->take(cnt, &d);
    if (!h) return LOB_ERR_NOMEM;
    int mmax = 1, i = 0;
    for (const lob_bjob& j : v)
      if (j.x2 == blas) { h[i++] = j; mmax = std::max(mmax, j.x0); }
    LOB_CUDA(cudaMemcpyAsync(d, h, cnt * sizeof(lob_bjob), cudaMemcpyHostToDevice, E->st));
    LOB_TRY(lob_rr_batch_launch(d, (int)cnt, mmax, blas == LOB_SPMM_MIXED, E->st));
  }
  return LOB_OK;
}

lob_bjob rr_job(const lob_ltask* t, int m, const double* G, const double* Mm, double* theta, double* C, int chol) {
  lob_bjob j{};
  j.x2 = t->rrb;
  j.x0 = m; j.x1 = chol; j.A = G; j.B = Mm; j.Y = theta; j.W0 = C; j.W1 = t->rrw;
  return j;
}

int sync(lob_engine* E) {
  const auto a = std::chrono::steady_clock::now();
  LOB_CUDA(cudaStreamSynchronize(E->st));
  E->wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
  return LOB_OK;
}

}  // namespace

// ---- engine API (internal) ----

int lob_engine_create(int cap, cudaStream_t st, lob_engine** out) {
  lob_engine* E = new lob_engine();
  E->st = st;
  E->cap = cap;
  for (int i = cap - 1; i >= 0; i--) E->free_slots.push_back(i);
  E->jcap = (size_t)cap * 40 + 1024;
  E->scap = cap;
  bool ok = cudaMalloc((void**)&E->d_relres, (size_t)cap * NBMAX * 8) == cudaSuccess &&
            cudaMalloc((void**)&E->d_theta, (size_t)cap * 3 * NBMAX * 8) == cudaSuccess &&
            cudaMalloc((void**)&E->d_info, (size_t)cap * 4 * 4) == cudaSuccess &&
            cudaHostAlloc((void**)&E->h_relres, (size_t)cap * NBMAX * 8, cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc((void**)&E->h_theta, (size_t)cap * 3 * NBMAX * 8, cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc((void**)&E->h_info, (size_t)cap * 4 * 4, cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc((void**)&E->jh, E->jcap * sizeof(lob_bjob), cudaHostAllocDefault) == cudaSuccess &&
            cudaMalloc((void**)&E->jd, E->jcap * sizeof(lob_bjob)) == cudaSuccess &&
            cudaHostAlloc((void**)&E->sh, (size_t)E->scap * sizeof(lob_spmm_job), cudaHostAllocDefault) == cudaSuccess &&
            cudaMalloc((void**)&E->sd, (size_t)E->scap * sizeof(lob_spmm_job)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lob_engine_destroy(E);
    return LOB_ERR_NOMEM;
  }
  *out = E;
  return LOB_OK;
}

void lob_engine_destroy(lob_engine* E) {
  if (!E) return;
  if (E->st) cudaStreamSynchronize(E->st);
  for (lob_ltask* t : E->tasks) {
    if (t->mem) cudaFreeAsync(t->mem, E->st);
    delete t;
  }
  cudaFree(E->d_relres); cudaFree(E->d_theta); cudaFree(E->d_info); cudaFree(E->jd); cudaFree(E->sd);
  cudaFreeHost(E->h_relres); cudaFreeHost(E->h_theta); cudaFreeHost(E->h_info); cudaFreeHost(E->jh);
  cudaFreeHost(E->sh);
  delete E;
}

size_t lob_engine_task_bytes(const lob_matrix* m, int nb, int64_t n_small) {
  int nch = 0;
  size_t d = task_doubles(m->T.n, nb, &nch);
  if (n_small >= 3 * nb) d *= 2;  // the guess child holds a second state of the same size
  return d * 8;
}

int lob_engine_free_slots(const lob_engine* E) { return (int)E->free_slots.size(); }

namespace {

int task_alloc(lob_engine* E, lob_ltask* t) {
  int nch = 0;
  const size_t d = task_doubles(t->n, t->nb, &nch);
  if (E->free_slots.empty()) return LOB_ERR_NOMEM;
  if (cudaMallocAsync(&t->mem, d * 8, E->st) != cudaSuccess) { cudaGetLastError(); t->mem = nullptr; return LOB_ERR_NOMEM; }
  t->slot = E->free_slots.back();
  E->free_slots.pop_back();
  double* p = reinterpret_cast<double*>(t->mem);
  const int64_t n = t->n;
  const int nb = t->nb, mm = 3 * nb;
  t->ldS = mm;
  auto take = [&](size_t c) { double* r = p; p += c; return r; };
  t->S = take((size_t)n * mm); t->HS = take((size_t)n * mm);
  t->P = take((size_t)n * nb); t->HP = take((size_t)n * nb); t->R = take((size_t)n * nb);
  t->W = take((size_t)n * nb); t->Tp = take((size_t)n * nb); t->THp = take((size_t)n * nb);
  t->G = take((size_t)mm * mm); t->Mm = take((size_t)mm * mm); t->Cc = take((size_t)mm * mm);
  t->Cx = take((size_t)mm * mm); t->C2 = take((size_t)mm * mm); t->Z = take((size_t)mm * mm);
  t->MmP = take((size_t)mm * mm); t->CcP = take((size_t)mm * mm);
  t->theta = E->d_theta + (size_t)t->slot * 3 * NBMAX;
  t->thw = take(mm); t->thP = take(mm); t->mu = take(mm);
  take(2 * mm);
  t->map = reinterpret_cast<int*>(take(32));
  t->nparts = (int)nblk(t->n_act);
  t->part = take((size_t)nblk(n) * 2 * nb);
  t->gw = take(2 * (size_t)nch * mm * mm);
  t->gw_half = (size_t)nch * mm * mm;
  t->rrw = take(lob_rr_work_doubles(mm));
  return LOB_OK;
}

void task_release(lob_engine* E, lob_ltask* t) {
  if (t->mem) cudaFreeAsync(t->mem, E->st);
  t->mem = nullptr;
  E->free_slots.push_back(t->slot);
}

int32_t* info_dev(lob_engine* E, lob_ltask* t, int i) { return E->d_info + (size_t)t->slot * 4 + i; }
int32_t info_host(lob_engine* E, lob_ltask* t, int i) { return E->h_info[(size_t)t->slot * 4 + i]; }
double* relres_dev(lob_engine* E, lob_ltask* t) { return E->d_relres + (size_t)t->slot * NBMAX; }
double relres_host(lob_engine* E, lob_ltask* t, int j) { return E->h_relres[(size_t)t->slot * NBMAX + j]; }

void set_phase(lob_ltask* t) {
  if (t->o.mode == LOB_MODE_MIXED && t->phase == 0) {
    t->run_tol = t->o.mixed_tol > 0.0 ? t->o.mixed_tol : (t->tol > LOB_MIXED_TOL ? t->tol : LOB_MIXED_TOL);
    t->run_max = t->max_iter;
  } else {
    t->run_tol = t->tol;
    t->run_max = t->o.mode == LOB_MODE_MIXED
                     ? (t->o.refine_iter > 0 ? t->o.refine_iter
                                             : (t->max_iter - t->iters_total > 50 ? t->max_iter - t->iters_total : 50))
                     : t->max_iter;
  }
  t->it = 0;
  t->best_res = 1e300;
  t->best_it = 0;
  t->pc_dropped = false;
  t->start = true;
  t->active = false;
  t->haveP = false;
}

int spmm_mode_of(const lob_ltask* t) {
  if (t->o.mode != LOB_MODE_MIXED) return LOB_SPMM_FP64;
  if (t->phase == 0) return LOB_SPMM_MIXED;
  return (t->o.refine_arith == LOB_ARITH_DF && t->M->T.v32lo) ? LOB_SPMM_DF64 : LOB_SPMM_FP64;
}

}  // namespace

// Create a solve (not yet iterating); with a guess, its child is created too. X0 random.
int lob_engine_add(lob_engine* E, lob_matrix* M, int32_t k, int32_t nb, double tol, const lob_solve_opts* o,
                   double* Xout, int64_t n_act, int64_t user, lob_ltask** out) {
  lob_ltask* t = new lob_ltask();
  t->M = M; t->n = M->T.n; t->n_act = n_act; t->nb = nb; t->k = k; t->tol = tol; t->o = *o; t->Xout = Xout;
  t->user = user;
  t->normH = o->norm_H > 0.0 ? o->norm_H : M->norm_inf;
  t->blas = o->mode == LOB_MODE_MIXED ? LOB_SPMM_MIXED : LOB_SPMM_FP64;
  t->rrb = (o->mode == LOB_MODE_MIXED && o->rr_arith == LOB_ARITH_DF) ? LOB_SPMM_MIXED : LOB_SPMM_FP64;
  t->max_iter = o->max_iter > 0 ? o->max_iter : 500;
  t->t0 = std::chrono::steady_clock::now();
  int rc = task_alloc(E, t);
  if (rc != LOB_OK) { delete t; return rc; }
  set_phase(t);
  // X0: seeded random columns in rows < n_act
  std::vector<lob_bjob> v(1);
  v[0].n = t->n; v[0].Y = t->S; v[0].ldy = t->ldS; v[0].x0 = 0; v[0].x1 = nb; v[0].x2 = (int32_t)n_act;
  v[0].x3 = (int32_t)(o->seed ? o->seed : 1);
  rc = launch_rows(E, v, [](const lob_bjob& j) { return (j.n * j.x1 + BS - 1) / BS; }, k_random_batch);
  if (rc != LOB_OK) { task_release(E, t); delete t; return rc; }
  E->tasks.push_back(t);
  if (o->n_small >= 3 * nb && o->n_small < n_act) {
    // eq. 12: the leading n_small block solved first (to LOB_GUESS_TOL), its vectors (zero-padded) become X0
    lob_solve_opts so = *o;
    so.n_small = 0;
    so.max_iter = 2000;
    so.refine_iter = 0;
    so.mixed_tol = 0.0;
    lob_ltask* c = nullptr;
    rc = lob_engine_add(E, M, nb, nb, LOB_GUESS_TOL, &so, t->W, o->n_small, -1, &c);
    if (rc == LOB_OK) {
      c->parent = t;
      t->child = c;
      t->waiting = true;
      LOB_CUDA(cudaMemsetAsync(t->W, 0, (size_t)t->n * nb * 8, E->st));
    }
  }
  *out = t;
  return LOB_OK;
}

// One round for every admitted solve. Finished solves (top-level ones) are appended to done.
static int engine_round(lob_engine* E, std::vector<lob_ltask*>& done);

int lob_engine_round(lob_engine* E, std::vector<lob_ltask*>& done) {
  const auto a = std::chrono::steady_clock::now();
  const double w0 = E->wait_ms;
  const int rc = engine_round(E, done);
  E->host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count() -
                (E->wait_ms - w0);
  return rc;
}

void lob_engine_times(const lob_engine* E, double* host_ms, double* wait_ms, long long* rounds) {
  *host_ms = E->host_ms;
  *wait_ms = E->wait_ms;
  *rounds = E->rounds;
}

static int engine_round(lob_engine* E, std::vector<lob_ltask*>& done) {
  E->joff = 0;
  E->rounds++;
  std::vector<lob_ltask*> iter, start;  // iterating this round; (re)starting with H X
  // ---- A: decisions
  std::vector<lob_bjob> j_shift, j_prec, j_gather, j_zg, j_proj, j_lcproj, j_cholg, j_pgather, j_rr1, j_xout;
  std::vector<lob_ltask*> j_tile;  // solves preconditioned on the diagonal tiles (one launch each)
  std::vector<lob_ltask*> finishing;
  for (lob_ltask* t : E->tasks) {
    if (t->finished || t->waiting) continue;
    if (t->start) { start.push_back(t); continue; }
    if (!t->active) continue;
    bool conv = true;
    t->na = 0;
    for (int j = 0; j < t->nb; j++) {
      const double r = relres_host(E, t, j);
      if (j < t->k && !(r <= t->run_tol)) conv = false;
      if (!(r <= t->run_tol)) t->hmap[t->na++] = j;
    }
    if (!conv && t->it >= t->run_max) { t->status = LOB_ERR_NOCONV; conv = true; }
    double worst = 0.0;
    for (int j = 0; j < t->k; j++) {
      const double r = relres_host(E, t, j);
      if (!(r <= t->run_tol)) worst = fmax(worst, r);
    }
    if (worst < 0.5 * t->best_res) { t->best_res = worst; t->best_it = t->it; }
    // MIXED, FP32-value phase: no halving of the worst residual in LOB_MIXED_STALL iterations -> the FP64-class
    // phase takes over from here
    if (!conv && t->o.mode == LOB_MODE_MIXED && t->phase == 0 && t->it - t->best_it >= LOB_MIXED_STALL) {
      t->status = LOB_ERR_NOCONV;
      conv = true;
    }
    if (conv) {
      t->iters_total += t->it;
      if (t->o.mode == LOB_MODE_MIXED && t->phase == 1) t->refine_its = t->it;
      // the FP64-class phase, unless the FP32-value phase already met the final tol
      if (t->o.mode == LOB_MODE_MIXED && t->phase == 0 && !(t->status == LOB_OK && t->run_tol <= t->tol)) {
        t->phase = 1;
        t->status = LOB_OK;
        set_phase(t);
        start.push_back(t);
        continue;
      }
      finishing.push_back(t);
      continue;
    }
    if (!t->pc_dropped && t->o.precond && t->it - t->best_it >= 40) {
      t->pc_dropped = true;
      if (!t->precond_dropped) t->precond_dropped = t->iters_total + t->it;
    }
    // Section 4.3: not in the first three iterations of the solve (across its phases), nor while the
    // first residual is above 1e-1
    t->pc_on = t->o.precond && !t->pc_dropped && t->M->P.bp > 0 && t->iters_total + t->it > 3 &&
               relres_host(E, t, 0) <= 1e-1;
    iter.push_back(t);
  }
  // finished solves: outputs
  for (lob_ltask* t : finishing) {
    if (t->Xout) {
      j_xout.push_back(cp_job(t->n, t->nb, t->S, t->ldS, nullptr, t->Xout, t->nb));
    }
  }
  LOB_TRY(copy_batch(E, j_xout));
  // active-column maps to the device, staged in the pinned job table
  for (lob_ltask* t : iter) {
    lob_bjob* dev = nullptr;
    lob_bjob* h = E->take(1, &dev);
    if (!h) return LOB_ERR_NOMEM;
    int* hm = reinterpret_cast<int*>(h);
    for (int i = 0; i < t->na; i++) hm[i] = t->hmap[i];
    LOB_CUDA(cudaMemcpyAsync(t->map, hm, t->na * sizeof(int), cudaMemcpyHostToDevice, E->st));
  }
  for (lob_ltask* t : iter) {
    if (t->pc_on) {
      lob_bjob s{};
      s.C = t->theta; s.D = relres_dev(E, t); s.Y = t->mu; s.x0 = t->nb; s.x1 = t->o.precond_shift; s.s0 = t->normH;
      j_shift.push_back(s);
      if (t->M->P.bp == LOB_TILE) {  // the diagonal tiles of the tile store: one launch for this solve
        j_tile.push_back(t);
      } else {
        lob_bjob a{};
        a.P0 = t->M->P.Q; a.P1 = t->M->P.lam; a.C = t->mu; a.A = t->R; a.Y = t->W; a.x0 = t->nb; a.x1 = t->M->P.bp;
        a.n = t->n_act; a.s0 = 1e-8 * t->M->norm_inf; a.x2 = t->o.precond_solve;
        a.x3 = t->o.precond_steps > 0 ? t->o.precond_steps : 3;
        j_prec.push_back(a);
      }
    }
    j_gather.push_back(cp_job(t->n_act, t->na, t->pc_on ? t->W : t->R, t->nb, t->map, t->S + t->nb, t->ldS));
    j_zg.push_back(gram_job(t, t->S, t->nb, t->S + t->nb, t->na, t->Z, t->gw, 0));
    lob_bjob pj{};
    pj.A = t->Z; pj.x0 = t->nb; pj.x1 = t->na; pj.Y = t->C2;
    j_proj.push_back(pj);
    j_lcproj.push_back(lc_job(t, t->n_act, t->S, t->ldS, t->nb + t->na, t->C2, t->na, t->S + t->nb, t->ldS));
    j_cholg.push_back(gram_job(t, t->S + t->nb, t->na, t->S + t->nb, t->na, t->Mm, t->gw, 1));
    lob_bjob r = rr_job(t, t->na, t->Mm, t->Mm, t->thw, t->Cc, 1);
    r.I0 = info_dev(E, t, 0);
    j_rr1.push_back(r);
    if (t->haveP) {
      j_pgather.push_back(cp_job(t->n_act, t->na, t->P, t->nb, t->map, t->S + t->nb + t->na, t->ldS));
      j_pgather.push_back(cp_job(t->n_act, t->na, t->HP, t->nb, t->map, t->HS + t->nb + t->na, t->ldS));
    }
  }
  const int blas = 0;  // each job carries its solve's arithmetic
  LOB_TRY(launch_per_job(E, j_shift, k_shifts_batch));
  for (lob_ltask* t : j_tile)
    LOB_TRY(lob_precond_launch(t->M, t->mu, t->R, t->W, t->nb, t->n_act, t->o.precond_solve,
                               t->o.precond_steps > 0 ? t->o.precond_steps : 3, E->st));
  if (!j_prec.empty()) {
    lob_bjob* dev = nullptr;
    lob_bjob* h = E->take(j_prec.size(), &dev);
    if (!h) return LOB_ERR_NOMEM;
    int bpmax = 1, nbmax = 1;
    for (size_t i = 0; i < j_prec.size(); i++) {
      h[i] = j_prec[i];
      bpmax = std::max(bpmax, j_prec[i].x1);
      nbmax = std::max(nbmax, j_prec[i].x0);
    }
    LOB_TRY(lob_precond_batch_launch(h, dev, (int)j_prec.size(), bpmax, nbmax, E->st));
  }
  LOB_TRY(copy_batch(E, j_gather));
  LOB_TRY(gram_batch(E, j_zg, blas));
  LOB_TRY(launch_per_job(E, j_proj, k_proj_batch));
  LOB_TRY(lincomb_batch(E, j_lcproj, blas));
  LOB_TRY(copy_batch(E, j_pgather));
  // Cholesky-QR Grams of W and of P (P's use the second half of the partial buffer)
  std::vector<lob_bjob> j_pcholg;
  for (lob_ltask* t : iter) {
    if (!t->haveP) continue;
    j_pcholg.push_back(gram_job(t, t->S + t->nb + t->na, t->na, t->S + t->nb + t->na, t->na, t->MmP,
                                t->gw + t->gw_half, 1));
    lob_bjob r = rr_job(t, t->na, t->MmP, t->MmP, t->thP, t->CcP, 1);
    r.I0 = info_dev(E, t, 1);
    j_rr1.push_back(r);
  }
  for (auto& j : j_pcholg) j_cholg.push_back(j);
  LOB_TRY(gram_batch(E, j_cholg, blas));
  LOB_TRY(rr_batch(E, j_rr1, blas));
  for (lob_ltask* t : finishing)
    LOB_CUDA(cudaMemcpyAsync(E->h_theta + (size_t)t->slot * 3 * NBMAX, t->theta, t->k * 8, cudaMemcpyDeviceToHost,
                             E->st));
  // ---- B: Cholesky-QR updates, SpMM, Rayleigh-Ritz -- enqueued on the assumption that the
  // factorisations succeeded; their statuses are read back with the Rayleigh-Ritz ones
  std::vector<lob_bjob> j_cfin, j_stage, j_post, j_g, j_rr;
  std::vector<lob_ltask*> rr_tasks;
  for (lob_ltask* t : iter) {
    t->pok = t->haveP;
    t->m = t->nb + t->na + (t->pok ? t->na : 0);
    j_cfin.push_back(lc_job(t, t->n_act, t->S + t->nb, t->ldS, t->na, t->Cc, t->na, t->S + t->nb, t->ldS));
    if (t->pok) {
      j_cfin.push_back(lc_job(t, t->n_act, t->S + t->nb + t->na, t->ldS, t->na, t->CcP, t->na, t->S + t->nb + t->na,
                              t->ldS));
      j_cfin.push_back(lc_job(t, t->n_act, t->HS + t->nb + t->na, t->ldS, t->na, t->CcP, t->na, t->HS + t->nb + t->na,
                              t->ldS));
    }
    rr_tasks.push_back(t);
  }
  for (lob_ltask* t : start) {
    t->m = t->nb;
    rr_tasks.push_back(t);
  }
  LOB_TRY(lincomb_batch(E, j_cfin, blas));
  // SpMM operands: W (iterating) or X (starting), contiguous in Tp
  std::vector<const lob_matrix*> ms;
  std::vector<const double*> Xs;
  std::vector<double*> Ys;
  std::vector<int> ncol, mode;
  std::vector<int64_t> nact;
  for (lob_ltask* t : rr_tasks) {
    const int c0 = t->start ? 0 : t->nb;
    const int w = t->start ? t->nb : t->na;
    j_stage.push_back(cp_job(t->n, w, t->S + c0, t->ldS, nullptr, t->Tp, w));
    j_post.push_back(cp_job(t->n, w, t->THp, w, nullptr, t->HS + c0, t->ldS));
    ms.push_back(t->M); Xs.push_back(t->Tp); Ys.push_back(t->THp); ncol.push_back(w); mode.push_back(spmm_mode_of(t));
    nact.push_back(t->n_act);
  }
  LOB_TRY(copy_batch(E, j_stage));
  if (!ms.empty()) {
    if ((int)ms.size() > E->scap) return LOB_ERR_NOMEM;
    int nk = 0;
    LOB_TRY(lob_spmm_batch_launch(ms.data(), Xs.data(), Ys.data(), ncol.data(), mode.data(), nact.data(),
                                  (int)ms.size(), E->sh, E->sd, E->st, &nk));
    E->spmm_launches += nk;
    E->spmm_products += (long long)ms.size();
  }
  LOB_TRY(copy_batch(E, j_post));
  for (lob_ltask* t : rr_tasks) {
    push_gm(j_g, t);
    lob_bjob r = rr_job(t, t->m, t->G, t->Mm, t->theta, t->Cc, 0);
    r.I0 = info_dev(E, t, 2);
    j_rr.push_back(r);
  }
  LOB_TRY(gram_batch(E, j_g, blas));
  LOB_TRY(rr_batch(E, j_rr, blas));
  LOB_CUDA(cudaMemcpyAsync(E->h_info, E->d_info, (size_t)E->cap * 16, cudaMemcpyDeviceToHost, E->st));
  LOB_TRY(sync(E));
  for (lob_ltask* t : finishing) t->finished = true;
  // statuses: a failed factor of W restarts the solve from X next round; a failed factor of P,
  // or a failed Rayleigh-Ritz with P, repeats the Rayleigh-Ritz step on [X W]
  std::vector<lob_bjob> j_g2, j_rr2;
  std::vector<lob_ltask*> retry, kept;
  for (lob_ltask* t : rr_tasks) {
    t->rrfail = info_host(E, t, 2) != 0;
    if (!t->start) {
      if (info_host(E, t, 0) != 0) {  // W lost rank
        t->restarts++;
        t->start = true;
        t->haveP = false;
        continue;
      }
      const bool pfail = t->pok && info_host(E, t, 1) != 0;
      if ((pfail || t->rrfail) && t->m > t->nb + t->na) {
        t->restarts++;
        t->pok = false;
        t->m = t->nb + t->na;
        push_gm(j_g2, t);
        lob_bjob r = rr_job(t, t->m, t->G, t->Mm, t->theta, t->Cc, 0);
        r.I0 = info_dev(E, t, 2);
        j_rr2.push_back(r);
        retry.push_back(t);
      }
    }
    kept.push_back(t);
  }
  rr_tasks.swap(kept);
  if (!retry.empty()) {
    LOB_TRY(gram_batch(E, j_g2, blas));
    LOB_TRY(rr_batch(E, j_rr2, blas));
    LOB_CUDA(cudaMemcpyAsync(E->h_info, E->d_info, (size_t)E->cap * 16, cudaMemcpyDeviceToHost, E->st));
    LOB_TRY(sync(E));
    for (lob_ltask* t : retry) t->rrfail = info_host(E, t, 2) != 0;
  }
  // ---- C: update, residuals
  std::vector<lob_bjob> j_cc, j_up1, j_up2, j_res, j_rel;
  for (lob_ltask* t : rr_tasks) {
    if (t->rrfail) {
      if (t->start) { t->status = LOB_ERR_BREAKDOWN; t->finished = true; finishing.push_back(t); continue; }
      t->restarts++;
      t->start = true;  // restart from X next round
      t->haveP = false;
      continue;
    }
    const int nb = t->nb, mm = t->m;
    if (mm == nb) {
      j_up2.push_back(lc_job(t, t->n_act, t->S, t->ldS, nb, t->Cc, nb, t->S, t->ldS));
      j_up2.push_back(lc_job(t, t->n_act, t->HS, t->ldS, nb, t->Cc, nb, t->HS, t->ldS));
    } else {
      j_cc.push_back(cp_job(mm - nb, nb, t->Cc + (size_t)nb * mm, mm, nullptr, t->C2, nb));
      j_cc.push_back(cp_job(nb, nb, t->Cc, mm, nullptr, t->Cx, nb));
      j_up1.push_back(lc_job(t, t->n_act, t->S + nb, t->ldS, mm - nb, t->C2, nb, t->P, nb));
      j_up1.push_back(lc_job(t, t->n_act, t->HS + nb, t->ldS, mm - nb, t->C2, nb, t->HP, nb));
      j_up2.push_back(lc_job(t, t->n_act, t->S, t->ldS, nb, t->Cx, nb, t->S, t->ldS, t->P, nb));
      j_up2.push_back(lc_job(t, t->n_act, t->HS, t->ldS, nb, t->Cx, nb, t->HS, t->ldS, t->HP, nb));
    }
    lob_bjob rj{};
    rj.A = t->S; rj.lda = t->ldS; rj.B = t->HS; rj.ldb = t->ldS; rj.C = t->theta; rj.Y = t->R; rj.W0 = t->part;
    rj.n = t->n_act; rj.x0 = nb; rj.s0 = 1.0 / t->normH;
    j_res.push_back(rj);
    lob_bjob rl{};
    rl.W0 = t->part; rl.x1 = (int32_t)nblk(t->n_act); rl.x0 = nb; rl.s0 = 1.0; rl.Y = relres_dev(E, t);
    j_rel.push_back(rl);
    if (t->start) {
      t->start = false;
      t->active = true;
      t->haveP = false;
      t->it = 1;
    } else {
      t->haveP = mm > nb;
      t->it++;
    }
  }
  LOB_TRY(copy_batch(E, j_cc));
  LOB_TRY(lincomb_batch(E, j_up1, blas));
  LOB_TRY(lincomb_batch(E, j_up2, blas));
  LOB_TRY(launch_rows(E, j_res, [](const lob_bjob& j) { return (j.n + BS - 1) / BS; }, k_resid_batch));
  LOB_TRY(launch_per_job(E, j_rel, k_relres_batch));
  LOB_CUDA(cudaMemcpyAsync(E->h_relres, E->d_relres, (size_t)E->cap * NBMAX * 8, cudaMemcpyDeviceToHost, E->st));
  LOB_TRY(sync(E));
  // retire finished solves; a finished guess child hands its vectors to its parent
  std::vector<lob_ltask*> keep;
  std::vector<lob_bjob> j_handoff;
  for (lob_ltask* t : E->tasks) {
    if (!t->finished) { keep.push_back(t); continue; }
    if (t->parent) {
      lob_ltask* p = t->parent;
      p->child = nullptr;
      p->waiting = false;
      if (t->status == LOB_OK || t->status == LOB_ERR_NOCONV)
        j_handoff.push_back(cp_job(p->n, p->nb, p->W, p->nb, nullptr, p->S, p->ldS));
      task_release(E, t);
      delete t;
      continue;
    }
    done.push_back(t);
  }
  E->tasks.swap(keep);
  LOB_TRY(copy_batch(E, j_handoff));
  return LOB_OK;
}

// Results of a finished solve; releases its state.
int lob_engine_result(lob_engine* E, lob_ltask* t, double* lambda, lob_stats* st, int64_t* user) {
  if (lambda)
    for (int i = 0; i < t->k; i++) lambda[i] = E->h_theta[(size_t)t->slot * 3 * NBMAX + i];
  if (st) {
    memset(st, 0, sizeof(*st));
    st->iterations = t->iters_total;
    st->refine_iterations = t->refine_its;
    st->restarts = t->restarts;
    st->precond_dropped = t->precond_dropped;
    for (int j = 0; j < t->nb; j++) st->residual[j] = E->h_relres[(size_t)t->slot * NBMAX + j];
    st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t->t0).count();
  }
  if (user) *user = t->user;
  const int rc = t->status;
  task_release(E, t);
  delete t;
  return rc;
}

long long lob_engine_spmm_launches(const lob_engine* E) { return E->spmm_launches; }
long long lob_engine_spmm_products(const lob_engine* E) { return E->spmm_products; }
int lob_engine_ntasks(const lob_engine* E) { return (int)E->tasks.size(); }
