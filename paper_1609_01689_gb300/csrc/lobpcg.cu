// LOBPCG (Section 3.1, Algorithm 1) with the block-diagonal preconditioner
// (Section 3.2, eq. 11), the robustness rules of Section 4.3, and the initial guess of
// Section 3.3.1 (eq. 12). All vectors stay on the device; the host orchestrates launches and
// reads back nb residual norms per iteration for the convergence test (step 5).
//
// The solver is a resumable task: lob_task_step() enqueues work on the task's stream until the
// host needs a value from the device (a convergence test or a factorisation status, returned as
// LOB_TASK_SYNC with an event to wait on) or until it needs H times a block (LOB_TASK_SPMM, which
// the driver runs either alone or batched with other tasks' products). lob_solve drives one task;
// the server drives many and shares the SpMM launches between them. Each iteration has three
// host synchronisations (residual norms; Cholesky-QR of W and P; Rayleigh-Ritz) and one SpMM.
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

#include <algorithm>
#include <chrono>
#include <mutex>
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

// eq. 13: X[r, :] -= W[r, :] for the rows r >= ns of the larger space only, where W = T^{-1} R is
// the block-preconditioned residual of the zero-padded guess (its rows below ns stay as they are).
__global__ void k_eq13_correct(int64_t n, int64_t ns, int nb, const double* __restrict__ W, double* __restrict__ X,
                               int ldx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (n - ns) * nb) return;
  const int64_t r = ns + t / nb;
  const int j = (int)(t % nb);
  X[r * ldx + j] -= W[r * nb + j];
}

// R = HX - X diag(theta); per-CTA partial column sums of r^2 and x^2 into part[blk][2*nb].
__global__ void __launch_bounds__(256) k_residual(int64_t n, int nb, const double* __restrict__ X, int ldx,
                                                  const double* __restrict__ HX, int ldh,
                                                  const double* __restrict__ theta, double inv_norm,
                                                  double* __restrict__ R, double* __restrict__ part) {
  __shared__ float sred[8 * 64];
  lob_residual_rows(n, nb, X, ldx, HX, ldh, theta, inv_norm, R, part, blockIdx.x, sred);
}

// relres_j = sqrt(sum r^2) / (normH sqrt(sum x^2)): one CTA per column, a strided pass over the
// partials then a fixed-order tree, so the result is deterministic. (The residual kernel's
// partials are already scaled by 1 / normH; it is then called with normH = 1.)
__global__ void __launch_bounds__(256) k_relres(int nparts, int nb, const double* __restrict__ part, double normH,
                                                double* __restrict__ out) {
  __shared__ double srr[256], sxx[256];
  const int j = blockIdx.x, tid = threadIdx.x;
  double rr = 0.0, xx = 0.0;
  for (int b = tid; b < nparts; b += 256) { rr += part[(int64_t)b * 2 * nb + j]; xx += part[(int64_t)b * 2 * nb + nb + j]; }
  srr[tid] = rr;
  sxx[tid] = xx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) { srr[tid] += srr[tid + o]; sxx[tid] += sxx[tid + o]; }
    __syncthreads();
  }
  if (tid == 0) out[j] = sqrt(srr[0]) / (normH * sqrt(sxx[0] > 0.0 ? sxx[0] : 1.0));
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

// Identity columns: out[(c0 + i) * ld + i] = 1 for i < ncol (after zeroing out).
__global__ void k_unit_cols(int64_t c0, int ncol, int ld, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncol) out[(c0 + i) * ld + i] = 1.0;
}

// C2 = [-Z; I] (rows: nb rows of -Z then na rows of the identity), for W - X Z as [X W] C2.
__global__ void k_proj_coef(int nb, int na, const double* __restrict__ Z, double* __restrict__ C2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (nb + na) * na) return;
  const int r = t / na, c = t % na;
  C2[t] = r < nb ? -Z[r * na + c] : (r - nb == c ? 1.0 : 0.0);
}

// Phase timing with CUDA events on the task's stream. Event pairs are recorded without
// synchronising and resolved in bulk whenever the task passes a synchronisation point anyway.
// Pairs recorded while a stage is captured belong to the stage's graph: the graph records them on
// every replay, and they are queued again (owned) after each launch.
struct PhaseClock {
  struct Pair { cudaEvent_t a, b; double* acc; bool owned; };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (pool.empty()) { cudaEvent_t e; cudaEventCreate(&e); return e; }
    cudaEvent_t e = pool.back(); pool.pop_back(); return e;
  }
  void resolve() {  // every recorded event has completed
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.acc) *p.acc += ms;
      else cudaGetLastError();
      if (!p.owned) { pool.push_back(p.a); pool.push_back(p.b); }
    }
    pending.clear();
  }
  ~PhaseClock() {
    for (auto& p : pending)
      if (!p.owned) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct Timer {
  PhaseClock* clk;
  cudaEvent_t a = nullptr;
  cudaStream_t st;
  double* acc;
  Timer(PhaseClock* c, cudaStream_t s, double* accum) : clk(c), st(s), acc(accum) {
    if (acc && clk) { a = clk->get(); cudaEventRecord(a, st); }
  }
  ~Timer() {
    if (a) {
      cudaEvent_t b = clk->get();
      cudaEventRecord(b, st);
      clk->pending.push_back({a, b, acc, false});
    }
  }
};

// Stream-ordered device buffer: allocation and release are ordered on the owning stream, so
// creating and retiring tasks never synchronises the device.
struct DBuf {
  double* p = nullptr;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { if (p) cudaFreeAsync(p, st); }
  int alloc(size_t n, cudaStream_t s) {
    st = s;
    if (cudaMallocAsync((void**)&p, (n ? n : 1) * sizeof(double), s) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return LOB_ERR_NOMEM;
    }
    return LOB_OK;
  }
};

// Pinned host words a task reads back asynchronously (residual norms, factorisation status,
// Ritz values) and the active-column map it uploads. Boxes come from a process-wide pool.
struct HostBox {
  double relres[64];
  double theta[64];
  int32_t info[4];
  int32_t map[64];
};
std::mutex g_box_mu;
std::vector<HostBox*> g_box_free;
HostBox* box_get() {
  std::lock_guard<std::mutex> g(g_box_mu);
  if (g_box_free.empty()) {
    HostBox* chunk = nullptr;
    if (cudaHostAlloc((void**)&chunk, 64 * sizeof(HostBox), cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = 0; i < 64; i++) g_box_free.push_back(chunk + i);
  }
  HostBox* b = g_box_free.back();
  g_box_free.pop_back();
  memset(b, 0, sizeof(*b));
  return b;
}
void box_put(HostBox* b) {
  if (!b) return;
  std::lock_guard<std::mutex> g(g_box_mu);
  g_box_free.push_back(b);
}

enum { PH_SPMM, PH_GRAM, PH_RR, PH_UPDATE, PH_PRECOND, PH_RESID, PH_ORTH, PH_GUESS };

// info slots in the host box
enum { SLOT_W = 0, SLOT_P = 1, SLOT_RR = 2 };

enum {
  PC_INIT, PC_GUESS_CHILD, PC_PHASE, PC_RUN_SPMM0, PC_RUN_RR0, PC_RUN_RR0_CHECK, PC_ITER_RESID, PC_ITER_DECIDE,
  PC_ITER_CHOL, PC_ITER_RR, PC_ITER_RR_CHECK, PC_RUN_END, PC_FINISH, PC_OUT, PC_END
};

size_t solver_doubles(int64_t n, int nb) {
  const size_t m = 3 * (size_t)nb;
  size_t d = 2 * (size_t)n * m + 7 * (size_t)n * nb;       // S, HS; P, HP, R, W, Tn, Tp, THp
  d += 11 * m * m + 3 * m + 2 * (size_t)nb;                 // G, M, C, Cx, C2, Z, M_P, C_P, ...
  d += lob_gram_work_doubles(n, 1, 1) * m * m;              // Gram chunk partials
  d += lob_rr_work_doubles((int)m);
  d += (size_t)nblk(n) * 2 * m;                             // residual partials
  return d;
}

}  // namespace

struct lob_task {
  // problem
  lob_matrix* M = nullptr;
  int64_t n = 0, n_act = 0;
  int nb = 0, k = 0;
  double tol = 0.0, normH = 0.0;
  lob_solve_opts o{};
  const double* X0 = nullptr;
  double* Xout = nullptr;
  cudaStream_t st = nullptr;
  bool timing = false;
  lob_stats stats{};
  PhaseClock clock;
  std::chrono::steady_clock::time_point t0;
  // device state
  int ldS = 0;
  DBuf S, HS, P, HP, R, W, Tn, Tp, THp, G, Mm, Cc, Cx, theta, thw, work, rrwork, part, relres_d, mu, C2, Z;
  DBuf MmP, CcP, thP, info_d, imap;
  DBuf gEc, gHEc, gG, gM, gth, gC, gwk;  // dense initial guess
  HostBox* hb = nullptr;
  cudaEvent_t ev = nullptr;
  // control
  int pc = PC_INIT, status = LOB_OK, run_status = LOB_OK, phase = 0;
  int spmm_mode = LOB_SPMM_FP64, blas_mode = LOB_SPMM_FP64, rr_mode = LOB_SPMM_FP64;
  double run_tol = 0.0;
  int run_max = 0, max_iter = 0;
  int it = 0, restarts = 0, na = 0, m = 0, iters_total = 0, restarts_total = 0;
  bool haveP = false, retry = false, wretry = false;
  bool eq13_done = false;  // the eq. 13 correction of the guess was applied
  // stagnation safeguard: the worst unconverged relative residual among the first k columns has
  // not halved for PC_STALL iterations -> the rest of the run goes without the preconditioner
  double best_res = 0.0;
  int best_it = 0;
  bool pc_dropped = false;
  // the SpMM the task waits for: Y = H X on contiguous n x ncol blocks, then Y copied to post
  const double* sp_x = nullptr;
  double* sp_y = nullptr;
  int sp_ncol = 0;
  double* sp_post = nullptr;
  int sp_post_ld = 0;
  lob_task* child = nullptr;
  // captured stages: one graph per stage shape (stage, active columns, P present, ...), replayed
  // as a single launch (phase timers inside a stage become event nodes of its graph)
  bool graphs = false;
  struct Staged { uint64_t key; cudaGraphExec_t exec; long long kernels; std::vector<PhaseClock::Pair> timers; };
  std::vector<Staged> gcache;

  ~lob_task() {
    delete child;
    for (auto& g : gcache) {
      cudaGraphExecDestroy(g.exec);
      for (auto& p : g.timers) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    }
    if (ev) cudaEventDestroy(ev);
    box_put(hb);
  }

  uint64_t skey(int stage_id, int a, int b, int c) const {
    return (uint64_t)stage_id | ((uint64_t)(a & 0xFFF) << 4) | ((uint64_t)(b & 0xFFF) << 16) |
           ((uint64_t)(c & 0xFF) << 28) | ((uint64_t)blas_mode << 36) | ((uint64_t)spmm_mode << 40);
  }

  // Enqueue a stage: replay its graph, or capture it on first use (falling back to plain launches
  // if capture is not possible).
  template <class F>
  int stage(uint64_t key, F&& enqueue) {
    if (!graphs) return enqueue();
    for (const Staged& g : gcache)
      if (g.key == key) {
        LOB_CUDA(cudaGraphLaunch(g.exec, st));
        g_lob_launches.fetch_add(g.kernels, std::memory_order_relaxed);
        for (const auto& p : g.timers) clock.pending.push_back(p);
        return LOB_OK;
      }
    const size_t p0 = clock.pending.size();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      graphs = false;
      return enqueue();
    }
    const long long k0 = g_lob_launches.load();
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    const long long nk = g_lob_launches.load() - k0;
    g_lob_launches.fetch_sub(nk, std::memory_order_relaxed);  // captured, not yet launched
    cudaGraphExec_t x = nullptr;
    if (rc != LOB_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      for (size_t i = p0; i < clock.pending.size(); i++) {  // recorded only in the abandoned capture
        clock.pool.push_back(clock.pending[i].a);
        clock.pool.push_back(clock.pending[i].b);
      }
      clock.pending.resize(p0);
      graphs = false;
      return rc != LOB_OK ? rc : enqueue();
    }
    cudaGraphDestroy(g);
    // timer pairs recorded during the capture now belong to the graph
    std::vector<PhaseClock::Pair> timers(clock.pending.begin() + p0, clock.pending.end());
    clock.pending.resize(p0);
    for (auto& p : timers) p.owned = true;
    gcache.push_back({key, x, nk, timers});
    LOB_CUDA(cudaGraphLaunch(x, st));
    g_lob_launches.fetch_add(nk, std::memory_order_relaxed);
    for (const auto& p : gcache.back().timers) clock.pending.push_back(p);
    return LOB_OK;
  }

  double* ph(int i) { return timing ? &stats.phase_ms[i] : nullptr; }
  PhaseClock* clk() { return timing ? &clock : nullptr; }

  int alloc() {
    ldS = 3 * nb;
    const size_t nS = (size_t)n * ldS, nv = (size_t)n * nb, mm = ldS;
    LOB_TRY(S.alloc(nS, st)); LOB_TRY(HS.alloc(nS, st));
    LOB_TRY(P.alloc(nv, st)); LOB_TRY(HP.alloc(nv, st)); LOB_TRY(R.alloc(nv, st)); LOB_TRY(W.alloc(nv, st));
    LOB_TRY(Tn.alloc(nv, st)); LOB_TRY(Tp.alloc(nv, st)); LOB_TRY(THp.alloc(nv, st));
    LOB_TRY(G.alloc(mm * mm, st)); LOB_TRY(Mm.alloc(mm * mm, st)); LOB_TRY(Cc.alloc(mm * mm, st));
    LOB_TRY(Cx.alloc(mm * mm, st)); LOB_TRY(theta.alloc(mm, st)); LOB_TRY(thw.alloc(mm, st));
    LOB_TRY(MmP.alloc(mm * mm, st)); LOB_TRY(CcP.alloc(mm * mm, st)); LOB_TRY(thP.alloc(mm, st));
    // bound over every (p, q) <= m, and the tensor-core Gram's partial sums
    LOB_TRY(work.alloc(std::max(lob_gram_work_doubles(n, 1, 1) * mm * mm, lob_gram_oz_work_doubles()), st));
    LOB_TRY(rrwork.alloc(lob_rr_work_doubles((int)mm), st));
    LOB_TRY(part.alloc((size_t)nblk(n) * 2 * mm, st));
    LOB_TRY(relres_d.alloc(nb, st)); LOB_TRY(mu.alloc(nb, st)); LOB_TRY(C2.alloc(mm * mm, st));
    LOB_TRY(Z.alloc(mm * mm, st));
    LOB_TRY(info_d.alloc(2, st));  // 4 int32 slots
    LOB_TRY(imap.alloc(32, st));   // 64 int32
    hb = box_get();
    if (!hb) return LOB_ERR_NOMEM;
    LOB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    return LOB_OK;
  }

  int32_t* info_slot(int s) { return reinterpret_cast<int32_t*>(info_d.p) + s; }
  int* map_d() { return reinterpret_cast<int*>(imap.p); }

  int sync_point() {
    LOB_CUDA(cudaEventRecord(ev, st));
    return LOB_TASK_SYNC;
  }

  // projected eigenproblem and Cholesky-QR factors in the task's small-solve arithmetic (native
  // FP64, or double-float when the options ask for it)
  // Arithmetic of the block products: native FP64, or in MIXED the FP64-class tensor-core kernels
  // (lob_gram_launch_ws / lob_lincomb_launch fall back to double-float beyond their shapes)
  int bmode() const { return blas_mode; }

  int rr(int mm, const double* Gp, const double* Mp, double* th, double* Cp, int slot, int chol_only) {
    if (rr_mode == LOB_SPMM_MIXED)
      return lob_rr_launch_df(mm, Gp, Mp, th, Cp, info_slot(slot), rrwork.p, st, chol_only);
    return lob_rr_launch(mm, Gp, Mp, th, Cp, info_slot(slot), rrwork.p, st, chol_only);
  }

  int read_info(int slot) {
    LOB_CUDA(cudaMemcpyAsync(&hb->info[slot], info_slot(slot), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return LOB_OK;
  }

  // Stage the operand of Y = H X (X, Y: ncol columns with leading dimensions ldx, ldy).
  int spmm_stage(const double* X, int ldx, int ncol) {
    if (ldx != ncol)
      (k_copy_cols<<<nblk(n * ncol), BS, 0, st>>>(n, ncol, X, ldx, nullptr, Tp.p, ncol), LOB_LAUNCHED());
    return LOB_OK;
  }

  // Register the product Y = H X (X, Y: ncol columns with leading dimensions ldx, ldy); the
  // operand must have been staged (spmm_stage) unless staged is false.
  int want_spmm(const double* X, int ldx, double* Y, int ldy, int ncol, bool staged = false) {
    if (!staged) LOB_TRY(spmm_stage(X, ldx, ncol));
    sp_x = ldx != ncol ? Tp.p : X;
    sp_y = ldy != ncol ? THp.p : Y;
    sp_post = ldy != ncol ? Y : nullptr;
    sp_post_ld = ldy;
    sp_ncol = ncol;
    stats.spmm_calls++;
    const double vb = spmm_mode == LOB_SPMM_MIXED ? 4.0 : 8.0;  // FP32 or FP64 (split pair) values
    const double bytes = (double)M->T.nnz * (vb + 4.0) + (double)M->T.ntiles * 12.0 + (double)n * ncol * 16.0;
    stats.spmm_bytes += bytes;
    stats.spmm_bytes_mode[spmm_mode] += bytes;
    stats.spmm_calls_mode[spmm_mode]++;
    LOB_CUDA(cudaGetLastError());
    return LOB_TASK_SPMM;
  }

  int spmm_post() {
    if (sp_post)
      (k_copy_cols<<<nblk(n * sp_ncol), BS, 0, st>>>(n, sp_ncol, sp_y, sp_ncol, nullptr, sp_post, sp_post_ld),
       LOB_LAUNCHED());
    return LOB_OK;
  }

  // G = S^T H S, M = S^T S on the first mm columns, then the Rayleigh-Ritz solve (status to SLOT_RR)
  int rr_begin(int mm) {
    {
      Timer t(clk(), st, ph(PH_GRAM));
      if (blas_mode == LOB_SPMM_MIXED && lob_oz_pays(mm, mm)) {
        // one tensor-core pass for both: M = S^T S and (H S)^T S, the transpose of G (equal to G for
        // the symmetric H; the solve reads the upper triangles)
        LOB_TRY(lob_gram_oz_launch(n_act, mm, S.p, ldS, HS.p, ldS, mm, S.p, ldS, Mm.p, G.p, work.p, st));
      } else {
        // both symmetric (H is): only their upper triangles are formed (and read by the solve)
        LOB_TRY(lob_gram_launch_ws(n_act, mm, S.p, ldS, mm, HS.p, ldS, G.p, bmode(), work.p, st, 1));
        LOB_TRY(lob_gram_launch_ws(n_act, mm, S.p, ldS, mm, S.p, ldS, Mm.p, bmode(), work.p, st, 1));
      }
    }
    Timer t(clk(), st, ph(PH_RR));
    LOB_TRY(rr(mm, G.p, Mm.p, theta.p, Cc.p, SLOT_RR, 0));
    return read_info(SLOT_RR);
  }

  // Y = A C (+ D) written to Y (leading dimension ldy), where Y may be columns of A's own rows:
  // with q <= 16 one CTA covers all output columns of its rows and loads them before writing, so
  // the product goes straight into place; wider products go through Tn.
  int lincomb_into(int p, const double* A, int lda, int q, const double* C, double* Y, int ldy,
                   const double* D = nullptr, int ldd = 0) {
    // one pass straight into place: one CTA covers all output columns of its rows (the tensor-core
    // kernel up to 64, the CUDA-core kernels up to 16)
    if (q <= 16 || (blas_mode == LOB_SPMM_MIXED && lob_oz_pays(p, q)))
      return lob_lincomb_launch(n_act, p, A, lda, q, C, Y, ldy, bmode(), st, D, ldd);
    LOB_TRY(lob_lincomb_launch(n_act, p, A, lda, q, C, Tn.p, q, bmode(), st, D, ldd));
    (k_copy_cols<<<nblk(n_act * q), BS, 0, st>>>(n_act, q, Tn.p, q, nullptr, Y, ldy), LOB_LAUNCHED());
    return LOB_OK;
  }

  // Cholesky-QR, first half: B^T B = L L^T for the ncol columns at S[:, col0]; C = L^{-T}.
  int cholqr_begin(int col0, int ncol, double* Mb, double* Cb, double* thb, int slot) {
    Timer t(clk(), st, ph(PH_ORTH));
    const double* B = S.p + col0;
    LOB_TRY(lob_gram_launch_ws(n_act, ncol, B, ldS, ncol, B, ldS, Mb, bmode(), work.p, st, 1));
    LOB_TRY(rr(ncol, Mb, Mb, thb, Cb, slot, 1));
    return read_info(slot);
  }

  // Cholesky-QR, second half: B <- B C (and the same on HS when withH).
  int cholqr_finish(int col0, int ncol, bool withH, const double* Cb) {
    Timer t(clk(), st, ph(PH_ORTH));
    LOB_TRY(lincomb_into(ncol, S.p + col0, ldS, ncol, Cb, S.p + col0, ldS));
    if (withH) LOB_TRY(lincomb_into(ncol, HS.p + col0, ldS, ncol, Cb, HS.p + col0, ldS));
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  int residual_begin() {
    Timer t(clk(), st, ph(PH_RESID));
    (k_residual<<<nblk(n_act), BS, 0, st>>>(n_act, nb, S.p, ldS, HS.p, ldS, theta.p, 1.0 / normH, R.p, part.p),
     LOB_LAUNCHED());
    (k_relres<<<nb, 256, 0, st>>>((int)nblk(n_act), nb, part.p, 1.0, relres_d.p), LOB_LAUNCHED());
    LOB_CUDA(cudaMemcpyAsync(hb->relres, relres_d.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    return LOB_OK;
  }

  // X <- S C[:, :nb], HX <- HS C[:, :nb]; P <- S[:, nb:mm] C[nb:mm, :nb], HP likewise. P is formed
  // first and reused: X <- X C[:nb, :nb] + P (and H X likewise), which saves the products of the
  // [W P] columns a second time.
  int update(int mm) {
    Timer t(clk(), st, ph(PH_UPDATE));
    if (mm == nb) {
      LOB_TRY(lincomb_into(nb, S.p, ldS, nb, Cc.p, S.p, ldS));
      LOB_TRY(lincomb_into(nb, HS.p, ldS, nb, Cc.p, HS.p, ldS));
    } else {
      // rows nb..mm-1 of C (row-major, leading dimension mm) -> compact (mm-nb) x nb block in C2;
      // rows 0..nb-1 -> Cx (nb x nb)
      (k_copy_cols<<<nblk((int64_t)(mm - nb) * nb), BS, 0, st>>>(mm - nb, nb, Cc.p + (size_t)nb * mm, mm, nullptr,
                                                                    C2.p, nb),
       LOB_LAUNCHED());
      (k_copy_cols<<<nblk((int64_t)nb * nb), BS, 0, st>>>(nb, nb, Cc.p, mm, nullptr, Cx.p, nb), LOB_LAUNCHED());
      LOB_TRY(lob_lincomb_launch(n_act, mm - nb, S.p + nb, ldS, nb, C2.p, P.p, nb, bmode(), st));
      LOB_TRY(lob_lincomb_launch(n_act, mm - nb, HS.p + nb, ldS, nb, C2.p, HP.p, nb, bmode(), st));
      LOB_TRY(lincomb_into(nb, S.p, ldS, nb, Cx.p, S.p, ldS, P.p, nb));
      LOB_TRY(lincomb_into(nb, HS.p, ldS, nb, Cx.p, HS.p, ldS, HP.p, nb));
    }
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  // eq. 12 for a tiny leading block (ns <= 3 nb): G = H_11 by SpMMs of unit columns, M = I,
  // Rayleigh-Ritz gives all its eigenpairs; X = [C[:, :nb]; 0], seeded random columns beyond ns.
  int guess_dense(int64_t ns, double* Xo) {
    const int nsi = (int)ns;
    const int cw = nsi < 64 ? nsi : 64;
    LOB_TRY(gEc.alloc((size_t)n * cw, st)); LOB_TRY(gHEc.alloc((size_t)n * cw, st));
    LOB_TRY(gG.alloc((size_t)nsi * nsi, st)); LOB_TRY(gM.alloc((size_t)nsi * nsi, st));
    LOB_TRY(gth.alloc(nsi, st)); LOB_TRY(gC.alloc((size_t)nsi * nsi, st));
    LOB_TRY(gwk.alloc(lob_rr_work_doubles(nsi), st));
    LOB_CUDA(cudaMemsetAsync(gM.p, 0, (size_t)nsi * nsi * 8, st));
    (k_unit_cols<<<1, 128, 0, st>>>(0, nsi, nsi, gM.p), LOB_LAUNCHED());
    for (int c0 = 0; c0 < nsi; c0 += 64) {
      const int w = nsi - c0 < 64 ? nsi - c0 : 64;
      LOB_CUDA(cudaMemsetAsync(gEc.p, 0, (size_t)n * w * 8, st));
      (k_unit_cols<<<1, 128, 0, st>>>(c0, w, w, gEc.p), LOB_LAUNCHED());
      LOB_TRY(lob_spmm_launch(M, LOB_SPMM_FP64, gEc.p, gHEc.p, w, ns, st));
      (k_copy_cols<<<nblk(ns * w), BS, 0, st>>>(ns, w, gHEc.p, w, nullptr, gG.p + c0, nsi), LOB_LAUNCHED());
    }
    LOB_TRY(lob_rr_launch(nsi, gG.p, gM.p, gth.p, gC.p, info_slot(3), gwk.p, st));
    (k_random<<<nblk(n * nb), BS, 0, st>>>(n, ns, nb, nb, 0, nb, o.seed ^ 0x1A5Eull, Xo), LOB_LAUNCHED());
    const int nc = nsi < nb ? nsi : nb;
    (k_copy_cols<<<nblk(ns * nc), BS, 0, st>>>(ns, nc, gC.p, nsi, nullptr, Xo, nb), LOB_LAUNCHED());
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }

  int step();
};

namespace {
int task_init(lob_task* t, lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0,
              const lob_solve_opts* o, double* X, int64_t n_act, cudaStream_t st, bool timing) {
  t->M = m; t->n = m->T.n; t->n_act = n_act; t->nb = nb; t->k = k; t->tol = tol; t->o = *o; t->X0 = X0;
  t->Xout = X; t->st = st; t->timing = timing;
  t->normH = o->norm_H > 0.0 ? o->norm_H : m->norm_inf;
  // block products: native FP64 in the plain solver, FP64-class double-float in MIXED
  t->blas_mode = o->mode == LOB_MODE_MIXED ? LOB_SPMM_MIXED : LOB_SPMM_FP64;
  t->rr_mode = (o->mode == LOB_MODE_MIXED && o->rr_arith == LOB_ARITH_DF) ? LOB_SPMM_MIXED : LOB_SPMM_FP64;
  t->max_iter = o->max_iter > 0 ? o->max_iter : 500;
  t->t0 = std::chrono::steady_clock::now();
  t->graphs = true;
  return t->alloc();
}
}  // namespace

int lob_task::step() {
  if (child) {
    const int r = child->step();
    if (r != LOB_TASK_DONE) return r;
    const int crc = child->status;
    delete child;
    child = nullptr;
    if (crc != LOB_OK && crc != LOB_ERR_NOCONV) { status = crc; pc = PC_END; return LOB_TASK_DONE; }
    (k_copy_cols<<<nblk(n * nb), BS, 0, st>>>(n, nb, W.p, nb, nullptr, S.p, ldS), LOB_LAUNCHED());
    pc = PC_PHASE;
  }
  for (;;) {
    switch (pc) {
      case PC_INIT: {
        Timer t(clk(), st, ph(PH_GUESS));
        if (X0) {
          (k_copy_cols<<<nblk(n * nb), BS, 0, st>>>(n, nb, X0, nb, nullptr, S.p, ldS), LOB_LAUNCHED());
        } else if (o.n_small > 0 && o.n_small < n_act) {
          // eq. 12: eigenvectors of the leading n_small x n_small block (the smaller
          // configuration space), zero-padded. The small problem is solved directly when it is
          // tiny, else by a child LOBPCG task from seeded random vectors (the multi-level use of
          // Section 3.3.1) to a moderate tolerance: the guess only needs the accuracy of eq. 12
          // itself, whose residual is set by the coupling ||H_21||.
          const int64_t ns = o.n_small;
          if (ns <= 3 * nb) {
            LOB_TRY(guess_dense(ns, W.p));
          } else {
            LOB_CUDA(cudaMemsetAsync(W.p, 0, (size_t)n * nb * 8, st));
            lob_solve_opts so = o;
            // multi-level: the leading-block solve takes its own eq. 12 guess from the inner block
            so.n_small = (o.n_small_inner > 0 && o.n_small_inner < ns) ? o.n_small_inner : 0;
            so.n_small_inner = 0;
            so.guess_correct = 0;
            so.max_iter = 2000;
            so.refine_iter = 0;
            so.mixed_tol = 0.0;
            so.verbose = 0;
            const double gtol = o.guess_tol > 0.0 ? o.guess_tol : LOB_GUESS_TOL;
            child = new lob_task();
            const int rc = task_init(child, M, nb, nb, gtol, nullptr, &so, W.p, ns, st, false);
            if (rc != LOB_OK) { delete child; child = nullptr; return rc; }
            pc = PC_GUESS_CHILD;
            return step();
          }
          (k_copy_cols<<<nblk(n * nb), BS, 0, st>>>(n, nb, W.p, nb, nullptr, S.p, ldS), LOB_LAUNCHED());
        } else {
          (k_random<<<nblk(n * nb), BS, 0, st>>>(n, n_act, nb, ldS, 0, nb, o.seed, S.p), LOB_LAUNCHED());
        }
        LOB_CUDA(cudaGetLastError());
        pc = PC_PHASE;
        continue;
      }
      case PC_GUESS_CHILD:
        return LOB_ERR_ARG;  // unreachable: the child is stepped above
      case PC_PHASE: {
        if (o.mode == LOB_MODE_MIXED && phase == 0) {
          // phase 1: FP32-value SpMM down to the FP32 floor
          spmm_mode = LOB_SPMM_MIXED;
          run_tol = o.mixed_tol > 0.0 ? o.mixed_tol : (tol > LOB_MIXED_TOL ? tol : LOB_MIXED_TOL);
          run_max = max_iter;
        } else if (o.mode == LOB_MODE_MIXED) {
          // phase 2: refinement products from the phase-1 vectors, FP64 values (or double-float
          // values and products when the options ask for it)
          spmm_mode = (o.refine_arith == LOB_ARITH_DF && M->T.v32lo) ? LOB_SPMM_DF64 : LOB_SPMM_FP64;
          run_tol = tol;
          run_max = o.refine_iter > 0 ? o.refine_iter : (max_iter - iters_total > 50 ? max_iter - iters_total : 50);
        } else {
          spmm_mode = LOB_SPMM_FP64;
          run_tol = tol;
          run_max = max_iter;
        }
        retry = false;
        it = 0;
        restarts = 0;
        best_res = 1e300;
        best_it = 0;
        pc_dropped = false;
        pc = PC_RUN_SPMM0;
        continue;
      }
      case PC_RUN_SPMM0:  // step 1: Rayleigh-Ritz on X alone (also orthonormalises it)
        pc = PC_RUN_RR0;
        return want_spmm(S.p, ldS, HS.p, ldS, nb);
      case PC_RUN_RR0:
        LOB_TRY(spmm_post());
        sp_post = nullptr;
        LOB_TRY(rr_begin(nb));
        pc = PC_RUN_RR0_CHECK;
        return sync_point();
      case PC_RUN_RR0_CHECK: {
        clock.resolve();
        if (hb->info[SLOT_RR]) {
          if (retry) { run_status = LOB_ERR_BREAKDOWN; pc = PC_RUN_END; continue; }
          retry = true;  // X0 rank-deficient: orthonormalise a randomised copy
          (k_random<<<nblk(n * nb), BS, 0, st>>>(n, n_act, nb, ldS, 0, nb, 0x5EEDull, S.p), LOB_LAUNCHED());
          pc = PC_RUN_SPMM0;
          continue;
        }
        LOB_TRY(update(nb));
        haveP = false;
        it = 1;
        pc = PC_ITER_RESID;
        continue;
      }
      case PC_ITER_RESID:
        if (it > run_max) { it = run_max; run_status = LOB_ERR_NOCONV; pc = PC_RUN_END; continue; }
        LOB_TRY(residual_begin());  // steps 4-5
        pc = PC_ITER_DECIDE;
        return sync_point();
      case PC_ITER_DECIDE: {
        clock.resolve();
        if (iters_total == 0 && it == 1) {
          // the first residuals of the solve: those of the initial guess (or of its eq. 13 correction)
          double g = 0.0;
          for (int j = 0; j < k; j++) g = fmax(g, hb->relres[j]);
          stats.guess_relres[eq13_done ? 1 : 0] = g;
          if (o.guess_correct && !eq13_done && !X0 && o.n_small > 0 && o.n_small < n_act) {
            // eq. 13 (Section 3.3.1): the block preconditioner with shifts mu_j = theta_j, applied to
            // the residual [~0; H_21 X_1] of the zero-padded guess, gives W ~ [0; (H_22 - theta I)^{-1}
            // H_21 X_1]; the guess becomes [X_1; -W_2] and the run restarts from it
            eq13_done = true;
            {
              Timer t(clk(), st, ph(PH_GUESS));
              (k_shifts<<<1, 32, 0, st>>>(nb, 0, theta.p, relres_d.p, normH, mu.p), LOB_LAUNCHED());
              LOB_TRY(lob_precond_launch(M, mu.p, R.p, W.p, nb, n_act, o.precond_solve,
                                         o.precond_steps > 0 ? o.precond_steps : 3, st));
              (k_eq13_correct<<<nblk((n_act - o.n_small) * nb), BS, 0, st>>>(n_act, o.n_small, nb, W.p, S.p, ldS),
               LOB_LAUNCHED());
              LOB_CUDA(cudaGetLastError());
            }
            pc = PC_RUN_SPMM0;
            continue;
          }
        }
        bool conv = true;
        na = 0;
        for (int j = 0; j < nb; j++) {
          if (j < k && !(hb->relres[j] <= run_tol)) conv = false;
          if (!(hb->relres[j] <= run_tol)) hb->map[na++] = j;
        }
        if (conv) { run_status = LOB_OK; pc = PC_RUN_END; continue; }
        {
          double worst = 0.0;
          for (int j = 0; j < k; j++)
            if (!(hb->relres[j] <= run_tol)) worst = fmax(worst, hb->relres[j]);
          if (worst < 0.5 * best_res) { best_res = worst; best_it = it; }
          // MIXED, FP32-value phase: no halving of the worst residual in LOB_MIXED_STALL iterations means the
          // FP32 products limit it (a near-degenerate pair at the edge of the block, say); the
          // FP64-class phase takes over from here
          if (o.mode == LOB_MODE_MIXED && phase == 0 && it - best_it >= LOB_MIXED_STALL) {
            run_status = LOB_ERR_NOCONV;
            pc = PC_RUN_END;
            continue;
          }
          if (!pc_dropped && o.precond && it - best_it >= 40) {
            pc_dropped = true;
            if (!stats.precond_dropped) stats.precond_dropped = iters_total + it;
          }
        }
        // W = T^{-1} R (step 6) with the rules of Section 4.3: no preconditioner in the first three
        // iterations of the solve (counted across its phases: the refinement phase continues the
        // same eigenpairs) nor while the first residual is above 1e-1
        const bool pc_on = o.precond && !pc_dropped && M->P.bp > 0 && iters_total + it > 3 && hb->relres[0] <= 1e-1;
        LOB_TRY(stage(skey(1, na, haveP ? 1 : 0, pc_on ? 1 : 0), [&]() -> int {
          {
            Timer t(clk(), st, ph(PH_PRECOND));
            if (pc_on) {
              (k_shifts<<<1, 32, 0, st>>>(nb, o.precond_shift, theta.p, relres_d.p, normH, mu.p), LOB_LAUNCHED());
              LOB_TRY(lob_precond_launch(M, mu.p, R.p, W.p, nb, n_act, o.precond_solve,
                                         o.precond_steps > 0 ? o.precond_steps : 3, st));
            }
            LOB_CUDA(cudaMemcpyAsync(map_d(), hb->map, na * sizeof(int), cudaMemcpyHostToDevice, st));
            (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, pc_on ? W.p : R.p, nb, map_d(), S.p + nb, ldS),
             LOB_LAUNCHED());
          }
          // W <- W - X (X^T W), then Cholesky-QR (step 7)
          {
            Timer t(clk(), st, ph(PH_ORTH));
            LOB_TRY(lob_gram_launch_ws(n_act, nb, S.p, ldS, na, S.p + nb, ldS, Z.p, bmode(), work.p, st));
            (k_proj_coef<<<nblk((nb + na) * na), BS, 0, st>>>(nb, na, Z.p, C2.p), LOB_LAUNCHED());
            LOB_TRY(lincomb_into(nb + na, S.p, ldS, na, C2.p, S.p + nb, ldS));
          }
          LOB_TRY(cholqr_begin(nb, na, Mm.p, Cc.p, thw.p, SLOT_W));
          if (haveP) {
            // P and H P restricted to the active columns, after [X W]; Cholesky-QR of P alongside W's
            (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, P.p, nb, map_d(), S.p + nb + na, ldS),
             LOB_LAUNCHED());
            (k_copy_cols<<<nblk(n_act * na), BS, 0, st>>>(n_act, na, HP.p, nb, map_d(), HS.p + nb + na, ldS),
             LOB_LAUNCHED());
            LOB_TRY(cholqr_begin(nb + na, na, MmP.p, CcP.p, thP.p, SLOT_P));
          }
          return LOB_OK;
        }));
        wretry = false;
        pc = PC_ITER_CHOL;
        return sync_point();
      }
      case PC_ITER_CHOL: {
        clock.resolve();
        if (hb->info[SLOT_W]) {
          if (wretry) { run_status = LOB_ERR_BREAKDOWN; pc = PC_RUN_END; continue; }
          // W lost rank: replace it by seeded random directions
          wretry = true;
          (k_random<<<nblk(n * na), BS, 0, st>>>(n, n_act, nb, ldS, nb, na, 0xB10Cull + it, S.p), LOB_LAUNCHED());
          LOB_TRY(cholqr_begin(nb, na, Mm.p, Cc.p, thw.p, SLOT_W));
          return sync_point();
        }
        m = nb + na;
        const bool pok = haveP && !hb->info[SLOT_P];
        if (haveP && !pok) restarts++;  // P lost rank: drop it for this iteration
        if (pok) m += na;
        LOB_TRY(stage(skey(2, na, pok ? 1 : 0, 0), [&]() -> int {
          LOB_TRY(cholqr_finish(nb, na, false, Cc.p));
          if (pok) LOB_TRY(cholqr_finish(nb + na, na, true, CcP.p));
          return spmm_stage(S.p + nb, ldS, na);
        }));
        pc = PC_ITER_RR;
        return want_spmm(S.p + nb, ldS, HS.p + nb, ldS, na, true);
      }
      case PC_ITER_RR:
        LOB_TRY(stage(skey(3, m, na, 0), [&]() -> int {
          LOB_TRY(spmm_post());
          return rr_begin(m);  // eq. 9, steps 7-8
        }));
        sp_post = nullptr;
        pc = PC_ITER_RR_CHECK;
        return sync_point();
      case PC_ITER_RR_CHECK: {
        clock.resolve();
        if (hb->info[SLOT_RR] && m > nb + na) {  // drop P and retry (restart)
          restarts++;
          m = nb + na;
          LOB_TRY(rr_begin(m));
          return sync_point();
        }
        if (hb->info[SLOT_RR]) { run_status = LOB_ERR_BREAKDOWN; pc = PC_RUN_END; continue; }
        haveP = true;
        it++;
        if (it > run_max) {
          LOB_TRY(update(m));
          pc = PC_ITER_RESID;
          continue;
        }
        // eq. 7, steps 9-10, then steps 4-5 of the next iteration
        LOB_TRY(stage(skey(4, m, 0, 0), [&]() -> int {
          LOB_TRY(update(m));
          return residual_begin();
        }));
        pc = PC_ITER_DECIDE;
        return sync_point();
      }
      case PC_RUN_END: {
        iters_total += it;
        restarts_total += restarts;
        if (o.mode == LOB_MODE_MIXED && phase == 1) stats.refine_iterations = it;
        if (run_status != LOB_OK && run_status != LOB_ERR_NOCONV) { status = run_status; pc = PC_END; continue; }
        // the FP64-class phase, unless the FP32-value phase already met the final tol
        if (o.mode == LOB_MODE_MIXED && phase == 0 && !(run_status == LOB_OK && run_tol <= tol)) {
          phase = 1;
          pc = PC_PHASE;
          continue;
        }
        status = run_status;
        pc = PC_FINISH;
        continue;
      }
      case PC_FINISH: {
        // outputs: X = S[:, :nb], lambda = theta[:k], final residuals
        LOB_TRY(residual_begin());
        if (Xout) {
          (k_copy_cols<<<nblk(n * nb), BS, 0, st>>>(n, nb, S.p, ldS, nullptr, Xout, nb), LOB_LAUNCHED());
          if (n_act < n) LOB_CUDA(cudaMemsetAsync(Xout + n_act * nb, 0, (size_t)(n - n_act) * nb * 8, st));
        }
        LOB_CUDA(cudaMemcpyAsync(hb->theta, theta.p, k * sizeof(double), cudaMemcpyDeviceToHost, st));
        pc = PC_OUT;
        return sync_point();
      }
      case PC_OUT: {
        clock.resolve();
        stats.iterations = iters_total;
        stats.restarts = restarts_total;
        for (int j = 0; j < nb && j < 64; j++) stats.residual[j] = hb->relres[j];
        stats.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        pc = PC_END;
        return LOB_TASK_DONE;
      }
      case PC_END:
      default:
        return LOB_TASK_DONE;
    }
  }
}

int lob_task_create(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0, const lob_solve_opts* o,
                    double* X, int64_t n_act, cudaStream_t st, bool timing, lob_task** out) {
  lob_task* t = new lob_task();
  const int rc = task_init(t, m, k, nb, tol, X0, o, X, n_act, st, timing);
  if (rc != LOB_OK) { delete t; return rc; }
  *out = t;
  return LOB_OK;
}

int lob_task_step(lob_task* t) { return t->step(); }

lob_task* lob_task_leaf(lob_task* t) {
  while (t->child) t = t->child;
  return t;
}

cudaEvent_t lob_task_event(const lob_task* leaf) { return leaf->ev; }

void lob_task_spmm_args(const lob_task* leaf, const lob_matrix** m, const double** X, double** Y, int* ncol,
                        int* mode, int64_t* n_act) {
  *m = leaf->M; *X = leaf->sp_x; *Y = leaf->sp_y; *ncol = leaf->sp_ncol; *mode = leaf->spmm_mode;
  *n_act = leaf->n_act;
}

int lob_task_spmm_direct(lob_task* leaf) {
  Timer t(leaf->clk(), leaf->st, leaf->ph(PH_SPMM));
  Timer tm(leaf->clk(), leaf->st, leaf->timing ? &leaf->stats.spmm_ms_mode[leaf->spmm_mode] : nullptr);
  return lob_spmm_launch(leaf->M, leaf->spmm_mode, leaf->sp_x, leaf->sp_y, leaf->sp_ncol, leaf->n_act, leaf->st);
}

int lob_task_result(const lob_task* t, double* lambda, lob_stats* st) {
  if (t->pc != PC_END) return LOB_ERR_ARG;
  if (t->status == LOB_OK || t->status == LOB_ERR_NOCONV)
    if (lambda) memcpy(lambda, t->hb->theta, t->k * sizeof(double));
  if (st) *st = t->stats;
  return t->status;
}

void lob_task_destroy(lob_task* t) { delete t; }

size_t lob_task_bytes(const lob_matrix* m, int nb, int64_t n_small) {
  const int64_t n = m->T.n;
  size_t d = solver_doubles(n, nb);
  if (n_small > 3 * nb) d += solver_doubles(n, nb);
  else if (n_small > 0) d += 2 * (size_t)n * 64 + 5 * 96 * 96;
  return d * sizeof(double);
}

int lob_solve_impl(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0, const lob_solve_opts* o,
                   double* lambda, double* X, lob_stats* st, int64_t n_act) {
  lob_solve_opts dflt;
  memset(&dflt, 0, sizeof(dflt));
  if (!o) o = &dflt;
  if (!m || !lambda || !X || k < 1 || nb < k || nb > 32 || !(tol > 0.0)) return LOB_ERR_ARG;
  if (n_act < 3 * nb) return LOB_ERR_ARG;
  if (o->mode != LOB_MODE_FP64 && o->mode != LOB_MODE_MIXED) return LOB_ERR_ARG;
  if (o->mode == LOB_MODE_MIXED && (!m->T.v32 || !m->T.v64)) return LOB_ERR_ARG;
  if (o->rr_arith < LOB_ARITH_FP64 || o->rr_arith > LOB_ARITH_DF || o->refine_arith < LOB_ARITH_FP64 ||
      o->refine_arith > LOB_ARITH_DF)
    return LOB_ERR_ARG;
  if (o->mode == LOB_MODE_FP64 && !m->T.v64) return LOB_ERR_ARG;
  if (o->precond && m->P.bp < 1) return LOB_ERR_ARG;
  if (o->n_small_inner < 0 || !(o->guess_tol >= 0.0 && o->guess_tol < 1.0)) return LOB_ERR_ARG;
  if (o->guess_correct < 0 || o->guess_correct > 1 || (o->guess_correct && m->P.bp < 1)) return LOB_ERR_ARG;
  if (o->precond_solve < LOB_PSOLVE_FOM || o->precond_solve > LOB_PSOLVE_ABS || o->precond_steps < 0 ||
      o->precond_steps > 3)
    return LOB_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)o->stream;
  lob_task* t = nullptr;
  LOB_TRY(lob_task_create(m, k, nb, tol, X0, o, X, n_act, stream, st != nullptr, &t));
  int rc = LOB_OK;
  for (;;) {
    const int r = lob_task_step(t);
    if (r < 0) { rc = r; break; }
    lob_task* leaf = lob_task_leaf(t);
    if (r == LOB_TASK_SYNC) {
      if (cudaEventSynchronize(leaf->ev) != cudaSuccess) { rc = LOB_ERR_CUDA; break; }
    } else if (r == LOB_TASK_SPMM) {
      rc = lob_task_spmm_direct(leaf);
      if (rc != LOB_OK) break;
    } else {
      rc = lob_task_result(t, lambda, st);
      break;
    }
  }
  lob_task_destroy(t);
  // a product that gave up on a bounded wait voids whatever the iteration made of it
  const int fault = lob_matrix_fault_take(m, stream) | lob_oz_fault_take(stream);
  if (fault != 0) {
    fprintf(stderr, "lob: an SpMM kernel gave up on a bounded wait; the result is not valid\n");
    rc = LOB_ERR_CUDA;
  }
  return rc;
}
