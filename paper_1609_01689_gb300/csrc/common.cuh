// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <vector>

#include "lob.h"

#define LOB_TILE 256
#define LOB_TILE_LOG 8
// Relative residual to which the eq. 12 guess (the leading n_small block's eigenvectors) is solved.
// The guess cannot be better than eq. 12 itself: on the n = 500,000 workload 1e-3 gives the
// main solve the same iteration count as 1e-4 (21) at a lower cost, and 1e-2 costs 6 more.
#define LOB_GUESS_TOL 1e-3
// Mixed solver, FP32-value phase: default target (relative residual) and the number of
// iterations without the worst residual halving after which it hands over to the FP64-class
// phase. The target sits near the floor of the FP32-value product (values and X rounded to FP32,
// FP32 products and in-tile sums: ~1e-7 of |H||X|); a solve that cannot reach it stalls and hands
// over after LOB_MIXED_STALL iterations instead.
#define LOB_MIXED_TOL 1e-7
#define LOB_MIXED_STALL 12
#define LOB_PERM_CHUNK 4096  // entries per SpMM chunk (column-order permutation granularity)
// Slack entries after every per-entry array of the tile store (and 16 bytes per slack entry
// after the chunk pointers): the SpMM copies 16-byte aligned windows around a chunk and may
// read up to 15 bytes past the last entry.
#define LOB_STORE_PAD 8

// Report a failed CUDA call and return LOB_ERR_CUDA from the enclosing function.
#define LOB_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      fprintf(stderr, "lob: CUDA error %s at %s:%d (%s)\n", cudaGetErrorString(e_), __FILE__,   \
              __LINE__, #call);                                                                 \
      return LOB_ERR_CUDA;                                                                      \
    }                                                                                           \
  } while (0)

// Count of kernel launches made by this library (diagnostic, lob_kernel_launches()).
extern std::atomic<long long> g_lob_launches;
#define LOB_LAUNCHED() g_lob_launches.fetch_add(1, std::memory_order_relaxed)

#define LOB_TRY(expr)       \
  do {                      \
    int rc_ = (expr);       \
    if (rc_ != LOB_OK) return rc_; \
  } while (0)

// Device tile store (canonical order: tiles by (tile row, tile col), entries by (r, c)).
struct lob_tiles {
  int64_t n = 0, nnz = 0, ntiles = 0, nt = 0;  // nt = number of tile rows
  int64_t* rowptr = nullptr;   // [nt+1] first tile of each tile row
  int32_t* tcol = nullptr;     // [ntiles] tile column
  int32_t* trow = nullptr;     // [ntiles] tile row (derived, for per-tile launches)
  int64_t* tptr = nullptr;     // [ntiles+1] first entry of each tile
  uint32_t* rc = nullptr;      // [nnz] (r << 16) | c
  double* v64 = nullptr;       // [nnz] FP64 values (may be null)
  float* v32 = nullptr;        // [nnz] FP32 values (may be null)
  float* v32lo = nullptr;      // [nnz] kernel-private: v64 - v32 rounded to FP32 (with both copies)
  uint2* rv = nullptr;         // [nnz] kernel-private: (rc, bits of v32) pairs (with FP32 values), so
                               // the SpMM reads an entry's position and value in one 8-byte load
  uint16_t* cperm = nullptr;   // [nnz] kernel-private: per chunk of LOB_PERM_CHUNK entries of a tile,
                               // the chunk-local indices of its entries in (c, r) order
  uint2* rvp = nullptr;        // [nnz] kernel-private: rv with every row segment of a chunk reordered
                               // so that entries whose column has the row's parity come first
  uint16_t* cpermp = nullptr;  // [nnz] kernel-private: per chunk, the rvp positions of its entries by
                               // column, each column's entries with the column's row parity first
                               // (two lane groups sharing a quarter-warp then gather X rows from
                               // different halves of the banks in most steps)
  int64_t nchunks = 0;
  int32_t* tchunk = nullptr;   // [ntiles+1] first chunk id of each tile
  uint16_t* cptrs = nullptr;   // [nchunks][2][257] kernel-private: start of each in-tile row in the
                               // chunk's (r, c) order, then of each in-tile column in (c, r) order
};

// Block-diagonal preconditioner of eq. 11: per block i (rows [i*bp, i*bp + m_i)),
// H~_[i] = Q_i diag(lam_i) Q_i^T; Q stored FP32, column-major per block (bp x bp slots).
struct lob_precond {
  int32_t bp = 0;          // block order; LOB_TILE: the diagonal tiles themselves, by Krylov steps
                           // on the tile store (no Q, lam)
  int64_t nblk = 0;
  float* Q = nullptr;      // [nblk * bp * bp]
  float* lam = nullptr;    // [nblk * bp]
  double* dblk = nullptr;  // [nblk * bp * bp] dense FP64 blocks (kept for the oracle-free self test)
};

struct lob_matrix {
  lob_tiles T;
  std::vector<int64_t> h_rowptr;  // host copy of T.rowptr
  lob_precond P;
  int32_t values = LOB_VALUES_BOTH;
  double norm_inf = 0.0;
  int device = 0;
  void* xs = nullptr;      // SpMM scratch: X rounded/staged per call (rows padded to whole tiles)
  size_t xs_bytes = 0;
  int* status = nullptr;   // device word: bit 0 set by an SpMM kernel that gave up on a bounded wait
  long long wait_limit = 1ll << 32;  // SM clocks any wait inside an SpMM kernel may take
  int wait_poison = 0;               // test mode: the first ring stage waits for bytes never sent
};

// One matrix's share of a batched SpMM launch (several matrices' tile rows in one grid).
struct lob_spmm_job {
  const int64_t* rowptr;
  const int32_t* tcol;
  const int64_t* tptr;
  const int32_t* tchunk;
  const uint32_t* rc;
  const void* vals;   // FP32 (MIXED, DF64 high part) or FP64 values
  const void* vlo;    // DF64 low parts
  const uint16_t* cperm;
  const uint16_t* cptrs;
  const void* Xs;     // staged X of this matrix
  double* Y;
  int32_t ldy, c0, w, pad;
  int64_t n_act;
  int64_t cta_begin;  // first CTA of this job in the grid
  // staging (one launch per class before the SpMM): X (n x w, leading dimension w) rounded into Xs
  // with rows >= n_act and columns >= w zeroed, rows padded to whole tiles; Y (n x w) zeroed
  const double* Xsrc;
  int64_t n_rows, rows_pad;
  int64_t stage_begin;  // first CTA of this job in the staging grid
};

// One job of a batched launch (lockstep engine): the fields each kernel uses are listed at the
// kernel; cta_begin is the job's first CTA in the grid (jobs sorted by it).
struct lob_bjob {
  const double* A;
  const double* B;
  const double* C;
  const double* D;
  double* Y;
  double* W0;
  double* W1;
  const void* P0;
  const void* P1;
  int32_t* I0;
  int64_t n;
  int32_t p, q, lda, ldb, ldy, ldd, x0, x1, x2, x3;
  double s0;
  int64_t cta_begin;
};

// ---- internal launchers (return LOB_OK or an error code) ----
// bnd (device, nblk + 1 entries) or null: variable square blocks [bnd[b], bnd[b + 1]) of at most
// LOB_TILE rows in place of the fixed LOB_TILE tiles; "tile row/column" then means block, and the
// in-tile offsets are relative to the block starts.
int lob_build_tiles(const lob_coo* H, int values, cudaStream_t st, lob_tiles* T, double* norm_inf,
                    const int64_t* bnd, int64_t nblk);
void lob_free_tiles(lob_tiles* T);
int lob_build_precond(const lob_coo* Hdev, int bp, int64_t n, cudaStream_t st, lob_precond* P);
void lob_free_precond(lob_precond* P);

// SMs of the current device (-1 if the query fails).
int lob_sm_count();
// Tensor-core FP64-class block products (ozaki.cu): p, q <= 64.
bool lob_oz_fits(int p, int q);
bool lob_oz_pays(int p, int q);
size_t lob_gram_oz_work_doubles();
int lob_gram_oz_launch(int64_t n, int p, const double* L0, int ld0, const double* L1, int ld1, int q,
                       const double* R, int ldr, double* G0, double* G1, double* work, cudaStream_t st);
int lob_lincomb_oz_launch(int64_t n, int p, const double* A, int lda, int q, const double* C, double* Y, int ldy,
                          cudaStream_t st, const double* D = nullptr, int ldd = 0);
int lob_oz_fault_take(cudaStream_t st);

// Grow the matrix's staged-X scratch to at least `need` bytes (synchronous allocation).
int lob_ensure_xs(const lob_matrix* m, size_t need);
// Y = H X over the active leading n_act x n_act block (n_act <= n; rows/cols >= n_act are
// treated as absent). Y is fully written (rows >= n_act get 0).
// Nonzero if an SpMM kernel on m gave up on a bounded wait since the last call (the word is then
// cleared), -1 if the read failed; synchronises st.
int lob_matrix_fault_take(const lob_matrix* m, cudaStream_t st);
int lob_spmm_launch(const lob_matrix* m, int mode, const double* X, double* Y, int nb, int64_t n_act,
                    cudaStream_t st);
// Y_j = H_j X_j for several matrices in as few launches as possible (one per arithmetic
// class); X_j, Y_j contiguous n_j x ncol_j, ncol_j <= 16; nact (nullable) restricts job j to
// its leading nact[j] x nact[j] block. Matrices must be distinct. jobs_dev: device buffer of at least
// njobs lob_spmm_job entries owned by the caller; jobs_host: pinned host buffer of the same size
// that the caller leaves untouched until the stream has passed this launch.
int lob_spmm_batch_launch(const lob_matrix* const* ms, const double* const* X, double* const* Y, const int* ncol,
                          const int* mode, const int64_t* nact, int njobs, lob_spmm_job* jobs_host,
                          lob_spmm_job* jobs_dev, cudaStream_t st, int* n_kernels = nullptr);
// ---- lockstep engine (lockstep.cu): many solves, one iteration per round for all ----
struct lob_engine;
struct lob_ltask;
int lob_engine_create(int cap, cudaStream_t st, lob_engine** out);
void lob_engine_destroy(lob_engine* E);
size_t lob_engine_task_bytes(const lob_matrix* m, int nb, int64_t n_small);
int lob_engine_free_slots(const lob_engine* E);
int lob_engine_add(lob_engine* E, lob_matrix* M, int32_t k, int32_t nb, double tol, const lob_solve_opts* o,
                   double* Xout, int64_t n_act, int64_t user, lob_ltask** out);
int lob_engine_round(lob_engine* E, std::vector<lob_ltask*>& done);
int lob_engine_result(lob_engine* E, lob_ltask* t, double* lambda, lob_stats* st, int64_t* user);
long long lob_engine_spmm_launches(const lob_engine* E);
long long lob_engine_spmm_products(const lob_engine* E);
int lob_engine_ntasks(const lob_engine* E);
void lob_engine_times(const lob_engine* E, double* host_ms, double* wait_ms, long long* rounds);

// ---- resumable LOBPCG task (lobpcg.cu) ----
#define LOB_TASK_SYNC 1  // wait for lob_task_event(leaf), then step again
#define LOB_TASK_SPMM 2  // run the leaf's SpMM (lob_task_spmm_args), then step again
#define LOB_TASK_DONE 3  // lob_task_result
struct lob_task;
int lob_task_create(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0, const lob_solve_opts* o,
                    double* X, int64_t n_act, cudaStream_t st, bool timing, lob_task** out);
int lob_task_step(lob_task* t);
lob_task* lob_task_leaf(lob_task* t);
cudaEvent_t lob_task_event(const lob_task* leaf);
void lob_task_spmm_args(const lob_task* leaf, const lob_matrix** m, const double** X, double** Y, int* ncol,
                        int* mode, int64_t* n_act);
int lob_task_spmm_direct(lob_task* leaf);
int lob_task_result(const lob_task* t, double* lambda, lob_stats* st);
void lob_task_destroy(lob_task* t);
size_t lob_task_bytes(const lob_matrix* m, int nb, int64_t n_small);

int lob_gram_launch(int64_t n, int p, const double* A, int lda, int q, const double* B, int ldb, double* G, int mode,
                    cudaStream_t st);
// Y = A C (+ D when D is given, n x q with leading dimension ldd).
int lob_lincomb_launch(int64_t n, int p, const double* A, int lda, int q, const double* C, double* Y, int ldy,
                       int mode, cudaStream_t st, const double* D = nullptr, int ldd = 0);
int lob_precond_launch(const lob_matrix* m, const double* mu, const double* R, double* W, int nb, int64_t n_act,
                       int solve, int steps, cudaStream_t st);
int lob_rr_launch(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                  cudaStream_t st, int chol_only = 0);
size_t lob_rr_work_doubles(int m);
// Batched block products for the lockstep engine. The launchers fill cta_begin and copy the
// host job tables (pinned, left untouched until the stream passes) to the device tables.
int lob_gram_chunks(int64_t n, int p, int q);
// pairs: use the 2 x 2-block kernel (every job with at most 1,024 blocks); else one tile of
// edge 16, 32 or 48 (pqmax). fused (pairs only): every job computes G = A^T B into Y and
// M = A^T A into D (partials W0 and W1; symmetric, p == q, at most 128 blocks); red_host must
// hold 2 njobs entries.
int lob_gram_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int pqmax, int mode,
                          lob_bjob* red_host, lob_bjob* red_dev, cudaStream_t st, int pairs = 0, int fused = 0);
int lob_lincomb_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int pmax, int qmax, int mode,
                             cudaStream_t st);
int lob_precond_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int bpmax, int nbmax,
                             cudaStream_t st);
// Rayleigh-Ritz / Cholesky-QR problems, one per job and CTA (fields at k_rr_batch).
int lob_rr_batch_launch(const lob_bjob* jobs_dev, int njobs, int mmax, int df, cudaStream_t st);
int lob_rr_launch_df(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                     cudaStream_t st, int chol_only = 0);
size_t lob_gram_work_doubles(int64_t n, int p, int q);
// sym: A^T B is known to be symmetric (p == q) and only its upper triangle is computed; the
// lower one is mirrored.
int lob_gram_launch_ws(int64_t n, int p, const double* A, int lda, int q, const double* B, int ldb, double* G,
                       int mode, double* work, cudaStream_t st, int sym = 0);
int lob_solve_impl(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0,
                              const lob_solve_opts* o, double* lambda, double* X, lob_stats* st, int64_t n_act);
