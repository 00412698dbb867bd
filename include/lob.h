/* lob.h -- C ABI of the GB300 block eigensolver library (liblob.so).
 *
 * The library computes the k smallest eigenpairs of a large sparse symmetric matrix H with
 * the preconditioned block LOBPCG method of Shao et al. (Section 3, Algorithm 1). Its hot
 * path is the symmetric sparse-matrix-times-block product Y = H X with only the upper
 * triangle of H stored in CSB-style tiles, each stored tile applied as H_ij and H_ij^T in
 * one pass (Sections 4.1-4.2).
 *
 * Conventions for every entry point:
 *  - Return value: LOB_OK (0) on success, otherwise a negative LOB_ERR_* code; no exception
 *    or abort crosses the ABI. lob_strerror() gives a message for a code.
 *  - "device" pointers are CUDA device (or managed) memory of the current device; "host"
 *    pointers are ordinary CPU memory. The caller owns every buffer it passes in; the library
 *    owns what lob_create allocates, until lob_destroy.
 *  - Block vectors are n x nb, row-major, leading dimension nb (element (i, j) at i*nb + j),
 *    FP64, as the paper stores its vector blocks (Section 4.2, row-major storage).
 *  - stream is a cudaStream_t (NULL = legacy default stream). Calls are asynchronous on it
 *    unless stated; host outputs are valid on return.
 *  - Not thread-safe on one lob_matrix; distinct matrices may be used concurrently.
 */
#ifndef LOB_H
#define LOB_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define LOB_OK 0
#define LOB_ERR_ARG (-1)       /* bad argument: sizes, null pointers, entry below the diagonal,
                                  out of range or duplicated, unsupported option */
#define LOB_ERR_NOMEM (-2)     /* device allocation failed (or an admission budget refused it) */
#define LOB_ERR_CUDA (-3)      /* a CUDA call failed; the CUDA error is logged to stderr */
#define LOB_ERR_NOCONV (-4)    /* iteration limit reached; outputs still hold the last iterate */
#define LOB_ERR_BREAKDOWN (-5) /* the projected Gram matrix stayed indefinite after the restarts */

typedef struct lob_matrix lob_matrix; /* opaque; owns the device tile store */

/* Upper triangle (row <= col) of symmetric H, including the diagonal, as COO. Entries may
 * come in any order; an entry below the diagonal, outside [0, n) or repeated is an error
 * (LOB_ERR_ARG), never summed. on_device = 1: the three arrays are device pointers. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t* row;
  const int64_t* col;
  const double* val;
  int32_t on_device;
} lob_coo;

/* Which value copies the tile store keeps. FP64 is needed by LOB_SPMM_FP64 and by the
 * FP64-class (refinement) products; FP32 by LOB_SPMM_MIXED (Section 4.4, footnote 5). */
#define LOB_VALUES_FP64 1
#define LOB_VALUES_FP32 2
#define LOB_VALUES_BOTH 3

typedef struct {
  int32_t tile;          /* CSB tile size b; 0 = 256. Must be 256 in this version. */
  int32_t values;        /* LOB_VALUES_*; 0 = BOTH */
  int32_t precond_block; /* b_p of the block-diagonal preconditioner (eq. 11), 1..64, dense
                            blocks eigendecomposed at create; 256: the diagonal tiles themselves,
                            solved by FOM or minimal-residual steps on the tile store at each
                            apply (Section 4.3; needs FP32 values; FOM or minimal-residual
                            solves only); 0 = none */
  int32_t wait_log2;     /* log2 of the SM clocks that any wait inside the persistent SpMM kernels
                            may take before the kernel gives up (1..40; 0 = 32, about 2 s). A
                            product that gives up leaves Y invalid and is reported by lob_check,
                            lob_solve or the server (LOB_ERR_CUDA); the context stays usable.
                            -1 is a test mode of that path: the first pipeline stage of every such
                            product waits for data that nothing sends (no copy is issued for it),
                            so the kernel gives up after 2^16 clocks every time. */
  void* stream;          /* cudaStream_t for the build */
} lob_create_opts;

/* Build the device tile store of H (Section 2.2 CSB blocks with fixed b x b tiles; Section
 * 4.2 COO inside each tile with 16-bit in-tile offsets packed as (r << 16) | c), the norm
 * ||H||_inf, and, if precond_block > 0, the block-diagonal preconditioner of eq. 11 (the
 * diagonal b_p x b_p blocks of H, each eigendecomposed once). Synchronous. *out receives the
 * handle. Errors: LOB_ERR_ARG (n < 1, nnz < 1, bad entry, duplicate, tile != 256,
 * precond_block outside [0, 64] and not 256, or 256 without FP32 values), LOB_ERR_NOMEM,
 * LOB_ERR_CUDA. */
int lob_create(const lob_coo* H, const lob_create_opts* opts, lob_matrix** out);

/* Free everything lob_create allocated. NULL is accepted. */
int lob_destroy(lob_matrix* m);

typedef struct {
  int64_t n, nnz, ntiles, n_tile_rows;
  int32_t tile, values, precond_block;
  int32_t perm_chunk;       /* entries per chunk of the kernel-private permutation (lob_export_perm) */
  double norm_inf;          /* max_i sum_j |h_ij| over the full symmetric H */
  int64_t store_bytes;      /* device bytes of the tile store (indices + values kept) */
  int64_t precond_bytes;    /* device bytes of the preconditioner */
} lob_matrix_info;

int lob_matrix_info_get(const lob_matrix* m, lob_matrix_info* out);

/* Copy the canonical tile store to host arrays (caller-allocated, sizes from
 * lob_matrix_info_get): tile_rowptr[n_tile_rows+1] (int64), tile_col[ntiles] (int32),
 * tile_ptr[ntiles+1] (int64), rc[nnz] (uint32), v64[nnz] (double, needs FP64 values),
 * v32[nnz] (float, needs FP32 values). Any pointer may be NULL to skip that array. */
int lob_export_tiles(const lob_matrix* m, int64_t* tile_rowptr, int32_t* tile_col, int64_t* tile_ptr, uint32_t* rc,
                     double* v64, float* v32);

/* Copy the kernel-private column-order permutation to a host uint16 array of nnz entries.
 * The SpMM walks each tile in chunks of perm_chunk entries (lob_matrix_info; the last chunk of a
 * tile may be shorter);
 * for the chunk starting at entry b, perm[b + j] is the chunk-local index of the j-th entry of
 * the chunk in (column, row) order. Derived from the canonical store at create time; exposed
 * so tests can check it against the canonical order. */
int lob_export_perm(const lob_matrix* m, uint16_t* perm);

/* Arithmetic of a product (Section 4.4, footnote 5 sets the paper's pattern). */
#define LOB_SPMM_FP64 0  /* FP64 values, FP64 X, FP64 products and sums (plain FP64) */
#define LOB_SPMM_MIXED 1 /* FP32 values, X rounded to FP32, FP32 products and in-tile sums,
                            tile partials summed across tiles in FP64, FP64 result */
#define LOB_SPMM_DF64 2  /* FP64-class: values and X as double-float pairs (~48 bits), every
                            product and sum in double-float on the FP32 pipes, FP64 result.
                            Needs LOB_VALUES_BOTH. (lob_spmm only.) */

/* Y = H X (Section 4.1: U_i = H_ij W_j and U_j = H_ij^T W_i for every stored tile, here in one
 * pass over the tiles). X, Y: device, n x nb, row-major FP64, must not overlap. 1 <= nb <= 64.
 * The requested value copy must have been kept at create. Asynchronous: a kernel that gives up on
 * a bounded wait (lob_create_opts.wait_log2) cannot be seen here; lob_check reports it. Errors:
 * LOB_ERR_ARG, LOB_ERR_CUDA (a launch failed). */
int lob_spmm(lob_matrix* m, int32_t mode, const double* X, double* Y, int32_t nb, void* stream);

/* Synchronise `stream` and report whether any SpMM kernel on m gave up on a bounded wait since
 * the last check (LOB_ERR_CUDA; the products it took part in are not valid; the flag is then
 * cleared) or not (LOB_OK). The flag belongs to the matrix: products of one matrix running on
 * several streams share it. The tensor-core block products (lob_gram, lob_lincomb) have one such
 * flag per device, checked here too; m may be NULL to check only that one. lob_solve checks both
 * itself. Errors: LOB_ERR_CUDA. */
int lob_check(lob_matrix* m, void* stream);

/* ---- the pieces of one LOBPCG iteration, each exposed for testing and reuse ---- */

/* Block inner product G = A^T B (Section 4.4, the tall-skinny X^T Y): A is n x p (leading
 * dimension lda), B is n x q (ldb), G is p x q row-major. All device. p, q <= 192.
 * mode: LOB_SPMM_FP64 for native FP64 fused multiply-adds; LOB_SPMM_MIXED for FP64-class
 * arithmetic (about 2^-44 relative to |A|^T |B|): on the tensor cores when p, q <= 64 and
 * p q >= 512 (below that the double-float kernel is faster; each
 * operand split exactly into seven bf16 digits per scaling group, the digit products summed
 * exactly in FP32 tensor memory, the levels combined in double-float; Ozaki et al.'s error-free
 * splitting), otherwise double-float on the FP32 pipes; LOB_SPMM_DF64 for that double-float
 * kernel always; LOB_BLAS_TC for the tensor-core kernel whenever p, q <= 64 (LOB_ERR_ARG beyond). The tensor-core path treats entries below 2^-126 of the scale of their group's
 * products as zero. */
int lob_gram(int64_t n, int32_t p, const double* A, int32_t lda, int32_t q, const double* B, int32_t ldb, double* G,
             int32_t mode, void* stream);

#define LOB_BLAS_TC 3 /* lob_gram / lob_lincomb only: the FP64-class tensor-core kernel */

/* Linear combination Y = A C (Section 4.4, eq. 7): A n x p (lda), C p x q row-major, Y n x q
 * (ldy). Device. p, q <= 192. Y must not overlap A. mode as lob_gram (LOB_SPMM_MIXED: tensor
 * cores for p, q <= 64 and p q >= 512, the scaling groups being the rows of A and the columns of
 * C). */
int lob_lincomb(int64_t n, int32_t p, const double* A, int32_t lda, int32_t q, const double* C, double* Y,
                int32_t ldy, int32_t mode, void* stream);

/* Solvers for the shifted block systems of eq. 11 (Sections 3.2, 4.3). */
#define LOB_PSOLVE_FOM 0     /* `steps` FOM iterations from a zero start (the paper's choice) */
#define LOB_PSOLVE_DIRECT 1  /* exact solve */
#define LOB_PSOLVE_MINRES 2  /* `steps` minimal-residual iterations from a zero start (GMRES for
                                a symmetric system) */
#define LOB_PSOLVE_ABS 3     /* |H~_[i] - mu_j I|^{-1}: the direct solve made positive definite */

/* Block-diagonal preconditioner apply of eq. 11: for each diagonal block [i*b_p, (i+1)*b_p)
 * of H and each column j, W_[i](:, j) = approximate solution of
 * (H~_[i] - mu_j I) w = R_[i](:, j) by `solve` (LOB_PSOLVE_*; steps 1..3 for the Krylov
 * solvers, ignored otherwise). All work in the eigendecomposition H~_[i] = Q diag(lambda) Q^T
 * made at create: Krylov spaces of (H~ - mu I, r) map exactly to those of (diag(lambda - mu),
 * Q^T r). FOM falls back to the minimal-residual iterate on a breakdown (a pivot of the
 * projected tridiagonal below 1e-4 of its largest entry). For DIRECT and ABS a shifted
 * eigenvalue with |lambda - mu_j| < 1e-8 ||H|| is replaced by +-1e-8 ||H|| keeping its sign.
 * With precond_block = 256 the blocks are the diagonal 256 x 256 tiles and nothing was
 * factorised: FOM and minimal residual run Lanczos (full reorthogonalisation) with products
 * taken from the tile store, then the same projected solve; DIRECT and ABS are LOB_ERR_ARG.
 * Arithmetic FP32 (Section 4.4, footnote 5), inputs/outputs FP64. R, W: device n x nb; mu:
 * device, nb. Needs precond_block > 0 at create. Errors: LOB_ERR_ARG. */
int lob_precond_apply(lob_matrix* m, const double* mu, const double* R, double* W, int32_t nb, int32_t solve,
                      int32_t steps, void* stream);

/* Rayleigh-Ritz of eq. 9 on the GPU: solve G c = theta M c for symmetric G and
 * positive-definite M (m x m, device, row-major; only the upper triangles are read) by
 * Cholesky M = L L^T, the standard problem L^{-1} G L^{-T}, and cyclic Jacobi. theta (device,
 * m) ascending, C (device, m x m) with C^T M C = I. *info (device int): 0, or j+1 if the
 * Cholesky pivot j was not positive. m <= 192. mode: LOB_SPMM_FP64 for native FP64,
 * LOB_SPMM_MIXED for double-float element arithmetic (FP64 scalars), as lob_gram. */
int lob_rayleigh_ritz(int32_t m, const double* G, const double* M, double* theta, double* C, int32_t* info,
                      int32_t mode, void* stream);

/* lob_rayleigh_ritz without any device allocation. The paper has no counterpart: this is for
 * callers that cannot call cudaMalloc -- code running under an allocator that owns the device
 * memory (a framework's caching allocator, a fixed memory budget), or a latency-critical loop
 * where an allocation's implicit device synchronisation is not acceptable. The caller still
 * passes every input and output (same meaning as lob_rayleigh_ritz). The workspace is a
 * file-scope device array sized for m <= 192 (five 192 x 192 FP64 matrices, 1,474,560 bytes),
 * held by every GPU that loads the library until the process exits; m outside [1, 192]
 * returns LOB_ERR_ARG. The first call on each device looks up the array's device address
 * (with that device current) and keeps it for the rest of the process; make that first call
 * before any stream capture. The kept addresses cover device ordinals 0..63 (a larger ordinal
 * returns LOB_ERR_ARG), and a cudaDeviceReset on a device leaves its kept address stale: do not
 * call this entry point on a device after resetting it. All calls share the array: each call
 * overwrites it completely before reading it, and calls that overlap on the GPU (other streams
 * or host threads using the same device) race on it. */
int lob_rayleigh_ritz_noalloc(int32_t m, const double* G, const double* M, double* theta, double* C,
                              int32_t* info, int32_t mode, void* stream);

/* ---- the solver (Algorithm 1) ---- */

#define LOB_MODE_FP64 0  /* every product in FP64 (the plain solver) */
#define LOB_MODE_MIXED 1 /* FP32-value SpMM with FP64 sums, FP64-class block products, FP64
                            Cholesky-QR factors and Rayleigh-Ritz solves, then refinement
                            iterations with the FP64-value SpMM (Section 4.4, footnote 5) */

/* Arithmetic choices inside LOB_MODE_MIXED (lob_solve_opts.rr_arith / refine_arith). */
#define LOB_ARITH_FP64 0 /* native FP64 (the default) */
#define LOB_ARITH_DF 1   /* double-float on the FP32 pipes (~48-bit significands): faster on this
                            GPU, whose FP64 rate is a small fraction of its FP32 rate */

typedef struct {
  int32_t mode;            /* LOB_MODE_* */
  int32_t precond;         /* 1: block-diagonal preconditioner (needs precond_block at create) */
  int32_t max_iter;        /* 0 = 500 */
  int32_t refine_iter;     /* MIXED: max FP64 refinement iterations; 0 = what max_iter leaves
                              after the FP32-value phase (at least 50) */
  double norm_H;           /* 0: use ||H||_inf */
  int64_t n_small;         /* X0 == NULL: if > 0, the initial guess of eq. 12 from the leading
                              n_small x n_small block (the smaller configuration space,
                              Section 3.3.1); else seeded random vectors */
  uint64_t seed;           /* seed of the random vectors the method draws */
  int32_t precond_shift;   /* 0: mu_j = theta_j; 1: the per-column rules of Section 4.3 */
  int32_t precond_solve;   /* LOB_PSOLVE_* for eq. 11; 0 = FOM (the paper's solver) */
  int32_t precond_steps;   /* Krylov steps for FOM / MINRES, 1..3; 0 = 3 */
  int32_t verbose;
  double mixed_tol;        /* MIXED: relative residual at which the FP32-value phase stops
                              (0 = max(tol, 1e-7); a phase that stalls near its FP32
                              floor hands over to the FP64-class phase earlier) */
  void* stream;
  int64_t n_small_inner;   /* multi-level guess (Section 3.3.1): if 0 < n_small_inner < n_small, the
                              solve on the leading n_small block that makes the eq. 12 guess
                              takes its own guess from the leading n_small_inner block (three
                              LOBPCG runs on nested configuration spaces); 0 = random start.
                              lob_solve only: the server's engine keeps the one-level guess */
  double guess_tol;        /* relative residual to which the leading-block solves of the guess
                              run, in [0, 1); 0 = 1e-3. A nested guess whose coupling
                              ||H_21|| / ||H|| is small pays off only with a tighter value.
                              lob_solve only */
  int32_t rr_arith;        /* MIXED: LOB_ARITH_* of the small dense solves -- the Cholesky factor of
                              Cholesky-QR and the 3nb x 3nb Rayleigh-Ritz eigenproblem (eq. 9) */
  int32_t refine_arith;    /* MIXED: LOB_ARITH_* of the refinement phase's SpMM (FP64 values, or
                              double-float values and products, LOB_SPMM_DF64) */
  int32_t guess_correct;   /* with the eq. 12 guess (n_small > 0, X0 == NULL): 1 = start instead from
                              the corrected guess of eq. 13, [X_1; Y_1] with column j of Y_1 equal to
                              -(H_22 - theta_j I)^{-1} H_21 x_j, the linear systems solved
                              approximately by the block-diagonal preconditioner (Section 3.3.1: its
                              W^(0) = -[0; Y_1]; needs precond_block at create, else LOB_ERR_ARG).
                              Costs one SpMM and one preconditioner application. lob_solve only: the
                              server's engines ignore it */
  int32_t reserved2;
} lob_solve_opts;

typedef struct {
  int32_t iterations;       /* total LOBPCG iterations (both phases) */
  int32_t refine_iterations;/* of which FP64 refinement iterations (MIXED) */
  int32_t spmm_calls;
  int32_t restarts;         /* times P was dropped after an indefinite Gram matrix */
  int32_t precond_dropped;  /* iteration at which stagnation turned the preconditioner off (the
                               worst unconverged relative residual of the first k columns had not
                               halved in 40 iterations; it stays off for the rest of that phase);
                               0 if it never happened */
  int32_t reserved;
  double time_ms;           /* wall time of lob_solve */
  double phase_ms[8];       /* device time per phase: spmm, gram, rr, update, precond,
                               residual, orth, guess */
  double spmm_bytes;        /* algorithmic bytes moved by all SpMMs */
  int32_t spmm_calls_mode[4];   /* per SpMM arithmetic (LOB_SPMM_*): launches, */
  double spmm_ms_mode[4];       /* device time (the Y reset, X staging and kernel), */
  double spmm_bytes_mode[4];    /* and algorithmic bytes */
  double residual[64];      /* final ||H x_j - theta_j x_j|| / (||H|| ||x_j||), FP64 */
  double guess_relres[2];   /* largest relative residual of the first k columns at the start of the
                               solve: [0] of the initial guess (after its Rayleigh-Ritz step), [1] of
                               the eq. 13 corrected guess (0 when guess_correct is off) */
} lob_stats;

/* k smallest eigenpairs of H (Section 3.1 eq. 6; Algorithm 1). 1 <= k <= nb <= 32 (nb - k
 * extra guard vectors, Section 5.2). tol: stop when every one of the first k columns has
 * ||H x_j - theta_j x_j|| <= tol ||H|| ||x_j|| (Section 5). X0: device n x nb or NULL (see
 * n_small). lambda: host, k values ascending. X: device n x nb; columns 0..k-1 are the
 * eigenvectors (unit 2-norm). st may be NULL. Synchronous. Errors: LOB_ERR_ARG,
 * LOB_ERR_NOMEM, LOB_ERR_CUDA, LOB_ERR_NOCONV (outputs hold the last iterate),
 * LOB_ERR_BREAKDOWN. */
int lob_solve(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0, const lob_solve_opts* opts,
              double* lambda, double* X, lob_stats* st);

/* ---- the Lanczos baseline ----
 * The legacy single-vector solver LOBPCG is compared against (Section 1; Section 5.2, Table 3),
 * on the GPU: FP64 SpMV through the tile store, full reorthogonalisation (classical Gram-Schmidt,
 * twice) against all previous Lanczos vectors, and every `check` steps (0 = 10) the k smallest
 * Ritz pairs of the tridiagonal (bisection + inverse iteration on the host); it stops when every
 * Ritz residual estimate beta_j |s_{j,i}| <= tol ||H||_inf, the relative residual lob_solve's
 * test uses. 1 <= k <= 16, max_steps > k (holds n x max_steps doubles). lambda: host, k values
 * ascending. X: device n x k row-major Ritz vectors, or NULL. Needs FP64 values. Errors:
 * LOB_ERR_ARG, LOB_ERR_NOMEM, LOB_ERR_CUDA, LOB_ERR_NOCONV (max_steps reached; outputs filled). */
typedef struct {
  int32_t steps;
  int32_t reserved;
  double time_ms;       /* wall time */
  double spmv_ms;       /* device time of one SpMV (the last one timed) */
  double device_bytes;  /* Lanczos basis bytes */
} lob_lanczos_stats;

int lob_lanczos(lob_matrix* H, int32_t k, double tol, int32_t max_steps, int32_t check, uint64_t seed,
                double* lambda, double* X, lob_lanczos_stats* stats, void* stream);

/* ---- serving: continuous batching of solves ----
 *
 * A server keeps the LOBPCG state of every admitted solve resident on the device (S = [X W P],
 * H S, R, the Ritz values) and advances all of them together. With the lockstep engine (the
 * default) each call of lob_server_progress() runs one iteration of every admitted solve, every
 * kernel of it as one launch over all solves (SpMMs: one launch per arithmetic and vector width,
 * lob_spmm_batch). With the stream engines each solve has its own CUDA stream and each call moves
 * every solve to its next host decision. Requests that arrive while others run are admitted
 * between progress calls as soon as a slot and enough of the device-memory budget are free (any
 * queued request that fits, in arrival order).
 *
 * A solve gives the same result in the mix as alone (lob_solve) up to the rounding of the
 * SpMM's atomic column sums, which are not ordered in either case. */

/* Y_j = H_j X_j for njobs distinct matrices in shared launches (one kernel per arithmetic and
 * vector width; each CTA finds its matrix and tile row in a job table). X[j], Y[j]: device,
 * n_j x nb[j] row-major, 1 <= nb[j] <= 16; mode[j]: LOB_SPMM_*. n_act (NULL: n_j) restricts job j
 * to the leading n_act[j] x n_act[j] block of H_j: rows of X_j at or beyond n_act[j] are never read
 * and rows of Y_j below n_act[j] get that block's product. Runs on `stream` and returns when the
 * products are complete. Errors: LOB_ERR_ARG (null pointers, nb or n_act out of range, a matrix
 * listed twice, missing value copy), LOB_ERR_NOMEM, LOB_ERR_CUDA. */
int lob_spmm_batch(int32_t njobs, lob_matrix* const* H, const double* const* X, double* const* Y,
                   const int32_t* nb, const int32_t* mode, const int64_t* n_act, void* stream);

typedef struct lob_server lob_server; /* opaque */

#define LOB_ENGINE_LOCKSTEP 0  /* every admitted solve advances one iteration per round; each kernel of
                                  the round is one launch for all solves (job tables); three host
                                  synchronisations per round whatever the number of solves */
#define LOB_ENGINE_SHARED 1    /* one CUDA stream per solve, stages replayed as CUDA graphs, SpMMs of
                                  solves that reach them together share launches */
#define LOB_ENGINE_STREAMS 2   /* one CUDA stream per solve, one SpMM launch per solve */

typedef struct {
  uint64_t budget_bytes;   /* device memory the admitted solves may hold (matrix + solver state);
                              0 = 60 GiB */
  int32_t max_active;      /* admitted solves at once; 0 = 64 */
  int32_t engine;          /* LOB_ENGINE_* (0 = lockstep) */
} lob_server_opts;

typedef struct {
  lob_matrix* H;           /* caller-owned; must stay valid until the request is finished */
  int32_t k, nb;           /* 1 <= k <= nb <= 16 */
  double tol;              /* as lob_solve */
  double* X;               /* device n x nb output (eigenvectors), or NULL */
  lob_solve_opts opts;     /* as lob_solve; opts.stream is ignored (the server owns the streams) */
} lob_request;

#define LOB_REQ_QUEUED 1
#define LOB_REQ_RUNNING 2
#define LOB_REQ_DONE 3

typedef struct {
  int32_t state;           /* LOB_REQ_* */
  int32_t rc;              /* when DONE: the solve's return code (as lob_solve) */
  double lambda[16];       /* when DONE: the k smallest eigenvalues */
  lob_stats stats;         /* when DONE: iterations, SpMM counts, final residuals (no phase times) */
  double t_submit_ms, t_admit_ms, t_done_ms; /* server clock (ms since lob_server_create) */
  uint64_t bytes;          /* device bytes charged against the budget */
} lob_result;

typedef struct {
  int64_t submitted, admitted, finished, active, queued;
  uint64_t bytes_in_use, bytes_peak;
  int64_t spmm_launches;   /* SpMM kernel launches made for the solves */
  int64_t spmm_products;   /* SpMM products they computed (one per solve per step) */
  int64_t progress_calls;
  int64_t rounds;          /* lockstep rounds */
  double host_ms;          /* lockstep: host time in rounds outside device waits */
  double wait_ms;          /* lockstep: time waiting for the device */
} lob_server_stats;

/* The server uses the current CUDA device. Errors: LOB_ERR_ARG, LOB_ERR_NOMEM, LOB_ERR_CUDA. */
int lob_server_create(const lob_server_opts* o, lob_server** out);
/* Queue a solve; *id identifies it. The request is copied. Errors: LOB_ERR_ARG (bad sizes, or a
 * solve that could never fit the budget). */
int lob_server_submit(lob_server* s, const lob_request* r, int64_t* id);
/* Admit what fits, then advance the admitted solves: lockstep, one iteration of all of them
 * (blocking); stream engines, each until it waits on the device (wait != 0: if no solve could
 * move, block until the oldest pending device step completes). *n_done (may be NULL) gets the
 * number of solves finished by this call. */
int lob_server_progress(lob_server* s, int32_t wait, int32_t* n_done);
/* State of a request; once DONE has been reported the record is released (the id becomes
 * unknown: LOB_ERR_ARG). */
int lob_server_poll(lob_server* s, int64_t id, lob_result* out);
int lob_server_stats_get(const lob_server* s, lob_server_stats* out);
/* Waits for the device work of every admitted solve, then frees the server. Queued and running
 * requests are dropped. */
int lob_server_destroy(lob_server* s);

/* ---- variable-size CSB blocks with 8 + 8-bit offsets ----
 *
 * A second, compact store of H (Section 2.2: blocks of at most beta rows aligned to the groups
 * of the basis; Section 4.2: two in-block offsets per stored entry). Each group [g_i, g_{i+1})
 * is cut into blocks of at most beta_max <= 256 rows starting at g_i, so no block straddles a
 * group boundary and an entry is one uint16 (r << 8) | c plus its FP32 value: 6 bytes, against
 * 8 for the fixed-tile store's (r << 16) | c and value. Nonzero blocks are kept in (block row,
 * block column) order, entries inside a block in (r, c) order. */
typedef struct lob_vmatrix lob_vmatrix; /* opaque; owns the device block store */

typedef struct {
  int64_t n, nnz, nblocks, ntiles;   /* ntiles: nonzero blocks of the upper triangle */
  int32_t beta_max, reserved;
  int64_t store_bytes;               /* rc16 and values (6 B per entry) + block tables */
  int64_t kernel_bytes;              /* the SpMM's private permutation and chunk pointers */
} lob_vmatrix_info;

/* Build the block store on the current device. group_starts: host, ngroups ascending row
 * indices, the first 0, all < n. H as for lob_create. Synchronous. Errors: LOB_ERR_ARG (bad
 * groups, beta_max outside [1, 256], a bad entry or duplicate), LOB_ERR_NOMEM, LOB_ERR_CUDA. */
int lob_vcreate(const lob_coo* H, const int64_t* group_starts, int32_t ngroups, int32_t beta_max, void* stream,
                lob_vmatrix** out);
int lob_vdestroy(lob_vmatrix* v);
int lob_vinfo(const lob_vmatrix* v, lob_vmatrix_info* out);
/* Copy the store to host arrays (caller-allocated; sizes from lob_vinfo; any may be NULL):
 * bounds[nblocks + 1] block starts, tile_rowptr[nblocks + 1] first nonzero block of each block
 * row, tile_col[ntiles] block column, tile_ptr[ntiles + 1] first entry of each block,
 * rc16[nnz] (r << 8) | c, v32[nnz] values rounded to FP32. */
int lob_vexport(const lob_vmatrix* v, int64_t* bounds, int64_t* tile_rowptr, int32_t* tile_col, int64_t* tile_ptr,
                uint16_t* rc16, float* v32);
/* Y = H X from the block store (Section 4.1: each stored block applied as H_IJ and H_IJ^T in one
 * pass) in the arithmetic of LOB_SPMM_MIXED: FP32 values, X rounded to FP32, FP32 products and
 * in-block sums, block partials summed in FP64. X, Y: device n x nb row-major FP64, 1 <= nb <= 16,
 * not overlapping. Asynchronous on stream. Errors: LOB_ERR_ARG, LOB_ERR_CUDA. */
int lob_vspmm(lob_vmatrix* v, const double* X, double* Y, int32_t nb, void* stream);

/* ---- batched small instances: one persistent schedule for many independent solves ----
 *
 * Many independent small matrices (each n <= 65,535), each solved for its k smallest
 * eigenpairs by the same LOBPCG iteration as lob_solve (Algorithm 1, without preconditioner),
 * all in ONE persistent kernel launch replayed from a CUDA graph: a CTA takes the next
 * instance from an atomic ticket (largest instances first) and runs that instance's whole solve
 * -- SpMM, Gram matrices, linear combinations, Cholesky-QR and the Rayleigh-Ritz solve of eq. 9
 * in FP64 -- then takes the next. The matrices are stored with both triangles in SELL slices
 * (16-bit instance-local column indices, FP32 and FP64 values). Instance results do not depend
 * on which CTA runs them or on the other instances; they do depend on the schedule's thread
 * count (the order of the Gram sums). */
typedef struct lob_batch lob_batch; /* opaque; owns the device store of all instances */

/* Build the store of `count` instances from the upper triangles H[0..count-1] (each as
 * lob_create's input: row <= col, in [0, n), no repeats; host or device per H[i].on_device).
 * 1 <= H[i].n <= 65,535. stream: cudaStream_t of the build. Synchronous. Errors: LOB_ERR_ARG
 * (count < 1, a bad size or entry), LOB_ERR_NOMEM, LOB_ERR_CUDA. */
int lob_batch_create(int32_t count, const lob_coo* H, void* stream, lob_batch** out);
int lob_batch_destroy(lob_batch* b);

typedef struct {
  int32_t k, nb;         /* 1 <= k <= nb <= 8 */
  int32_t mode;          /* LOB_MODE_FP64: FP64 values, products and sums throughout.
                            LOB_MODE_MIXED: an FP32 phase (FP32 values and X in the SpMM, FP32
                            products in the Gram matrices, summed in FP32 over at most 32 rows
                            and in double-float beyond, FP32 linear combinations) until the first k relative residuals reach mixed_tol or
                            stall for 12 iterations, then an FP64-class phase from those vectors to
                            tol: double-float values (the FP32 value and its FP32-rounded
                            remainder), products and sums, ~48 significant bits on the FP32 pipes.
                            The Cholesky factors and Rayleigh-Ritz solves are FP64 in both. */
  int32_t max_iter;      /* per instance, both phases together; 0 = 500 */
  double tol;            /* stop when every one of the first k columns has
                            ||H x_j - theta_j x_j|| <= tol ||H||_inf ||x_j|| */
  double mixed_tol;      /* target of the FP32 phase; 0 = max(tol, 1e-6) */
  uint64_t seed;         /* the random starting blocks (a counter-based hash of seed, instance,
                            row and column) */
  int32_t tile;          /* SELL slice height 8, 16 or 32; 0 = autotuned */
  int32_t threads;       /* threads per CTA, 64..512, a multiple of 32; 0 = autotuned */
  int32_t per_sm;        /* CTAs launched per SM (at most what fits); 0 = autotuned */
  int32_t tune_iter;     /* iterations each candidate schedule runs while the autotuner times it
                            (all instances, mode as requested); 0 = 4 */
  void* stream;
} lob_batch_opts;

typedef struct {
  int32_t tile, threads, per_sm;  /* the schedule that ran */
  int32_t candidates;      /* schedules the autotuner timed in this call (0: none; the batch keeps
                              the first tuned choice for later calls with the same k, nb, mode) */
  double tune_ms;          /* wall time of that tuning */
  double kernel_ms;        /* device time of the schedule (CUDA events around the graph launch) */
  double wall_ms;          /* wall time of the whole call */
  int64_t rows;            /* sum of the instances' n */
  int64_t entries;         /* SELL entries of the slice height used (both triangles, padding) */
  int64_t work_bytes;      /* device workspace of the schedule */
} lob_batch_stats;

/* Solve every instance. Outputs (device, caller-owned): lambda[count][k] ascending per
 * instance; status[count] (LOB_OK, LOB_ERR_NOCONV: the iteration budget ran out, outputs hold
 * the last iterate; LOB_ERR_BREAKDOWN); iters[count][2] (iterations, of which in the phase that
 * ends at tol: FP64-class in MIXED, all in FP64) or
 * NULL; X (rows x nb, row-major, instance i's rows starting at the sum of the earlier n; unit
 * 2-norm columns, the first k the eigenvectors) or NULL. Returns when the schedule is done.
 * st may be NULL. Errors: LOB_ERR_ARG, LOB_ERR_NOMEM, LOB_ERR_CUDA. */
int lob_batch_solve(lob_batch* b, const lob_batch_opts* o, double* lambda, int32_t* status, int32_t* iters,
                    double* X, lob_batch_stats* st);

const char* lob_strerror(int code);

/* Size in bytes of the ABI struct with the given type name ("lob_solve_opts", "lob_stats",
 * ...), so that a binding can check its own layout; 0 for an unknown name or NULL. Host only. */
int64_t lob_struct_size(const char* name);

/* Number of CUDA kernels this library has launched in this process so far (all devices,
 * all threads). Diagnostic: a benchmark reads it before and after a timed region. */
long long lob_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif
