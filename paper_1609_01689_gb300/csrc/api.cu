// C ABI entry points (lob.h): argument checks, ownership, and dispatch to the launchers.
#include <string.h>

#include "common.cuh"

std::atomic<long long> g_lob_launches{0};

extern "C" {

long long lob_kernel_launches(void) { return g_lob_launches.load(); }

int64_t lob_struct_size(const char* name) {
  if (!name) return 0;
  struct E { const char* n; int64_t s; };
  static const E table[] = {
      {"lob_coo", sizeof(lob_coo)},
      {"lob_create_opts", sizeof(lob_create_opts)},
      {"lob_matrix_info", sizeof(lob_matrix_info)},
      {"lob_solve_opts", sizeof(lob_solve_opts)},
      {"lob_stats", sizeof(lob_stats)},
      {"lob_lanczos_stats", sizeof(lob_lanczos_stats)},
      {"lob_server_opts", sizeof(lob_server_opts)},
      {"lob_request", sizeof(lob_request)},
      {"lob_result", sizeof(lob_result)},
      {"lob_server_stats", sizeof(lob_server_stats)},
      {"lob_batch_opts", sizeof(lob_batch_opts)},
      {"lob_batch_stats", sizeof(lob_batch_stats)},
      {"lob_vmatrix_info", sizeof(lob_vmatrix_info)},
  };
  for (const E& e : table)
    if (strcmp(e.n, name) == 0) return e.s;
  return 0;
}

const char* lob_strerror(int code) {
  switch (code) {
    case LOB_OK: return "ok";
    case LOB_ERR_ARG: return "invalid argument";
    case LOB_ERR_NOMEM: return "device memory allocation failed";
    case LOB_ERR_CUDA: return "CUDA error";
    case LOB_ERR_NOCONV: return "iteration limit reached before convergence";
    case LOB_ERR_BREAKDOWN: return "projected Gram matrix indefinite (breakdown)";
    default: return "unknown error";
  }
}

int lob_create(const lob_coo* H, const lob_create_opts* opts, lob_matrix** out) {
  if (!H || !out || H->n < 1 || H->nnz < 1 || !H->row || !H->col || !H->val) return LOB_ERR_ARG;
  lob_create_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.tile != 0 && o.tile != LOB_TILE) return LOB_ERR_ARG;
  const int values = o.values ? o.values : LOB_VALUES_BOTH;
  if (values < 1 || values > 3) return LOB_ERR_ARG;
  if (o.precond_block < 0 || (o.precond_block > 64 && o.precond_block != LOB_TILE)) return LOB_ERR_ARG;
  if (o.precond_block == LOB_TILE && !(values & LOB_VALUES_FP32)) return LOB_ERR_ARG;  // tile mode runs on FP32 values
  if (o.wait_log2 < -1 || o.wait_log2 > 40) return LOB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)o.stream;
  *out = nullptr;

  // one device copy of the COO, shared by the tile build and the preconditioner setup
  lob_coo D = *H;
  int64_t *dr = nullptr, *dc = nullptr;
  double* dv = nullptr;
  if (!H->on_device) {
    if (cudaMalloc(&dr, H->nnz * 8) != cudaSuccess || cudaMalloc(&dc, H->nnz * 8) != cudaSuccess ||
        cudaMalloc(&dv, H->nnz * 8) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(dr); cudaFree(dc); cudaFree(dv);
      return LOB_ERR_NOMEM;
    }
    cudaMemcpyAsync(dr, H->row, H->nnz * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dc, H->col, H->nnz * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dv, H->val, H->nnz * 8, cudaMemcpyHostToDevice, st);
    D.row = dr; D.col = dc; D.val = dv; D.on_device = 1;
  }
  lob_matrix* m = new lob_matrix();
  cudaGetDevice(&m->device);
  m->values = values;
  m->wait_limit = o.wait_log2 > 0 ? (1ll << o.wait_log2) : (o.wait_log2 < 0 ? (1ll << 16) : (1ll << 32));
  m->wait_poison = o.wait_log2 < 0;
  int rc = LOB_OK;
  if (cudaMalloc((void**)&m->status, sizeof(int)) != cudaSuccess || cudaMemset(m->status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rc = LOB_ERR_NOMEM;
  }
  if (rc == LOB_OK) rc = lob_build_tiles(&D, values, st, &m->T, &m->norm_inf, nullptr, 0);
  if (rc == LOB_OK) {
    m->h_rowptr.resize(m->T.nt + 1);
    if (cudaMemcpy(m->h_rowptr.data(), m->T.rowptr, (m->T.nt + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = LOB_ERR_CUDA;
  }
  if (rc == LOB_OK && o.precond_block > 0) rc = lob_build_precond(&D, o.precond_block, H->n, st, &m->P);
  cudaFree(dr); cudaFree(dc); cudaFree(dv);
  if (rc != LOB_OK) {
    lob_free_tiles(&m->T);
    lob_free_precond(&m->P);
    cudaFree(m->status);
    delete m;
    return rc;
  }
  *out = m;
  return LOB_OK;
}

int lob_destroy(lob_matrix* m) {
  if (!m) return LOB_OK;
  cudaFree(m->xs);
  cudaFree(m->status);
  lob_free_tiles(&m->T);
  lob_free_precond(&m->P);
  delete m;
  return LOB_OK;
}

int lob_matrix_info_get(const lob_matrix* m, lob_matrix_info* out) {
  if (!m || !out) return LOB_ERR_ARG;
  memset(out, 0, sizeof(*out));
  out->n = m->T.n; out->nnz = m->T.nnz; out->ntiles = m->T.ntiles; out->n_tile_rows = m->T.nt;
  out->tile = LOB_TILE; out->values = m->values; out->precond_block = m->P.bp; out->perm_chunk = LOB_PERM_CHUNK;
  out->norm_inf = m->norm_inf;
  out->store_bytes = (m->T.nt + 1) * 8 + m->T.ntiles * (4 + 4 + 8) + 8 + m->T.nnz * 4 +
                     (m->T.v64 ? m->T.nnz * 8 : 0) + (m->T.v32 ? m->T.nnz * 4 : 0);  // canonical arrays only
  out->precond_bytes = m->P.Q ? m->P.nblk * (int64_t)m->P.bp * m->P.bp * 4 + m->P.nblk * (int64_t)m->P.bp * 4 : 0;
  return LOB_OK;
}

int lob_export_tiles(const lob_matrix* m, int64_t* tile_rowptr, int32_t* tile_col, int64_t* tile_ptr, uint32_t* rc,
                     double* v64, float* v32) {
  if (!m) return LOB_ERR_ARG;
  const lob_tiles& T = m->T;
  if ((v64 && !T.v64) || (v32 && !T.v32)) return LOB_ERR_ARG;
  if (tile_rowptr) LOB_CUDA(cudaMemcpy(tile_rowptr, T.rowptr, (T.nt + 1) * 8, cudaMemcpyDeviceToHost));
  if (tile_col) LOB_CUDA(cudaMemcpy(tile_col, T.tcol, T.ntiles * 4, cudaMemcpyDeviceToHost));
  if (tile_ptr) LOB_CUDA(cudaMemcpy(tile_ptr, T.tptr, (T.ntiles + 1) * 8, cudaMemcpyDeviceToHost));
  if (rc) LOB_CUDA(cudaMemcpy(rc, T.rc, T.nnz * 4, cudaMemcpyDeviceToHost));
  if (v64) LOB_CUDA(cudaMemcpy(v64, T.v64, T.nnz * 8, cudaMemcpyDeviceToHost));
  if (v32) LOB_CUDA(cudaMemcpy(v32, T.v32, T.nnz * 4, cudaMemcpyDeviceToHost));
  return LOB_OK;
}

int lob_export_perm(const lob_matrix* m, uint16_t* perm) {
  if (!m || !perm || !m->T.cperm) return LOB_ERR_ARG;
  LOB_CUDA(cudaMemcpy(perm, m->T.cperm, m->T.nnz * 2, cudaMemcpyDeviceToHost));
  return LOB_OK;
}

int lob_spmm(lob_matrix* m, int32_t mode, const double* X, double* Y, int32_t nb, void* stream) {
  if (!m || !X || !Y) return LOB_ERR_ARG;
  return lob_spmm_launch(m, mode, X, Y, nb, m->T.n, (cudaStream_t)stream);
}

int lob_check(lob_matrix* m, void* stream) {
  const int fm = m ? lob_matrix_fault_take(m, (cudaStream_t)stream) : 0;
  const int fo = lob_oz_fault_take((cudaStream_t)stream);
  if (fm < 0 || fo < 0) return LOB_ERR_CUDA;
  if (fm || fo) {
    fprintf(stderr, "lob: a %s kernel gave up on a bounded wait; its product is not valid\n",
            fm ? "SpMM" : "tensor-core block");
    return LOB_ERR_CUDA;
  }
  return LOB_OK;
}

int lob_gram(int64_t n, int32_t p, const double* A, int32_t lda, int32_t q, const double* B, int32_t ldb, double* G,
             int32_t mode, void* stream) {
  return lob_gram_launch(n, p, A, lda, q, B, ldb, G, mode, (cudaStream_t)stream);
}

int lob_lincomb(int64_t n, int32_t p, const double* A, int32_t lda, int32_t q, const double* C, double* Y,
                int32_t ldy, int32_t mode, void* stream) {
  return lob_lincomb_launch(n, p, A, lda, q, C, Y, ldy, mode, (cudaStream_t)stream);
}

int lob_precond_apply(lob_matrix* m, const double* mu, const double* R, double* W, int32_t nb, int32_t solve,
                      int32_t steps, void* stream) {
  if (!m || !mu || !R || !W) return LOB_ERR_ARG;
  if (solve == LOB_PSOLVE_DIRECT || solve == LOB_PSOLVE_ABS) steps = 1;
  return lob_precond_launch(m, mu, R, W, nb, m->T.n, solve, steps, (cudaStream_t)stream);
}

int lob_rayleigh_ritz(int32_t m, const double* G, const double* M, double* theta, double* C, int32_t* info,
                      int32_t mode, void* stream) {
  if (m < 1 || m > 192 || !G || !M || !theta || !C || !info) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_FP64 && mode != LOB_SPMM_MIXED) return LOB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* work = nullptr;
  LOB_CUDA(cudaMallocAsync((void**)&work, lob_rr_work_doubles(m) * sizeof(double), st));
  int rc = mode == LOB_SPMM_MIXED ? lob_rr_launch_df(m, G, M, theta, C, info, work, st)
                                  : lob_rr_launch(m, G, M, theta, C, info, work, st);
  cudaFreeAsync(work, st);
  return rc;
}

int lob_solve(lob_matrix* m, int32_t k, int32_t nb, double tol, const double* X0, const lob_solve_opts* opts,
              double* lambda, double* X, lob_stats* st) {
  if (!m) return LOB_ERR_ARG;
  return lob_solve_impl(m, k, nb, tol, X0, opts, lambda, X, st, m->T.n);
}

}  // extern "C"
