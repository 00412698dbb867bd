// Rayleigh-Ritz step of LOBPCG (eq. 9, Algorithm 1 steps 7-8): the generalised symmetric
// eigenproblem G c = theta M c of order m = 3 nb on one CTA -- the kernels and their launchers.
// The device code (rr.cuh): Cholesky M = L L^T (a non-positive pivot j reports info = j + 1),
// A = L^{-1} G L^{-T}, the eigenpairs of A (FP64: FP32 Jacobi refined in FP64; double-float:
// FP32 Jacobi finished by double-float Jacobi), ascending order, C = L^{-T} V. The matrices live
// in shared memory up to m = 64, else in a global workspace of 5 m^2 doubles.
#include <mutex>

#include "common.cuh"
#include "df.cuh"
#include "rr.cuh"

namespace {

constexpr int RR_THREADS = 544;  // at most (every 2x2 block of a round has its thread up to m = 64)

template <bool SMEM>
__global__ void __launch_bounds__(RR_THREADS) k_rayleigh_ritz(int m, const double* __restrict__ G,
                                                              const double* __restrict__ Mi, double* __restrict__ theta,
                                                              double* __restrict__ C, int32_t* __restrict__ info,
                                                              double* __restrict__ work, int chol_only) {
  extern __shared__ __align__(16) unsigned char rr_sm[];
  rr_body<SMEM>(m, G, Mi, theta, C, info, work, chol_only, rr_sm);
}

template <bool SMEM>
__global__ void __launch_bounds__(RR_THREADS) k_rayleigh_ritz_df(int m, const double* __restrict__ G,
                                                                 const double* __restrict__ Mi,
                                                                 double* __restrict__ theta, double* __restrict__ C,
                                                                 int32_t* __restrict__ info, double* __restrict__ work,
                                                                 int chol_only) {
  extern __shared__ __align__(16) unsigned char rr_sm[];
  rr_body_df<SMEM>(m, G, Mi, theta, C, info, work, chol_only, rr_sm);
}

// One Rayleigh-Ritz (or Cholesky-QR) problem per CTA: job j gives m (x0), chol_only (x1), G (A),
// M (B), theta (Y), C (W0), info (I0) and a global workspace (W1, used when m > 64).
template <bool DF, bool SMEM>
__global__ void __launch_bounds__(RR_THREADS) k_rr_batch(const lob_bjob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char rr_sm[];
  const lob_bjob& j = jobs[blockIdx.x];
  if (DF) rr_body_df<SMEM>(j.x0, j.A, j.B, j.Y, j.W0, j.I0, j.W1, j.x1, rr_sm);
  else rr_body<SMEM>(j.x0, j.A, j.B, j.Y, j.W0, j.I0, j.W1, j.x1, rr_sm);
}

}  // namespace

// The m x m matrices live in shared memory when they fit (m <= 64), else in the caller's global
// workspace (L1-cached). Rows padded to m + 1; the FP64 solve keeps five FP64 matrices, the
// double-float one five double-float matrices and one FP32 one.
static size_t rr_smem_bytes(int m, bool df = false) {
  return (df ? 5ull * 8 + 4 : 5ull * 8) * m * (m + 1);
}
static const size_t RR_SMEM_MAX = 200 * 1024;

// Threads for order m: one per 2x2 block of the upper triangle of a Jacobi round, 128 to 512 --
// the kernel is barrier-latency bound, and fewer warps make each barrier cheaper.
static int rr_threads(int m) {
  const int np = (m + 1) / 2;
  int t = ((np * (np + 1) / 2 + 31) / 32) * 32;
  return t < 128 ? 128 : (t > RR_THREADS ? RR_THREADS : t);
}

int lob_rr_launch_df(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                     cudaStream_t st, int chol_only) {
  if (m < 1 || m > 192) return LOB_ERR_ARG;
  const size_t sb = rr_smem_bytes(m, true);
  if (sb <= RR_SMEM_MAX) {
    LOB_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    (k_rayleigh_ritz_df<true><<<1, rr_threads(m), sb, st>>>(m, G, M, theta, C, info, work, chol_only), LOB_LAUNCHED());
  } else {
    (k_rayleigh_ritz_df<false><<<1, rr_threads(m), 0, st>>>(m, G, M, theta, C, info, work, chol_only), LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

size_t lob_rr_work_doubles(int m) { return 5ull * m * m; }

int lob_rr_launch(int m, const double* G, const double* M, double* theta, double* C, int32_t* info, double* work,
                  cudaStream_t st, int chol_only) {
  if (m < 1 || m > 192) return LOB_ERR_ARG;
  const size_t sb = rr_smem_bytes(m);
  if (sb <= RR_SMEM_MAX) {
    LOB_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    (k_rayleigh_ritz<true><<<1, rr_threads(m), sb, st>>>(m, G, M, theta, C, info, work, chol_only), LOB_LAUNCHED());
  } else {
    (k_rayleigh_ritz<false><<<1, rr_threads(m), 0, st>>>(m, G, M, theta, C, info, work, chol_only), LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

// ---- Rayleigh-Ritz without allocation -------------------------------------------------------
// A fixed workspace for lob_rayleigh_ritz_noalloc: five 192 x 192 FP64 matrices (1,474,560 bytes)
// in a file-scope device array, so the call needs no cudaMalloc. Every GPU that loads this
// library holds it until the process exits. All calls share it: the kernel fills it from its
// inputs before reading it, and calls that overlap on the GPU (different streams, or different
// host threads on one device) race on it.
#define LOB_RR_NOALLOC_MAX_M 192
static __device__ __align__(256) double g_rr_scratch[5 * LOB_RR_NOALLOC_MAX_M * LOB_RR_NOALLOC_MAX_M];

namespace {
std::mutex g_rr_scratch_mu;
void* g_rr_scratch_ptr[64] = {nullptr};  // device address of g_rr_scratch, per device ordinal
}  // namespace

extern "C" int lob_rayleigh_ritz_noalloc(int32_t m, const double* G, const double* M, double* theta, double* C,
                                         int32_t* info, int32_t mode, void* stream) {
  if (m < 1 || m > LOB_RR_NOALLOC_MAX_M || !G || !M || !theta || !C || !info) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_FP64 && mode != LOB_SPMM_MIXED) return LOB_ERR_ARG;
  int dev = 0;
  LOB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return LOB_ERR_ARG;
  double* work = nullptr;
  {
    // first call on a device: look up the array's device address with that device current
    std::lock_guard<std::mutex> lock(g_rr_scratch_mu);
    if (!g_rr_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_rr_scratch);
      if (e != cudaSuccess || !ptr) {
        fprintf(stderr, "lob: cudaGetSymbolAddress of the Rayleigh-Ritz workspace failed: %s\n", cudaGetErrorString(e));
        return LOB_ERR_CUDA;
      }
      g_rr_scratch_ptr[dev] = ptr;
    }
    work = static_cast<double*>(g_rr_scratch_ptr[dev]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  return mode == LOB_SPMM_MIXED ? lob_rr_launch_df(m, G, M, theta, C, info, work, st)
                                : lob_rr_launch(m, G, M, theta, C, info, work, st);
}

int lob_rr_batch_launch(const lob_bjob* jobs_dev, int njobs, int mmax, int df, cudaStream_t st) {
  if (njobs <= 0) return LOB_OK;
  if (mmax < 1 || mmax > 192) return LOB_ERR_ARG;
  const size_t sb = rr_smem_bytes(mmax, df != 0);
  const int nt = rr_threads(mmax);
  if (sb <= RR_SMEM_MAX) {
    if (df) {
      LOB_CUDA(cudaFuncSetAttribute(k_rr_batch<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
      (k_rr_batch<true, true><<<njobs, nt, sb, st>>>(jobs_dev), LOB_LAUNCHED());
    } else {
      LOB_CUDA(cudaFuncSetAttribute(k_rr_batch<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
      (k_rr_batch<false, true><<<njobs, nt, sb, st>>>(jobs_dev), LOB_LAUNCHED());
    }
  } else {
    if (df) (k_rr_batch<true, false><<<njobs, nt, 0, st>>>(jobs_dev), LOB_LAUNCHED());
    else (k_rr_batch<false, false><<<njobs, nt, 0, st>>>(jobs_dev), LOB_LAUNCHED());
  }
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}
