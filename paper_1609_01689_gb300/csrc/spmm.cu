// Symmetric SpMM Y = H X over the upper-triangle tile store (Sections 4.1-4.2).
//
// Every stored tile T_IJ contributes Y_I += T_IJ X_J and, off the diagonal tile, also
// Y_J += T_IJ^T X_I -- the paper's row pass and column pass over the CSB pointer array,
// here fused into a single pass over the tiles so the matrix streams from HBM once. On a
// diagonal tile the entries with r != c are applied both ways and the diagonal once.
//
// One CTA per tile. The two 256-row slices of X the tile touches are staged in shared
// memory, the tile's entries stream from global memory with one group of NBC lanes per
// entry (one lane per vector column), and both products accumulate into shared-memory
// partials which are flushed to Y with one global atomic per touched (row, column).
//
// MIXED: FP32 values, X rounded to FP32, FP32 products and in-tile sums; the tile partials
// are converted to FP64 and summed across tiles in FP64 (footnote 5 of Section 4.4).
// FP64: every operation in FP64.
#include "common.cuh"

namespace {

template <typename S>
__device__ __forceinline__ void smem_add(S* p, S v) { atomicAdd(p, v); }

template <bool MIXED, int NBC>
__global__ void __launch_bounds__(256) k_spmm_tile(const int32_t* __restrict__ trow, const int32_t* __restrict__ tcol,
                                                   const int64_t* __restrict__ tptr, const uint32_t* __restrict__ rc,
                                                   const double* __restrict__ v64, const float* __restrict__ v32,
                                                   const double* __restrict__ X, double* __restrict__ Y, int nb,
                                                   int64_t n_act) {
  using S = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* XI = reinterpret_cast<S*>(smem_raw);
  S* XJ = XI + LOB_TILE * NBC;
  S* YI = XJ + LOB_TILE * NBC;
  S* YJ = YI + LOB_TILE * NBC;

  const int t = blockIdx.x;
  const int64_t I = trow[t], J = tcol[t];
  if (J * LOB_TILE >= n_act) return;  // tile entirely outside the active leading block
  const int64_t p0 = tptr[t], p1 = tptr[t + 1];
  const bool diag = (I == J);
  const int tid = threadIdx.x;
  const int lane_k = tid % NBC;  // vector column handled by this lane
  const int group = tid / NBC;
  constexpr int GROUPS = 256 / NBC;

  for (int c0 = 0; c0 < nb; c0 += NBC) {
    const int w = (nb - c0) < NBC ? (nb - c0) : NBC;
    for (int idx = tid; idx < LOB_TILE * NBC; idx += 256) {
      const int r = idx / NBC, k = idx % NBC;
      const int64_t gj = J * LOB_TILE + r, gi = I * LOB_TILE + r;
      double xj = (k < w && gj < n_act) ? X[gj * nb + c0 + k] : 0.0;
      XJ[idx] = (S)xj;
      if (!diag) {
        double xi = (k < w && gi < n_act) ? X[gi * nb + c0 + k] : 0.0;
        XI[idx] = (S)xi;
      }
      YI[idx] = (S)0;
      YJ[idx] = (S)0;
    }
    __syncthreads();
    const S* xi_src = diag ? XJ : XI;
    if (lane_k < w) {
      for (int64_t e = p0 + group; e < p1; e += GROUPS) {
        const uint32_t p = rc[e];
        const int r = (int)(p >> 16), c = (int)(p & 0xFFFFu);
        if (I * LOB_TILE + r >= n_act || J * LOB_TILE + c >= n_act) continue;
        const S v = MIXED ? (S)v32[e] : (S)v64[e];
        smem_add(&YI[r * NBC + lane_k], v * XJ[c * NBC + lane_k]);
        if (!diag || r != c) smem_add(&YJ[c * NBC + lane_k], v * xi_src[r * NBC + lane_k]);
      }
    }
    __syncthreads();
    for (int idx = tid; idx < LOB_TILE * NBC; idx += 256) {
      const int r = idx / NBC, k = idx % NBC;
      if (k >= w) continue;
      if (diag) {
        const int64_t g = I * LOB_TILE + r;
        const double s = (double)YI[idx] + (double)YJ[idx];
        if (g < n_act && s != 0.0) atomicAdd(&Y[g * nb + c0 + k], s);
      } else {
        const int64_t gi = I * LOB_TILE + r, gj = J * LOB_TILE + r;
        const double si = (double)YI[idx], sj = (double)YJ[idx];
        if (gi < n_act && si != 0.0) atomicAdd(&Y[gi * nb + c0 + k], si);
        if (gj < n_act && sj != 0.0) atomicAdd(&Y[gj * nb + c0 + k], sj);
      }
    }
    __syncthreads();
  }
}

template <bool MIXED, int NBC>
int launch(const lob_matrix* m, const double* X, double* Y, int nb, int64_t n_act, cudaStream_t st) {
  using S = typename std::conditional<MIXED, float, double>::type;
  const size_t smem = 4ull * LOB_TILE * NBC * sizeof(S);
  auto kern = k_spmm_tile<MIXED, NBC>;
  LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const lob_tiles& T = m->T;
  // tiles of the tile rows that intersect the active leading block
  const int64_t nt_act = (n_act + LOB_TILE - 1) / LOB_TILE;
  const int64_t ntl = m->h_rowptr[nt_act];
  if (ntl > 0)
    (kern<<<(unsigned)ntl, 256, smem, st>>>(T.trow, T.tcol, T.tptr, T.rc, T.v64, T.v32, X, Y, nb, n_act), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

}  // namespace

int lob_spmm_launch(const lob_matrix* m, int mode, const double* X, double* Y, int nb, int64_t n_act,
                    cudaStream_t st) {
  if (nb < 1 || nb > 64 || n_act < 0 || n_act > m->T.n) return LOB_ERR_ARG;
  if (mode == LOB_SPMM_MIXED && !m->T.v32) return LOB_ERR_ARG;
  if (mode == LOB_SPMM_FP64 && !m->T.v64) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_MIXED && mode != LOB_SPMM_FP64) return LOB_ERR_ARG;
  LOB_CUDA(cudaMemsetAsync(Y, 0, (size_t)m->T.n * nb * sizeof(double), st));
  if (mode == LOB_SPMM_MIXED) return nb <= 8 ? launch<true, 8>(m, X, Y, nb, n_act, st) : launch<true, 16>(m, X, Y, nb, n_act, st);
  return nb <= 8 ? launch<false, 8>(m, X, Y, nb, n_act, st) : launch<false, 16>(m, X, Y, nb, n_act, st);
}
