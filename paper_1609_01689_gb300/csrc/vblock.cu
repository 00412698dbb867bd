// Variable-size CSB blocks with 8 + 8-bit in-block offsets (Section 2.2: blocks of at most beta
// rows aligned to the groups of the basis; Section 4.2: each stored entry addressed by its two
// offsets inside the block). The groups here are given by the caller (for the synthetic
// Hamiltonians, the starts of the truncation levels); each group is cut into blocks of at most
// beta_max <= 256 rows, so no block straddles a group boundary and both offsets fit in 8 bits.
//
// Store (all derived on the device from the upper-triangle COO by the tile builder run on the
// block boundaries): nonzero blocks in (block row, block column) order; inside a block the entries
// in (r, c) order, each as one uint16 (r << 8) | c and its FP32 value: 6 bytes per stored entry
// against the fixed-tile store's 4-byte (r << 16) | c. The SpMM's kernel-private column-order
// permutation (2 bytes per entry) and per-chunk row and column starts are kept too.
//
// Product (FP32 values, X rounded to FP32, FP32 products and in-block sums, block partials added
// in FP64, FP64 result -- LOB_SPMM_MIXED's arithmetic): one CTA per block row, the lane group of 4
// owning in-block row g and column g, the row pass over the block's entries in (r, c) order and
// the column pass through the permutation, as the fixed-tile kernel; X_I and X_J are the staged X
// rows from the blocks' starts.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "df.cuh"

struct lob_vmatrix {
  lob_tiles T;                   // block store (tile = block); rc and rv freed after rc16 is derived
  int64_t* bnd = nullptr;        // device [nblk + 1] block starts
  uint16_t* rc16 = nullptr;      // device [nnz + pad] (r << 8) | c
  std::vector<int64_t> h_bnd;
  int64_t nblk = 0;
  int32_t beta_max = 0;
  float* xs = nullptr;           // staged X: (n + 256) x 16 FP32
  size_t xs_bytes = 0;
  int device = 0;
};

namespace {

constexpr int VB_NB = 16;                 // vector columns staged per launch (nb <= 16)
constexpr int VB_G = 4;                   // lanes per group (4 columns each)
constexpr int VB_THREADS = LOB_TILE * VB_G;
constexpr int VB_CH = LOB_PERM_CHUNK;
constexpr int VB_PTRS = 2 * (LOB_TILE + 1);
constexpr size_t VB_XV = sizeof(float) * LOB_TILE * VB_NB;
constexpr size_t VB_XI = 0;
constexpr size_t VB_XJ = VB_XI + VB_XV;                       // 2 buffers
constexpr size_t VB_RC = VB_XJ + 2 * VB_XV;                   // 2 x (CH + 8) uint16
constexpr size_t VB_VV = VB_RC + 2 * 2 * (VB_CH + 8);         // 2 x CH floats
constexpr size_t VB_PM = VB_VV + 2 * 4 * VB_CH;               // 2 x (CH + 8) uint16
constexpr size_t VB_PT = VB_PM + 2 * 2 * (VB_CH + 8);         // 2 x PTRS uint16
constexpr size_t VB_BYTES = VB_PT + 2 * 2 * VB_PTRS;

__device__ __forceinline__ void vb_cp4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void vb_cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void vb_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void vb_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void vb_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__global__ void k_vb_rc16(int64_t nnz, const uint32_t* __restrict__ rc, uint16_t* __restrict__ rc16) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) rc16[k] = (uint16_t)(((rc[k] >> 16) << 8) | (rc[k] & 0xFFu));
}

// Xs (rows x 16 FP32, rounded to nearest) from columns [0, nb) of X (n x nb FP64); zero elsewhere.
__global__ void k_vb_stage(int64_t n, int64_t rows, int nb, const double* __restrict__ X, float* __restrict__ Xs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * VB_NB) return;
  const int64_t i = t / VB_NB;
  const int j = (int)(t % VB_NB);
  Xs[t] = (j < nb && i < n) ? __double2float_rn(X[i * nb + j]) : 0.f;
}

__device__ __forceinline__ void vb_fma(float4& a, float v, const float4& x) {
  a.x = fmaf(v, x.x, a.x); a.y = fmaf(v, x.y, a.y); a.z = fmaf(v, x.z, a.z); a.w = fmaf(v, x.w, a.w);
}

// One CTA per block row I. Group g owns in-block row g and column g:
//   row pass    acc_t += v X_J[c] over row g's entries of the chunk; at block end acc_t is added
//               to the row accumulator (double-float);
//   column pass acc_c += v X_I[r] over column g's entries (through the permutation); at block end
//               it goes to Y_J with FP64 atomics, or, on the diagonal block, into the row accumulator.
__global__ void __launch_bounds__(VB_THREADS, 1)
    k_vspmm(const int64_t* __restrict__ bnd, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol,
            const int64_t* __restrict__ tptr, const int32_t* __restrict__ tchunk, const uint16_t* __restrict__ rc16,
            const float* __restrict__ vals, const uint16_t* __restrict__ cperm, const uint16_t* __restrict__ cptrs,
            const float* __restrict__ Xs, double* __restrict__ Y, int nb) {
  constexpr int XN = LOB_TILE * VB_NB;
  extern __shared__ __align__(16) unsigned char sm[];
  float* XI = reinterpret_cast<float*>(sm + VB_XI);
  float* XJb = reinterpret_cast<float*>(sm + VB_XJ);
  uint16_t* RCb = reinterpret_cast<uint16_t*>(sm + VB_RC);
  float* VVb = reinterpret_cast<float*>(sm + VB_VV);
  uint16_t* PMb = reinterpret_cast<uint16_t*>(sm + VB_PM);
  uint16_t* PTb = reinterpret_cast<uint16_t*>(sm + VB_PT);
  const int64_t I = blockIdx.x;
  const int64_t row0 = bnd[I];
  const int sizeI = (int)(bnd[I + 1] - row0);
  const int tid = threadIdx.x, g = tid / VB_G, gl = tid % VB_G;
  const int64_t t0 = rowptr[I], t1 = rowptr[I + 1];

  // X_I: the 256 staged rows from the block start (rows past the block are never used)
  for (int e = tid * 4; e < XN; e += VB_THREADS * 4) vb_cp16(&XI[e], &Xs[row0 * VB_NB + e]);
  vb_commit();

  auto issue = [&](int64_t t, int64_t k, int buf, int xbuf) {
    const int64_t J = tcol[t];
    if (k == 0 && J != I) {
      float* XJ = XJb + xbuf * XN;
      const float* src = Xs + bnd[J] * VB_NB;
      for (int e = tid * 4; e < XN; e += VB_THREADS * 4) vb_cp16(&XJ[e], &src[e]);
    }
    const int64_t base = tptr[t] + k * VB_CH;
    const int64_t rem = tptr[t + 1] - base;
    const int cnt = (int)(rem < VB_CH ? rem : VB_CH);
    // 16-bit arrays as 32-bit words from the even entry at or below base
    const int64_t wb = base & ~(int64_t)1;
    const int nwords = (int)((base + cnt - wb + 1) / 2);
    uint32_t* RC32 = reinterpret_cast<uint32_t*>(RCb + buf * (VB_CH + 8));
    uint32_t* PM32 = reinterpret_cast<uint32_t*>(PMb + buf * (VB_CH + 8));
    const uint32_t* src_rc = reinterpret_cast<const uint32_t*>(rc16 + wb);
    const uint32_t* src_pm = reinterpret_cast<const uint32_t*>(cperm + wb);
    for (int i = tid; i < nwords; i += VB_THREADS) {
      vb_cp4(&RC32[i], &src_rc[i]);
      vb_cp4(&PM32[i], &src_pm[i]);
    }
    float* VVs = VVb + buf * VB_CH;
    for (int i = tid; i < cnt; i += VB_THREADS) vb_cp4(&VVs[i], &vals[base + i]);
    uint32_t* PT32 = reinterpret_cast<uint32_t*>(PTb + buf * VB_PTRS);
    const uint32_t* srcp = reinterpret_cast<const uint32_t*>(cptrs + (int64_t)(tchunk[t] + k) * VB_PTRS);
    for (int i = tid; i < VB_PTRS / 2; i += VB_THREADS) vb_cp4(&PT32[i], &srcp[i]);
    vb_commit();
  };

  float4 acc_t = make_float4(0.f, 0.f, 0.f, 0.f), acc_c = make_float4(0.f, 0.f, 0.f, 0.f);
  float rh[4] = {0.f, 0.f, 0.f, 0.f}, rl[4] = {0.f, 0.f, 0.f, 0.f};
  int64_t t = t0, k = 0;
  int tl = 0, buf = 0;
  if (t < t1) issue(t, 0, 0, 0);
  while (t < t1) {
    const int64_t J = tcol[t];
    const bool diag = (J == I);
    const bool last = (tptr[t] + (k + 1) * VB_CH >= tptr[t + 1]);
    int64_t tn = t, kn = k + 1;
    int tln = tl;
    if (last) { tn = t + 1; kn = 0; tln = tl + 1; }
    if (tn < t1) { issue(tn, kn, buf ^ 1, tln & 1); vb_wait_1(); } else { vb_wait_all(); }
    __syncthreads();
    const int64_t base = tptr[t] + k * VB_CH;
    const uint16_t* RCs = RCb + buf * (VB_CH + 8) + (int)(base & 1);
    const float* VVs = VVb + buf * VB_CH;
    const uint16_t* PM = PMb + buf * (VB_CH + 8) + (int)(base & 1);
    const uint16_t* PR = PTb + buf * VB_PTRS;
    const uint16_t* PC = PR + (LOB_TILE + 1);
    const float* xj = diag ? XI : XJb + (tl & 1) * XN;
    {  // row pass
      const int s = PR[g], e = PR[g + 1];
#pragma unroll 4
      for (int i = s; i < e; i++) {
        const int c = RCs[i] & 0xFF;
        const float4 x = *reinterpret_cast<const float4*>(&xj[c * VB_NB + gl * 4]);
        vb_fma(acc_t, VVs[i], x);
      }
    }
    {  // column pass
      const int s = PC[g], e = PC[g + 1];
#pragma unroll 4
      for (int i = s; i < e; i++) {
        const int q = PM[i] & (VB_CH - 1);
        const int r = RCs[q] >> 8;
        if (diag && r == g) continue;  // the diagonal entry is applied once (row pass)
        const float4 xi = *reinterpret_cast<const float4*>(&XI[r * VB_NB + gl * 4]);
        vb_fma(acc_c, VVs[q], xi);
      }
    }
    if (last) {
      const float* ta = reinterpret_cast<const float*>(&acc_t);
      const float* ca = reinterpret_cast<const float*>(&acc_c);
      const int sizeJ = (int)(bnd[J + 1] - bnd[J]);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        df_add(rh[q], rl[q], ta[q], 0.f);
        if (diag) df_add(rh[q], rl[q], ca[q], 0.f);
        const int kk = gl * 4 + q;
        if (!diag && kk < nb && g < sizeJ && ca[q] != 0.f)
          atomicAdd(&Y[(bnd[J] + g) * nb + kk], f32_to_f64(ca[q]));
      }
      acc_t = make_float4(0.f, 0.f, 0.f, 0.f);
      acc_c = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();  // this buffer is refilled two chunks from now
    t = tn; k = kn; tl = tln; buf ^= 1;
  }
  vb_wait_all();
  if (g < sizeI) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int kk = gl * 4 + q;
      if (kk >= nb) continue;
      if (rh[q] != 0.f) atomicAdd(&Y[(row0 + g) * nb + kk], f32_to_f64(rh[q]));
      if (rl[q] != 0.f) atomicAdd(&Y[(row0 + g) * nb + kk], f32_to_f64(rl[q]));
    }
  }
}

void vb_release(lob_vmatrix* v) {
  if (!v) return;
  lob_free_tiles(&v->T);
  if (v->bnd) cudaFree(v->bnd);
  if (v->rc16) cudaFree(v->rc16);
  if (v->xs) cudaFree(v->xs);
  delete v;
}

}  // namespace

extern "C" int lob_vcreate(const lob_coo* H, const int64_t* group_starts, int32_t ngroups, int32_t beta_max,
                           void* stream, lob_vmatrix** out) {
  if (!H || !out || !group_starts || ngroups < 1 || beta_max < 1 || beta_max > LOB_TILE) return LOB_ERR_ARG;
  if (H->n < 1 || H->nnz < 1 || !H->row || !H->col || !H->val) return LOB_ERR_ARG;
  if (group_starts[0] != 0) return LOB_ERR_ARG;
  for (int i = 1; i < ngroups; i++)
    if (group_starts[i] <= group_starts[i - 1] || group_starts[i] >= H->n) return LOB_ERR_ARG;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  lob_vmatrix* v = new lob_vmatrix();
  v->beta_max = beta_max;
  cudaGetDevice(&v->device);
  // every group cut into blocks of at most beta_max rows, from the group's start
  for (int i = 0; i < ngroups; i++) {
    const int64_t e = i + 1 < ngroups ? group_starts[i + 1] : H->n;
    for (int64_t b = group_starts[i]; b < e; b += beta_max) v->h_bnd.push_back(b);
  }
  v->h_bnd.push_back(H->n);
  v->nblk = (int64_t)v->h_bnd.size() - 1;
  if (cudaMalloc(&v->bnd, sizeof(int64_t) * (v->nblk + 1)) != cudaSuccess) {
    cudaGetLastError();
    vb_release(v);
    return LOB_ERR_NOMEM;
  }
  if (cudaMemcpyAsync(v->bnd, v->h_bnd.data(), sizeof(int64_t) * (v->nblk + 1), cudaMemcpyHostToDevice, st) !=
      cudaSuccess) {
    vb_release(v);
    return LOB_ERR_CUDA;
  }
  double norm = 0.0;
  int rc = lob_build_tiles(H, LOB_VALUES_FP32, st, &v->T, &norm, v->bnd, v->nblk);
  if (rc != LOB_OK) {
    v->T = lob_tiles();
    vb_release(v);
    return rc;
  }
  const int64_t nnz = v->T.nnz;
  if (cudaMalloc(&v->rc16, (nnz + LOB_STORE_PAD) * 2) != cudaSuccess) {
    cudaGetLastError();
    vb_release(v);
    return LOB_ERR_NOMEM;
  }
  cudaMemsetAsync(v->rc16 + nnz, 0, LOB_STORE_PAD * 2, st);
  k_vb_rc16<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, v->T.rc, v->rc16);
  LOB_LAUNCHED();
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    vb_release(v);
    return LOB_ERR_CUDA;
  }
  // the 32-bit records and the (record, value) pairs of the fixed-tile kernels are not kept
  cudaFree(v->T.rc);
  v->T.rc = nullptr;
  if (v->T.rv) {
    cudaFree(v->T.rv);
    v->T.rv = nullptr;
  }
  v->xs_bytes = sizeof(float) * (size_t)(H->n + LOB_TILE) * VB_NB;
  if (cudaMalloc(&v->xs, v->xs_bytes) != cudaSuccess) {
    cudaGetLastError();
    vb_release(v);
    return LOB_ERR_NOMEM;
  }
  if (cudaFuncSetAttribute(k_vspmm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)VB_BYTES) != cudaSuccess) {
    vb_release(v);
    return LOB_ERR_CUDA;
  }
  *out = v;
  return LOB_OK;
}

extern "C" int lob_vdestroy(lob_vmatrix* v) {
  if (v) {
    cudaDeviceSynchronize();
    vb_release(v);
  }
  return LOB_OK;
}

extern "C" int lob_vinfo(const lob_vmatrix* v, lob_vmatrix_info* o) {
  if (!v || !o) return LOB_ERR_ARG;
  o->n = v->T.n;
  o->nnz = v->T.nnz;
  o->nblocks = v->nblk;
  o->ntiles = v->T.ntiles;
  o->beta_max = v->beta_max;
  o->reserved = 0;
  o->store_bytes = v->T.nnz * 6 + v->T.ntiles * 12 + (v->nblk + 1) * 16;
  o->kernel_bytes = v->T.nnz * 2 + v->T.nchunks * (int64_t)VB_PTRS * 2 + (v->T.ntiles + 1) * 4;
  return LOB_OK;
}

extern "C" int lob_vexport(const lob_vmatrix* v, int64_t* bounds, int64_t* tile_rowptr, int32_t* tile_col,
                           int64_t* tile_ptr, uint16_t* rc16, float* v32) {
  if (!v) return LOB_ERR_ARG;
  const lob_tiles& T = v->T;
  if (bounds) memcpy(bounds, v->h_bnd.data(), sizeof(int64_t) * (v->nblk + 1));
  if (tile_rowptr) LOB_CUDA(cudaMemcpy(tile_rowptr, T.rowptr, (T.nt + 1) * 8, cudaMemcpyDeviceToHost));
  if (tile_col) LOB_CUDA(cudaMemcpy(tile_col, T.tcol, T.ntiles * 4, cudaMemcpyDeviceToHost));
  if (tile_ptr) LOB_CUDA(cudaMemcpy(tile_ptr, T.tptr, (T.ntiles + 1) * 8, cudaMemcpyDeviceToHost));
  if (rc16) LOB_CUDA(cudaMemcpy(rc16, v->rc16, T.nnz * 2, cudaMemcpyDeviceToHost));
  if (v32) LOB_CUDA(cudaMemcpy(v32, T.v32, T.nnz * 4, cudaMemcpyDeviceToHost));
  return LOB_OK;
}

extern "C" int lob_vspmm(lob_vmatrix* v, const double* X, double* Y, int32_t nb, void* stream) {
  if (!v || !X || !Y || nb < 1 || nb > VB_NB) return LOB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = v->T.n, rows = n + LOB_TILE;
  k_vb_stage<<<(unsigned)((rows * VB_NB + 255) / 256), 256, 0, st>>>(n, rows, nb, X, v->xs);
  LOB_LAUNCHED();
  LOB_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * n * nb, st));
  k_vspmm<<<(unsigned)v->nblk, VB_THREADS, VB_BYTES, st>>>(v->bnd, v->T.rowptr, v->T.tcol, v->T.tptr, v->T.tchunk,
                                                            v->rc16, v->T.v32, v->T.cperm, v->T.cptrs, v->xs, Y, nb);
  LOB_LAUNCHED();
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}
