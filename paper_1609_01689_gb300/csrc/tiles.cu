// Device build of the CSB-style tile store (Sections 2.2 and 4.2).
//
// Input: upper-triangle COO (row <= col) in any order. Output (canonical order): nonzero
// 256 x 256 tiles sorted by (tile row, tile col); inside a tile the entries sorted by (r, c),
// each with one uint32 (r << 16) | c -- the paper's two 16-bit in-block offsets -- and its
// value in FP64 and/or FP32. One radix sort on a key that concatenates
// (tile row, tile col, r, c) gives this order directly.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_scan.cuh>

#include "common.cuh"

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

template <class T>
int dalloc(DevBuf& b, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc(&b.p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return LOB_ERR_NOMEM;
  }
  return LOB_OK;
}

__global__ void k_keys(int64_t nnz, int64_t n, const int64_t* __restrict__ row, const int64_t* __restrict__ col,
                       int bits_t, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx, int* __restrict__ err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  int64_t i = row[t], j = col[t];
  if (i < 0 || j < 0 || i >= n || j >= n || i > j) {
    atomicOr(err, 1);
    i = 0; j = 0;
  }
  uint64_t tr = (uint64_t)(i >> LOB_TILE_LOG), tc = (uint64_t)(j >> LOB_TILE_LOG);
  uint64_t r = (uint64_t)(i & (LOB_TILE - 1)), c = (uint64_t)(j & (LOB_TILE - 1));
  keys[t] = (tr << (bits_t + 2 * LOB_TILE_LOG)) | (tc << (2 * LOB_TILE_LOG)) | (r << LOB_TILE_LOG) | c;
  idx[t] = (uint32_t)t;
}

__global__ void k_flags(int64_t nnz, const uint64_t* __restrict__ keys, int32_t* __restrict__ flag,
                        int* __restrict__ err) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  uint64_t key = keys[k];
  int f = 1;
  if (k > 0) {
    uint64_t prev = keys[k - 1];
    if (prev == key) atomicOr(err, 2);
    f = (prev >> (2 * LOB_TILE_LOG)) != (key >> (2 * LOB_TILE_LOG));
  }
  flag[k] = f;
}

__global__ void k_fill(int64_t nnz, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx,
                       const int32_t* __restrict__ flag, const int32_t* __restrict__ tid, const double* __restrict__ val,
                       int bits_t, uint32_t* __restrict__ rc, double* __restrict__ v64, float* __restrict__ v32,
                       int64_t* __restrict__ tptr, int32_t* __restrict__ tcol, int32_t* __restrict__ trow) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  uint64_t key = keys[k];
  uint32_t r = (uint32_t)((key >> LOB_TILE_LOG) & (LOB_TILE - 1)), c = (uint32_t)(key & (LOB_TILE - 1));
  rc[k] = (r << 16) | c;
  double v = val[idx[k]];
  if (v64) v64[k] = v;
  if (v32) v32[k] = __double2float_rn(v);
  if (flag[k]) {
    int32_t t = tid[k];
    tptr[t] = k;
    uint64_t tt = key >> (2 * LOB_TILE_LOG);
    tcol[t] = (int32_t)(tt & ((1ull << bits_t) - 1));
    trow[t] = (int32_t)(tt >> bits_t);
  }
}

__global__ void k_rowptr(int64_t nt, int64_t ntiles, const int32_t* __restrict__ trow, int64_t* __restrict__ rowptr,
                         int64_t* __restrict__ tptr, int64_t nnz) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > nt) return;
  // first tile whose row >= r (tiles are sorted by row)
  int64_t lo = 0, hi = ntiles;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (trow[mid] < r) lo = mid + 1; else hi = mid;
  }
  rowptr[r] = lo;
  if (r == 0) tptr[ntiles] = nnz;
}

__global__ void k_absrow(int64_t nnz, const int64_t* __restrict__ row, const int64_t* __restrict__ col,
                         const double* __restrict__ val, double* __restrict__ s) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  double a = fabs(val[t]);
  atomicAdd(&s[row[t]], a);
  if (row[t] != col[t]) atomicAdd(&s[col[t]], a);
}

inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void lob_free_tiles(lob_tiles* T) {
  cudaFree(T->rowptr); cudaFree(T->tcol); cudaFree(T->trow); cudaFree(T->tptr);
  cudaFree(T->rc); cudaFree(T->v64); cudaFree(T->v32);
  *T = lob_tiles();
}

int lob_build_tiles(const lob_coo* H, int values, cudaStream_t st, lob_tiles* T, double* norm_inf) {
  const int64_t n = H->n, nnz = H->nnz;
  if (nnz >= (int64_t)0xFFFFFFFFll) return LOB_ERR_ARG;
  const int64_t nt = (n + LOB_TILE - 1) / LOB_TILE;
  int bits_t = 1;
  while ((1ll << bits_t) < nt) bits_t++;
  if (2 * bits_t + 2 * LOB_TILE_LOG > 64) return LOB_ERR_ARG;
  const int bs = 256;

  // inputs on the device
  DevBuf in_r, in_c, in_v;
  const int64_t *row = H->row, *col = H->col;
  const double* val = H->val;
  if (!H->on_device) {
    LOB_TRY(dalloc<int64_t>(in_r, nnz)); LOB_TRY(dalloc<int64_t>(in_c, nnz)); LOB_TRY(dalloc<double>(in_v, nnz));
    LOB_CUDA(cudaMemcpyAsync(in_r.p, H->row, nnz * 8, cudaMemcpyHostToDevice, st));
    LOB_CUDA(cudaMemcpyAsync(in_c.p, H->col, nnz * 8, cudaMemcpyHostToDevice, st));
    LOB_CUDA(cudaMemcpyAsync(in_v.p, H->val, nnz * 8, cudaMemcpyHostToDevice, st));
    row = (const int64_t*)in_r.p; col = (const int64_t*)in_c.p; val = (const double*)in_v.p;
  }

  DevBuf keys0, keys1, idx0, idx1, flag, tid, err, tmp, rows_abs, dmax;
  LOB_TRY(dalloc<uint64_t>(keys0, nnz)); LOB_TRY(dalloc<uint64_t>(keys1, nnz));
  LOB_TRY(dalloc<uint32_t>(idx0, nnz)); LOB_TRY(dalloc<uint32_t>(idx1, nnz));
  LOB_TRY(dalloc<int>(err, 1));
  LOB_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  (k_keys<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, n, row, col, bits_t, (uint64_t*)keys0.p, (uint32_t*)idx0.p, (int*)err.p), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());

  cub::DoubleBuffer<uint64_t> dk((uint64_t*)keys0.p, (uint64_t*)keys1.p);
  cub::DoubleBuffer<uint32_t> dv((uint32_t*)idx0.p, (uint32_t*)idx1.p);
  const int end_bit = 2 * bits_t + 2 * LOB_TILE_LOG;
  size_t tsort = 0, tscan = 0, tmax = 0;
  LOB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tsort, dk, dv, (int)nnz, 0, end_bit, st));
  LOB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tscan, (int32_t*)nullptr, (int32_t*)nullptr, (int)nnz, st));
  LOB_CUDA(cub::DeviceReduce::Max(nullptr, tmax, (double*)nullptr, (double*)nullptr, (int)n, st));
  size_t tb = tsort > tscan ? tsort : tscan;
  tb = tb > tmax ? tb : tmax;
  LOB_TRY(dalloc<char>(tmp, tb));
  LOB_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, dk, dv, (int)nnz, 0, end_bit, st));
  const uint64_t* skeys = dk.Current();
  const uint32_t* sidx = dv.Current();

  LOB_TRY(dalloc<int32_t>(flag, nnz)); LOB_TRY(dalloc<int32_t>(tid, nnz));
  (k_flags<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, skeys, (int32_t*)flag.p, (int*)err.p), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  LOB_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, tb, (int32_t*)flag.p, (int32_t*)tid.p, (int)nnz, st));
  int32_t last_flag = 0, last_tid = 0;
  int herr = 0;
  LOB_CUDA(cudaMemcpyAsync(&last_flag, (int32_t*)flag.p + nnz - 1, 4, cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaMemcpyAsync(&last_tid, (int32_t*)tid.p + nnz - 1, 4, cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
  LOB_CUDA(cudaStreamSynchronize(st));
  if (herr) return LOB_ERR_ARG;
  const int64_t ntiles = (int64_t)last_tid + last_flag;

  lob_tiles R;
  R.n = n; R.nnz = nnz; R.ntiles = ntiles; R.nt = nt;
  bool ok = cudaMalloc(&R.rowptr, (nt + 1) * 8) == cudaSuccess && cudaMalloc(&R.tcol, ntiles * 4) == cudaSuccess &&
            cudaMalloc(&R.trow, ntiles * 4) == cudaSuccess && cudaMalloc(&R.tptr, (ntiles + 1) * 8) == cudaSuccess &&
            cudaMalloc(&R.rc, nnz * 4) == cudaSuccess;
  if (ok && (values & LOB_VALUES_FP64)) ok = cudaMalloc(&R.v64, nnz * 8) == cudaSuccess;
  if (ok && (values & LOB_VALUES_FP32)) ok = cudaMalloc(&R.v32, nnz * 4) == cudaSuccess;
  if (!ok) { cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM; }
  (k_fill<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, skeys, sidx, (const int32_t*)flag.p, (const int32_t*)tid.p, val,
                                          bits_t, R.rc, R.v64, R.v32, R.tptr, R.tcol, R.trow), LOB_LAUNCHED());
  (k_rowptr<<<nblocks(nt + 1, bs), bs, 0, st>>>(nt, ntiles, R.trow, R.rowptr, R.tptr, nnz), LOB_LAUNCHED());

  // ||H||_inf over the full symmetric matrix
  if (dalloc<double>(rows_abs, n) != LOB_OK || dalloc<double>(dmax, 1) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; }
  cudaMemsetAsync(rows_abs.p, 0, n * 8, st);
  (k_absrow<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, row, col, val, (double*)rows_abs.p), LOB_LAUNCHED());
  cub::DeviceReduce::Max(tmp.p, tb, (double*)rows_abs.p, (double*)dmax.p, (int)n, st);
  double hmax = 0.0;
  cudaMemcpyAsync(&hmax, dmax.p, 8, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    fprintf(stderr, "lob: tile build failed: %s\n", cudaGetErrorString(e));
    lob_free_tiles(&R);
    return LOB_ERR_CUDA;
  }
  *norm_inf = hmax;
  *T = R;
  return LOB_OK;
}
