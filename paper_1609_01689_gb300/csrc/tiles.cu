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

// block of index i under the boundaries bnd[0..nb] (bnd[0] = 0, ascending, gaps <= LOB_TILE):
// the last b with bnd[b] <= i
__device__ __forceinline__ int64_t block_of(const int64_t* __restrict__ bnd, int64_t nb, int64_t i) {
  int64_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (bnd[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Sort key of entry t: (tile row, tile col, r, c). Fixed tiles: tile = i / 256, r = i % 256.
// Variable blocks (bnd != null, nb blocks): tile = the block holding i, r = i - its start.
__global__ void k_keys(int64_t nnz, int64_t n, const int64_t* __restrict__ row, const int64_t* __restrict__ col,
                       int bits_t, const int64_t* __restrict__ bnd, int64_t nb, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx, int* __restrict__ err) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  int64_t i = row[t], j = col[t];
  if (i < 0 || j < 0 || i >= n || j >= n || i > j) {
    atomicOr(err, 1);
    i = 0; j = 0;
  }
  uint64_t tr, tc, r, c;
  if (bnd) {
    const int64_t bi = block_of(bnd, nb, i), bj = block_of(bnd, nb, j);
    tr = (uint64_t)bi; tc = (uint64_t)bj;
    r = (uint64_t)(i - bnd[bi]); c = (uint64_t)(j - bnd[bj]);
  } else {
    tr = (uint64_t)(i >> LOB_TILE_LOG); tc = (uint64_t)(j >> LOB_TILE_LOG);
    r = (uint64_t)(i & (LOB_TILE - 1)); c = (uint64_t)(j & (LOB_TILE - 1));
  }
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

// Key of entry k for the column-order permutation of its chunk: chunks are CH consecutive
// entries of a tile, starting at the tile's first entry; within a chunk, order by (c, r).
__global__ void k_perm_keys(int64_t nnz, const int32_t* __restrict__ flag, const int32_t* __restrict__ tid,
                            const int64_t* __restrict__ tptr, const uint32_t* __restrict__ rc,
                            uint64_t* __restrict__ keys, uint16_t* __restrict__ vals) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int64_t t0 = tptr[tid[k] + flag[k] - 1];  // tile of entry k (tid is the exclusive count of tile starts)
  const int64_t base = t0 + ((k - t0) / LOB_PERM_CHUNK) * LOB_PERM_CHUNK;
  const uint32_t p = rc[k];
  const uint64_t c = p & 0xFFFFu, r = p >> 16;
  keys[k] = ((uint64_t)base << 16) | (c << 8) | r;
  vals[k] = (uint16_t)(k - base);
}

// Keys of the parity orders of the FP32-value ring kernel, per chunk (base = the chunk's first
// entry): rows = (r, [c's parity differs from r's], c), columns = (c, [r's parity differs from c's],
// r). values: the entry (rows) or its rvp position relative to the chunk (columns).
__global__ void k_parity_keys(int64_t nnz, const int32_t* __restrict__ flag, const int32_t* __restrict__ tid,
                              const int64_t* __restrict__ tptr, const uint32_t* __restrict__ rc,
                              const uint32_t* __restrict__ inv, uint64_t* __restrict__ keys,
                              uint32_t* __restrict__ vals32, uint16_t* __restrict__ vals16) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int64_t t0 = tptr[tid[k] + flag[k] - 1];
  const int64_t base = t0 + ((k - t0) / LOB_PERM_CHUNK) * LOB_PERM_CHUNK;
  const uint32_t p = rc[k];
  const uint64_t c = p & 0xFFFFu, r = p >> 16, mm = (r ^ c) & 1u;
  if (!inv) {
    keys[k] = ((uint64_t)base << 17) | (r << 9) | (mm << 8) | c;
    vals32[k] = (uint32_t)k;
  } else {
    keys[k] = ((uint64_t)base << 17) | (c << 9) | (mm << 8) | r;
    vals16[k] = (uint16_t)(inv[k] - (uint32_t)base);
  }
}

// rvp[pos] = rv[perm[pos]] and inv[perm[pos]] = pos
__global__ void k_parity_gather(int64_t nnz, const uint32_t* __restrict__ perm, const uint2* __restrict__ rv,
                                uint2* __restrict__ rvp, uint32_t* __restrict__ inv) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nnz) return;
  const uint32_t k = perm[pos];
  rvp[pos] = rv[k];
  inv[k] = (uint32_t)pos;
}

// Number of SpMM chunks of each tile and the first chunk id of every tile.
__global__ void k_chunk_counts(int64_t ntiles, const int64_t* __restrict__ tptr, int32_t* __restrict__ cnt) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  cnt[t] = (int32_t)((tptr[t + 1] - tptr[t] + LOB_PERM_CHUNK - 1) / LOB_PERM_CHUNK);
}

// One CTA per chunk: where each in-tile row starts in the chunk's (r, c) order and where each
// in-tile column starts in its (c, r) order (exclusive prefix sums of the row and column counts).
__global__ void k_chunk_ptrs(int64_t ntiles, const int64_t* __restrict__ tptr, const int32_t* __restrict__ tchunk,
                             const uint32_t* __restrict__ rc, uint16_t* __restrict__ ptrs) {
  __shared__ int hr[LOB_TILE], hc[LOB_TILE];
  const int64_t ch = blockIdx.x;
  // tile of this chunk: last t with tchunk[t] <= ch
  int64_t lo = 0, hi = ntiles - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (tchunk[mid] <= ch) lo = mid; else hi = mid - 1;
  }
  const int64_t t = lo;
  const int64_t b = tptr[t] + (ch - tchunk[t]) * (int64_t)LOB_PERM_CHUNK;
  const int64_t e = (tptr[t + 1] - b) < LOB_PERM_CHUNK ? tptr[t + 1] : b + LOB_PERM_CHUNK;
  for (int i = threadIdx.x; i < LOB_TILE; i += blockDim.x) { hr[i] = 0; hc[i] = 0; }
  __syncthreads();
  for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) {
    const uint32_t p = rc[k];
    atomicAdd(&hr[p >> 16], 1);
    atomicAdd(&hc[p & 0xFFFFu], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint16_t* pr = ptrs + ch * (2 * (LOB_TILE + 1));
    uint16_t* pc = pr + (LOB_TILE + 1);
    int sr = 0, sc = 0;
    for (int i = 0; i < LOB_TILE; i++) {
      pr[i] = (uint16_t)sr; sr += hr[i];
      pc[i] = (uint16_t)sc; sc += hc[i];
    }
    pr[LOB_TILE] = (uint16_t)sr;
    pc[LOB_TILE] = (uint16_t)sc;
  }
}

// Low parts of the values: v64 - v32, rounded to FP32 (so v32 + v32lo carries ~48 bits).
__global__ void k_value_lo(int64_t nnz, const double* __restrict__ v64, const float* __restrict__ v32,
                           float* __restrict__ lo) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  lo[k] = __double2float_rn(v64[k] - (double)v32[k]);
}

__global__ void k_pack_rv(int64_t nnz, const uint32_t* __restrict__ rc, const float* __restrict__ v32,
                          uint2* __restrict__ rv) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  rv[k] = make_uint2(rc[k], __float_as_uint(v32[k]));
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
  cudaFree(T->rc); cudaFree(T->v64); cudaFree(T->v32); cudaFree(T->cperm);
  cudaFree(T->tchunk); cudaFree(T->cptrs); cudaFree(T->v32lo); cudaFree(T->rv);
  cudaFree(T->rvp); cudaFree(T->cpermp);
  *T = lob_tiles();
}

int lob_build_tiles(const lob_coo* H, int values, cudaStream_t st, lob_tiles* T, double* norm_inf,
                    const int64_t* bnd, int64_t nblk) {
  const int64_t n = H->n, nnz = H->nnz;
  if (nnz >= (int64_t)0xFFFFFFFFll) return LOB_ERR_ARG;
  const int64_t nt = bnd ? nblk : (n + LOB_TILE - 1) / LOB_TILE;
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
  (k_keys<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, n, row, col, bits_t, bnd, nblk, (uint64_t*)keys0.p, (uint32_t*)idx0.p,
                                           (int*)err.p),
   LOB_LAUNCHED());
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
            cudaMalloc(&R.rc, (nnz + LOB_STORE_PAD) * 4) == cudaSuccess;
  if (ok && (values & LOB_VALUES_FP64)) ok = cudaMalloc(&R.v64, (nnz + LOB_STORE_PAD) * 8) == cudaSuccess;
  if (ok && (values & LOB_VALUES_FP32)) ok = cudaMalloc(&R.v32, (nnz + LOB_STORE_PAD) * 4) == cudaSuccess;
  if (!ok) { cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM; }
  (k_fill<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, skeys, sidx, (const int32_t*)flag.p, (const int32_t*)tid.p, val,
                                          bits_t, R.rc, R.v64, R.v32, R.tptr, R.tcol, R.trow), LOB_LAUNCHED());
  (k_rowptr<<<nblocks(nt + 1, bs), bs, 0, st>>>(nt, ntiles, R.trow, R.rowptr, R.tptr, nnz), LOB_LAUNCHED());

  // kernel-private column-order permutation of every chunk (derived from the canonical store)
  if (cudaMalloc(&R.cperm, (nnz + LOB_STORE_PAD) * 2) != cudaSuccess) { cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM; }
  {
    // reuse the sort buffers: keys0/keys1 (uint64) and idx0/idx1 (32-bit slots, used as uint16)
    uint64_t* pk0 = (uint64_t*)keys0.p;
    uint64_t* pk1 = (uint64_t*)keys1.p;
    uint16_t* pv0 = (uint16_t*)idx0.p;
    uint16_t* pv1 = (uint16_t*)idx1.p;
    // the sorted keys/indices still referenced above are no longer needed after k_fill
    LOB_CUDA(cudaStreamSynchronize(st));
    (k_perm_keys<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, (const int32_t*)flag.p, (const int32_t*)tid.p, R.tptr, R.rc, pk0, pv0), LOB_LAUNCHED());
    int ebits = 16;
    while (ebits < 64 && (((uint64_t)nnz) << 16) >> ebits) ebits++;
    cub::DoubleBuffer<uint64_t> pk(pk0, pk1);
    cub::DoubleBuffer<uint16_t> pv(pv0, pv1);
    size_t tp = 0;
    LOB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tp, pk, pv, (int)nnz, 0, ebits, st));
    DevBuf tmp2;
    if (tp > tb) { if (dalloc<char>(tmp2, tp) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; } }
    void* tpp = tp > tb ? tmp2.p : tmp.p;
    size_t tpb = tp > tb ? tp : tb;
    LOB_CUDA(cub::DeviceRadixSort::SortPairs(tpp, tpb, pk, pv, (int)nnz, 0, ebits, st));
    LOB_CUDA(cudaMemcpyAsync(R.cperm, pv.Current(), nnz * 2, cudaMemcpyDeviceToDevice, st));
    LOB_CUDA(cudaStreamSynchronize(st));
  }
  // per-chunk row and column start pointers (kernel-private, derived from the canonical store)
  {
    DevBuf ccount;
    if (dalloc<int32_t>(ccount, ntiles) != LOB_OK || cudaMalloc(&R.tchunk, (ntiles + 1) * 4) != cudaSuccess) {
      cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM;
    }
    (k_chunk_counts<<<nblocks(ntiles, bs), bs, 0, st>>>(ntiles, R.tptr, (int32_t*)ccount.p), LOB_LAUNCHED());
    size_t ts = 0;
    LOB_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, ts, (int32_t*)ccount.p, R.tchunk, (int)ntiles, st));
    DevBuf tmp3;
    if (dalloc<char>(tmp3, ts) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; }
    LOB_CUDA(cub::DeviceScan::ExclusiveSum(tmp3.p, ts, (int32_t*)ccount.p, R.tchunk, (int)ntiles, st));
    int32_t lastc = 0, lastt = 0;
    LOB_CUDA(cudaMemcpyAsync(&lastc, (int32_t*)ccount.p + ntiles - 1, 4, cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaMemcpyAsync(&lastt, R.tchunk + ntiles - 1, 4, cudaMemcpyDeviceToHost, st));
    LOB_CUDA(cudaStreamSynchronize(st));
    const int32_t total_chunks = lastc + lastt;
    R.nchunks = total_chunks;
    LOB_CUDA(cudaMemcpyAsync(R.tchunk + ntiles, &total_chunks, 4, cudaMemcpyHostToDevice, st));
    if (cudaMalloc(&R.cptrs, (size_t)R.nchunks * 2 * (LOB_TILE + 1) * 2 + 16 * LOB_STORE_PAD) != cudaSuccess) {
      cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM;
    }
    (k_chunk_ptrs<<<(unsigned)R.nchunks, 256, 0, st>>>(ntiles, R.tptr, R.tchunk, R.rc, R.cptrs), LOB_LAUNCHED());
    LOB_CUDA(cudaStreamSynchronize(st));
  }

  if (R.v32) {
    if (cudaMalloc(&R.rv, (nnz + LOB_STORE_PAD) * 8) != cudaSuccess) { cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM; }
    (k_pack_rv<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, R.rc, R.v32, R.rv), LOB_LAUNCHED());
  }
  if (R.rv && !bnd) {  // the parity orders of the FP32-value ring kernel (fixed tiles only)
    if (cudaMalloc(&R.rvp, (nnz + LOB_STORE_PAD) * 8) != cudaSuccess ||
        cudaMalloc(&R.cpermp, (nnz + LOB_STORE_PAD) * 2) != cudaSuccess) {
      cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM;
    }
    LOB_CUDA(cudaMemsetAsync(R.rvp + nnz, 0, LOB_STORE_PAD * 8, st));
    LOB_CUDA(cudaMemsetAsync(R.cpermp + nnz, 0, LOB_STORE_PAD * 2, st));
    DevBuf inv;
    if (dalloc<uint32_t>(inv, nnz) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; }
    uint64_t* pk0 = (uint64_t*)keys0.p;
    uint64_t* pk1 = (uint64_t*)keys1.p;
    int ebits = 17;
    while (ebits < 64 && (((uint64_t)nnz) << 17) >> ebits) ebits++;
    // rows: sort (chunk, r, parity mismatch, c) -> entry
    {
      uint32_t* pv0 = (uint32_t*)idx0.p;
      uint32_t* pv1 = (uint32_t*)idx1.p;
      (k_parity_keys<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, (const int32_t*)flag.p, (const int32_t*)tid.p, R.tptr,
                                                      R.rc, nullptr, pk0, pv0, nullptr),
       LOB_LAUNCHED());
      cub::DoubleBuffer<uint64_t> pk(pk0, pk1);
      cub::DoubleBuffer<uint32_t> pv(pv0, pv1);
      size_t tp = 0;
      LOB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tp, pk, pv, (int)nnz, 0, ebits, st));
      DevBuf tmp4;
      if (dalloc<char>(tmp4, tp) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; }
      LOB_CUDA(cub::DeviceRadixSort::SortPairs(tmp4.p, tp, pk, pv, (int)nnz, 0, ebits, st));
      (k_parity_gather<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, pv.Current(), R.rv, R.rvp, (uint32_t*)inv.p),
       LOB_LAUNCHED());
      LOB_CUDA(cudaStreamSynchronize(st));
    }
    // columns: sort (chunk, c, parity mismatch, r) -> rvp position in the chunk
    {
      uint16_t* pv0 = (uint16_t*)idx0.p;
      uint16_t* pv1 = (uint16_t*)idx1.p;
      (k_parity_keys<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, (const int32_t*)flag.p, (const int32_t*)tid.p, R.tptr,
                                                      R.rc, (const uint32_t*)inv.p, pk0, nullptr, pv0),
       LOB_LAUNCHED());
      cub::DoubleBuffer<uint64_t> pk(pk0, pk1);
      cub::DoubleBuffer<uint16_t> pv(pv0, pv1);
      size_t tp = 0;
      LOB_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tp, pk, pv, (int)nnz, 0, ebits, st));
      DevBuf tmp4;
      if (dalloc<char>(tmp4, tp) != LOB_OK) { lob_free_tiles(&R); return LOB_ERR_NOMEM; }
      LOB_CUDA(cub::DeviceRadixSort::SortPairs(tmp4.p, tp, pk, pv, (int)nnz, 0, ebits, st));
      LOB_CUDA(cudaMemcpyAsync(R.cpermp, pv.Current(), nnz * 2, cudaMemcpyDeviceToDevice, st));
      LOB_CUDA(cudaStreamSynchronize(st));
    }
  }
  if (R.v64 && R.v32) {
    if (cudaMalloc(&R.v32lo, (nnz + LOB_STORE_PAD) * 4) != cudaSuccess) { cudaGetLastError(); lob_free_tiles(&R); return LOB_ERR_NOMEM; }
    (k_value_lo<<<nblocks(nnz, bs), bs, 0, st>>>(nnz, R.v64, R.v32, R.v32lo), LOB_LAUNCHED());
  }

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
