/* Device generator of the seeded synthetic Hamiltonian; same entries as synth_host.c. */
#include <cuda_runtime.h>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>
#include "synth.h"

#define SYN_INVALID 0xFFFFFFFFFFFFFFFFull

__global__ void syn_k_candidates(syn_layout L, int64_t m, uint64_t* keys) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = L.n * (m + 1);
  if (t >= total) return;
  int64_t i = t / (m + 1), d = t % (m + 1);
  uint64_t key;
  if (d == m) {
    key = ((uint64_t)i << 32) | (uint64_t)i;
  } else {
    int64_t j = syn_partner(&L, i, d);
    if (j < 0) key = SYN_INVALID;
    else {
      int64_t a = i < j ? i : j, b = i < j ? j : i;
      key = ((uint64_t)a << 32) | (uint64_t)b;
    }
  }
  keys[t] = key;
}

__global__ void syn_k_values(syn_layout L, const uint64_t* keys, int64_t nnz, int64_t* rows, int64_t* cols, double* vals) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  uint64_t k = keys[t];
  int64_t i = (int64_t)(k >> 32), j = (int64_t)(k & 0xFFFFFFFFull);
  rows[t] = i;
  cols[t] = j;
  vals[t] = (i == j) ? syn_diag(&L, i) : syn_offdiag(L.seed, i, j);
}

extern "C" int64_t syn_generate_device(const syn_layout* Lp, int64_t* rows, int64_t* cols, double* vals, int64_t cap, void* stream_) {
  if (!Lp || !rows || !cols || !vals) return -1;
  syn_layout L = *Lp;
  cudaStream_t st = (cudaStream_t)stream_;
  int64_t m = syn_draws(&L);
  int64_t total = L.n * (m + 1);
  if (cap < total) return -1;
  uint64_t *k0 = nullptr, *k1 = nullptr;
  int64_t* d_num = nullptr;
  void* tmp = nullptr;
  size_t tmp_sort = 0, tmp_sel = 0;
  int64_t nnz = -3;
  if (cudaMalloc(&k0, (size_t)total * 8) != cudaSuccess || cudaMalloc(&k1, (size_t)total * 8) != cudaSuccess ||
      cudaMalloc(&d_num, sizeof(int64_t)) != cudaSuccess) { nnz = -2; goto done; }
  {
    int bs = 256;
    syn_k_candidates<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(L, m, k0);
    cub::DoubleBuffer<uint64_t> db(k0, k1);
    if (cub::DeviceRadixSort::SortKeys(nullptr, tmp_sort, db, total, 0, 64, st) != cudaSuccess) goto done;
    if (cub::DeviceSelect::Unique(nullptr, tmp_sel, k0, k1, d_num, total, st) != cudaSuccess) goto done;
    size_t tb = tmp_sort > tmp_sel ? tmp_sort : tmp_sel;
    if (cudaMalloc(&tmp, tb) != cudaSuccess) { nnz = -2; goto done; }
    if (cub::DeviceRadixSort::SortKeys(tmp, tb, db, total, 0, 64, st) != cudaSuccess) goto done;
    uint64_t* sorted = db.Current();
    uint64_t* uniq = (sorted == k0) ? k1 : k0;
    if (cub::DeviceSelect::Unique(tmp, tb, sorted, uniq, d_num, total, st) != cudaSuccess) goto done;
    int64_t nsel = 0;
    if (cudaMemcpyAsync(&nsel, d_num, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess) goto done;
    if (cudaStreamSynchronize(st) != cudaSuccess) goto done;
    /* the invalid marker sorts last and is unique: drop it if present */
    uint64_t last = 0;
    if (nsel > 0) {
      if (cudaMemcpyAsync(&last, uniq + nsel - 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) goto done;
      if (cudaStreamSynchronize(st) != cudaSuccess) goto done;
      if (last == SYN_INVALID) nsel--;
    }
    if (nsel > 0) syn_k_values<<<(unsigned)((nsel + bs - 1) / bs), bs, 0, st>>>(L, uniq, nsel, rows, cols, vals);
    if (cudaStreamSynchronize(st) != cudaSuccess) goto done;
    if (cudaGetLastError() != cudaSuccess) goto done;
    nnz = nsel;
  }
done:
  cudaFree(k0); cudaFree(k1); cudaFree(d_num); cudaFree(tmp);
  return nnz;
}
