/* Seeded synthetic Hamiltonian generator: host and device entry points.
 * Output: the upper triangle (row <= col) including the full diagonal, as COO sorted by
 * (row, col), rows/cols int64, values float64. Host and device outputs are identical.
 * Arrays are caller-owned and must hold syn_candidate_cap(L) entries; the return value is
 * the number of stored entries (negative on error). */
#ifndef SYNTH_H
#define SYNTH_H
#include <stdint.h>
#include "synth_core.h"
#ifdef __cplusplus
extern "C" {
#endif
int syn_layout_init(syn_layout* L, int64_t n, int32_t Q, int32_t nu, int32_t w_min, int32_t w_div, uint64_t seed);
int64_t syn_draws_per_row(const syn_layout* L);
int64_t syn_candidate_cap(const syn_layout* L);
int64_t syn_generate_host(const syn_layout* L, int64_t* rows, int64_t* cols, double* vals, int64_t cap);
/* Device variant: rows/cols/vals are device pointers; stream is a cudaStream_t (may be 0).
 * Returns nnz, or -1 (bad argument), -2 (device allocation failed), -3 (CUDA error). */
int64_t syn_generate_device(const syn_layout* L, int64_t* rows, int64_t* cols, double* vals, int64_t cap, void* stream);
#ifdef __cplusplus
}
#endif
#endif
