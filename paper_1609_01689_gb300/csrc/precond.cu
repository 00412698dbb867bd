// Block-diagonal preconditioner T_j = H~ - mu_j I of Section 3.2 (eq. 11), with H~ the
// diagonal b_p x b_p blocks of H (Section 4.3 builds it from diagonal tiles; here fixed-size
// blocks, the last one partial).
//
// Setup, once per matrix: gather each diagonal block (both triangles) densely and compute
// H~_[i] = Q_i diag(lambda_i) Q_i^T by cyclic Jacobi, one CTA per block, in FP32 -- the paper
// runs the preconditioner in single precision (footnote 5 of Section 4.4). Any solve of eq. 11
// for any shift then works in the block's eigenbasis: W_[i] = Q_i f(Lambda_i - mu_j I) Q_i^T R_[i]
// with f(D) = D^{-1} for a direct solve, or the polynomial that m steps of FOM or of a
// minimal-residual method (the paper's iterative solvers, Sections 3.2 and 4.3, "two or three
// iterations") produce from a zero start -- two small products per block in every case.
#include "common.cuh"
#include "df.cuh"

namespace {

__global__ void k_gather_blocks(int64_t nnz, const int64_t* __restrict__ row, const int64_t* __restrict__ col,
                                const double* __restrict__ val, int bp, double* __restrict__ blk) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  const int64_t i = row[t], j = col[t];
  const int64_t b = i / bp;
  if (j / bp != b) return;
  const int64_t o = b * bp;
  double* B = blk + b * (int64_t)bp * bp;
  B[(i - o) * bp + (j - o)] = val[t];
  B[(j - o) * bp + (i - o)] = val[t];
}

// One CTA per block: FP32 cyclic Jacobi (round-robin order) on the bp x bp block in shared
// memory. Q (column k = eigenvector k) and lambda written per block.
__global__ void __launch_bounds__(256) k_block_eig(int bp, const double* __restrict__ blk, float* __restrict__ Q,
                                                   float* __restrict__ lam) {
  extern __shared__ float sm[];
  float* A = sm;            // bp x bp
  float* V = A + bp * bp;   // bp x bp
  __shared__ float cs_c[32], cs_s[32];
  __shared__ int pr_p[32], pr_q[32];
  __shared__ float red[8];
  __shared__ float s_off, s_fro;
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x, mm = bp * bp;
  const double* B = blk + b * (int64_t)mm;
  for (int e = tid; e < mm; e += nt) {
    A[e] = __double2float_rn(B[e]);
    V[e] = (e / bp == e % bp) ? 1.f : 0.f;
  }
  __syncthreads();
  const int mp = bp + (bp & 1), np = mp / 2;
  for (int sweep = 0; sweep < 30; sweep++) {
    float off = 0.f, fro = 0.f;
    for (int e = tid; e < mm; e += nt) {
      const float x = A[e];
      fro += x * x;
      if (e / bp != e % bp) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) { off += __shfl_down_sync(0xFFFFFFFFu, off, o); fro += __shfl_down_sync(0xFFFFFFFFu, fro, o); }
    if (tid % 32 == 0) red[tid / 32] = off;
    __syncthreads();
    if (tid == 0) { float s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_off = s; }
    __syncthreads();
    if (tid % 32 == 0) red[tid / 32] = fro;
    __syncthreads();
    if (tid == 0) { float s = 0; for (int w = 0; w < nt / 32; w++) s += red[w]; s_fro = s; }
    __syncthreads();
    if (s_off <= 1e-13f * s_fro || s_off == 0.f) break;
    for (int round = 0; round < mp - 1; round++) {
      for (int k = tid; k < np; k += nt) {
        int p = k == 0 ? 0 : 1 + (k - 1 + round) % (mp - 1);
        const int pos = mp - 1 - k;
        int q = pos == 0 ? 0 : 1 + (pos - 1 + round) % (mp - 1);
        if (p > q) { int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < bp) {
          const float apq = A[p * bp + q];
          if (apq != 0.f) {
            const float tau = (A[q * bp + q] - A[p * bp + p]) / (2.f * apq);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        }
        pr_p[k] = p; pr_q[k] = q; cs_c[k] = c; cs_s[k] = s;
      }
      __syncthreads();
      for (int e = tid; e < np * bp; e += nt) {
        const int k = e / bp, col = e % bp, p = pr_p[k], q = pr_q[k];
        if (q >= bp || cs_s[k] == 0.f) continue;
        const float c = cs_c[k], s = cs_s[k], ap = A[p * bp + col], aq = A[q * bp + col];
        A[p * bp + col] = c * ap - s * aq;
        A[q * bp + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = tid; e < np * bp; e += nt) {
        const int k = e / bp, r = e % bp, p = pr_p[k], q = pr_q[k];
        if (q >= bp || cs_s[k] == 0.f) continue;
        const float c = cs_c[k], s = cs_s[k];
        const float ap = A[r * bp + p], aq = A[r * bp + q];
        A[r * bp + p] = c * ap - s * aq;
        A[r * bp + q] = s * ap + c * aq;
        const float vp = V[r * bp + p], vq = V[r * bp + q];
        V[r * bp + p] = c * vp - s * vq;
        V[r * bp + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  float* Qb = Q + b * (int64_t)mm;
  for (int e = tid; e < mm; e += nt) {
    const int k = e / bp, i = e % bp;  // column-major: Qb[k*bp + i] = V[i][k]
    Qb[e] = V[i * bp + k];
  }
  for (int k = tid; k < bp; k += nt) lam[b * bp + k] = A[k * bp + k];
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// Coefficients y of the Krylov iterate w = V y after m Lanczos steps (T = tridiag(al, be),
// be[m-1] coupling to the next vector): FOM solves T y = beta0 e1 by elimination without
// pivoting, and a pivot below 1e-4 max_i(|al_i| + be_i) counts as a FOM breakdown; then, and for
// the minimal-residual solve, y minimises || beta0 e1 - T_bar y || (Givens rotations on the
// (m+1) x m T_bar).
__device__ __forceinline__ void krylov_coeffs(int solve, int m, const float al[3], const float be[3], float beta0, float y[3]) {
  constexpr int KM = 3;
  // tridiagonal T (m x m): diagonal al, off-diagonal be[0..m-2]; T_bar adds the row be[m-1] e_m^T
#pragma unroll
  for (int i = 0; i < KM; i++) y[i] = 0.f;
  bool ok = false;
  float tmax = 0.f;
#pragma unroll
  for (int i = 0; i < KM; i++)
    if (i < m) tmax = fmaxf(tmax, fabsf(al[i]) + be[i]);
  if (solve == LOB_PSOLVE_FOM) {
    // Galerkin: T y = beta0 e1 by elimination without pivoting; a small pivot is a FOM breakdown
    float dg[KM], rhs[KM];
#pragma unroll
    for (int i = 0; i < KM; i++) { dg[i] = 1.f; rhs[i] = i == 0 ? beta0 : 0.f; }
    ok = true;
#pragma unroll
    for (int i = 0; i < KM; i++) {
      if (i >= m) continue;
      dg[i] = al[i];
      if (i > 0) {
        const int ip = i > 0 ? i - 1 : 0;
        const float l = be[ip] / dg[ip];
        dg[i] -= l * be[ip];
        rhs[i] -= l * rhs[ip];
      }
      if (!(fabsf(dg[i]) > 1e-4f * tmax)) ok = false;
    }
    if (ok) {
#pragma unroll
      for (int i = KM - 1; i >= 0; i--) {
        if (i >= m) continue;
        const int in = i + 1 < KM ? i + 1 : i;
        y[i] = (rhs[i] - (i + 1 < m ? be[i] * y[in] : 0.f)) / dg[i];
      }
    }
  }
  if (!ok) {
    // minimal residual: min || beta0 e1 - T_bar y || by Givens rotations on the (m+1) x m T_bar
    float R[KM + 1][KM], g[KM + 1];
#pragma unroll
    for (int i = 0; i <= KM; i++) {
      g[i] = i == 0 ? beta0 : 0.f;
#pragma unroll
      for (int j = 0; j < KM; j++) R[i][j] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < KM; i++) {
      if (i >= m) continue;
      R[i][i] = al[i];
      R[i + 1][i] = be[i];
      if (i + 1 < m) R[i][i + 1 < KM ? i + 1 : i] = be[i];
    }
#pragma unroll
    for (int i = 0; i < KM; i++) {
      if (i >= m) continue;
      const float a = R[i][i], b = R[i + 1][i];
      const float r = sqrtf(a * a + b * b);
      if (!(r > 0.f)) continue;
      const float cs = a / r, sn = b / r;
#pragma unroll
      for (int j = 0; j < KM; j++) {
        if (j < i || j >= m) continue;
        const float p = R[i][j], q = R[i + 1][j];
        R[i][j] = cs * p + sn * q;
        R[i + 1][j] = -sn * p + cs * q;
      }
      const float p = g[i], q = g[i + 1];
      g[i] = cs * p + sn * q;
      g[i + 1] = -sn * p + cs * q;
    }
#pragma unroll
    for (int i = KM - 1; i >= 0; i--) {
      if (i >= m) continue;
      float s2 = g[i];
#pragma unroll
      for (int j = 0; j < KM; j++)
        if (j > i && j < m) s2 -= R[i][j] * y[j];
      y[i] = fabsf(R[i][i]) > 1e-6f * tmax ? s2 / R[i][i] : 0.f;
    }
  }
}

// x = f(D) c for one right-hand side in a block's eigenbasis (D = Lambda - mu I diagonal,
// c = Q^T r), one warp, entries k = lane and lane + 32. The Krylov solvers of eq. 11 with a
// zero start reduce to this basis exactly: K_m(A, r) = Q K_m(D, c), so Lanczos on (D, c)
// gives the FOM (Galerkin) or minimal-residual iterate of (H~ - mu I) w = r after m steps.
__device__ void block_solve(int solve, int steps, float guard, const float d[2], const float c[2], float x[2]) {
  if (solve == LOB_PSOLVE_DIRECT || solve == LOB_PSOLVE_ABS) {
#pragma unroll
    for (int u = 0; u < 2; u++) {
      float dd = d[u];
      if (solve == LOB_PSOLVE_ABS) dd = fabsf(dd);
      if (fabsf(dd) < guard) dd = dd < 0.f ? -guard : guard;
      x[u] = c[u] / dd;
    }
    return;
  }
  // All loops below run to the fixed bound KM = 3 (the most Krylov steps) and test the runtime
  // count inside, so every small array is indexed by constants and stays in registers.
  constexpr int KM = 3;
  x[0] = x[1] = 0.f;
  const float beta0 = sqrtf(warp_sum(c[0] * c[0] + c[1] * c[1]));
  if (!(beta0 > 0.f)) return;
  // Lanczos on (D, c), full reorthogonalisation (at most 3 vectors)
  float v[KM][2], al[KM], be[KM];
#pragma unroll
  for (int i = 0; i < KM; i++) { v[i][0] = v[i][1] = 0.f; al[i] = be[i] = 0.f; }
  v[0][0] = c[0] / beta0;
  v[0][1] = c[1] / beta0;
  int m = 0;
  bool done = false;  // warp-uniform: it depends on warp sums only
#pragma unroll
  for (int i = 0; i < KM; i++) {
    if (done || i >= steps) continue;
    float w[2] = {d[0] * v[i][0], d[1] * v[i][1]};
    al[i] = warp_sum(v[i][0] * w[0] + v[i][1] * w[1]);
    m = i + 1;
#pragma unroll
    for (int t = 0; t < KM; t++) {
      if (t > i) continue;
      const float h = warp_sum(v[t][0] * w[0] + v[t][1] * w[1]);
      w[0] -= h * v[t][0];
      w[1] -= h * v[t][1];
    }
    be[i] = sqrtf(warp_sum(w[0] * w[0] + w[1] * w[1]));
    const float scale = fabsf(al[i]) + (i > 0 ? be[i > 0 ? i - 1 : 0] : 0.f);
    if (i + 1 == steps || !(be[i] > 1e-6f * scale)) {
      if (!(be[i] > 1e-6f * scale)) be[i] = 0.f;  // invariant subspace: both iterates are exact
      done = true;
    } else if (i + 1 < KM) {
      v[i + 1 < KM ? i + 1 : i][0] = w[0] / be[i];
      v[i + 1 < KM ? i + 1 : i][1] = w[1] / be[i];
    }
  }
  float y[KM];
  krylov_coeffs(solve, m, al, be, beta0, y);
#pragma unroll
  for (int i = 0; i < KM; i++) {
    if (i >= m) continue;
    x[0] += y[i] * v[i][0];
    x[1] += y[i] * v[i][1];
  }
}

// W_[i] = Q f(Lambda - mu_j) Q^T R_[i], FP32 arithmetic. f is the exact inverse (a direct solve
// of eq. 11), its absolute value, or the FOM / minimal-residual polynomial of the given number of
// Krylov steps (the paper's iterative solve, Section 4.3). The block is handled by nt threads
// (tid = 0 .. nt-1, whole warps) of the CTA; valid = false makes them pass the barriers only.
__device__ __forceinline__ void block_apply_body(int bp, int64_t n_act, const float* __restrict__ Q,
                                                 const float* __restrict__ lam, const double* __restrict__ mu,
                                                 float guard, const double* __restrict__ R, double* __restrict__ W,
                                                 int nb, int solve, int steps, int64_t b, float* sm, int tid, int nt,
                                                 bool valid) {
  float* Qs = sm;             // bp x bp, column-major (Qs[k*bp + i])
  float* Rs = Qs + bp * bp;   // bp x nb
  float* Ts = Rs + bp * nb;   // bp x nb
  const int64_t o = b * bp;
  if (valid) {
    const float* Qb = Q + b * (int64_t)bp * bp;
    for (int e = tid; e < bp * bp; e += nt) Qs[e] = Qb[e];
    for (int e = tid; e < bp * nb; e += nt) {
      const int i = e / nb, j = e % nb;
      Rs[e] = (o + i < n_act) ? f64_to_f32_rz(R[(o + i) * nb + j]) : 0.f;
    }
  }
  __syncthreads();
  if (valid)
    for (int e = tid; e < bp * nb; e += nt) {  // C = Q^T R
      const int k = e / nb, j = e % nb;
      float sum = 0.f;
      for (int i = 0; i < bp; i++) sum = fmaf(Qs[k * bp + i], Rs[i * nb + j], sum);
      Ts[e] = sum;
    }
  __syncthreads();
  const int warp = tid / 32, lane = tid % 32, nw = nt / 32;
  if (valid)
    for (int j = warp; j < nb; j += nw) {  // T[:, j] = f(Lambda - mu_j) C[:, j], one warp per column
      const float2 m = df_split(mu[j]);
      float d[2], c[2], x[2];
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int k = lane + 32 * u;
        d[u] = k < bp ? __fsub_rn(__fsub_rn(lam[b * bp + k], m.x), m.y) : 0.f;
        c[u] = k < bp ? Ts[k * nb + j] : 0.f;
      }
      block_solve(solve, steps, guard, d, c, x);
#pragma unroll
      for (int u = 0; u < 2; u++) {
        const int k = lane + 32 * u;
        if (k < bp) Ts[k * nb + j] = x[u];
      }
    }
  __syncthreads();
  if (valid)
    for (int e = tid; e < bp * nb; e += nt) {  // W = Q T
      const int i = e / nb, j = e % nb;
      if (o + i >= n_act) continue;
      float sum = 0.f;
      for (int k = 0; k < bp; k++) sum = fmaf(Qs[k * bp + i], Ts[k * nb + j], sum);
      W[(o + i) * nb + j] = f32_to_f64(sum);
    }
}

__global__ void __launch_bounds__(256) k_block_apply(int bp, int64_t n_act, const float* __restrict__ Q,
                                                     const float* __restrict__ lam, const double* __restrict__ mu,
                                                     float guard, const double* __restrict__ R, double* __restrict__ W,
                                                     int nb, int solve, int steps) {
  extern __shared__ float sm[];
  block_apply_body(bp, n_act, Q, lam, mu, guard, R, W, nb, solve, steps, blockIdx.x, sm, threadIdx.x, blockDim.x,
                   true);
}

// Blocks per CTA of the batched apply: with nb <= 8 a block takes 32 nb threads (one warp per
// column in the Krylov solve, one thread per element in the products), and 8 / nb blocks share a
// 256-thread CTA, as many as fit in 48 KB of shared memory.
__host__ __device__ inline int blocks_per_cta(int bp, int nb) {
  if (nb > 8) return 1;
  int k = 8 / nb;
  const int per = (bp * bp + 2 * bp * nb) * 4;
  while (k > 1 && k * per > 48 * 1024) k--;
  return k;
}

// Batched apply: job fields P0 (Q), P1 (lambda), C (mu), A (R), Y (W), x0 (nb), x1 (bp), n (rows),
// s0 (guard), x2 (solve), x3 (steps); ceil(n / bp) CTAs.
__global__ void __launch_bounds__(256) k_block_apply_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  extern __shared__ float sm[];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].cta_begin <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const lob_bjob& j = jobs[lo];
  const int bp = j.x1, nb = j.x0;
  const int bpc = blocks_per_cta(bp, nb);
  const int tpb = nb > 8 ? 256 : 32 * nb;  // threads of one block
  const int sub = threadIdx.x / tpb;
  const int64_t b = ((int64_t)blockIdx.x - j.cta_begin) * bpc + sub;
  const bool valid = sub < bpc && b * bp < j.n;
  block_apply_body(bp, j.n, reinterpret_cast<const float*>(j.P0), reinterpret_cast<const float*>(j.P1), j.C,
                   (float)j.s0, j.A, j.Y, nb, j.x2, j.x3, b, sm + (sub < bpc ? sub : 0) * (bp * bp + 2 * bp * nb),
                   threadIdx.x % tpb, tpb, valid);
}

// Eq. 11 on the diagonal CSB tiles (Sections 3.2 and 4.3: the block-diagonal preconditioner built
// from the diagonal tiles of H, each shifted system solved by two or three FOM iterations from a
// zero start, the iterations of all right-hand sides fused into one tile product each). One CTA per diagonal tile I, 1,024 threads: the lane group g of four lanes owns in-tile
// row g, each lane four of the NB = 16 columns of one pass. A product with the tile uses the tile
// store's own layout -- the row pass over the chunk's row pointers and the column pass through
// its column-order permutation, the stored diagonal applied once -- in FP32 (footnote 5), with
// the pass's Lanczos vectors in shared memory. Per column j: Lanczos on (H~_I - mu_j I, r_j) with
// full reorthogonalisation (classical Gram-Schmidt against the at most three vectors), the
// invariant-subspace test and the projected solve of the eigenbasis path (krylov_coeffs), then
// w_j = V y. Rows at or beyond n_act are outside the operator: their r is zero and every product
// is cut to the active rows.
template <int NB>
struct CfgTF {
  static constexpr int VW = 4, G = NB / VW, THREADS = LOB_TILE * G, NW = THREADS / 32, KM = 3;
  static constexpr size_t V = 0;                                      // [KM][TILE][NB] Lanczos vectors
  static constexpr size_t PART = V + sizeof(float) * KM * LOB_TILE * NB;  // [NW][KM][NB] warp partial sums
  static constexpr size_t RES = PART + sizeof(float) * NW * KM * NB;      // [KM][NB] CTA sums
  static constexpr size_t AL = RES + sizeof(float) * KM * NB;             // [KM][NB]
  static constexpr size_t BE = AL + sizeof(float) * KM * NB;              // [KM][NB]
  static constexpr size_t Y = BE + sizeof(float) * KM * NB;               // [KM][NB]
  static constexpr size_t B0 = Y + sizeof(float) * KM * NB;               // [NB]
  static constexpr size_t MC = B0 + sizeof(float) * NB;                   // [NB] steps taken per column
  static constexpr size_t BYTES = MC + sizeof(int) * NB;
  static_assert(VW * G == NB && THREADS <= 1024, "launch shape");
};

// Sums over the CTA's rows, per column, of KV values a thread holds for its four columns:
// xor-shuffles over the eight groups of a warp, then a fixed-order sum over the warps.
template <int NB, int KV>
__device__ __forceinline__ void tile_col_sums(float (&x)[KV][4], float* part, float* res) {
  using C = CfgTF<NB>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < KV; k++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float v = x[k][q];
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 4);
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
      v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
      if (lane < C::G) part[(warp * C::KM + k) * NB + lane * 4 + q] = v;
    }
  __syncthreads();
  if (tid < KV * NB) {
    const int k = tid / NB, j = tid % NB;
    float sum = 0.f;
    for (int w2 = 0; w2 < C::NW; w2++) sum += part[(w2 * C::KM + k) * NB + j];
    res[k * NB + j] = sum;
  }
  __syncthreads();
}

template <int NB>
__global__ void __launch_bounds__(CfgTF<NB>::THREADS, 1)
    k_tile_fom(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ tcol,
               const int64_t* __restrict__ tptr, const int32_t* __restrict__ tchunk,
               const uint2* __restrict__ rv, const uint16_t* __restrict__ cperm,
               const uint16_t* __restrict__ cptrs, const double* __restrict__ mu, const double* __restrict__ R,
               double* __restrict__ W, int nb, int c0, int w, int64_t n_act, int solve, int steps) {
  using C = CfgTF<NB>;
  constexpr int KM = C::KM, CH = LOB_PERM_CHUNK, PTRS = 2 * (LOB_TILE + 1);
  extern __shared__ __align__(16) unsigned char smt[];
  float* V = reinterpret_cast<float*>(smt + C::V);
  float* part = reinterpret_cast<float*>(smt + C::PART);
  float* res = reinterpret_cast<float*>(smt + C::RES);
  float* al = reinterpret_cast<float*>(smt + C::AL);
  float* be = reinterpret_cast<float*>(smt + C::BE);
  float* ys = reinterpret_cast<float*>(smt + C::Y);
  float* b0 = reinterpret_cast<float*>(smt + C::B0);
  int* mc = reinterpret_cast<int*>(smt + C::MC);
  const int tid = threadIdx.x, g = tid / C::G, gl = tid % C::G;
  const int64_t I = blockIdx.x, o = I * LOB_TILE;
  const int m_act = (int)((n_act - o) < LOB_TILE ? (n_act - o) : LOB_TILE);
  const bool live = g < m_act;
  const int64_t t0 = rowptr[I];
  const bool has_diag = t0 < rowptr[I + 1] && tcol[t0] == (int32_t)I;
  const int nk = has_diag ? tchunk[t0 + 1] - tchunk[t0] : 0;

  float r[4], muf[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int j = gl * 4 + q;
    r[q] = (live && j < w) ? (float)R[(o + g) * nb + c0 + j] : 0.f;
    muf[q] = j < w ? (float)mu[c0 + j] : 0.f;
  }
  {  // beta0 = ||r_j|| over the tile's rows
    float x[1][4];
#pragma unroll
    for (int q = 0; q < 4; q++) x[0][q] = r[q] * r[q];
    tile_col_sums<NB, 1>(x, part, res);
  }
  if (tid < NB) {
    b0[tid] = sqrtf(res[tid]);
    mc[tid] = 0;
  }
  if (tid < KM * NB) al[tid] = be[tid] = 0.f;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float bb = b0[gl * 4 + q];
    V[g * NB + gl * 4 + q] = bb > 0.f ? r[q] / bb : 0.f;
  }
  __syncthreads();

  for (int i = 0; i < steps; i++) {
    const float* Vi = V + (size_t)i * LOB_TILE * NB;
    // u = (H~_I - mu I) v_i on this group's row
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < nk; k++) {
      const int64_t base = tptr[t0] + (int64_t)k * CH;
      const uint16_t* PR = cptrs + (int64_t)(tchunk[t0] + k) * PTRS;
      const uint16_t* PC = PR + (LOB_TILE + 1);
      const int rs = __ldg(&PR[g]), re = __ldg(&PR[g + 1]);
      for (int e = rs; e < re; e++) {
        const uint2 ent = __ldg(&rv[base + e]);
        const float val = __uint_as_float(ent.y);
        const float4 x = *reinterpret_cast<const float4*>(&Vi[(int)(ent.x & 0xFFFFu) * NB + gl * 4]);
        u[0] = fmaf(val, x.x, u[0]); u[1] = fmaf(val, x.y, u[1]); u[2] = fmaf(val, x.z, u[2]); u[3] = fmaf(val, x.w, u[3]);
      }
      const int cs = __ldg(&PC[g]), ce = __ldg(&PC[g + 1]);
      for (int e = cs; e < ce; e++) {
        const uint2 ent = __ldg(&rv[base + (__ldg(&cperm[base + e]) & (CH - 1))]);
        const int rr = (int)(ent.x >> 16);
        if (rr == g) continue;  // the diagonal entry is applied once (row pass)
        const float val = __uint_as_float(ent.y);
        const float4 x = *reinterpret_cast<const float4*>(&Vi[rr * NB + gl * 4]);
        u[0] = fmaf(val, x.x, u[0]); u[1] = fmaf(val, x.y, u[1]); u[2] = fmaf(val, x.z, u[2]); u[3] = fmaf(val, x.w, u[3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) u[q] = live ? fmaf(-muf[q], Vi[g * NB + gl * 4 + q], u[q]) : 0.f;
    // h_t = v_t . u for t <= i (classical Gram-Schmidt); alpha_i = h_i
    {
      float x[KM][4];
#pragma unroll
      for (int t = 0; t < KM; t++)
#pragma unroll
        for (int q = 0; q < 4; q++) x[t][q] = t <= i ? V[((size_t)t * LOB_TILE + g) * NB + gl * 4 + q] * u[q] : 0.f;
      tile_col_sums<NB, KM>(x, part, res);
    }
#pragma unroll
    for (int t = 0; t < KM; t++) {
      if (t > i) continue;
#pragma unroll
      for (int q = 0; q < 4; q++) u[q] = fmaf(-res[t * NB + gl * 4 + q], V[((size_t)t * LOB_TILE + g) * NB + gl * 4 + q], u[q]);
    }
    if (tid < NB) al[i * NB + tid] = res[i * NB + tid];
    {
      float x[1][4];
#pragma unroll
      for (int q = 0; q < 4; q++) x[0][q] = u[q] * u[q];
      tile_col_sums<NB, 1>(x, part, res);  // its first barrier also orders the al writes above
    }
    if (tid < NB && mc[tid] == 0 && b0[tid] > 0.f) {
      float bi = sqrtf(res[tid]);
      const float scale = fabsf(al[i * NB + tid]) + (i > 0 ? be[(i - 1) * NB + tid] : 0.f);
      const bool brk = !(bi > 1e-6f * scale);
      if (brk) bi = 0.f;  // invariant subspace: the iterate is exact
      be[i * NB + tid] = bi;
      if (brk || i + 1 == steps) mc[tid] = i + 1;
    }
    __syncthreads();
    if (i + 1 < steps) {
      float* Vn = V + (size_t)(i + 1) * LOB_TILE * NB;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int j = gl * 4 + q;
        const bool stop = mc[j] != 0 || !(b0[j] > 0.f);
        Vn[g * NB + j] = stop ? 0.f : u[q] / be[i * NB + j];
      }
      __syncthreads();
    }
  }
  if (tid < NB) {
    float a3[KM], b3[KM], y3[KM];
#pragma unroll
    for (int t = 0; t < KM; t++) { a3[t] = al[t * NB + tid]; b3[t] = be[t * NB + tid]; }
    const int m = mc[tid];
    if (m > 0) {
      krylov_coeffs(solve, m, a3, b3, b0[tid], y3);
    } else {
#pragma unroll
      for (int t = 0; t < KM; t++) y3[t] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < KM; t++) ys[t * NB + tid] = t < m ? y3[t] : 0.f;
  }
  __syncthreads();
  if (!live) return;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int j = gl * 4 + q;
    if (j >= w) continue;
    const int m = mc[j];  // Lanczos vectors past the column's last step were never written
    float x = 0.f;
#pragma unroll
    for (int t = 0; t < KM; t++)
      if (t < m) x = fmaf(ys[t * NB + j], V[((size_t)t * LOB_TILE + g) * NB + j], x);
    W[(o + g) * nb + c0 + j] = (double)x;
  }
}

}  // namespace

void lob_free_precond(lob_precond* P) {
  cudaFree(P->Q); cudaFree(P->lam); cudaFree(P->dblk);
  *P = lob_precond();
}

int lob_build_precond(const lob_coo* H, int bp, int64_t n, cudaStream_t st, lob_precond* P) {
  if (bp == LOB_TILE) {  // the diagonal tiles of the tile store are the blocks: nothing to build
    lob_precond R;
    R.bp = LOB_TILE;
    R.nblk = (n + LOB_TILE - 1) / LOB_TILE;
    *P = R;
    return LOB_OK;
  }
  if (bp < 1 || bp > 64 || !H->on_device) return LOB_ERR_ARG;
  lob_precond R;
  R.bp = bp;
  R.nblk = (n + bp - 1) / bp;
  const size_t mm = (size_t)bp * bp;
  if (cudaMalloc(&R.dblk, R.nblk * mm * 8) != cudaSuccess || cudaMalloc(&R.Q, R.nblk * mm * 4) != cudaSuccess ||
      cudaMalloc(&R.lam, R.nblk * bp * 4) != cudaSuccess) {
    cudaGetLastError();
    lob_free_precond(&R);
    return LOB_ERR_NOMEM;
  }
  cudaMemsetAsync(R.dblk, 0, R.nblk * mm * 8, st);
  (k_gather_blocks<<<(unsigned)((H->nnz + 255) / 256), 256, 0, st>>>(H->nnz, H->row, H->col, H->val, bp, R.dblk), LOB_LAUNCHED());
  const size_t smem = 2 * mm * sizeof(float);
  (k_block_eig<<<(unsigned)R.nblk, 256, smem, st>>>(bp, R.dblk, R.Q, R.lam), LOB_LAUNCHED());
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    fprintf(stderr, "lob: preconditioner setup failed: %s\n", cudaGetErrorString(e));
    lob_free_precond(&R);
    return LOB_ERR_CUDA;
  }
  cudaFree(R.dblk);  // the dense blocks are only needed for the factorisation
  R.dblk = nullptr;
  *P = R;
  return LOB_OK;
}

int lob_precond_launch(const lob_matrix* m, const double* mu, const double* R, double* W, int nb, int64_t n_act,
                       int solve, int steps, cudaStream_t st) {
  const lob_precond& P = m->P;
  if (P.bp < 1 || nb < 1 || nb > 64) return LOB_ERR_ARG;
  if (solve < LOB_PSOLVE_FOM || solve > LOB_PSOLVE_ABS || steps < 1 || steps > 3) return LOB_ERR_ARG;
  if (P.bp == LOB_TILE) {  // FOM / minimal residual on the diagonal tiles
    if ((solve != LOB_PSOLVE_FOM && solve != LOB_PSOLVE_MINRES) || !m->T.rv) return LOB_ERR_ARG;
    constexpr int NB = 16;
    using C = CfgTF<NB>;
    const int64_t nt_act = (n_act + LOB_TILE - 1) / LOB_TILE;
    if (n_act < m->T.n) LOB_CUDA(cudaMemsetAsync(W + n_act * nb, 0, (size_t)(m->T.n - n_act) * nb * 8, st));
    if (nt_act == 0) return LOB_OK;
    LOB_CUDA(cudaFuncSetAttribute(k_tile_fom<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
    const lob_tiles& T = m->T;
    for (int c0 = 0; c0 < nb; c0 += NB) {
      const int w = (nb - c0) < NB ? (nb - c0) : NB;
      (k_tile_fom<NB><<<(unsigned)nt_act, C::THREADS, C::BYTES, st>>>(T.rowptr, T.tcol, T.tptr, T.tchunk, T.rv,
                                                                      T.cperm, T.cptrs, mu, R, W, nb, c0, w, n_act,
                                                                      solve, steps),
       LOB_LAUNCHED());
    }
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  }
  const int bp = P.bp;
  const size_t smem = ((size_t)bp * bp + 2ull * bp * nb) * sizeof(float);
  const int64_t nblk = (n_act + bp - 1) / bp;
  if (n_act < m->T.n) LOB_CUDA(cudaMemsetAsync(W + n_act * nb, 0, (size_t)(m->T.n - n_act) * nb * 8, st));
  if (nblk > 0)
    (k_block_apply<<<(unsigned)nblk, 256, smem, st>>>(bp, n_act, P.Q, P.lam, mu, (float)(1e-8 * m->norm_inf), R, W, nb,
                                                      solve, steps),
     LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

int lob_precond_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int bpmax, int nbmax,
                             cudaStream_t st) {
  if (njobs <= 0) return LOB_OK;
  int64_t ctas = 0;
  size_t smem = 0;
  for (int i = 0; i < njobs; i++) {
    lob_bjob& j = jobs_host[i];
    if (j.x1 < 1 || j.x1 > 64 || j.x0 < 1 || j.x0 > 64) return LOB_ERR_ARG;
    const int bpc = blocks_per_cta(j.x1, j.x0);
    j.cta_begin = ctas;
    ctas += ((j.n + j.x1 - 1) / j.x1 + bpc - 1) / bpc;
    const size_t need = (size_t)bpc * ((size_t)j.x1 * j.x1 + 2ull * j.x1 * j.x0) * sizeof(float);
    if (need > smem) smem = need;
  }
  if (ctas == 0) return LOB_OK;
  (void)bpmax;
  (void)nbmax;
  LOB_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, njobs * sizeof(lob_bjob), cudaMemcpyHostToDevice, st));
  (k_block_apply_batch<<<(unsigned)ctas, 256, smem, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}
