// Device code of the Rayleigh-Ritz step (eq. 9, Algorithm 1 steps 7-8) for one CTA: the FP64
// solve (rr_body) and the double-float one (rr_body_df), with the cyclic Jacobi they share.
// Included by the single-solve and batched kernels (dense.cu) and by the persistent batched
// small-instance solver (batch.cu); every function is internal to the including file.
#pragma once
#include "common.cuh"
#include "df.cuh"

namespace {

// ---- cyclic Jacobi with 2x2-block updates (double-float and FP32 eigensolvers) ----
// Round r of the round-robin order pairs the indices as (p_k, q_k), k < m/2, all disjoint.
// A <- J^T A J with J the product of the round's rotations; for the 2x2 block of rows {p1, q1}
// and columns {p2, q2} the new values depend only on that block, so one thread updates a whole
// block (left rotation k1, then right rotation k2) and the round needs no barrier between its
// row and column halves. V <- V J touches no value the angles depend on, so V's rotations of
// round r run in the next round's first phase, beside the angle computation:
//   phase 1: warp 0 computes round r's angles | the other warps rotate V by round r-1's
//   barrier
//   phase 2: all threads update the 2x2 blocks of A by round r's rotations
//   barrier
// Angles and pairs are double-buffered by round parity.
__device__ __forceinline__ void rot2(d2& x, d2& y, d2 c, d2 s) { d2_rot(x, y, c, s); }
__device__ __forceinline__ void rot2(float& x, float& y, float c, float s) {
  const float u = fmaf(c, x, -s * y), v = fmaf(s, x, c * y);
  x = u;
  y = v;
}
__device__ __forceinline__ double hi64(float x) { return (double)x; }
__device__ __forceinline__ bool nonzero(float x) { return x != 0.f; }
__device__ __forceinline__ float ident_one(float) { return 1.f; }
__device__ __forceinline__ float ident_zero(float) { return 0.f; }
__device__ __forceinline__ double hi64(d2 x) { return d2_hi64(x); }
__device__ __forceinline__ bool nonzero(d2 x) { return x.hi != 0.f; }
__device__ __forceinline__ d2 ident_one(d2) { return d2{1.f, 0.f}; }
__device__ __forceinline__ d2 ident_zero(d2) { return d2{0.f, 0.f}; }

// rotation (c, s) that zeros a_pq (GVL 8.5: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) /
// (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c). FP32: all in FP32. Double-float:
// the angle in FP32 from a double-float difference, then c, s in double-float from that exact t.
__device__ __forceinline__ void jac_angle(float app, float aqq, float apq, float& c, float& s) {
  c = 1.f; s = 0.f;
  if (apq == 0.f) return;
  const float tau = (aqq - app) / (2.f * apq);
  const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  c = rsqrtf(1.f + t * t);
  s = t * c;
}
__device__ __forceinline__ void jac_angle(d2 app, d2 aqq, d2 apq, d2& c, d2& s) {
  c = d2{1.f, 0.f}; s = d2{0.f, 0.f};
  apq = d2_norm(apq);
  if (apq.hi == 0.f) return;
  const d2 diff = d2_add(aqq, d2_neg(app));
  const float tau = diff.hi / (2.f * apq.hi);
  const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
  if (t == 0.f) return;
  const d2 tt{t, 0.f};
  c = d2_rsqrt(d2_add(d2{1.f, 0.f}, d2_mul(tt, tt)));
  s = d2_mul(tt, c);
}

// b-th pair (k1 <= k2) of an np x np array, row by row over its upper triangle
__device__ __forceinline__ void tri_index(int b, int np, int& k1, int& k2) {
  const float t = (float)(2 * np + 1);
  int r = (int)floorf(0.5f * (t - sqrtf(fmaxf(t * t - 8.f * (float)b, 0.f))));
  auto first = [np](int x) { return x * np - x * (x - 1) / 2; };  // index of (x, x)
  if (r < 0) r = 0;
  if (r > np - 1) r = np - 1;
  while (r > 0 && first(r) > b) r--;
  while (r < np - 1 && first(r + 1) <= b) r++;
  k1 = r;
  k2 = r + (b - first(r));
}

// position -> index in round r (circle method: position 0 fixed, the others rotate by one)
__device__ __forceinline__ int rr_index(int pos, int round, int mp) {
  if (pos == 0) return 0;
  int x = pos - 1 + round;  // < 2 (mp - 1)
  if (x >= mp - 1) x -= mp - 1;
  return 1 + x;
}

// Cyclic Jacobi on A (m x m, symmetric), accumulating the rotations into V. cs_c, cs_s, pr_p,
// pr_q hold two rounds of 96 pairs each.
template <typename E>
__device__ void jacobi_blocks(int m, int ld, E* A, E* V, double stop_ratio, E* cs_c, E* cs_s, int* pr_p, int* pr_q,
                              double* red, double* s_off, double* s_fro) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m;
  const int mp = m + (m & 1), np = mp / 2;
  int pend = -1;  // buffer of the round whose V rotations are still to be applied
  auto rotate_v = [&](int b, int t0, int ts) {
    for (int e = t0; e < np * m; e += ts) {
      const int row = e / np, k = e % np;  // neighbouring threads: one row, neighbouring pairs
      const int q = pr_q[b * 96 + k];
      if (q >= m || !nonzero(cs_s[b * 96 + k])) continue;
      rot2(V[row * ld + pr_p[b * 96 + k]], V[row * ld + q], cs_c[b * 96 + k], cs_s[b * 96 + k]);
    }
  };
  // This thread's work items are the same in every round: its block (k1, k2) of the upper
  // triangle and up to VMAX (row, pair) rotations of V; found once, when they fit.
  constexpr int VMAX = 4;
  const int nA = np * (np + 1) / 2, nV = np * m;
  const bool afix = nA <= nt;
  const bool vfix = nt > 32 && nV <= VMAX * (nt - 32);
  int ak1 = -1, ak2 = 0;
  if (afix && tid < nA) tri_index(tid, np, ak1, ak2);
  int vrow[VMAX], vk[VMAX];
#pragma unroll
  for (int u = 0; u < VMAX; u++) {
    const int e = (tid - 32) + u * (nt - 32);
    const bool ok = vfix && tid >= 32 && e < nV;
    vrow[u] = ok ? (e / np) * ld : -1;
    vk[u] = ok ? e % np : 0;
  }
  auto rotate_v_fixed = [&](int b) {
#pragma unroll
    for (int u = 0; u < VMAX; u++) {
      if (vrow[u] < 0) continue;
      const int k = vk[u];
      const int q = pr_q[b * 96 + k];
      if (q >= m || !nonzero(cs_s[b * 96 + k])) continue;
      rot2(V[vrow[u] + pr_p[b * 96 + k]], V[vrow[u] + q], cs_c[b * 96 + k], cs_s[b * 96 + k]);
    }
  };
  int rcount = 0;
  double prev = 0.0;
  for (int sweep = 0; sweep < 40; sweep++) {
    double off = 0.0, fro = 0.0;
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      const double x = hi64(A[i * ld + j]);
      fro += x * x;
      if (i != j) off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) { off += __shfl_down_sync(0xFFFFFFFFu, off, o); fro += __shfl_down_sync(0xFFFFFFFFu, fro, o); }
    if (tid % 32 == 0) { red[tid / 32] = off; red[32 + tid / 32] = fro; }
    __syncthreads();
    if (tid == 0) {
      double so = 0, sf = 0;
      for (int w = 0; w < nt / 32; w++) { so += red[w]; sf += red[32 + w]; }
      *s_off = so; *s_fro = sf;
    }
    __syncthreads();
    if (*s_off <= stop_ratio * *s_fro || *s_off == 0.0) break;
    // near the arithmetic's floor a sweep that no longer reduces ||off||^2 fourfold ends it
    if (sweep > 0 && *s_off <= 1e-8 * *s_fro && *s_off > 0.25 * prev) break;
    prev = *s_off;
    for (int round = 0; round < mp - 1; round++, rcount++) {
      const int b = rcount & 1;
      E* cc = cs_c + b * 96;
      E* ss = cs_s + b * 96;
      int* pp = pr_p + b * 96;
      int* qq = pr_q + b * 96;
      if (tid < 32) {
        for (int k = tid; k < np; k += 32) {
          int p = rr_index(k, round, mp), q = rr_index(mp - 1 - k, round, mp);
          if (p > q) { const int t = p; p = q; q = t; }
          E c = ident_one(E{}), sn = ident_zero(E{});
          if (q < m) jac_angle(A[p * ld + p], A[q * ld + q], A[p * ld + q], c, sn);
          pp[k] = p; qq[k] = q; cc[k] = c; ss[k] = sn;
        }
      } else if (pend >= 0) {
        if (vfix) rotate_v_fixed(pend);
        else rotate_v(pend, tid - 32, nt - 32);
      }
      __syncthreads();
      // 2x2 blocks of A: block (k1, k2) = rows {p1, q1} x columns {p2, q2}, k1 <= k2; the block
      // (k2, k1) is its transpose and is written by the same thread, so A stays exactly symmetric
      auto block = [&](int k1, int k2) {
        const int p1 = pp[k1], q1 = qq[k1], p2 = pp[k2], q2 = qq[k2];
        const bool r1 = q1 < m, r2 = q2 < m;  // second index valid (not the dummy)
        E a11 = A[p1 * ld + p2];
        E a12 = r2 ? A[p1 * ld + q2] : ident_zero(E{});
        E a21 = r1 ? A[q1 * ld + p2] : ident_zero(E{});
        E a22 = (r1 && r2) ? A[q1 * ld + q2] : ident_zero(E{});
        if (r1 && nonzero(ss[k1])) { rot2(a11, a21, cc[k1], ss[k1]); rot2(a12, a22, cc[k1], ss[k1]); }
        if (r2 && nonzero(ss[k2])) { rot2(a11, a12, cc[k2], ss[k2]); rot2(a21, a22, cc[k2], ss[k2]); }
        A[p1 * ld + p2] = a11;
        if (r2) A[p1 * ld + q2] = a12;
        if (r1) A[q1 * ld + p2] = a21;
        if (r1 && r2) A[q1 * ld + q2] = a22;
        if (k1 != k2) {
          A[p2 * ld + p1] = a11;
          if (r2) A[q2 * ld + p1] = a12;
          if (r1) A[p2 * ld + q1] = a21;
          if (r1 && r2) A[q2 * ld + q1] = a22;
        }
      };
      if (afix) {
        if (ak1 >= 0) block(ak1, ak2);
      } else {
        for (int bb = tid; bb < nA; bb += nt) {
          int k1, k2;
          tri_index(bb, np, k1, k2);
          block(k1, k2);
        }
      }
      __syncthreads();
      pend = b;
    }
  }
  if (pend >= 0) {
    rotate_v(pend, tid, nt);
    __syncthreads();
  }
}

// ---- FP64 Rayleigh-Ritz (eq. 9): G c = theta M c for one CTA ----
// GB300's FP64 pipe retires about 1.6 multiply-adds per clock per SM, so a dependent chain of FP64
// scalar operations (a QL recurrence, a Jacobi angle per rotation) stalls for tens of clocks at every
// step. The solve therefore keeps its FP64 work in parallel products and does the iterative part in
// FP32:
//   1. M = L L^T and A = L^{-1} G L^{-T} in FP64 (right-looking, every thread at every step);
//   2. cyclic Jacobi on fl32(A) gives an approximate eigenbasis X (FP32 accuracy);
//   3. iterative refinement of X in FP64 (Ogita and Aishima, "Iterative refinement for symmetric
//      eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018): with R = I - X^T X and
//      S = X^T A X, the Ritz values are l_i = s_ii / (1 - r_ii), and X <- X + X E with
//      e_ij = (s_ij + l_j r_ij) / (l_j - l_i) for |l_i - l_j| > d, e_ij = r_ij / 2 otherwise
//      (e_ii = r_ii / 2), d = 2 (||S - diag(l)|| + ||A|| ||R||) (Frobenius norms). The error
//      squares at every step, so two steps take FP32 accuracy to FP64's. Two safeguards keep the
//      iteration from oscillating on pairs that FP32 could not separate: d never falls below an
//      earlier step's, and a pair whose first-order correction exceeds 1e-3 is treated as close;
//   4. close pairs are not separated by step 3: where S (of the final X) still couples two
//      columns, FP64 Jacobi rotations on S and X separate them (skipped when S is diagonal to
//      rounding);
//   5. C = L^{-T} X, columns in ascending order of the Ritz values.
// The FP64 multiply-adds are about m^3 (1 + 2 per refinement step); X E runs in FP32, as E is
// small (its rounding error is below the next step's or the final accuracy).
// Storage: A, L, X, T and SR (m x m each, row stride ld); SR holds S above its diagonal and R below.
template <bool SMEM>
__device__ __forceinline__ void rr_body(int m, const double* __restrict__ G, const double* __restrict__ Mi,
                                        double* __restrict__ theta, double* __restrict__ C,
                                        int32_t* __restrict__ info, double* __restrict__ work, int chol_only,
                                        unsigned char* rr_sm) {
  const int ld = SMEM ? m + 1 : m;  // padded rows in shared memory: column walks hit distinct banks
  double* base = SMEM ? reinterpret_cast<double*>(rr_sm) : work;
  double* A = base;
  double* L = A + m * ld;
  double* X = L + m * ld;
  double* T = X + m * ld;
  double* SR = T + m * ld;
  __shared__ float cs_c[192], cs_s[192];
  __shared__ int pr_p[192], pr_q[192];
  __shared__ double red[64];
  __shared__ double inv[192], lam[192], rdg[192];
  __shared__ int rk[192];
  __shared__ unsigned pmask[192 * 192 / 32];
  __shared__ int s_fail;
  __shared__ double s_off, s_fro, s_sc[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m, ntri = m * (m + 1) / 2;
  // element (r, c) updates of the right-looking loops: thread = (R0, C0), RS rows at a time
  // (the launch gives nt >= m threads)
  const int RS = nt / m, R0 = tid / m, C0 = tid % m;
  const bool upd = tid < RS * m;
  // sums over the CTA of one or two per-thread values (every thread gets the result)
  auto sum2 = [&](double a, double b, double& ra, double& rb) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xFFFFFFFFu, a, o);
      b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5] = a; red[32 + (tid >> 5)] = b; }
    __syncthreads();
    if (tid == 0) {
      double x = 0.0, y = 0.0;
      for (int w = 0; w < (nt + 31) / 32; w++) { x += red[w]; y += red[32 + w]; }
      s_sc[0] = x; s_sc[1] = y;
    }
    __syncthreads();
    ra = s_sc[0]; rb = s_sc[1];
    __syncthreads();
  };
  auto max1 = [&](double a) -> double {
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xFFFFFFFFu, a, o));
    if ((tid & 31) == 0) red[tid >> 5] = a;
    __syncthreads();
    if (tid == 0) {
      double x = 0.0;
      for (int w = 0; w < (nt + 31) / 32; w++) x = fmax(x, red[w]);
      s_sc[2] = x;
    }
    __syncthreads();
    const double r = s_sc[2];
    __syncthreads();
    return r;
  };
  // Xm <- L^{-T} Xm for all columns (right-looking back substitution)
  auto back_sub = [&](double* Xm) {
    for (int i = m - 1; i >= 0; i--) {
      if (tid < m) Xm[i * ld + tid] *= inv[i];
      __syncthreads();
      if (upd)
        for (int r = R0; r < i; r += RS) Xm[r * ld + C0] -= L[i * ld + r] * Xm[i * ld + C0];
      __syncthreads();
    }
  };

  // symmetric copies from the upper triangles
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    const int a = i < j ? i : j, b = i < j ? j : i;
    A[i * ld + j] = G[a * m + b];
    L[i * ld + j] = Mi[a * m + b];
    X[i * ld + j] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) s_fail = 0;
  __syncthreads();

  // 1. right-looking Cholesky in place on L (lower part), inv[j] = 1 / L_jj
  for (int j = 0; j < m; j++) {
    if (tid == 0) {
      const double d = L[j * ld + j];
      if (!(d > 0.0)) {
        s_fail = j + 1;
      } else {
        const double r = sqrt(d);
        L[j * ld + j] = r;
        inv[j] = 1.0 / r;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double ij = inv[j];
    for (int i = j + 1 + tid; i < m; i += nt) L[i * ld + j] *= ij;
    __syncthreads();
    if (upd && C0 > j)
      for (int i = j + 1 + R0; i < m; i += RS)
        if (C0 <= i) L[i * ld + C0] -= L[i * ld + j] * L[C0 * ld + j];
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) *info = s_fail;
    return;
  }
  if (chol_only) {  // Cholesky-QR: C = L^{-T}
    back_sub(X);
    for (int e = tid; e < mm; e += nt) C[e] = X[(e / m) * ld + e % m];
    for (int j = tid; j < m; j += nt) theta[j] = 1.0;
    if (tid == 0) *info = 0;
    return;
  }
  // 2. A <- L^{-1} A L^{-T} (right-looking: row i, then column i, is final once the earlier ones
  // have been subtracted), made exactly symmetric
  for (int i = 0; i < m; i++) {
    if (tid < m) A[i * ld + tid] *= inv[i];
    __syncthreads();
    if (upd)
      for (int r = i + 1 + R0; r < m; r += RS) A[r * ld + C0] -= L[r * ld + i] * A[i * ld + C0];
    __syncthreads();
  }
  for (int i = 0; i < m; i++) {
    if (tid < m) A[tid * ld + i] *= inv[i];
    __syncthreads();
    if (upd)
      for (int c = i + 1 + R0; c < m; c += RS) A[C0 * ld + c] -= A[C0 * ld + i] * L[c * ld + i];
    __syncthreads();
  }
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    if (i < j) {
      const double s = 0.5 * (A[i * ld + j] + A[j * ld + i]);
      A[i * ld + j] = s;
      A[j * ld + i] = s;
    }
  }
  __syncthreads();
  // 3. approximate eigenbasis: cyclic Jacobi on fl32(A) to ||off|| <= 3e-7 ||A|| or FP32's floor
  // (F and VF in T's space)
  {
    float* F = reinterpret_cast<float*>(T);
    float* VF = F + m * ld;
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      F[i * ld + j] = (float)A[i * ld + j];
      VF[i * ld + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_blocks<float>(m, ld, F, VF, 1e-13, cs_c, cs_s, pr_p, pr_q, red, &s_off, &s_fro);
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      X[i * ld + j] = (double)VF[i * ld + j];
    }
  }
  double nA;
  {
    double a2 = 0.0, z = 0.0;
    for (int e = tid; e < mm; e += nt) {
      const double x = A[(e / m) * ld + e % m];
      a2 += x * x;
    }
    sum2(a2, 0.0, a2, z);  // (its barriers also order X's writes above)
    nA = sqrt(a2);
  }
  // 4. refinement: R = I - X^T X, S = X^T A X, then X <- X + X E
  double* X32s = T;  // FP32 copies of X and E for the correction product (T's space, free by then)
  double dl = 0.0, cmax = 0.0;
  for (int it = 0; it < 6; it++) {
    for (int e = tid; e < mm; e += nt) {  // T = A X
      const int i = e / m, j = e % m;
      double s = 0.0;
      for (int k = 0; k < m; k++) s = fma(A[i * ld + k], X[k * ld + j], s);
      T[i * ld + j] = s;
    }
    __syncthreads();
    for (int b = tid; b < ntri; b += nt) {  // S (upper), R (lower; its diagonal in rdg)
      int i, j;
      tri_index(b, m, i, j);
      double s = 0.0, r = 0.0;
      for (int k = 0; k < m; k++) {
        const double xi = X[k * ld + i];
        s = fma(xi, T[k * ld + j], s);
        r = fma(xi, X[k * ld + j], r);
      }
      SR[i * ld + j] = s;
      if (i < j) SR[j * ld + i] = -r;
      else rdg[i] = 1.0 - r;
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) lam[i] = SR[i * ld + i] / (1.0 - rdg[i]);
    __syncthreads();
    double so = 0.0, sr = 0.0;
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      if (i < j) {
        const double s = SR[i * ld + j], r = SR[j * ld + i];
        so += 2.0 * s * s;
        sr += 2.0 * r * r;
      } else if (i == j) {
        const double s = SR[i * ld + i] - lam[i];
        so += s * s;
        sr += rdg[i] * rdg[i];
      }
    }
    sum2(so, sr, so, sr);
    dl = fmax(dl, 2.0 * (sqrt(so) + nA * sqrt(sr)));  // never below an earlier step's
    // E, written as FP32 into the second half of T's space, X as FP32 into the first half
    float* X32 = reinterpret_cast<float*>(X32s);
    float* E32 = X32 + m * ld;
    double emax = 0.0, cmx = 0.0;  // largest correction; largest coupling between close pairs
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      X32[i * ld + j] = (float)X[i * ld + j];
      if (i > j) continue;
      if (i == j) {
        const double d = 0.5 * rdg[i];
        E32[i * ld + i] = (float)d;
        emax = fmax(emax, fabs(d));
        continue;
      }
      const double s = SR[i * ld + j], r = SR[j * ld + i];
      double eij = 0.0, eji = 0.0;
      bool sep = fabs(lam[i] - lam[j]) > dl;
      if (sep) {
        eij = (s + lam[j] * r) / (lam[j] - lam[i]);
        eji = (s + lam[i] * r) / (lam[i] - lam[j]);
        sep = fmax(fabs(eij), fabs(eji)) <= 1e-3;  // a larger first-order step would not converge
      }
      if (!sep) {
        eij = 0.5 * r;
        eji = eij;
        cmx = fmax(cmx, fabs(s));
      }
      E32[i * ld + j] = (float)eij;
      E32[j * ld + i] = (float)eji;
      emax = fmax(emax, fmax(fabs(eij), fabs(eji)));
    }
    emax = max1(emax);  // (its barriers also order the FP32 copies)
    cmax = max1(cmx);
    for (int e = tid; e < mm; e += nt) {  // X + X E into SR's space
      const int i = e / m, j = e % m;
      float s = 0.f;
      for (int k = 0; k < m; k++) s = fmaf(X32[i * ld + k], E32[k * ld + j], s);
      SR[i * ld + j] = X[i * ld + j] + (double)s;
    }
    __syncthreads();
    double* t = X; X = SR; SR = t;
    if (emax <= 1e-9) break;  // the update just made leaves an error of order emax^2
  }
  // 5. close pairs still coupled: FP64 Jacobi rotations on S = X^T A X (of the final X) and on X,
  // pair by pair, wherever |s_pq| exceeds the rounding level of S
  const double thr = 32.0 * 1.1102230246251565e-16 * nA;
  if (cmax > thr) {
    for (int e = tid; e < mm; e += nt) {  // T = A X
      const int i = e / m, j = e % m;
      double s = 0.0;
      for (int k = 0; k < m; k++) s = fma(A[i * ld + k], X[k * ld + j], s);
      T[i * ld + j] = s;
    }
    __syncthreads();
    for (int b = tid; b < ntri; b += nt) {  // S, both triangles
      int i, j;
      tri_index(b, m, i, j);
      double s = 0.0;
      for (int k = 0; k < m; k++) s = fma(X[k * ld + i], T[k * ld + j], s);
      SR[i * ld + j] = s;
      SR[j * ld + i] = s;
    }
    __syncthreads();
    // each sweep: flag the coupled pairs (bit p m + q of pmask, p < q) in parallel, then rotate
    // them in row-major order, skipping a pair that earlier rotations of the sweep decoupled
    const int nw = (mm + 31) / 32;
    for (int sweep = 0; sweep < 10; sweep++) {
      for (int w = tid; w < nw; w += nt) {
        unsigned bits = 0u;
        for (int b = 0; b < 32; b++) {
          const int e = w * 32 + b;
          if (e >= mm) break;
          const int p = e / m, q = e % m;
          if (p < q && fabs(SR[p * ld + q]) > thr) bits |= 1u << b;
        }
        pmask[w] = bits;
      }
      __syncthreads();
      bool any = false;  // uniform: every thread reads the same values after the same barriers
      for (int w = 0; w < nw; w++) {
        unsigned bits = pmask[w];
        while (bits) {
          const int e = w * 32 + __ffs(bits) - 1;
          bits &= bits - 1u;
          const int p = e / m, q = e % m;
          const double spq = SR[p * ld + q];
          if (!(fabs(spq) > thr)) continue;
          any = true;
          const double spp = SR[p * ld + p], sqq = SR[q * ld + q];
          const double tau = (sqq - spp) / (2.0 * spq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
          __syncthreads();  // every thread has read S before any writes
          for (int k = tid; k < m; k += nt) {
            if (k == p) {
              SR[p * ld + p] = spp - t * spq;
              SR[q * ld + q] = sqq + t * spq;
              SR[p * ld + q] = 0.0;
              SR[q * ld + p] = 0.0;
            } else if (k != q) {
              const double a = SR[k * ld + p], b = SR[k * ld + q];
              const double na = c * a - sn * b, nb = sn * a + c * b;
              SR[k * ld + p] = na;
              SR[p * ld + k] = na;
              SR[k * ld + q] = nb;
              SR[q * ld + k] = nb;
            }
            const double xa = X[k * ld + p], xb = X[k * ld + q];
            X[k * ld + p] = c * xa - sn * xb;
            X[k * ld + q] = sn * xa + c * xb;
          }
          __syncthreads();
        }
      }
      __syncthreads();  // pmask is rewritten by the next sweep
      if (!any) break;
    }
    for (int i = tid; i < m; i += nt) lam[i] = SR[i * ld + i];
    __syncthreads();
  }
  // 6. rank sort of the Ritz values (ties by index), C = L^{-T} X in that order
  for (int j = tid; j < m; j += nt) {
    const double wj = lam[j];
    int rank = 0;
    for (int i = 0; i < m; i++) {
      const double wi = lam[i];
      rank += (wi < wj) || (wi == wj && i < j);
    }
    theta[rank] = wj;
    rk[j] = rank;
  }
  back_sub(X);  // (its first barrier orders the ranks before their use below)
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    C[i * m + rk[j]] = X[i * ld + j];
  }
  if (tid == 0) *info = 0;
}

// The same Rayleigh-Ritz step in double-float (df.cuh): every element operation of the
// Cholesky factorisation, the triangular solves and the Jacobi rotations runs on the FP32
// pipes with ~48-bit significands; only scalar work per pivot or per rotation (square roots,
// reciprocals, rotation angles, convergence sums) is done in FP64. The workspace holds the
// three m x m matrices as (hi, lo) pairs.
template <bool SMEM>
__device__ __forceinline__ void rr_body_df(int m, const double* __restrict__ G, const double* __restrict__ Mi,
                                           double* __restrict__ theta, double* __restrict__ C,
                                           int32_t* __restrict__ info, double* __restrict__ work, int chol_only,
                                           unsigned char* rr_sm) {
  const int ld = SMEM ? m + 1 : m;  // padded rows in shared memory: column walks hit distinct banks
  d2* A = SMEM ? reinterpret_cast<d2*>(rr_sm) : reinterpret_cast<d2*>(work);
  d2* L = A + m * ld;
  d2* V = L + m * ld;
  // shared-memory path only: a temporary, the Cholesky factor of V32^T V32, and V32 (FP32)
  d2* T = V + m * ld;
  d2* Lb = T + m * ld;
  float* VF = reinterpret_cast<float*>(Lb + m * ld);
  __shared__ d2 cs_c[192], cs_s[192];
  __shared__ int pr_p[192], pr_q[192];
  __shared__ d2 inv[192], inv2[192];
  __shared__ int rk[192];
  __shared__ double red[64];
  __shared__ int s_fail;
  __shared__ double s_off, s_fro;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mm = m * m;
  // element (r, c) updates of the right-looking loops: thread = (R0, C0), RS rows at a time
  // (the launch gives nt >= m threads)
  const int RS = nt / m, R0 = tid / m, C0 = tid % m;
  const bool upd = tid < RS * m;

  // Cholesky (right-looking) of the symmetric Lm in place: lower factor, iv[j] = 1 / L_jj.
  // Returns 0, or j + 1 for a non-positive pivot j.
  auto cholesky = [&](d2* Lm, d2* iv) -> int {
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int j = 0; j < m; j++) {
      if (tid == 0) {
        const d2 d = d2_norm(Lm[j * ld + j]);
        if (!(d.hi > 0.f)) s_fail = j + 1;
        else {
          const d2 ri = d2_rsqrt(d);  // 1 / sqrt(d)
          Lm[j * ld + j] = d2_mul(d, ri);
          iv[j] = ri;
        }
      }
      __syncthreads();
      if (s_fail) break;
      const d2 ij = iv[j];
      for (int i = j + 1 + tid; i < m; i += nt) Lm[i * ld + j] = d2_mul(Lm[i * ld + j], ij);
      __syncthreads();
      if (upd && C0 > j)
        for (int i = j + 1 + R0; i < m; i += RS) {
          if (C0 > i) continue;
          d2 x = Lm[i * ld + C0];
          const d2 a = Lm[i * ld + j], b = Lm[C0 * ld + j];
          df_mac(x.hi, x.lo, -a.hi, -a.lo, b.hi, b.lo);
          Lm[i * ld + C0] = d2_norm(x);
        }
      __syncthreads();
    }
    return s_fail;
  };
  // Am <- Lm^{-1} Am Lm^{-T} (right-looking: row i, then column i, is final once the earlier
  // ones have been subtracted), made exactly symmetric
  auto congruence = [&](d2* Am, const d2* Lm, const d2* iv) {
    for (int i = 0; i < m; i++) {
      if (tid < m) Am[i * ld + tid] = d2_mul(d2_norm(Am[i * ld + tid]), iv[i]);
      __syncthreads();
      if (upd)
        for (int r = i + 1 + R0; r < m; r += RS) {
          d2 x = Am[r * ld + C0];
          const d2 l = Lm[r * ld + i], a = Am[i * ld + C0];
          df_mac(x.hi, x.lo, -l.hi, -l.lo, a.hi, a.lo);
          Am[r * ld + C0] = d2_norm(x);
        }
      __syncthreads();
    }
    for (int i = 0; i < m; i++) {
      if (tid < m) Am[tid * ld + i] = d2_mul(d2_norm(Am[tid * ld + i]), iv[i]);
      __syncthreads();
      if (upd)
        for (int c = i + 1 + R0; c < m; c += RS) {
          d2 x = Am[C0 * ld + c];
          const d2 a = Am[C0 * ld + i], l = Lm[c * ld + i];
          df_mac(x.hi, x.lo, -a.hi, -a.lo, l.hi, l.lo);
          Am[C0 * ld + c] = d2_norm(x);
        }
      __syncthreads();
    }
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      if (i < j) {
        d2 sum = d2_add(Am[i * ld + j], Am[j * ld + i]);
        sum.hi *= 0.5f; sum.lo *= 0.5f;  // exact
        Am[i * ld + j] = sum;
        Am[j * ld + i] = sum;
      }
    }
    __syncthreads();
  };
  // Xm <- Lm^{-T} Xm for all columns (right-looking back substitution)
  auto back_sub = [&](const d2* Lm, const d2* iv, d2* Xm) {
    for (int i = m - 1; i >= 0; i--) {
      if (tid < m) Xm[i * ld + tid] = d2_mul(d2_norm(Xm[i * ld + tid]), iv[i]);
      __syncthreads();
      if (upd)
        for (int r = R0; r < i; r += RS) {
          d2 x = Xm[r * ld + C0];
          const d2 l = Lm[i * ld + r], a = Xm[i * ld + C0];
          df_mac(x.hi, x.lo, -l.hi, -l.lo, a.hi, a.lo);
          Xm[r * ld + C0] = d2_norm(x);
        }
      __syncthreads();
    }
  };

  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    const int a = i < j ? i : j, b = i < j ? j : i;
    A[i * ld + j] = d2_from(G[a * m + b]);
    L[i * ld + j] = d2_from(Mi[a * m + b]);
    V[i * ld + j] = d2{(i == j) ? 1.f : 0.f, 0.f};
  }
  __syncthreads();
  // 1. M = L L^T
  const int fail = cholesky(L, inv);
  if (fail) {
    if (tid == 0) *info = fail;
    return;
  }
  if (chol_only) {  // Cholesky-QR: C = L^{-T}
    back_sub(L, inv, V);
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      C[i * m + j] = d2_to(V[i * ld + j]);
    }
    for (int j = tid; j < m; j += nt) theta[j] = 1.0;
    if (tid == 0) *info = 0;
    return;
  }
  // 2. A <- L^{-1} G L^{-T}
  congruence(A, L, inv);
  // 3. A = W diag(theta) W^T. Double-float carries ~48 significant bits, so the off-diagonal part
  // cannot fall much below 2^-46 of the whole; the Jacobi sweeps stop at ||off|| <= 1e-10 ||A||
  // (quadratic convergence: the Ritz values then carry errors of order ||off||^2 / gap).
  d2* W = V;  // eigenvectors of the step-2 matrix
  if (!SMEM) {
    jacobi_blocks<d2>(m, ld, A, V, 1e-20, cs_c, cs_s, pr_p, pr_q, red, &s_off, &s_fro);
  } else {
    // Two stages. (a) Cyclic Jacobi on an FP32 copy of A, to ||off|| <= 1e-5 ||A||, gives V32 with
    // V32^T A V32 nearly diagonal -- most sweeps run at FP32 cost. (b) In double-float, with
    // V32^T V32 = Lb Lb^T: A <- Lb^{-1} V32^T A V32 Lb^{-T}, an exact congruence by
    // Q = V32 Lb^{-T} (Q^T Q = I), finished by Jacobi sweeps from V = I (one or two, as A starts
    // nearly diagonal); the eigenvectors of the step-2 matrix are W = Q V.
    float* F = reinterpret_cast<float*>(T);  // FP32 copy of A, in T's space until (b)
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      F[i * ld + j] = __fadd_rn(A[i * ld + j].hi, A[i * ld + j].lo);
      VF[i * ld + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_blocks<float>(m, ld, F, VF, 1e-10, reinterpret_cast<float*>(cs_c), reinterpret_cast<float*>(cs_s), pr_p,
                         pr_q, red, &s_off, &s_fro);
    // T = A V32 (double-float times FP32)
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      float h = 0.f, l = 0.f;
      for (int k = 0; k < m; k++) {
        const d2 a = A[i * ld + k];
        df_mac(h, l, a.hi, a.lo, VF[k * ld + j], 0.f);
      }
      T[i * ld + j] = d2_norm(d2{h, l});
    }
    __syncthreads();
    // upper triangles of A <- V32^T T and Lb <- V32^T V32, mirrored
    for (int e = tid; e < mm; e += nt) {
      const int i = e / m, j = e % m;
      if (i > j) continue;
      float h = 0.f, l = 0.f, bh = 0.f, bl = 0.f;
      for (int k = 0; k < m; k++) {
        const float vki = VF[k * ld + i];
        const d2 t = T[k * ld + j];
        df_mac(h, l, vki, 0.f, t.hi, t.lo);
        df_mac(bh, bl, vki, 0.f, VF[k * ld + j], 0.f);
      }
      const d2 av = d2_norm(d2{h, l}), bv = d2_norm(d2{bh, bl});
      A[i * ld + j] = av;
      A[j * ld + i] = av;
      Lb[i * ld + j] = bv;
      Lb[j * ld + i] = bv;
      V[i * ld + j] = d2{(i == j) ? 1.f : 0.f, 0.f};
      V[j * ld + i] = d2{(i == j) ? 1.f : 0.f, 0.f};
    }
    __syncthreads();
    if (cholesky(Lb, inv2)) {  // V32 lost rank: cannot happen for a finite A
      if (tid == 0) *info = m + 1;
      return;
    }
    congruence(A, Lb, inv2);
    jacobi_blocks<d2>(m, ld, A, V, 1e-20, cs_c, cs_s, pr_p, pr_q, red, &s_off, &s_fro);
    back_sub(Lb, inv2, V);  // V <- Lb^{-T} V
    for (int e = tid; e < mm; e += nt) {  // W = V32 V
      const int i = e / m, j = e % m;
      float h = 0.f, l = 0.f;
      for (int k = 0; k < m; k++) {
        const d2 t = V[k * ld + j];
        df_mac(h, l, VF[i * ld + k], 0.f, t.hi, t.lo);
      }
      T[i * ld + j] = d2_norm(d2{h, l});
    }
    W = T;
    __syncthreads();
  }
  // 4. rank sort of the Ritz values (ties by index), C = L^{-T} W in that order
  for (int j = tid; j < m; j += nt) {
    const double wj = d2_to(A[j * ld + j]);
    int rank = 0;
    for (int i = 0; i < m; i++) {
      const double wi = d2_to(A[i * ld + i]);
      rank += (wi < wj) || (wi == wj && i < j);
    }
    theta[rank] = wj;
    rk[j] = rank;
  }
  back_sub(L, inv, W);  // (its first barrier orders the ranks before their use below)
  for (int e = tid; e < mm; e += nt) {
    const int i = e / m, j = e % m;
    C[i * m + rk[j]] = d2_to(W[i * ld + j]);
  }
  if (tid == 0) *info = 0;
}

}  // namespace
