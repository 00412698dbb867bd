// Tall-skinny block kernels of one LOBPCG iteration (Section 4.4): the block inner product
// G = A^T B ("X^T Y") and the linear combination Y = A C (eq. 7).
//
// The paper splits the tall matrices into row blocks, forms small products per block and
// aggregates them (Section 4.4). Here each CTA owns a chunk of rows and a 48 x 48 tile of G,
// keeps its partial in registers (3 x 3 per thread), and a second kernel sums the chunk
// partials in a fixed order, so the result is deterministic.
//
// Arithmetic (mode): LOB_SPMM_FP64 -- native FP64 fused multiply-adds.
//                    LOB_SPMM_MIXED -- double-float (df.cuh) on the FP32 pipes: operands split
//                    on load (|x - (hi+lo)| <= 2^-48 |x|), products exact in their hi parts,
//                    sums error-free in hi; relative error per accumulated term ~2^-46.
#include "common.cuh"
#include "df.cuh"

namespace {

constexpr int TG = 48;  // largest output tile edge
constexpr int RB = 16;  // rows staged per step

template <bool DF>
struct Ar;
template <>
struct Ar<false> {
  using in_t = double;
  struct acc_t { double v; };
  __device__ static in_t load(double x) { return x; }
  __device__ static in_t zero_in() { return 0.0; }
  __device__ static void zero(acc_t& a) { a.v = 0.0; }
  __device__ static void init(acc_t& a, double x) { a.v = x; }
  __device__ static void mac(acc_t& a, in_t x, in_t y) { a.v = fma(x, y, a.v); }
  __device__ static double out(acc_t a) { return a.v; }
};
template <>
struct Ar<true> {
  using in_t = float2;
  struct acc_t { float hi, lo; };
  __device__ static in_t load(double x) { return df_split(x); }
  __device__ static in_t zero_in() { return make_float2(0.f, 0.f); }
  __device__ static void zero(acc_t& a) { a.hi = 0.f; a.lo = 0.f; }
  __device__ static void init(acc_t& a, double x) { const float2 s = df_split(x); a.hi = s.x; a.lo = s.y; }
  __device__ static void mac(acc_t& a, in_t x, in_t y) { df_mac(a.hi, a.lo, x.x, x.y, y.x, y.y); }
  __device__ static double out(acc_t a) { df_renorm(a.hi, a.lo); return df_join_int(a.hi, a.lo); }
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

// U = tile edge / 16 outputs per thread along each dimension (1, 2 or 3): small Gram matrices
// (16 x 16, 32 x 32) use a matching tile instead of a zero-padded 48 x 48 one.
// TRI: only the upper triangle of a symmetric result is needed -- the thread skips its
// sub-blocks below the diagonal (3 of 9 at U = 3); the reduction mirrors them.
// Rows arrive by cp.async into a double-buffered raw FP64 stage (Ra, Rb): the next RB rows load
// while the current ones are converted (to double-float for DF) and multiplied.
template <bool DF, int U, bool TRI>
__device__ __forceinline__ void gram_body(int64_t r0, int64_t r1, int p, const double* __restrict__ A, int lda, int q,
                                          const double* __restrict__ B, int ldb, int a0, int b0,
                                          typename Ar<DF>::in_t (*As)[16 * U], typename Ar<DF>::in_t (*Bs)[16 * U],
                                          double (*Ra)[RB][16 * U], double (*Rb)[RB][16 * U],
                                          typename Ar<DF>::acc_t (&acc)[U][U]) {
  using R = Ar<DF>;
  using in_t = typename R::in_t;
  constexpr int TGU = 16 * U;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  auto fetch = [&](int64_t rr, int buf) {
    for (int idx = tid; idx < RB * TGU; idx += 256) {
      const int i = idx / TGU, a = idx % TGU;
      const int64_t r = rr + i;
      if (r < r1 && a0 + a < p) cp_async8(&Ra[buf][i][a], &A[r * lda + a0 + a]);
      else Ra[buf][i][a] = 0.0;
      if (r < r1 && b0 + a < q) cp_async8(&Rb[buf][i][a], &B[r * ldb + b0 + a]);
      else Rb[buf][i][a] = 0.0;
    }
    cp_async_commit();
  };
  if (r0 < r1) fetch(r0, 0);
  int buf = 0;
  for (int64_t rr = r0; rr < r1; rr += RB, buf ^= 1) {
    if (rr + RB < r1) {
      fetch(rr + RB, buf ^ 1);
      cp_async_wait_1();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();  // this step's rows have landed; the previous step's products are done
    for (int idx = tid; idx < RB * TGU; idx += 256) {
      const int i = idx / TGU, a = idx % TGU;
      As[i][a] = R::load(Ra[buf][i][a]);
      Bs[i][a] = R::load(Rb[buf][i][a]);
    }
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < RB; i++) {
      in_t av[U], bv[U];
#pragma unroll
      for (int u = 0; u < U; u++) { av[u] = As[i][ty + 16 * u]; bv[u] = Bs[i][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < U; v++)
          if (!TRI || u <= v) R::mac(acc[u][v], av[u], bv[v]);
    }
  }
}

template <bool DF, int U>
__global__ void __launch_bounds__(256) k_gram(int64_t n, int p, const double* __restrict__ A, int lda, int q,
                                              const double* __restrict__ B, int ldb, double* __restrict__ part,
                                              int64_t rpc, int sym) {
  using R = Ar<DF>;
  using in_t = typename R::in_t;
  constexpr int TGU = 16 * U;
  __shared__ in_t As[RB][TGU];
  __shared__ in_t Bs[RB][TGU];
  __shared__ __align__(16) double Ra[2][RB][TGU];
  __shared__ __align__(16) double Rb[2][RB][TGU];
  const int chunk = blockIdx.x;
  if (sym && blockIdx.y > blockIdx.z) return;  // below-diagonal tile: mirrored by the reduction
  const int a0 = blockIdx.y * TGU, b0 = blockIdx.z * TGU;
  const int64_t r0 = (int64_t)chunk * rpc;
  const int64_t r1 = (r0 + rpc) < n ? (r0 + rpc) : n;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const bool tri = sym && blockIdx.y == blockIdx.z;
  typename R::acc_t acc[U][U];
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) R::zero(acc[i][j]);
  if (tri) gram_body<DF, U, true>(r0, r1, p, A, lda, q, B, ldb, a0, b0, As, Bs, Ra, Rb, acc);
  else gram_body<DF, U, false>(r0, r1, p, A, lda, q, B, ldb, a0, b0, As, Bs, Ra, Rb, acc);
#pragma unroll
  for (int u = 0; u < U; u++)
#pragma unroll
    for (int v = 0; v < U; v++) {
      if (tri && u > v) continue;
      const int a = a0 + ty + 16 * u, b = b0 + tx + 16 * v;
      if (a < p && b < q) part[(int64_t)chunk * p * q + (int64_t)a * q + b] = R::out(acc[u][v]);
    }
}

// G[e] = sum over chunks of part[chunk][e], one warp per entry, fixed order. With sym (p == q)
// an entry below the diagonal whose partial was not computed takes its mirror's: the tiles
// below the diagonal were skipped, and inside diagonal tiles so were the 16 x 16 sub-blocks
// below the diagonal; entries of diagonal sub-blocks were computed on both sides.
__global__ void k_gram_reduce(int nchunks, int pq, int q, int sym, int tge, const double* __restrict__ part,
                              double* __restrict__ G) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= pq) return;
  int src = warp;
  if (sym) {
    const int a = warp / q, b = warp % q;
    if (a / 16 > b / 16 || a / tge > b / tge) src = b * q + a;  // not computed: use the mirror
  }
  double s = 0.0;
  for (int c = lane; c < nchunks; c += 32) s += part[(int64_t)c * pq + src];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) G[warp] = s;
}

// Y = A C (+ D): RM 256/QT rows x QT output columns per CTA; thread (rl, j) computes rows
// rl, rl + 256/QT, ... (RM of them) of output column j, so each staged value of C feeds RM
// independent accumulators. The CTA loads its rows of A (all p columns) into shared memory
// before writing any output, so with a single column block (q <= QT) the output may be columns
// of A's own rows (used in place by the solver).
template <bool DF, int QT, int RM>
__device__ __forceinline__ void lincomb_body(int64_t n, int p, const double* __restrict__ A, int lda, int q,
                                             const double* __restrict__ C, double* __restrict__ Y, int ldy,
                                             const double* __restrict__ D, int ldd, int64_t rb, int cb,
                                             unsigned char* sm) {
  using R = Ar<DF>;
  using in_t = typename R::in_t;
  constexpr int RT = 256 / QT;             // rows per pass of the CTA's threads
  constexpr int RPC = RT * RM;             // rows per CTA
  const int lp = p | 1;                    // odd row stride: the warp's rows fall in different banks
  in_t* As = reinterpret_cast<in_t*>(sm);  // [RPC][lp]
  in_t* Cs = As + RPC * lp;                // [p][QT]
  const int64_t r0 = rb * RPC;
  const int j0 = cb * QT;
  const int tid = threadIdx.x, rl = tid / QT, j = tid % QT;
  for (int idx = tid; idx < RPC * p; idx += 256) {
    const int i = idx / p, a = idx % p;
    const int64_t r = r0 + i;
    As[i * lp + a] = r < n ? R::load(A[r * lda + a]) : R::zero_in();
  }
  for (int idx = tid; idx < QT * p; idx += 256) {
    const int a = idx / QT, jj = idx % QT;
    Cs[idx] = (j0 + jj < q) ? R::load(C[(int64_t)a * q + j0 + jj]) : R::zero_in();
  }
  __syncthreads();
  typename R::acc_t acc[RM];
#pragma unroll
  for (int u = 0; u < RM; u++) {
    R::zero(acc[u]);
    const int64_t r = r0 + rl + RT * u;
    if (D && r < n && j0 + j < q) R::init(acc[u], D[r * ldd + j0 + j]);  // Y = A C + D
  }
#pragma unroll 2
  for (int a = 0; a < p; a++) {
    const in_t c = Cs[a * QT + j];
#pragma unroll
    for (int u = 0; u < RM; u++) R::mac(acc[u], As[(rl + RT * u) * lp + a], c);
  }
#pragma unroll
  for (int u = 0; u < RM; u++) {
    const int64_t r = r0 + rl + RT * u;
    if (r < n && j0 + j < q) Y[r * ldy + j0 + j] = R::out(acc[u]);
  }
}

template <bool DF, int RM>
__global__ void __launch_bounds__(256) k_lincomb(int64_t n, int p, const double* __restrict__ A, int lda, int q,
                                                 const double* __restrict__ C, double* __restrict__ Y, int ldy,
                                                 const double* __restrict__ D, int ldd) {
  extern __shared__ __align__(16) unsigned char sm[];
  lincomb_body<DF, 16, RM>(n, p, A, lda, q, C, Y, ldy, D, ldd, blockIdx.x, blockIdx.y, sm);
}

__device__ __forceinline__ int find_job(const lob_bjob* __restrict__ jobs, int njobs, int64_t b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].cta_begin <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Batched Y = A C (+ D), q <= QT: job fields A, lda, p, C, q, Y, ldy, D, ldd, n; ceil(n / (lb_rm 256 /
// QT)) CTAs. Narrow blocks (QT = 1, 2, 4, 8) put more rows in a CTA instead of idle output columns.
// rows a thread: 4 (1 or 2 for the one- and two-column classes, whose CTAs already span 256
// or 128 rows a pass)
__host__ __device__ constexpr int lb_rm(int QT) { return QT >= 4 ? 4 : QT; }
template <bool DF, int QT>
__global__ void __launch_bounds__(256) k_lincomb_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  extern __shared__ __align__(16) unsigned char sm[];
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  lincomb_body<DF, QT, lb_rm(QT)>(j.n, j.p, j.A, j.lda, j.q, j.C, j.Y, j.ldy, j.D, j.ldd,
                                  (int64_t)blockIdx.x - j.cta_begin, 0, sm);
}

// Batched Gram products, one output tile (p, q <= 16 U): job fields A, lda, p, B, ldb, q, n,
// W0 (chunk partials), x0 (chunks), x1 (sym); x0 CTAs.
template <bool DF, int U>
__global__ void __launch_bounds__(256) k_gram_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  using R = Ar<DF>;
  using in_t = typename R::in_t;
  constexpr int TGU = 16 * U;
  __shared__ in_t As[RB][TGU];
  __shared__ in_t Bs[RB][TGU];
  __shared__ __align__(16) double Ra[2][RB][TGU];
  __shared__ __align__(16) double Rb[2][RB][TGU];
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  const int chunk = (int)((int64_t)blockIdx.x - j.cta_begin);
  const int64_t rpc = (j.n + j.x0 - 1) / j.x0;
  const int64_t r0 = (int64_t)chunk * rpc;
  const int64_t r1 = (r0 + rpc) < j.n ? (r0 + rpc) : j.n;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  typename R::acc_t acc[U][U];
#pragma unroll
  for (int a = 0; a < U; a++)
#pragma unroll
    for (int b = 0; b < U; b++) R::zero(acc[a][b]);
  if (j.x1) gram_body<DF, U, true>(r0, r1, j.p, j.A, j.lda, j.q, j.B, j.ldb, 0, 0, As, Bs, Ra, Rb, acc);
  else gram_body<DF, U, false>(r0, r1, j.p, j.A, j.lda, j.q, j.B, j.ldb, 0, 0, As, Bs, Ra, Rb, acc);
  const int pq = j.p * j.q;
#pragma unroll
  for (int u = 0; u < U; u++)
#pragma unroll
    for (int v = 0; v < U; v++) {
      if (j.x1 && u > v) continue;
      const int a = ty + 16 * u, b = tx + 16 * v;
      if (a < j.p && b < j.q) j.W0[(int64_t)chunk * pq + (int64_t)a * j.q + b] = R::out(acc[u][v]);
    }
}

// Batched Gram products by 2 x 2 output blocks, for at most 1,024 blocks (ceil(p/2) ceil(q/2), or
// the upper triangle of blocks when symmetric), so little work goes to padding and each
// multiply-add costs one shared-memory load. With many blocks thread t owns blocks t, t + 256,
// t + 512, t + 768 over all rows of the chunk; with P <= 128 blocks the 256 threads form
// G = floor(256 / P) groups of P that split the rows, and the groups' sums are added in a fixed
// order at the end. Job fields as k_gram_batch.
// FUSED: G = A^T B and M = A^T A of a symmetric pair in one pass (p == q, sym, at most 128
// blocks): the staged rows of A serve as M's second operand, so M costs no staging of its own.
// M's partials go to W1.
template <bool DF, bool FUSED>
__global__ void __launch_bounds__(256) k_gram_pairs_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  using R = Ar<DF>;
  using in_t = typename R::in_t;
  using acc_t = typename R::acc_t;
  constexpr int PMAX = 48;
  constexpr int PER = FUSED ? 1 : 4;  // blocks a thread at most
  __shared__ in_t As[RB * PMAX];
  __shared__ in_t Bs[RB * PMAX];
  __shared__ double gsum[4][256];
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  const int chunk = (int)((int64_t)blockIdx.x - j.cta_begin);
  const int64_t rpc = (j.n + j.x0 - 1) / j.x0;
  const int64_t r0 = (int64_t)chunk * rpc;
  const int64_t r1 = (r0 + rpc) < j.n ? (r0 + rpc) : j.n;
  const int p = j.p, q = j.q, tid = threadIdx.x;
  const int bp = (p + 1) / 2, bq = (q + 1) / 2, pe = 2 * bp, qe = 2 * bq;
  const int nblocks = j.x1 ? bp * (bp + 1) / 2 : bp * bq;
  const int P = nblocks;                           // threads of a row group
  const int G = nblocks <= 128 ? 256 / P : 1;      // row groups (threads past G P idle)
  const int slot = G > 1 ? tid % P : tid, grp = G > 1 ? tid / P : 0;
  const int per = G > 1 ? 1 : PER;
  int ba[PER], bb[PER];
  acc_t acc[PER][4], acm[PER][4];
#pragma unroll
  for (int u = 0; u < PER; u++) {
#pragma unroll
    for (int e = 0; e < 4; e++) { R::zero(acc[u][e]); R::zero(acm[u][e]); }
    int idx = slot + 256 * u;
    ba[u] = -1;
    bb[u] = 0;
    if (u < per && idx < nblocks && grp < G) {
      if (j.x1) {  // idx-th block (A, B), A <= B, row-major over the upper triangle of blocks
        int a = 0;
        while (idx >= bp - a) { idx -= bp - a; a++; }
        ba[u] = 2 * a;
        bb[u] = 2 * (a + idx);
      } else {
        ba[u] = 2 * (idx / bq);
        bb[u] = 2 * (idx % bq);
      }
    }
  }
  // rows staged per step: the shared arrays hold RB rows of 48 columns, so narrow blocks stage
  // proportionally more rows (each row group then has several rows per barrier)
  const int RS = (RB * PMAX) / (pe > qe ? pe : qe);
  for (int64_t rr = r0; rr < r1; rr += RS) {
    for (int idx = tid; idx < RS * pe; idx += 256) {
      const int i = idx / pe, a = idx % pe;
      const int64_t r = rr + i;
      As[idx] = (r < r1 && a < p) ? R::load(j.A[r * j.lda + a]) : R::zero_in();
    }
    for (int idx = tid; idx < RS * qe; idx += 256) {
      const int i = idx / qe, a = idx % qe;
      const int64_t r = rr + i;
      Bs[idx] = (r < r1 && a < q) ? R::load(j.B[r * j.ldb + a]) : R::zero_in();
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; u++) {
      if (ba[u] < 0) continue;
      for (int i = grp; i < RS; i += G) {
        const in_t* ar = As + i * pe;
        const in_t* br = Bs + i * qe;
        const in_t a0 = ar[ba[u]], a1 = ar[ba[u] + 1], b0 = br[bb[u]], b1 = br[bb[u] + 1];
        R::mac(acc[u][0], a0, b0);
        R::mac(acc[u][1], a0, b1);
        R::mac(acc[u][2], a1, b0);
        R::mac(acc[u][3], a1, b1);
        if (FUSED) {
          const in_t c0 = ar[bb[u]], c1 = ar[bb[u] + 1];
          R::mac(acm[u][0], a0, c0);
          R::mac(acm[u][1], a0, c1);
          R::mac(acm[u][2], a1, c0);
          R::mac(acm[u][3], a1, c1);
        }
      }
    }
    __syncthreads();
  }
  const int pq = p * q;
  if (G > 1) {
    // fixed-order sum over the row groups (FP64 values of each group's partials)
    for (int out = 0; out < (FUSED ? 2 : 1); out++) {
      acc_t* ac = out == 0 ? acc[0] : acm[0];
      double* W = out == 0 ? j.W0 : j.W1;
      if (out) __syncthreads();  // the first product's sums have been read
#pragma unroll
      for (int e = 0; e < 4; e++) gsum[e][tid] = ba[0] >= 0 ? R::out(ac[e]) : 0.0;
      __syncthreads();
      if (grp == 0 && ba[0] >= 0) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int a = ba[0] + e / 2, b = bb[0] + e % 2;
          if (a >= p || b >= q) continue;
          double sum = 0.0;
          for (int g = 0; g < G; g++) sum += gsum[e][g * P + slot];
          W[(int64_t)chunk * pq + (int64_t)a * q + b] = sum;
        }
      }
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < PER; u++) {
    if (ba[u] < 0) continue;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int a = ba[u] + e / 2, b = bb[u] + e % 2;
      if (a < p && b < q) {
        j.W0[(int64_t)chunk * pq + (int64_t)a * q + b] = R::out(acc[u][e]);
        if (FUSED) j.W1[(int64_t)chunk * pq + (int64_t)a * q + b] = R::out(acm[u][e]);
      }
    }
  }
}

// Batched fixed-order sum of the chunk partials: job fields W0, x0 (chunks), p, q, x1 (sym),
// x3 (which entries of a symmetric result were formed: 0 = the tile kernel's, entries with
// a / 16 > b / 16 missing; 1 = the pair kernel's, a > b missing), Y; ceil(p q 32 / 256) CTAs.
__global__ void k_gram_reduce_batch(const lob_bjob* __restrict__ jobs, int njobs) {
  const lob_bjob& j = jobs[find_job(jobs, njobs, blockIdx.x)];
  const int64_t lb = (int64_t)blockIdx.x - j.cta_begin;
  const int e = (int)((lb * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
  const int pq = j.p * j.q;
  if (e >= pq) return;
  int src = e;
  if (j.x1) {
    const int a = e / j.q, b = e % j.q;
    if (j.x3 ? a > b : a / 16 > b / 16) src = b * j.q + a;
  }
  double s = 0.0;
  for (int c = lane; c < j.x0; c += 32) s += j.W0[(int64_t)c * pq + src];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) j.Y[e] = s;
}

// Row chunks of one Gram product: one full wave of CTAs over all output tiles -- as many CTAs as
// fit on an SM by registers (8 for 16 x 16 tiles, 6 for 32 x 32, 5 for 48 x 48) -- with at least
// 64 rows each.
inline int nchunks_for(int64_t n, int tiles, int edge) {
  int64_t c = ((edge == 16 ? 8 : (edge == 32 ? 6 : 5)) * 152 + tiles - 1) / tiles;
  int64_t maxc = (n + 63) / 64;
  if (c > maxc) c = maxc;
  return (int)(c < 1 ? 1 : c);
}

}  // namespace

static int gram_edge(int p, int q) {
  const int mx = p > q ? p : q;
  return mx <= 16 ? 16 : (mx <= 32 ? 32 : TG);
}

size_t lob_gram_work_doubles(int64_t n, int p, int q) {
  const int e = gram_edge(p, q);
  const int tiles = ((p + e - 1) / e) * ((q + e - 1) / e);
  return (size_t)nchunks_for(n, tiles, e) * p * q;
}

template <bool DF>
static void gram_go(dim3 grid, cudaStream_t st, int U, int64_t n, int p, const double* A, int lda, int q,
                    const double* B, int ldb, double* work, int64_t rpc, int sym) {
  if (U == 1) (k_gram<DF, 1><<<grid, 256, 0, st>>>(n, p, A, lda, q, B, ldb, work, rpc, sym), LOB_LAUNCHED());
  else if (U == 2) (k_gram<DF, 2><<<grid, 256, 0, st>>>(n, p, A, lda, q, B, ldb, work, rpc, sym), LOB_LAUNCHED());
  else (k_gram<DF, 3><<<grid, 256, 0, st>>>(n, p, A, lda, q, B, ldb, work, rpc, sym), LOB_LAUNCHED());
}

int lob_gram_launch_ws(int64_t n, int p, const double* A, int lda, int q, const double* B, int ldb, double* G,
                       int mode, double* work, cudaStream_t st, int sym) {
  if (sym && p != q) return LOB_ERR_ARG;
  // FP64-class products go to the tensor cores (ozaki.cu) when they fit; LOB_SPMM_DF64 keeps the
  // double-float CUDA-core kernel
  if ((mode == LOB_SPMM_MIXED && lob_oz_pays(p, q)) || mode == LOB_BLAS_TC)
    return lob_gram_oz_launch(n, p, A, lda, nullptr, 0, q, B, ldb, G, nullptr, work, st);
  const int e = gram_edge(p, q);
  const int ta = (p + e - 1) / e, tb = (q + e - 1) / e;
  const int nch = nchunks_for(n, sym ? ta * (ta + 1) / 2 : ta * tb, e);
  const int64_t rpc = (n + nch - 1) / nch;
  dim3 grid(nch, ta, tb);
  if (mode != LOB_SPMM_FP64) gram_go<true>(grid, st, e / 16, n, p, A, lda, q, B, ldb, work, rpc, sym);
  else gram_go<false>(grid, st, e / 16, n, p, A, lda, q, B, ldb, work, rpc, sym);
  const int pq = p * q;
  (k_gram_reduce<<<(pq * 32 + 255) / 256, 256, 0, st>>>(nch, pq, q, sym, e, work, G), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

int lob_gram_launch(int64_t n, int p, const double* A, int lda, int q, const double* B, int ldb, double* G, int mode,
                    cudaStream_t st) {
  if (n < 1 || p < 1 || q < 1 || p > 192 || q > 192 || lda < p || ldb < q || !A || !B || !G) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_FP64 && mode != LOB_SPMM_MIXED && mode != LOB_SPMM_DF64 && mode != LOB_BLAS_TC)
    return LOB_ERR_ARG;
  if (mode == LOB_BLAS_TC && !lob_oz_fits(p, q)) return LOB_ERR_ARG;
  double* work = nullptr;
  const size_t wd = lob_gram_work_doubles(n, p, q), wo = lob_gram_oz_work_doubles();
  LOB_CUDA(cudaMallocAsync((void**)&work, (wd > wo ? wd : wo) * sizeof(double), st));
  int rc = lob_gram_launch_ws(n, p, A, lda, q, B, ldb, G, mode, work, st);
  cudaFreeAsync(work, st);
  return rc;
}

int lob_lincomb_launch(int64_t n, int p, const double* A, int lda, int q, const double* C, double* Y, int ldy,
                       int mode, cudaStream_t st, const double* D, int ldd) {
  if (n < 1 || p < 1 || q < 1 || p > 192 || q > 192 || lda < p || ldy < q || !A || !C || !Y) return LOB_ERR_ARG;
  if (mode != LOB_SPMM_FP64 && mode != LOB_SPMM_MIXED && mode != LOB_SPMM_DF64 && mode != LOB_BLAS_TC)
    return LOB_ERR_ARG;
  if (mode == LOB_BLAS_TC && !lob_oz_fits(p, q)) return LOB_ERR_ARG;
  if ((mode == LOB_SPMM_MIXED && lob_oz_pays(p, q)) || mode == LOB_BLAS_TC)
    return lob_lincomb_oz_launch(n, p, A, lda, q, C, Y, ldy, st, D, ldd);
  // four rows a thread when the CTA's rows of A fit comfortably in shared memory, else one
  const int RM = p <= 64 ? 4 : 1;
  dim3 grid((unsigned)((n + 16 * RM - 1) / (16 * RM)), (q + 15) / 16);
  const size_t smem = (16ull * RM * (p | 1) + 16ull * p) * (mode != LOB_SPMM_FP64 ? sizeof(float2) : sizeof(double));
  auto go = [&](auto kern) -> int {
    LOB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    (kern<<<grid, 256, smem, st>>>(n, p, A, lda, q, C, Y, ldy, D, ldd), LOB_LAUNCHED());
    LOB_CUDA(cudaGetLastError());
    return LOB_OK;
  };
  if (mode != LOB_SPMM_FP64) return RM == 4 ? go(k_lincomb<true, 4>) : go(k_lincomb<true, 1>);
  return RM == 4 ? go(k_lincomb<false, 4>) : go(k_lincomb<false, 1>);
}

int lob_gram_chunks(int64_t n, int p, int q) {
  const int e = gram_edge(p, q);
  return nchunks_for(n, ((p + e - 1) / e) * ((q + e - 1) / e), e);
}

int lob_gram_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int pqmax, int mode,
                          lob_bjob* red_host, lob_bjob* red_dev, cudaStream_t st, int pairs, int fused) {
  if (njobs <= 0) return LOB_OK;
  if (pqmax > TG) return LOB_ERR_ARG;
  for (int i = 0; pairs && i < njobs; i++) {
    const lob_bjob& j = jobs_host[i];
    const int bp = (j.p + 1) / 2, bq = (j.q + 1) / 2;
    const int nbl = j.x1 ? bp * (bp + 1) / 2 : bp * bq;
    if (nbl > 1024 || j.p > 48 || j.q > 48) return LOB_ERR_ARG;
    if (fused && (nbl > 128 || j.p != j.q || !j.x1 || !j.W1 || !j.D)) return LOB_ERR_ARG;
  }
  if (fused && !pairs) return LOB_ERR_ARG;
  // reductions: one per product (two per fused job: G from W0 into Y, M from W1 into D)
  int64_t ctas = 0, rctas = 0;
  int nred = 0;
  for (int i = 0; i < njobs; i++) {
    lob_bjob& j = jobs_host[i];
    j.cta_begin = ctas;
    ctas += j.x0;
    for (int o = 0; o < (fused ? 2 : 1); o++) {
      lob_bjob rj = j;
      if (o == 1) { rj.W0 = j.W1; rj.Y = const_cast<double*>(j.D); }  // a fused job carries M's output in D
      rj.cta_begin = rctas;
      rj.x3 = pairs ? 1 : 0;  // which entries of a symmetric result were formed
      red_host[nred++] = rj;
      rctas += ((int64_t)j.p * j.q * 32 + 255) / 256;
    }
  }
  LOB_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, njobs * sizeof(lob_bjob), cudaMemcpyHostToDevice, st));
  LOB_CUDA(cudaMemcpyAsync(red_dev, red_host, nred * sizeof(lob_bjob), cudaMemcpyHostToDevice, st));
  const int U = pqmax <= 16 ? 1 : (pqmax <= 32 ? 2 : 3);
  if (pairs) {
    if (mode == LOB_SPMM_MIXED) {
      if (fused) (k_gram_pairs_batch<true, true><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
      else (k_gram_pairs_batch<true, false><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    } else {
      if (fused) (k_gram_pairs_batch<false, true><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
      else (k_gram_pairs_batch<false, false><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    }
  } else if (mode == LOB_SPMM_MIXED) {
    if (U == 1) (k_gram_batch<true, 1><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    else if (U == 2) (k_gram_batch<true, 2><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    else (k_gram_batch<true, 3><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
  } else {
    if (U == 1) (k_gram_batch<false, 1><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    else if (U == 2) (k_gram_batch<false, 2><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
    else (k_gram_batch<false, 3><<<(unsigned)ctas, 256, 0, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
  }
  (k_gram_reduce_batch<<<(unsigned)rctas, 256, 0, st>>>(red_dev, nred), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

template <bool DF, int QT>
static int lincomb_batch_go(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int pmax, cudaStream_t st) {
  constexpr int RPC = lb_rm(QT) * 256 / QT;
  int64_t ctas = 0;
  for (int i = 0; i < njobs; i++) {
    jobs_host[i].cta_begin = ctas;
    ctas += (jobs_host[i].n + RPC - 1) / RPC;
  }
  if (ctas == 0) return LOB_OK;
  LOB_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, njobs * sizeof(lob_bjob), cudaMemcpyHostToDevice, st));
  const size_t smem = ((size_t)RPC * (pmax | 1) + (size_t)QT * pmax) * (DF ? sizeof(float2) : sizeof(double));
  LOB_CUDA(cudaFuncSetAttribute(k_lincomb_batch<DF, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  (k_lincomb_batch<DF, QT><<<(unsigned)ctas, 256, smem, st>>>(jobs_dev, njobs), LOB_LAUNCHED());
  LOB_CUDA(cudaGetLastError());
  return LOB_OK;
}

// All jobs of one call must share the output width class (q <= 1, 2, 4, 8 or 16; qmax selects).
int lob_lincomb_batch_launch(lob_bjob* jobs_host, lob_bjob* jobs_dev, int njobs, int pmax, int qmax, int mode,
                             cudaStream_t st) {
  if (njobs <= 0) return LOB_OK;
  if (qmax > 16 || pmax > 64) return LOB_ERR_ARG;
  const bool df = mode == LOB_SPMM_MIXED;
  if (qmax <= 1)
    return df ? lincomb_batch_go<true, 1>(jobs_host, jobs_dev, njobs, pmax, st)
              : lincomb_batch_go<false, 1>(jobs_host, jobs_dev, njobs, pmax, st);
  if (qmax <= 2)
    return df ? lincomb_batch_go<true, 2>(jobs_host, jobs_dev, njobs, pmax, st)
              : lincomb_batch_go<false, 2>(jobs_host, jobs_dev, njobs, pmax, st);
  if (qmax <= 4)
    return df ? lincomb_batch_go<true, 4>(jobs_host, jobs_dev, njobs, pmax, st)
              : lincomb_batch_go<false, 4>(jobs_host, jobs_dev, njobs, pmax, st);
  if (qmax <= 8)
    return df ? lincomb_batch_go<true, 8>(jobs_host, jobs_dev, njobs, pmax, st)
              : lincomb_batch_go<false, 8>(jobs_host, jobs_dev, njobs, pmax, st);
  return df ? lincomb_batch_go<true, 16>(jobs_host, jobs_dev, njobs, pmax, st)
            : lincomb_batch_go<false, 16>(jobs_host, jobs_dev, njobs, pmax, st);
}
