// Preconditioned conjugate gradients on t right-hand sides at once (mBCG; the
// footnote to Sec. 4.4 runs y and every probe through one CG call).
//
// Per column c (independent scalars, shared kernel launches):
//   x = 0, r = b, z = P^-1 r, p = z, rho = r^T z
//   repeat: q = K_hat p; alpha = rho / p^T q; x += alpha p; r -= alpha q
//           (every R steps r = b - K_hat x); stop on ||r|| <= tol ||b|| or the cap
//           z = P^-1 r; rho' = r^T z; beta = rho' / rho; p = z + beta p
// P^-1 r = sigma^-2 (r - L C^-1 L^T r) with C = sigma^2 I + L^T L (matrix
// inversion lemma, Sec. 2.2): L^T r and the final product in the problem
// precision, C^-1 (L^T r) in FP64.
//
// Every launch reads the device count of active columns and returns at once when
// it is zero, so the host can enqueue several iterations between convergence polls.
// When the stream is being captured into a CUDA graph, the iteration loop is a
// conditional WHILE node instead: the body is one iteration, the kernels read the
// iteration index and the residual-recompute flag from a device control block
// (ctl), and a one-thread kernel at the end of the body advances it and sets the
// loop condition (columns still active and j < max_iter).  Both paths launch the
// same kernels in the same order, so they give identical results.
// Column-wise reductions write per-block partials; a small kernel with one block per
// column (alpha_combine, update_decide, rho_finish) sums them in a fixed order
// (deterministic) and takes the column's scalar step, so the combines of all columns
// run side by side instead of in the last block of the reduction.
#include "ops.h"

namespace gp {
namespace {

constexpr int kThreads = 256;

template <class T>
struct Dev {
  T *X, *R, *Z, *P, *Q, *Sp;
  const T* B;
  int64_t ldb;
  double *rho, *rho0, *bnorm2, *alpha, *beta, *part, *S;
  int *active, *caps, *iters, *n_active, *status;
  unsigned* counter;
  const int* ctl;   // null (host loop) or {j, recompute, recompute gate}
};

template <class T>
Dev<T> dev_of(const CgBufs<T>& cb, const T* B, int64_t ldb) {
  Dev<T> d;
  d.X = cb.X; d.R = cb.R; d.Z = cb.Z; d.P = cb.P; d.Q = cb.Q; d.Sp = cb.Sp;
  d.B = B; d.ldb = ldb;
  d.rho = cb.rho; d.rho0 = cb.rho0; d.bnorm2 = cb.bnorm2; d.alpha = cb.alpha; d.beta = cb.beta;
  d.part = cb.part; d.S = cb.S;
  d.active = cb.active; d.caps = cb.caps; d.iters = cb.iters; d.n_active = cb.n_active;
  d.status = cb.status; d.counter = cb.counter;
  d.ctl = nullptr;
  return d;
}

// Each block owns one contiguous chunk of rows; inside it, warp w handles columns
// w, w + 8, ... so every column is read as coalesced 128-byte segments and reduced
// with warp shuffles (no block barrier per column).  The per-block partials are
// combined in a fixed order by one block per column (cg_init: by its last block).
__device__ __forceinline__ void row_chunk(int64_t n, int64_t* r0, int64_t* r1) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  *r0 = blockIdx.x * per;
  *r1 = min(n, *r0 + per);
}

// Dot-product accumulator of the column reductions.  FP64 arithmetic is slow on this
// part, so the FP32 path accumulates with the compensated "Dot2" scheme of Ogita,
// Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// each product is split exactly into p + e (TwoProduct via FMA) and each addition
// into s + q (Knuth's TwoSum); the error terms are summed separately, which gives the
// accuracy of a twice-as-precise accumulation.  The warp combine uses the same TwoSum
// (exact, so every lane of the butterfly ends with the same pair), and only the
// per-warp result is converted to FP64.  __fmul_rn / __fadd_rn keep the compiler from
// fusing the steps, which the error-free transformations rely on.
template <class T>
struct DotAcc {
  T s = T(0);
  __device__ __forceinline__ void add(T x, T y) { s = fma(x, y, s); }
  __device__ __forceinline__ double warp_total() { return warp_sum(s); }
};
template <>
struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void two_sum(float a, float b, float& sum, float& err) {
    sum = __fadd_rn(a, b);
    const float z = __fadd_rn(sum, -a);
    err = __fadd_rn(__fadd_rn(a, -__fadd_rn(sum, -z)), __fadd_rn(b, -z));
  }
  __device__ __forceinline__ void add(float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);              // x y = p + e exactly
    float q;
    two_sum(s, p, s, q);
    c = __fadd_rn(c, __fadd_rn(q, e));
  }
  __device__ __forceinline__ double warp_total() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
      const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
      float q;
      two_sum(s, s2, s, q);
      c = __fadd_rn(__fadd_rn(c, c2), q);
    }
    return (double)s + (double)c;
  }
};

// Sum of the nb per-block partials of column c, by one warp: lane-strided FP64 sums in
// four independent chains (four loads in flight per lane), combined in a fixed order,
// then a shuffle tree (deterministic); the result is in every lane.
__device__ __forceinline__ double warp_col_sum(const double* part, int nb, int c) {
  const int lane = threadIdx.x & 31;
  const double* pc = part + (size_t)c * nb;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int b = lane;
  for (; b + 96 < nb; b += 128) {
    s0 += pc[b];
    s1 += pc[b + 32];
    s2 += pc[b + 64];
    s3 += pc[b + 96];
  }
  for (; b < nb; b += 32) s0 += pc[b];
  return warp_sum((s0 + s1) + (s2 + s3));
}

// Sum of the nb per-block partials of column c by a whole block: thread-strided FP64
// sums and block_sum's fixed tree (deterministic); the result is in warp 0.
__device__ __forceinline__ double block_col_sum(const double* part, int nb, int c,
                                                double* sh) {
  const double* pc = part + (size_t)c * nb;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += pc[b];
  return block_sum(s, sh);
}

// Blocks of the column reductions and of the preconditioner's z pass: two 256-thread
// blocks per SM (one wave), so each column has 2 x SMs per-block partials.
int cg_grid() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      sms = 152;
  }
  return 2 * sms;
}

// x = 0, r = b, ||b||^2, caps, active set.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_init(int64_t n, int t, int max_iter,
                                                   const int* __restrict__ iters_override,
                                                   Dev<T> g) {
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int c = warp; c < t; c += kThreads / 32) {
    DotAcc<T> acc;
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      const T b = g.B[a + c * g.ldb];
      g.X[a + c * n] = T(0);
      g.R[a + c * n] = b;
      acc.add(b, b);
    }
    const double sum = acc.warp_total();
    if (lane == 0) g.part[c * nb + blockIdx.x] = sum;
  }
  if (last_block_arrived(g.counter)) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = warp; c < t; c += kThreads / 32) {
      const double s = warp_col_sum(g.part, nb, c);
      if (lane != 0) continue;
      g.bnorm2[c] = s;
      int cap = max_iter;
      int act;
      if (iters_override) {
        cap = min(max(iters_override[c], 0), max_iter);
        act = cap > 0;
      } else {
        act = s > 0.0;
      }
      g.caps[c] = cap;
      g.active[c] = act;
      g.iters[c] = 0;
      g.rho[c] = 0.0;
      g.rho0[c] = 0.0;
      if (act) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *g.n_active = cnt;
  }
}

// ---- preconditioner P^-1 R = sigma^-2 (R - L C^-1 L^T R) ------------------------------
// One application streams L (n x k) twice, with two small steps in between:
//   (1) S_part[b] = L^T R over the rows of part b               ltr_partial
//   (2) S = sum of the parts in part order (FP64)                s_reduce
//   (3) Sp = C^-1 S (FP64)                                       cinv_apply
//   (4) Z = sigma^-2 (R - L Sp), r^T z partials per column          precond_rho
//   (5) rho (and beta, or a column stops), one block per column       rho_finish
// The two n-long products keep a register tile per thread and stage tiles of L and of
// the right-hand sides in shared memory.  The lanes of a warp own pivots (1) or rows
// (4) 32 apart, so their shared-memory reads of L are conflict-free; the eight warps
// own disjoint groups of CPW = TC / 8 columns.  A warp's columns sit in an 8-wide,
// 32-byte aligned slot of the staged tile, which every lane reads as one broadcast of
// 16-byte loads.  Per row (1) or pivot (4) a warp issues MI (or RI) + 2 shared-memory
// wavefronts for MI (or RI) x CPW FMAs.

// The CPW values of a warp's column slot (16-byte aligned), by 16-byte broadcast loads.
template <class T, int CPW>
__device__ __forceinline__ void slot_read(const T* p, T (&v)[CPW]) {
  constexpr int V = 16 / (int)sizeof(T);
  constexpr int NV = (CPW + V - 1) / V;
  T buf[NV * V];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if constexpr (sizeof(T) == 4) {
      const float4 x = reinterpret_cast<const float4*>(p)[q];
      buf[4 * q] = x.x;
      buf[4 * q + 1] = x.y;
      buf[4 * q + 2] = x.z;
      buf[4 * q + 3] = x.w;
    } else {
      const double2 x = reinterpret_cast<const double2*>(p)[q];
      buf[2 * q] = x.x;
      buf[2 * q + 1] = x.y;
    }
  }
#pragma unroll
  for (int j = 0; j < CPW; ++j) v[j] = buf[j];
}

// Slot position of column c in a staged tile of TC columns.
template <int TC>
__device__ __forceinline__ int col_slot(int c) {
  constexpr int CPW = TC / 8;
  return (c / CPW) * 8 + c % CPW;
}

// (1) Lane l of warp w owns pivots m0 + l + 32 i (i < MI) and columns w CPW .. w CPW +
//     CPW - 1 of a slice of 32 MI pivots.  Rows go through shared memory in stages of
//     RS; the next stage is loaded into registers while the current one is multiplied.
//     Each part sums its rows in order, so the partials do not depend on the slicing.
constexpr int kLtrParts = 304;    // row parts (two blocks per SM with one slice); x slices
constexpr int kLtrThreads = 256;
template <class T>
__host__ __device__ constexpr int ltr_rows() { return sizeof(T) == 4 ? 32 : 16; }
template <class T, int TC, int MI>
__global__ void __launch_bounds__(kLtrThreads) ltr_partial(int64_t n, int t,
                                                          const T* __restrict__ L, int64_t ldl,
                                                          int k, Dev<T> g) {
  if (*g.n_active == 0) return;
  constexpr int CPW = TC / 8;
  constexpr int RS = ltr_rows<T>();
  constexpr int MS = 32 * MI;                                     // pivots of the slice
  constexpr int LP = MS + 1;                      // odd pitch: conflict-free staging stores
  constexpr int NL = RS * MS / kLtrThreads;                       // L values per thread
  constexpr int NR = (RS * TC + kLtrThreads - 1) / kLtrThreads;   // R values per thread
  static_assert(RS * MS % kLtrThreads == 0, "stage must split evenly over the threads");
  __shared__ T sL[RS][LP];
  __shared__ __align__(16) T sR[RS][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m0 = blockIdx.x * MS;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = blockIdx.y * per, r1 = min(n, r0 + per);
  T acc[MI][CPW];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < CPW; ++j) acc[i][j] = T(0);
  // element e of a stage: row e % RS (consecutive threads on consecutive rows:
  // coalesced), pivot or column e / RS
  T pl[NL], pr[NR];
  auto fetch = [&](int64_t rb) {
    const int rn = (int)min((int64_t)RS, r1 - rb);
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      const int rr = e % RS, mm = e / RS;
      pl[q] = (rr < rn && m0 + mm < k) ? L[rb + rr + (int64_t)(m0 + mm) * ldl] : T(0);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      const int rr = e % RS, c = e / RS;
      pr[q] = (e < RS * TC && rr < rn && c < t) ? g.R[rb + rr + (int64_t)c * n] : T(0);
    }
  };
  if (r0 < r1) fetch(r0);
  for (int64_t rb = r0; rb < r1; rb += RS) {
    __syncthreads();                 // the previous stage has been read
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      sL[e % RS][e / RS] = pl[q];
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      if (e < RS * TC) sR[e % RS][col_slot<TC>(e / RS)] = pr[q];
    }
    __syncthreads();
    if (rb + RS < r1) fetch(rb + RS);   // in flight during the FMAs below
#pragma unroll 4
    for (int rr = 0; rr < RS; ++rr) {
      T lv[MI], rv[CPW];
#pragma unroll
      for (int i = 0; i < MI; ++i) lv[i] = sL[rr][lane + 32 * i];
      slot_read<T, CPW>(&sR[rr][w * 8], rv);
#pragma unroll
      for (int j = 0; j < CPW; ++j)
#pragma unroll
        for (int i = 0; i < MI; ++i) acc[i][j] = fma(lv[i], rv[j], acc[i][j]);
    }
  }
  double* out = g.S + (size_t)blockIdx.y * k * t;     // per-part partials (t x k)
#pragma unroll
  for (int i = 0; i < MI; ++i) {
    const int m = m0 + lane + 32 * i;
    if (m >= k) continue;
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      const int col = w * CPW + j;
      if (col < t) out[(size_t)col * k + m] = (double)acc[i][j];
    }
  }
}

// (2) S[e] = sum over parts b of part[b][e], e = c k + m < tc k, in part order.  Block:
//     32 consecutive e (lanes); warp w sums parts w, w + 8, ... with two chains, and
//     warp 0 adds the eight warp sums in warp order (deterministic).
__global__ void __launch_bounds__(256) s_reduce(int64_t ne, int nparts,
                                                const double* __restrict__ part,
                                                double* __restrict__ S,
                                                const int* __restrict__ n_active) {
  if (*n_active == 0) return;
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  double a0 = 0.0, a1 = 0.0;
  if (e < ne) {
    int b = w;
    for (; b + 8 < nparts; b += 16) {
      a0 += part[(int64_t)b * ne + e];
      a1 += part[(int64_t)(b + 8) * ne + e];
    }
    if (b < nparts) a0 += part[(int64_t)b * ne + e];
  }
  sh[w][lane] = a0 + a1;
  __syncthreads();
  if (w == 0 && e < ne) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += sh[q][lane];
    S[e] = s;
  }
}

// (3) Sp[i][c] = sum_m C^-1[m][i] S[c][m] for the active columns (C^-1 is exactly
//     symmetric: formed as Gc^-T Gc^-1 with one summation order).  Block (i-tile of
//     32, column c): lane = i, warp w takes m = w, w + 8, ... (coalesced rows of C^-1,
//     S broadcast), warp 0 adds the eight warp sums in warp order.
template <class T>
__global__ void __launch_bounds__(256) cinv_apply(int k, int ldsp,
                                                  const double* __restrict__ Cinv,
                                                  const double* __restrict__ S, Dev<T> g) {
  if (*g.n_active == 0) return;
  const int c = blockIdx.y;
  if (!g.active[c]) return;          // block-uniform
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const double* Sc = S + (size_t)c * k;
  double a0 = 0.0, a1 = 0.0;
  if (i < k) {
    int m = w;
    for (; m + 8 < k; m += 16) {
      a0 += Cinv[(int64_t)m * k + i] * Sc[m];
      a1 += Cinv[(int64_t)(m + 8) * k + i] * Sc[m + 8];
    }
    if (m < k) a0 += Cinv[(int64_t)m * k + i] * Sc[m];
  }
  sh[w][lane] = a0 + a1;
  __syncthreads();
  if (w == 0 && i < k) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += sh[q][lane];
    g.Sp[(int64_t)i * ldsp + c] = (T)s;
  }
}

// rho (mode 0: rho = rho0 = r^T z) or beta_j = r^T z / rho and rho = r^T z (mode 1) for
// the active column c0 + blockIdx.x, from the per-block partials of precond_rho.  One
// block per column, so the columns' combines run on as many SMs.
template <class T>
__global__ void __launch_bounds__(kThreads) rho_finish(int c0, int nb, int mode, int j,
                                                      int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl && mode != 0) j = g.ctl[0];
  const int c = c0 + blockIdx.x;
  if (!g.active[c]) return;          // block-uniform
  __shared__ double sh[32];
  const double s = block_col_sum(g.part, nb, c, sh);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    g.rho[c] = s;
    g.rho0[c] = s;
    return;
  }
  if (!(s > 0.0) || !isfinite(s)) {
    // r^T P^-1 r <= 0 only happens once r is at the rounding floor of the
    // preconditioner solve: the column stops here (no beta_j, m = j + 1 nodes)
    g.active[c] = 0;
    g.iters[c] = j + 1;
    atomicSub(g.n_active, 1);
    return;
  }
  double be = s / g.rho[c];
  if (!isfinite(be)) { raise_status(g.status, GP_ERR_NUMERIC); be = 0.0; }
  g.beta[(int64_t)c * max_iter + j] = be;
  g.rho[c] = s;
}

// (4) Tiles of 32 RI rows, visited by the blocks in a grid-stride loop (one wave of
//     cg_grid() blocks).  Lane l of warp w owns rows a0 + l + 32 i (i < RI) of the tile
//     and columns w CPW .. w CPW + CPW - 1.  Pivots go through shared memory
//     in chunks of MC; the next chunk of L and Sp is loaded into registers while the
//     current one is multiplied.  Then z, and r^T z summed over the block's rows per
//     column (compensated FP32 within the block, FP64 across blocks, in rho_finish).
constexpr int kPrRI = 4;
constexpr int kPrRows = 32 * kPrRI;
template <class T>
__host__ __device__ constexpr int pr_chunk() { return sizeof(T) == 4 ? 32 : 16; }
template <class T, int TC>
__global__ void __launch_bounds__(kThreads, 2) precond_rho(int64_t n, int t, int c0,
                                                       const T* __restrict__ L, int64_t ldl,
                                                       int k, const double* __restrict__ theta,
                                                       int D, Dev<T> g) {
  if (*g.n_active == 0) return;
  constexpr int CPW = TC / 8;
  constexpr int RI = kPrRI;
  constexpr int RT = kPrRows;
  constexpr int MC = pr_chunk<T>();
  constexpr int NL = MC * RT / kThreads;                        // L values per thread
  constexpr int NS = (MC * TC + kThreads - 1) / kThreads;       // Sp values per thread
  static_assert(MC * RT % kThreads == 0, "chunk must split evenly over the threads");
  __shared__ __align__(16) T sL[MC][RT];
  __shared__ __align__(16) T sSp[MC][64];
  __shared__ double swarp[kThreads / 32][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tc = min(TC, t - c0);
  const T inv_s2 = (T)(1.0 / theta[D + 1]);
  const int64_t ntiles = (n + RT - 1) / RT;
  DotAcc<T> rz[CPW];                 // r^T z over this block's rows, per column
  T acc[RI][CPW];
  int64_t a0 = 0;
  // L element e of a chunk: row e % RT (coalesced), pivot e / RT; Sp element e:
  // pivot e / TC, column e % TC
  T pl[NL], ps[NS];
  auto fetch = [&](int m0) {
    const int mn = min(MC, k - m0);
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kThreads;
      const int rr = e % RT, mm = e / RT;
      const int64_t a = a0 + rr;
      pl[q] = (mm < mn && a < n) ? L[a + (int64_t)(m0 + mm) * ldl] : T(0);
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int e = threadIdx.x + q * kThreads;
      const int mm = e / TC, c = e % TC;
      ps[q] = (e < MC * TC && mm < mn && c < tc) ? g.Sp[(int64_t)(m0 + mm) * t + c0 + c]
                                                 : T(0);
    }
  };
  auto step = [&](int mm) {
    T lv[RI], sv[CPW];
#pragma unroll
    for (int i = 0; i < RI; ++i) lv[i] = sL[mm][lane + 32 * i];
    slot_read<T, CPW>(&sSp[mm][w * 8], sv);
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
      for (int i = 0; i < RI; ++i) acc[i][q] = fma(lv[i], sv[q], acc[i][q]);
  };
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  a0 = tile * RT;
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int q = 0; q < CPW; ++q) acc[i][q] = T(0);
  if (k > 0) fetch(0);
  for (int m0 = 0; m0 < k; m0 += MC) {
    __syncthreads();                 // the previous chunk has been read
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kThreads;
      sL[e / RT][e % RT] = pl[q];
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int e = threadIdx.x + q * kThreads;
      if (e < MC * TC) sSp[e / TC][col_slot<TC>(e % TC)] = ps[q];
    }
    __syncthreads();
    const int mn = min(MC, k - m0);
    if (m0 + MC < k) fetch(m0 + MC);   // in flight during the FMAs below
    if (mn == MC) {
#pragma unroll 8
      for (int mm = 0; mm < MC; ++mm) step(mm);
    } else {
      for (int mm = 0; mm < mn; ++mm) step(mm);
    }
  }
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int col = w * CPW + q;
    if (col < tc && g.active[c0 + col]) {      // warp-uniform
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const int64_t row = a0 + lane + 32 * i;
        if (row < n) {
          const int64_t off = row + (int64_t)(c0 + col) * n;
          const T r = g.R[off];
          const T z = (r - acc[i][q]) * inv_s2;
          g.Z[off] = z;
          rz[q].add(r, z);
        }
      }
    }
  }
  __syncthreads();                   // the next tile's first stores reuse sL / sSp
  }
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const double rzw = rz[q].warp_total();
    if (lane == 0) swarp[w][q] = rzw;
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int col = threadIdx.x; col < tc; col += blockDim.x)
    g.part[(size_t)(c0 + col) * nb + blockIdx.x] = swarp[col / CPW][col % CPW];
}

// p = z (start) and optionally PinvB = z.
template <class T>
__global__ void p_start(int64_t n, int t, Dev<T> g, T* PinvB, int64_t ldpb) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * t) return;
  int c = (int)(e / n);
  int64_t a = e % n;
  T z = g.active[c] ? g.Z[e] : T(0);
  g.P[e] = z;
  if (PinvB) PinvB[a + c * ldpb] = z;
}

// The column reductions below visit four columns per warp pass (w, w + 8, w + 16,
// w + 24, then + 32 ...) and issue the loads of all four before their sums, so each
// lane keeps 8 (alpha) to 16 (update) loads in flight.
constexpr int kColGroup = 4;

// p^T q per column, as per-block partials (alpha_combine forms alpha_j = rho / p^T q).
template <class T>
__global__ void __launch_bounds__(kThreads) cg_alpha(int64_t n, int t, Dev<T> g) {
  if (*g.n_active == 0) return;
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int cb = warp; cb < t; cb += 8 * kColGroup) {
    bool act[kColGroup];
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) act[q] = cb + 8 * q < t && g.active[cb + 8 * q];
    DotAcc<T> acc[kColGroup];
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      T pv[kColGroup], qv[kColGroup];
#pragma unroll
      for (int q = 0; q < kColGroup; ++q) {
        const int64_t off = a + (int64_t)(cb + 8 * q) * n;
        pv[q] = act[q] ? g.P[off] : T(0);
        qv[q] = act[q] ? g.Q[off] : T(0);
      }
#pragma unroll
      for (int q = 0; q < kColGroup; ++q)
        if (act[q]) acc[q].add(pv[q], qv[q]);
    }
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) {
      if (!act[q]) continue;                     // warp-uniform
      const double sum = acc[q].warp_total();
      if (lane == 0) g.part[(cb + 8 * q) * nb + blockIdx.x] = sum;
    }
  }
}

// alpha_j = rho / p^T q for the active column blockIdx.x, from cg_alpha's partials.
template <class T>
__global__ void __launch_bounds__(kThreads) alpha_combine(int nb, int j, int max_iter,
                                                         Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) j = g.ctl[0];
  const int c = blockIdx.x;
  if (!g.active[c]) return;          // block-uniform
  __shared__ double sh[32];
  const double pq = block_col_sum(g.part, nb, c, sh);
  if (threadIdx.x != 0) return;
  const double al = g.rho[c] / pq;
  if (!(pq > 0.0) || !isfinite(al)) {
    // breakdown: the operator is not positive definite in this precision (or the
    // iterates overflowed); the column stops with the j steps it has
    raise_status(g.status, GP_ERR_NUMERIC);
    g.alpha[(int64_t)c * max_iter + j] = 0.0;
    g.active[c] = 0;
    g.iters[c] = j;
    atomicSub(g.n_active, 1);
    return;
  }
  g.alpha[(int64_t)c * max_iter + j] = al;
}

// The stopping decision for the active column blockIdx.x from the ||r||^2 partials of
// cg_update (from_update = 1) or cg_resid (0): stop when ||r|| <= tol ||b||, at the
// column's cap (iteration overrides) or at max_iter.  Under graph capture the
// recompute flag ctl[1] selects which of the two launches decides this step.
template <class T>
__global__ void __launch_bounds__(kThreads) update_decide(int nb, int j, int max_iter,
                                                         double tol2, int use_caps,
                                                         int from_update, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) {
    if ((g.ctl[1] != 0) == (from_update != 0)) return;
    j = g.ctl[0];
  }
  const int c = blockIdx.x;
  if (!g.active[c]) return;          // block-uniform
  bool stop, capped = false;
  if (use_caps) {
    if (threadIdx.x != 0) return;
    stop = (j + 1) >= g.caps[c];
  } else {
    __shared__ double sh[32];
    const double s = block_col_sum(g.part, nb, c, sh);
    if (threadIdx.x != 0) return;
    const bool conv = s <= tol2 * g.bnorm2[c];
    capped = !conv && (j + 1 >= max_iter);
    stop = conv || capped;
  }
  // the iteration cap ended a column above the tolerance: results are written, with a
  // warning (with per-column caps from the caller the stop is deliberate)
  if (capped) raise_status(g.status, GP_WARN_NOT_CONVERGED);
  if (stop) {
    g.active[c] = 0;
    g.iters[c] = j + 1;
    atomicSub(g.n_active, 1);
  }
}

// x += alpha p; r -= alpha q (active columns); ||r||^2 per column as per-block partials
// unless this step recomputes the residual (update_decide takes the stopping decision).
template <class T>
__global__ void __launch_bounds__(kThreads) cg_update(int64_t n, int t, int j, int max_iter,
                                                     int recompute, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) {
    j = g.ctl[0];
    recompute = g.ctl[1];
  }
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int cb = warp; cb < t; cb += 8 * kColGroup) {
    bool act[kColGroup];
    T al[kColGroup];
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) {
      const int c = cb + 8 * q;
      act[q] = c < t && g.active[c];
      al[q] = act[q] ? (T)g.alpha[(int64_t)c * max_iter + j] : T(0);
    }
    DotAcc<T> acc[kColGroup];
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      T xv[kColGroup], pv[kColGroup], qv[kColGroup], rv[kColGroup];
#pragma unroll
      for (int q = 0; q < kColGroup; ++q) {
        const int64_t off = a + (int64_t)(cb + 8 * q) * n;
        if (act[q]) {
          xv[q] = g.X[off];
          pv[q] = g.P[off];
          qv[q] = g.Q[off];
          rv[q] = g.R[off];
        }
      }
#pragma unroll
      for (int q = 0; q < kColGroup; ++q) {
        if (!act[q]) continue;
        const int64_t off = a + (int64_t)(cb + 8 * q) * n;
        g.X[off] = fma(al[q], pv[q], xv[q]);
        const T r = fma(-al[q], qv[q], rv[q]);
        g.R[off] = r;
        acc[q].add(r, r);
      }
    }
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) {
      if (!act[q]) continue;                     // warp-uniform
      const double sum = acc[q].warp_total();
      if (lane == 0 && !recompute) g.part[(cb + 8 * q) * nb + blockIdx.x] = sum;
    }
  }
}

// r = b - K_hat x (Q holds K_hat x) and ||r||^2 per column, as per-block partials
// (update_decide takes the stopping decision).
template <class T>
__global__ void __launch_bounds__(kThreads) cg_resid(int64_t n, int t, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl && !g.ctl[1]) return;    // not a residual-recompute step
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int cb = warp; cb < t; cb += 8 * kColGroup) {
    bool act[kColGroup];
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) act[q] = cb + 8 * q < t && g.active[cb + 8 * q];
    DotAcc<T> acc[kColGroup];
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      T bv[kColGroup], qv[kColGroup];
#pragma unroll
      for (int q = 0; q < kColGroup; ++q) {
        const int c = cb + 8 * q;
        bv[q] = act[q] ? g.B[a + (int64_t)c * g.ldb] : T(0);
        qv[q] = act[q] ? g.Q[a + (int64_t)c * n] : T(0);
      }
#pragma unroll
      for (int q = 0; q < kColGroup; ++q) {
        if (!act[q]) continue;
        const T r = bv[q] - qv[q];
        g.R[a + (int64_t)(cb + 8 * q) * n] = r;
        acc[q].add(r, r);
      }
    }
#pragma unroll
    for (int q = 0; q < kColGroup; ++q) {
      if (!act[q]) continue;                     // warp-uniform
      const double sum = acc[q].warp_total();
      if (lane == 0) g.part[(cb + 8 * q) * nb + blockIdx.x] = sum;
    }
  }
}

// p = z + beta_j p for active columns; four consecutive elements of the n x t arrays
// per thread (16-byte loads for FP32; the workspace arrays are 256-byte aligned).
constexpr int kPupV = 4;
template <class T>
__global__ void cg_pupdate(int64_t n, int t, int j, int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) j = g.ctl[0];
  const int64_t total = n * t;
  const int64_t e0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kPupV;
  if (e0 >= total) return;
  T pv[kPupV], zv[kPupV];
  const bool full = e0 + kPupV <= total;
  if constexpr (sizeof(T) == 4) {
    if (full) {
      const float4 p4 = *reinterpret_cast<const float4*>(g.P + e0);
      const float4 z4 = *reinterpret_cast<const float4*>(g.Z + e0);
      pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
      zv[0] = z4.x; zv[1] = z4.y; zv[2] = z4.z; zv[3] = z4.w;
    }
  } else {
    if (full) {
#pragma unroll
      for (int v = 0; v < kPupV; v += 2) {
        const double2 p2 = *reinterpret_cast<const double2*>(g.P + e0 + v);
        const double2 z2 = *reinterpret_cast<const double2*>(g.Z + e0 + v);
        pv[v] = p2.x; pv[v + 1] = p2.y;
        zv[v] = z2.x; zv[v + 1] = z2.y;
      }
    }
  }
  if (!full) {
#pragma unroll
    for (int v = 0; v < kPupV; ++v) {
      pv[v] = e0 + v < total ? g.P[e0 + v] : T(0);
      zv[v] = e0 + v < total ? g.Z[e0 + v] : T(0);
    }
  }
  int c = (int)(e0 / n);
  int64_t a = e0 - (int64_t)c * n;
#pragma unroll
  for (int v = 0; v < kPupV; ++v) {
    if (c < t && g.active[c]) pv[v] = fma((T)g.beta[(int64_t)c * max_iter + j], pv[v], zv[v]);
    if (++a == n) { a = 0; ++c; }
  }
  if (full) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(g.P + e0) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    } else {
#pragma unroll
      for (int v = 0; v < kPupV; v += 2)
        *reinterpret_cast<double2*>(g.P + e0 + v) = make_double2(pv[v], pv[v + 1]);
    }
  } else {
#pragma unroll
    for (int v = 0; v < kPupV; ++v)
      if (e0 + v < total) g.P[e0 + v] = pv[v];
  }
}

// Device loop control: ctl = {j, recompute step?, recompute gate (= n_active on a
// recompute step, else 0)}.  ctl_init sets j = 0; ctl_step advances j after an
// iteration.  Both set the WHILE condition: some column active and j < max_iter.
__device__ __forceinline__ void ctl_set(int* ctl, int j, int R, int max_iter, const int* n_active,
                                        cudaGraphConditionalHandle h) {
  const int rec = (R > 0 && (j + 1) % R == 0) ? 1 : 0;
  ctl[0] = j;
  ctl[1] = rec;
  ctl[2] = rec ? *n_active : 0;
  cudaGraphSetConditional(h, (*n_active > 0 && j < max_iter) ? 1u : 0u);
}
__global__ void ctl_init_kernel(int* ctl, int R, int max_iter, const int* n_active,
                                cudaGraphConditionalHandle h) {
  ctl_set(ctl, 0, R, max_iter, n_active, h);
}
__global__ void ctl_step_kernel(int* ctl, int R, int max_iter, const int* n_active,
                                cudaGraphConditionalHandle h) {
  ctl_set(ctl, ctl[0] + 1, R, max_iter, n_active, h);
}

// T_diag / T_off from the CG coefficients (Sec. S1.2).
__global__ void tridiag_kernel(int t, int max_iter, const double* alpha, const double* beta,
                               const int* iters, double* T_diag, double* T_off) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= t * max_iter) return;
  int c = e / max_iter, jj = e % max_iter;
  int m = iters[c];
  double dg = 0.0, of = 0.0;
  if (jj < m) {
    const double* al = alpha + (int64_t)c * max_iter;
    const double* be = beta + (int64_t)c * max_iter;
    dg = 1.0 / al[jj];
    if (jj > 0) dg += be[jj - 1] / al[jj - 1];
    if (jj < m - 1) of = sqrt(be[jj]) / al[jj];
  }
  T_diag[e] = dg;
  T_off[e] = of;
}

template <class T>
__global__ void __launch_bounds__(kThreads) dot_kernel(int64_t n, const T* a, const T* b,
                                                      double* part, unsigned* counter,
                                                      double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads)
    acc += (double)a[i] * (double)b[i];
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block_arrived(counter)) {
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (unsigned q = 0; q < gridDim.x; ++q) r += part[q];
      *out = r;
    }
  }
}

// A non-blocking stream per host thread and device on which the body of the
// captured iteration loop is recorded (cudaStreamBeginCaptureToGraph).
cudaStream_t capture_body_stream() {
  struct BodyStream {
    cudaStream_t s = nullptr;
    int device = -1;
  };
  static thread_local BodyStream bs;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (bs.s == nullptr || bs.device != dev) {
    if (cudaStreamCreateWithFlags(&bs.s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    bs.device = dev;
  }
  return bs.s;
}

int pick_tc16(int t) { return t <= 16 ? 16 : t <= 32 ? 32 : t <= 40 ? 40 : t <= 48 ? 48 : 64; }

#define GP_TC_DISPATCH(TCv, ...)                        \
  switch (TCv) {                                        \
    case 16: { constexpr int TC = 16; __VA_ARGS__; } break; \
    case 32: { constexpr int TC = 32; __VA_ARGS__; } break; \
    case 40: { constexpr int TC = 40; __VA_ARGS__; } break; \
    case 48: { constexpr int TC = 48; __VA_ARGS__; } break; \
    default: { constexpr int TC = 64; __VA_ARGS__; } break; \
  }

// Pivots per lane of ltr_partial: 7 (224-pivot slices) where that pads k less than 4
// (128-pivot slices) and the column tile is at most 40 wide (register tile); FP64
// always uses 4.
template <class T>
int ltr_mi(int k, int tcp) {
  if (sizeof(T) != 4 || tcp > 40) return 4;
  return cdiv(k, 224) * 224 < cdiv(k, 128) * 128 ? 7 : 4;
}

template <class T>
gp_status precond_apply(int64_t n, int t, const T* L, int64_t ldl, int k, const double* Cinv,
                        const double* theta, int D, int mode, int j, int max_iter,
                        const CgBufs<T>& cb, Dev<T>& g, cudaStream_t st) {
  if (k > 0) {
    // S = L^T R and Sp = C^-1 S, in column chunks of at most 64
    for (int c0 = 0; c0 < t; c0 += 64) {
      const int tc = std::min(64, t - c0);
      Dev<T> gc = g;                 // this chunk's columns; part partials into atb_part
      gc.R = g.R + (int64_t)c0 * n;
      gc.S = cb.atb_part;
      const int tcp = pick_tc16(tc);
      const int mi = ltr_mi<T>(k, tcp);
      const dim3 grid((unsigned)cdiv(k, 32 * mi), (unsigned)kLtrParts);
      if constexpr (sizeof(T) == 4) {
        if (mi == 7) {               // tcp <= 40 (ltr_mi)
          if (tcp == 16) {
            ltr_partial<T, 16, 7><<<grid, kLtrThreads, 0, st>>>(n, tc, L, ldl, k, gc);
          } else if (tcp == 32) {
            ltr_partial<T, 32, 7><<<grid, kLtrThreads, 0, st>>>(n, tc, L, ldl, k, gc);
          } else {
            ltr_partial<T, 40, 7><<<grid, kLtrThreads, 0, st>>>(n, tc, L, ldl, k, gc);
          }
        } else {
          GP_TC_DISPATCH(tcp, (ltr_partial<T, TC, 4><<<grid, kLtrThreads, 0, st>>>(
                                  n, tc, L, ldl, k, gc)));
        }
      } else {
        GP_TC_DISPATCH(tcp, (ltr_partial<T, TC, 4><<<grid, kLtrThreads, 0, st>>>(
                                n, tc, L, ldl, k, gc)));
      }
      GP_LAUNCH_CHECK();
      const int64_t ne = (int64_t)tc * k;
      s_reduce<<<(unsigned)cdiv(ne, 32), 256, 0, st>>>(ne, kLtrParts, cb.atb_part, cb.S,
                                                       g.n_active);
      GP_LAUNCH_CHECK();
      Dev<T> gs = g;                 // Sp columns c0.. (leading dimension t)
      gs.active = g.active + c0;
      gs.Sp = g.Sp + c0;
      cinv_apply<T><<<dim3((unsigned)cdiv(k, 32), (unsigned)tc), 256, 0, st>>>(k, t, Cinv,
                                                                              cb.S, gs);
      GP_LAUNCH_CHECK();
    }
  }
  // z = sigma^-2 (r - L Sp) and r^T z, then rho / beta per column.  The row tiles are
  // spread evenly over at most cg_grid() blocks (every block takes the same number).
  const int64_t ntiles = cdiv(n, kPrRows);
  const int nbp = (int)cdiv(ntiles, cdiv(ntiles, cg_grid()));
  for (int c0 = 0; c0 < t; c0 += 64) {
    const int tc = std::min(64, t - c0);
    GP_TC_DISPATCH(pick_tc16(tc), (precond_rho<T, TC><<<nbp, kThreads, 0, st>>>(
                                      n, t, c0, L, ldl, k, theta, D, g)));
    GP_LAUNCH_CHECK();
    rho_finish<T><<<tc, kThreads, 0, st>>>(c0, nbp, mode, j, max_iter, g);
    GP_LAUNCH_CHECK();
  }
  return GP_OK;
}

}  // namespace

template <class T>
gp_status cg_solve(const Prob& pb, MvmOp& mvm, const T* L, int64_t ldl, int k,
                   const double* Cinv, const T* B, int64_t ldb, int t,
                   const int* iters_override, const gp_opts& o, const CgBufs<T>& cb,
                   T* PinvB, int64_t ldpb, int* host_status, cudaStream_t st) {
  const int64_t n = pb.n;
  Dev<T> g = dev_of(cb, B, ldb);
  const int nb = (int)std::min<int64_t>(cg_grid(), cdiv(n, 128));
  const int use_caps = iters_override ? 1 : 0;
  const double tol2 = o.cg_tol * o.cg_tol;
  const int R = o.recompute_every;
  int check = o.check_every > 0 ? o.check_every : 4;

  cg_init<T><<<nb, kThreads, 0, st>>>(n, t, o.max_iter, iters_override, g);
  GP_LAUNCH_CHECK();
  GP_TRY(precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 0, 0, o.max_iter, cb, g, st));
  p_start<T><<<(unsigned)cdiv(n * t, 256), 256, 0, st>>>(n, t, g, PinvB, ldpb);
  GP_LAUNCH_CHECK();

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusActive) (void)capture_body_stream();   // create it early
  if (cap == cudaStreamCaptureStatusActive) {
    // graph capture: the iteration loop becomes a conditional WHILE node
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    GP_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cap, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h;
    GP_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, graph, 0, 0));
    ctl_init_kernel<<<1, 1, 0, st>>>(cb.ctl, R, o.max_iter, g.n_active, h);
    GP_LAUNCH_CHECK();
    GP_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cap, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    GP_CUDA_TRY(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    GP_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
    cudaStream_t bs = capture_body_stream();
    if (!bs) return GP_ERR_CUDA;
    GP_CUDA_TRY(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
    Dev<T> gd = g;
    gd.ctl = cb.ctl;
    gp_status rs = GP_OK;
    do {
      rs = mvm.apply(gd.P, n, t, gd.Q, n, gd.n_active, bs);
      if (rs != GP_OK) break;
      cg_alpha<T><<<nb, kThreads, 0, bs>>>(n, t, gd);
      alpha_combine<T><<<t, kThreads, 0, bs>>>(nb, 0, o.max_iter, gd);
      cg_update<T><<<nb, kThreads, 0, bs>>>(n, t, 0, o.max_iter, 0, gd);
      update_decide<T><<<t, kThreads, 0, bs>>>(nb, 0, o.max_iter, tol2, use_caps, 1, gd);
      if (R > 0) {
        rs = mvm.apply(gd.X, n, t, gd.Q, n, cb.ctl + 2, bs);   // gated: recompute steps only
        if (rs != GP_OK) break;
        cg_resid<T><<<nb, kThreads, 0, bs>>>(n, t, gd);
        update_decide<T><<<t, kThreads, 0, bs>>>(nb, 0, o.max_iter, tol2, use_caps, 0, gd);
      }
      rs = precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 1, 0, o.max_iter, cb, gd, bs);
      if (rs != GP_OK) break;
      cg_pupdate<T><<<(unsigned)cdiv(n * t, 256 * kPupV), 256, 0, bs>>>(n, t, 0, o.max_iter,
                                                                          gd);
      ctl_step_kernel<<<1, 1, 0, bs>>>(cb.ctl, R, o.max_iter, g.n_active, h);
    } while (false);
    cudaGraph_t body_out = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(bs, &body_out);
    if (rs != GP_OK) return rs;
    GP_CUDA_TRY(ec);
    GP_LAUNCH_CHECK();
    *host_status = 0;   // the status stays on the device (read after the graph runs)
    return GP_OK;
  }

  const bool timed = mvm_timing_enabled();
  for (int j = 0; j < o.max_iter; ++j) {
    if (timed) mvm_timing_begin(st);
    GP_TRY(mvm.apply(g.P, n, t, g.Q, n, g.n_active, st));
    if (timed) mvm_timing_end(st);
    if (timed) mvm_timing_begin(st, 2);
    cg_alpha<T><<<nb, kThreads, 0, st>>>(n, t, g);
    GP_LAUNCH_CHECK();
    alpha_combine<T><<<t, kThreads, 0, st>>>(nb, j, o.max_iter, g);
    GP_LAUNCH_CHECK();
    const int rec = (R > 0 && (j + 1) % R == 0) ? 1 : 0;
    cg_update<T><<<nb, kThreads, 0, st>>>(n, t, j, o.max_iter, rec, g);
    GP_LAUNCH_CHECK();
    if (!rec) {
      update_decide<T><<<t, kThreads, 0, st>>>(nb, j, o.max_iter, tol2, use_caps, 1, g);
      GP_LAUNCH_CHECK();
    }
    if (timed) mvm_timing_end(st, 2);
    if (rec) {
      if (timed) mvm_timing_begin(st);
      GP_TRY(mvm.apply(g.X, n, t, g.Q, n, g.n_active, st));
      if (timed) mvm_timing_end(st);
      cg_resid<T><<<nb, kThreads, 0, st>>>(n, t, g);
      GP_LAUNCH_CHECK();
      update_decide<T><<<t, kThreads, 0, st>>>(nb, j, o.max_iter, tol2, use_caps, 0, g);
      GP_LAUNCH_CHECK();
    }
    if (timed) mvm_timing_begin(st, 2);
    GP_TRY(precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 1, j, o.max_iter, cb, g, st));
    cg_pupdate<T><<<(unsigned)cdiv(n * t, 256 * kPupV), 256, 0, st>>>(n, t, j, o.max_iter, g);
    GP_LAUNCH_CHECK();
    if (timed) mvm_timing_end(st, 2);
    if ((j + 1) % check == 0 || j + 1 == o.max_iter) {
      int h = 0;
      GP_CUDA_TRY(cudaMemcpyAsync(&h, g.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      if (h == 0) break;
    }
  }
  int hs = 0;
  GP_CUDA_TRY(cudaMemcpyAsync(&hs, g.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  *host_status = hs;
  return GP_OK;
}

size_t cg_atb_part_elems(int64_t n, int k, int t) {
  (void)n;
  return (size_t)kLtrParts * std::max(k, 1) * std::min(std::max(t, 1), 64);
}
size_t cg_part_elems(int64_t n, int t) {
  return (size_t)std::max<int64_t>(kCgBlocks, cdiv(n, kPrRows)) * std::max(t, 1);
}

template <class T>
gp_status cg_tridiag(int t, int max_iter, const CgBufs<T>& cb, double* T_diag, double* T_off,
                     cudaStream_t st) {
  int total = t * max_iter;
  tridiag_kernel<<<(unsigned)cdiv(total, 256), 256, 0, st>>>(t, max_iter, cb.alpha, cb.beta,
                                                            cb.iters, T_diag, T_off);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template <class T>
gp_status dot_into(int64_t n, const T* a, const T* b, double* part, unsigned* counter,
                   double* out, cudaStream_t st) {
  int nb = (int)std::min<int64_t>(kCgBlocks, cdiv(n, kThreads));
  dot_kernel<T><<<nb, kThreads, 0, st>>>(n, a, b, part, counter, out);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

#define GP_INST(T)                                                                          \
  template gp_status cg_solve<T>(const Prob&, MvmOp&, const T*, int64_t, int, const double*, \
                                 const T*, int64_t, int, const int*, const gp_opts&,        \
                                 const CgBufs<T>&, T*, int64_t, int*, cudaStream_t);         \
  template gp_status cg_tridiag<T>(int, int, const CgBufs<T>&, double*, double*,            \
                                   cudaStream_t);                                           \
  template gp_status dot_into<T>(int64_t, const T*, const T*, double*, unsigned*, double*,   \
                                 cudaStream_t);
GP_INST(float)
GP_INST(double)
#undef GP_INST

}  // namespace gp
