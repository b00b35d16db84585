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
// Column-wise reductions use per-block partials combined by the last block in
// block order (deterministic).
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
// with warp shuffles (no block barrier per column).  The last block to finish
// combines the per-block partials in block order (deterministic).
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

// Sum of the nb per-block partials of column c, by one warp: lane-strided FP64 sums
// and a shuffle tree (fixed order, so deterministic); the result is in every lane.
__device__ __forceinline__ double warp_col_sum(const double* part, int nb, int c) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[(size_t)c * nb + b];
  return warp_sum(s);
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
// Both n-long products are skinny GEMMs streaming L (n x k) once from HBM: tiles of
// L and of the right-hand sides are staged in shared memory with coalesced loads,
// and each thread keeps a small register tile of the result.

// (1) S_part[b] = L[rows of part b]^T R[rows of part b] for a 128-pivot slice of S.
//     256 threads; thread (tm, tc) of a 32 x 8 grid owns pivots 4 tm .. 4 tm + 3 and
//     columns CPT tc .. CPT tc + CPT - 1 (CPT = TC / 8).  Rows go through shared memory
//     in stages of 32; the next stage is loaded into registers while the current one is
//     multiplied, so the loads of L and R overlap the FMAs.  Each part sums its rows in
//     order, so the partials do not depend on the slicing.
constexpr int kLtrRows = 32;
constexpr int kLtrM = 128;
constexpr int kLtrParts = 152;    // row parts; x (k / 128) slices
constexpr int kLtrThreads = 256;
template <class T, int TC>
__global__ void __launch_bounds__(kLtrThreads) ltr_partial(int64_t n, int t,
                                                          const T* __restrict__ L, int64_t ldl,
                                                          int k, Dev<T> g) {
  if (*g.n_active == 0) return;
  constexpr int CPT = TC / 8;
  constexpr int LP = kLtrM + 16 / (int)sizeof(T);   // row pitch: 16-byte aligned rows
  constexpr int RP = TC + 2;
  constexpr int NL = kLtrRows * kLtrM / kLtrThreads;                   // 16 L values
  constexpr int NR = (kLtrRows * TC + kLtrThreads - 1) / kLtrThreads;  // <= CPT R values
  __shared__ __align__(16) T sL[kLtrRows][LP];
  __shared__ __align__(16) T sR[kLtrRows][RP];
  const int tm = threadIdx.x & 31, tcol = threadIdx.x >> 5;
  const int m0 = blockIdx.x * kLtrM;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = blockIdx.y * per, r1 = min(n, r0 + per);
  T acc[4][CPT];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[a][c] = T(0);
  // element e of a stage: row e % 32 (consecutive threads on consecutive rows: coalesced),
  // pivot / column e / 32
  T pl[NL], pr[NR];
  auto fetch = [&](int64_t rb) {
    const int rn = (int)min((int64_t)kLtrRows, r1 - rb);
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      const int rr = e % kLtrRows, mm = e / kLtrRows;
      pl[q] = (rr < rn && m0 + mm < k) ? L[rb + rr + (int64_t)(m0 + mm) * ldl] : T(0);
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      const int rr = e % kLtrRows, c = e / kLtrRows;
      pr[q] = (e < kLtrRows * TC && rr < rn && c < t) ? g.R[rb + rr + (int64_t)c * n] : T(0);
    }
  };
  if (r0 < r1) fetch(r0);
  for (int64_t rb = r0; rb < r1; rb += kLtrRows) {
    __syncthreads();                 // the previous stage has been read
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      sL[e % kLtrRows][e / kLtrRows] = pl[q];
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int e = threadIdx.x + q * kLtrThreads;
      if (e < kLtrRows * TC) sR[e % kLtrRows][e / kLtrRows] = pr[q];
    }
    __syncthreads();
    if (rb + kLtrRows < r1) fetch(rb + kLtrRows);   // in flight during the FMAs below
#pragma unroll 4
    for (int rr = 0; rr < kLtrRows; ++rr) {
      T lv[4], rv[CPT];
#pragma unroll
      for (int a = 0; a < 4; ++a) lv[a] = sL[rr][tm * 4 + a];
#pragma unroll
      for (int c = 0; c < CPT; ++c) rv[c] = sR[rr][tcol * CPT + c];
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][c] = fma(lv[a], rv[c], acc[a][c]);
    }
  }
  double* out = g.S + (size_t)blockIdx.y * k * t;     // per-part partials (t x k)
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int m = m0 + tm * 4 + a;
    if (m >= k) continue;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int col = tcol * CPT + c;
      if (col < t) out[(size_t)col * k + m] = (double)acc[a][c];
    }
  }
}

// (2) S = sum of the part partials (FP64), Sp = C^-1 S (FP64), for active columns.
//     C^-1 is exactly symmetric (formed as Gc^-T Gc^-1 with one summation order), so
//     Sp_i = sum_m C^-1[m][i] S_m reads rows of C^-1 coalesced across threads i.
template <class T>
__global__ void reduce_cinv(int k, int t, int ldsp, int nparts, const double* __restrict__ Cinv,
                            const double* __restrict__ part, Dev<T> g) {
  if (*g.n_active == 0) return;
  extern __shared__ double sS[];    // k doubles: column c of S
  const int c = blockIdx.y;
  if (!g.active[c]) return;
  // eight independent chains (fixed order), so eight loads are in flight per thread
  constexpr int CH = 8;
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    double sc[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) sc[q] = 0.0;
    int b = 0;
    for (; b + CH <= nparts; b += CH) {
#pragma unroll
      for (int q = 0; q < CH; ++q) sc[q] += part[((size_t)(b + q) * t + c) * k + m];
    }
    for (; b < nparts; ++b) sc[0] += part[((size_t)b * t + c) * k + m];
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < CH; ++q) s += sc[q];
    sS[m] = s;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double ac[CH];
#pragma unroll
  for (int q = 0; q < CH; ++q) ac[q] = 0.0;
  int m = 0;
  for (; m + CH <= k; m += CH) {
#pragma unroll
    for (int q = 0; q < CH; ++q) ac[q] += Cinv[(int64_t)(m + q) * k + i] * sS[m + q];
  }
  for (; m < k; ++m) ac[0] += Cinv[(int64_t)m * k + i] * sS[m];
  double a = 0.0;
#pragma unroll
  for (int q = 0; q < CH; ++q) a += ac[q];
  g.Sp[(int64_t)i * ldsp + c] = (T)a;
}

// (3) z = sigma^-2 (r - L Sp) and the partial sums of r^T z for active columns, one
//     128-row tile per block.  Thread (tr, tc) of a 32 x 8 grid owns rows
//     4 tr .. 4 tr + 3 and columns CPT tc .. CPT tc + CPT - 1.  Pivots go through shared
//     memory in chunks of 32; the next chunk of L and Sp is loaded into registers while
//     the current one is multiplied.
constexpr int kPrRows = 128;
constexpr int kPrM = 32;
template <class T, int TC>
__global__ void __launch_bounds__(kThreads) precond_rho(int64_t n, int t, int c0,
                                                       const T* __restrict__ L, int64_t ldl,
                                                       int k, const double* __restrict__ theta,
                                                       int D, Dev<T> g) {
  if (*g.n_active == 0) return;
  constexpr int CPT = TC / 8;
  constexpr int NL = kPrM * kPrRows / kThreads;                  // 16 L values
  constexpr int NS = (kPrM * TC + kThreads - 1) / kThreads;      // <= CPT Sp values
  __shared__ __align__(16) T sL[kPrM][kPrRows];
  __shared__ T sSp[kPrM][TC];
  __shared__ double swarp[kThreads / 32][TC];
  const int tr = threadIdx.x & 31, tcol = threadIdx.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int64_t a0 = blockIdx.x * (int64_t)kPrRows;
  const int tc = min(TC, t - c0);
  const T inv_s2 = (T)(1.0 / theta[D + 1]);
  T acc[4][CPT];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[a][c] = T(0);
  // L element e of a chunk: row e % 128 (coalesced), pivot e / 128; Sp element e:
  // pivot e / TC, column e % TC
  T pl[NL], ps[NS];
  auto fetch = [&](int m0) {
    const int mn = min(kPrM, k - m0);
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kThreads;
      const int rr = e % kPrRows, mm = e / kPrRows;
      const int64_t a = a0 + rr;
      pl[q] = (mm < mn && a < n) ? L[a + (int64_t)(m0 + mm) * ldl] : T(0);
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int e = threadIdx.x + q * kThreads;
      const int mm = e / TC, c = e % TC;
      ps[q] = (e < kPrM * TC && mm < mn && c < tc) ? g.Sp[(int64_t)(m0 + mm) * t + c0 + c]
                                                   : T(0);
    }
  };
  fetch(0);
  for (int m0 = 0; m0 < k; m0 += kPrM) {
    __syncthreads();                 // the previous chunk has been read
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * kThreads;
      sL[e / kPrRows][e % kPrRows] = pl[q];
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int e = threadIdx.x + q * kThreads;
      if (e < kPrM * TC) sSp[e / TC][e % TC] = ps[q];
    }
    __syncthreads();
    if (m0 + kPrM < k) fetch(m0 + kPrM);   // in flight during the FMAs below
#pragma unroll 8
    for (int mm = 0; mm < kPrM; ++mm) {
      T lv[4], sv[CPT];
#pragma unroll
      for (int a = 0; a < 4; ++a) lv[a] = sL[mm][tr * 4 + a];
#pragma unroll
      for (int c = 0; c < CPT; ++c) sv[c] = sSp[mm][tcol * CPT + c];
#pragma unroll
      for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][c] = fma(lv[a], sv[c], acc[a][c]);
    }
  }
  // z, and r^T z summed over this block's rows per column (compensated FP32 within
  // the block, FP64 across blocks)
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int col = tcol * CPT + c;
    DotAcc<T> rz;
    if (col < tc && g.active[c0 + col]) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t row = a0 + tr * 4 + a;
        if (row < n) {
          const int64_t off = row + (int64_t)(c0 + col) * n;
          const T r = g.R[off];
          const T z = (r - acc[a][c]) * inv_s2;
          g.Z[off] = z;
          rz.add(r, z);
        }
      }
    }
    const double rzw = rz.warp_total();           // the warp's 32 threads share column col
    if (tr == 0) swarp[warp][c] = rzw;            // warp index == tcol
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int col = threadIdx.x; col < tc; col += blockDim.x) {
    // column col is owned by warp (col / CPT), slot (col % CPT)
    g.part[(size_t)(c0 + col) * nb + blockIdx.x] = swarp[col / CPT][col % CPT];
  }
}

// Combine the r^T z partials of all blocks (one small launch).
template <class T>
__global__ void rho_combine(int t, int nb, int mode, int j, int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl && mode != 0) j = g.ctl[0];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < t; c += blockDim.x >> 5) {
    if (!g.active[c]) continue;
    const double s = warp_col_sum(g.part, nb, c);
    if (lane != 0) continue;
    if (mode == 0) {
      g.rho[c] = s;
      g.rho0[c] = s;
    } else {
      if (!(s > 0.0) || !isfinite(s)) {
        // r^T P^-1 r <= 0 only happens once r is at the rounding floor of the
        // preconditioner solve: the column stops here (no beta_j, m = j + 1 nodes)
        g.active[c] = 0;
        g.iters[c] = j + 1;
        atomicSub(g.n_active, 1);
        continue;
      }
      double be = s / g.rho[c];
      if (!isfinite(be)) { raise_status(g.status, GP_ERR_NUMERIC); be = 0.0; }
      g.beta[(int64_t)c * max_iter + j] = be;
      g.rho[c] = s;
    }
  }
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

// alpha_j = rho / p^T q  for active columns.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_alpha(int64_t n, int t, int j, int max_iter,
                                                    Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) j = g.ctl[0];
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int c = warp; c < t; c += kThreads / 32) {
    if (!g.active[c]) continue;
    DotAcc<T> acc;
    for (int64_t a = r0 + lane; a < r1; a += 32) acc.add(g.P[a + c * n], g.Q[a + c * n]);
    const double sum = acc.warp_total();
    if (lane == 0) g.part[c * nb + blockIdx.x] = sum;
  }
  if (last_block_arrived(g.counter)) {
    for (int c = warp; c < t; c += kThreads / 32) {
      if (!g.active[c]) continue;
      const double pq = warp_col_sum(g.part, nb, c);
      if (lane != 0) continue;
      double al = g.rho[c] / pq;
      if (!(pq > 0.0) || !isfinite(al)) {
        // breakdown: the operator is not positive definite in this precision (or
        // the iterates overflowed); the column stops with the j steps it has
        raise_status(g.status, GP_ERR_NUMERIC);
        g.alpha[(int64_t)c * max_iter + j] = 0.0;
        g.active[c] = 0;
        g.iters[c] = j;
        atomicSub(g.n_active, 1);
        continue;
      }
      g.alpha[(int64_t)c * max_iter + j] = al;
    }
  }
}

__device__ void decide(int t, int j, const double* rnorm2_part, int nb, double tol2,
                       int use_caps, int max_iter, int* active, const int* caps, int* iters,
                       const double* bnorm2, int* n_active, int* status) {
  __shared__ int cnt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int c = warp; c < t; c += blockDim.x >> 5) {
    if (!active[c]) continue;
    bool stop, capped = false;
    if (use_caps) {
      stop = (j + 1) >= caps[c];
    } else {
      const double s = warp_col_sum(rnorm2_part, nb, c);
      const bool conv = s <= tol2 * bnorm2[c];
      capped = !conv && (j + 1 >= max_iter);
      stop = conv || capped;
    }
    if (lane != 0) continue;
    // the iteration cap ended a column above the tolerance: results are written, with a
    // warning (with per-column caps from the caller the stop is deliberate)
    if (capped) raise_status(status, GP_WARN_NOT_CONVERGED);
    if (stop) {
      active[c] = 0;
      iters[c] = j + 1;
    } else {
      atomicAdd(&cnt, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *n_active = cnt;
}

// x += alpha p; r -= alpha q (active columns); ||r||^2 and the stopping decision
// unless this step recomputes the residual.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_update(int64_t n, int t, int j, int max_iter,
                                                     double tol2, int use_caps, int recompute,
                                                     Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) {
    j = g.ctl[0];
    recompute = g.ctl[1];
  }
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int c = warp; c < t; c += kThreads / 32) {
    if (!g.active[c]) continue;
    const T al = (T)g.alpha[(int64_t)c * max_iter + j];
    DotAcc<T> acc;
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      const int64_t off = a + c * n;
      g.X[off] = fma(al, g.P[off], g.X[off]);
      const T r = fma(-al, g.Q[off], g.R[off]);
      g.R[off] = r;
      acc.add(r, r);
    }
    const double sum = acc.warp_total();
    if (lane == 0 && !recompute) g.part[c * nb + blockIdx.x] = sum;
  }
  if (recompute) return;
  if (last_block_arrived(g.counter))
    decide(t, j, g.part, nb, tol2, use_caps, max_iter, g.active, g.caps, g.iters, g.bnorm2,
           g.n_active, g.status);
}

// r = b - K_hat x (Q holds K_hat x), ||r||^2, stopping decision.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_resid(int64_t n, int t, int j, int max_iter,
                                                    double tol2, int use_caps, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) {
    if (!g.ctl[1]) return;   // not a residual-recompute step
    j = g.ctl[0];
  }
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r0, r1;
  row_chunk(n, &r0, &r1);
  for (int c = warp; c < t; c += kThreads / 32) {
    if (!g.active[c]) continue;
    DotAcc<T> acc;
    for (int64_t a = r0 + lane; a < r1; a += 32) {
      const int64_t off = a + c * n;
      const T r = g.B[a + c * g.ldb] - g.Q[off];
      g.R[off] = r;
      acc.add(r, r);
    }
    const double sum = acc.warp_total();
    if (lane == 0) g.part[c * nb + blockIdx.x] = sum;
  }
  if (last_block_arrived(g.counter))
    decide(t, j, g.part, nb, tol2, use_caps, max_iter, g.active, g.caps, g.iters, g.bnorm2,
           g.n_active, g.status);
}

// p = z + beta_j p for active columns.
template <class T>
__global__ void cg_pupdate(int64_t n, int t, int j, int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  if (g.ctl) j = g.ctl[0];
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * t) return;
  int c = (int)(e / n);
  if (!g.active[c]) return;
  const T be = (T)g.beta[(int64_t)c * max_iter + j];
  g.P[e] = fma(be, g.P[e], g.Z[e]);
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

template <class T>
gp_status precond_apply(int64_t n, int t, const T* L, int64_t ldl, int k, const double* Cinv,
                        const double* theta, int D, int mode, int j, int max_iter,
                        const CgBufs<T>& cb, Dev<T>& g, int nb, cudaStream_t st) {
  (void)nb;
  if (k > 0) {
    // L^T R, in column chunks of at most 64
    for (int c0 = 0; c0 < t; c0 += 64) {
      const int tc = std::min(64, t - c0);
      Dev<T> gc = g;                 // this chunk's columns; part partials into atb_part
      gc.R = g.R + (int64_t)c0 * n;
      gc.S = cb.atb_part;
      dim3 grid((unsigned)cdiv(k, kLtrM), (unsigned)kLtrParts);
      GP_TC_DISPATCH(pick_tc16(tc),
                     (ltr_partial<T, TC><<<grid, kLtrThreads, 0, st>>>(n, tc, L, ldl, k, gc)));
      GP_LAUNCH_CHECK();
      Dev<T> gs = g;                 // Sp columns c0.. (leading dimension t)
      gs.active = g.active + c0;
      gs.Sp = g.Sp + c0;
      dim3 g2((unsigned)cdiv(k, 256), (unsigned)tc);
      reduce_cinv<T><<<g2, 256, sizeof(double) * k, st>>>(k, tc, t, kLtrParts, Cinv,
                                                         cb.atb_part, gs);
      GP_LAUNCH_CHECK();
    }
  }
  const int nbp = (int)cdiv(n, kPrRows);
  for (int c0 = 0; c0 < t; c0 += 64) {
    const int tc = std::min(64, t - c0);
    GP_TC_DISPATCH(pick_tc16(tc), (precond_rho<T, TC><<<nbp, kThreads, 0, st>>>(
                                      n, t, c0, L, ldl, k, theta, D, g)));
    GP_LAUNCH_CHECK();
  }
  rho_combine<T><<<1, 256, 0, st>>>(t, nbp, mode, j, max_iter, g);
  GP_LAUNCH_CHECK();
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
  const int nb = (int)std::min<int64_t>(kCgBlocks, cdiv(n, kThreads));
  const int use_caps = iters_override ? 1 : 0;
  const double tol2 = o.cg_tol * o.cg_tol;
  const int R = o.recompute_every;
  int check = o.check_every > 0 ? o.check_every : 4;

  cg_init<T><<<nb, kThreads, 0, st>>>(n, t, o.max_iter, iters_override, g);
  GP_LAUNCH_CHECK();
  GP_TRY(precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 0, 0, o.max_iter, cb, g, nb, st));
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
      cg_alpha<T><<<nb, kThreads, 0, bs>>>(n, t, 0, o.max_iter, gd);
      cg_update<T><<<nb, kThreads, 0, bs>>>(n, t, 0, o.max_iter, tol2, use_caps, 0, gd);
      if (R > 0) {
        rs = mvm.apply(gd.X, n, t, gd.Q, n, cb.ctl + 2, bs);   // gated: recompute steps only
        if (rs != GP_OK) break;
        cg_resid<T><<<nb, kThreads, 0, bs>>>(n, t, 0, o.max_iter, tol2, use_caps, gd);
      }
      rs = precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 1, 0, o.max_iter, cb, gd, nb,
                            bs);
      if (rs != GP_OK) break;
      cg_pupdate<T><<<(unsigned)cdiv(n * t, 256), 256, 0, bs>>>(n, t, 0, o.max_iter, gd);
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
    cg_alpha<T><<<nb, kThreads, 0, st>>>(n, t, j, o.max_iter, g);
    GP_LAUNCH_CHECK();
    const int rec = (R > 0 && (j + 1) % R == 0) ? 1 : 0;
    cg_update<T><<<nb, kThreads, 0, st>>>(n, t, j, o.max_iter, tol2, use_caps, rec, g);
    GP_LAUNCH_CHECK();
    if (rec) {
      if (timed) mvm_timing_begin(st);
      GP_TRY(mvm.apply(g.X, n, t, g.Q, n, g.n_active, st));
      if (timed) mvm_timing_end(st);
      cg_resid<T><<<nb, kThreads, 0, st>>>(n, t, j, o.max_iter, tol2, use_caps, g);
      GP_LAUNCH_CHECK();
    }
    GP_TRY(precond_apply<T>(n, t, L, ldl, k, Cinv, pb.theta, pb.D, 1, j, o.max_iter, cb, g, nb,
                            st));
    cg_pupdate<T><<<(unsigned)cdiv(n * t, 256), 256, 0, st>>>(n, t, j, o.max_iter, g);
    GP_LAUNCH_CHECK();
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
