// Greedy partial pivoted Cholesky of the noise-free kernel matrix (the paper's
// "partial Cholesky" preconditioner, Prop. "Cholesky approximation quality").
//
// One launch per rank-one step.  Each step kernel
//   1. reads the pivot pi_m chosen by the previous launch and its residual d,
//   2. forms column m for every row a:
//        L[a, m] = (k(x_a, x_pi) - L[a, :m] . L[pi, :m]) / sqrt(d)
//      (FP32 or FP64 GEMV; rows of earlier pivots are exactly 0, the pivot row sqrt(d)),
//   3. downdates the residual diagonal in FP64 and finds the next pivot: the
//      largest residual among unchosen rows, lowest index on exact ties, by a
//      block reduction whose partials the last block to finish combines in block
//      order (deterministic).
// The stopping tests (rank k reached, residual trace <= tol * tr K, best residual
// <= n u max_i K_ii) are taken on the device; later step kernels see the stop flag
// and return.  The last test is the default rank rule of LAPACK's pivoted Cholesky
// (xPSTRF; Lucas, "LAPACK-style codes for level 2 and 3 pivoted Cholesky
// factorizations", 2004), with u the unit roundoff of the precision L is formed in
// (2^-24 for FP32, 2^-53 for FP64).  A residual below it is rounding error of the
// earlier columns: the column it would normalise is noise, and the frozen-pivot
// derivative of the factor (L = K[:, piv] L[piv, :]^-T) no longer holds for it.
// The factor stops there with rank < k and the caller reports the rank deficiency.
#include "ops.h"

namespace gp {
namespace {

constexpr int kThreads = 256;

struct Best {
  double v;
  int i;
};
__device__ __forceinline__ Best better(Best a, Best b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i && b.i >= 0)) return b;
  if (a.i < 0) return b;
  return a;
}

__device__ Best block_best(Best x, double* sv, int* si) {
  for (int o = 16; o > 0; o >>= 1) {
    Best y;
    y.v = __shfl_xor_sync(0xffffffffu, x.v, o);
    y.i = __shfl_xor_sync(0xffffffffu, x.i, o);
    x = better(x, y);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { sv[w] = x.v; si[w] = x.i; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    Best y{-1.0, -1};
    if (lane < nw) { y.v = sv[lane]; y.i = si[lane]; }
    for (int o = 16; o > 0; o >>= 1) {
      Best z;
      z.v = __shfl_xor_sync(0xffffffffu, y.v, o);
      z.i = __shfl_xor_sync(0xffffffffu, y.i, o);
      y = better(y, z);
    }
    x = y;
  }
  return x;
}

// Final combine for step m (or the initial diagonal, m = -1): choose pivot m+1.
// trace0 = {tr K, max_i K_ii}, both of the initial diagonal; floor_rel = n u.
__device__ void choose_next(int64_t n, int m, int k, double tol, double floor_rel,
                            const int* piv_override, const double* dres, const double* pval,
                            const int* pidx, const double* psum, int nblk, int* piv,
                            double* dval, double* trace0, int* stop, int* rank) {
  if (threadIdx.x != 0) return;
  Best b{-1.0, -1};
  double sum = 0.0;
  for (int q = 0; q < nblk; ++q) {
    b = better(b, Best{pval[q], pidx[q]});
    sum += psum[q];
  }
  if (m < 0) {
    trace0[0] = sum;
    trace0[1] = b.v;
  }
  const int next = m + 1;
  if (next >= k) { *rank = k; *stop = 1; return; }
  if (sum <= tol * trace0[0]) { *rank = next; *stop = 1; return; }
  int pi = piv_override ? piv_override[next] : b.i;
  double dv = (pi >= 0 && pi < n) ? dres[pi] : -1.0;   // an out-of-range override stops
  if (!(dv > 0.0) || dv <= floor_rel * trace0[1]) { *rank = next; *stop = 1; return; }
  piv[next] = pi;
  dval[next] = dv;
  *rank = next + 1;   // provisional: column `next` will be formed
}

template <class T>
__global__ void __launch_bounds__(kThreads) pivchol_init(
    int64_t n, int d, int kind, int D, const double* __restrict__ theta, int k, double tol,
    double floor_rel, const int* __restrict__ piv_override, PivBufs b, int* piv, int* rank) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const double s = theta[D];
  // k(x, x) = k(r^2 = 0): every stationary kernel here gives s.
  const double diag = (double)kval<T>(kind, T(0), (T)s);
  Best best{-1.0, -1};
  double sum = 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    b.dres[a] = diag;
    best = better(best, Best{diag, (int)a});
    sum += diag;
  }
  Best bb = block_best(best, sv, si);
  double bs = block_sum(sum, sv);
  if (threadIdx.x == 0) {
    b.pval[blockIdx.x] = bb.v;
    b.pidx[blockIdx.x] = bb.i;
    b.psum[blockIdx.x] = bs;
  }
  if (last_block_arrived(b.counter)) {
    if (threadIdx.x == 0) *b.stop = 0;
    choose_next(n, -1, k, tol, floor_rel, piv_override, b.dres, b.pval, b.pidx, b.psum,
                gridDim.x, piv, b.dval, b.trace0, b.stop, rank);
  }
}

template <class T>
__global__ void __launch_bounds__(kThreads) pivchol_step(
    int64_t n, int d, int kind, int D, const double* __restrict__ theta, int m, int k,
    double tol, double floor_rel, const int* __restrict__ piv_override,
    const T* __restrict__ Xs,
    T* __restrict__ L, int64_t ldl, PivBufs b, int* piv, int* rank) {
  if (*b.stop) return;
  extern __shared__ unsigned char smem_raw[];
  T* lrow = reinterpret_cast<T*>(smem_raw);          // m entries of L[pi, :m]
  __shared__ T xp[kMaxD];
  __shared__ double sv[32];
  __shared__ int si[32];
  const int pi = piv[m];
  const double dpi = b.dval[m];
  const double root = sqrt(dpi);
  const T inv_root = (T)(1.0 / root);
  for (int j = threadIdx.x; j < m; j += blockDim.x) lrow[j] = L[pi + (int64_t)j * ldl];
  for (int q = threadIdx.x; q < d; q += blockDim.x) xp[q] = Xs[(int64_t)pi * d + q];
  __syncthreads();
  const T s = (T)theta[D];
  Best best{-1.0, -1};
  double sum = 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    double da = b.dres[a];
    T col;
    if (a == pi) {
      col = (T)root;
      da = -1.0;
    } else if (da < 0.0) {
      col = T(0);
    } else {
      T r2 = T(0);
      for (int q = 0; q < d; ++q) {
        T df = Xs[a * d + q] - xp[q];
        r2 = fma(df, df, r2);
      }
      T acc = kval<T>(kind, r2, s);
      const T* La = L + a;
      for (int j = 0; j < m; ++j) acc = fma(-La[(int64_t)j * ldl], lrow[j], acc);
      col = acc * inv_root;
      double c2 = (double)col * (double)col;
      da = da - c2;
      if (da < 0.0) da = 0.0;
    }
    L[a + (int64_t)m * ldl] = col;
    b.dres[a] = da;
    if (da >= 0.0) {
      best = better(best, Best{da, (int)a});
      sum += da;
    }
  }
  Best bb = block_best(best, sv, si);
  double bs = block_sum(sum, sv);
  if (threadIdx.x == 0) {
    b.pval[blockIdx.x] = bb.v;
    b.pidx[blockIdx.x] = bb.i;
    b.psum[blockIdx.x] = bs;
  }
  if (last_block_arrived(b.counter))
    choose_next(n, m, k, tol, floor_rel, piv_override, b.dres, b.pval, b.pidx, b.psum,
                gridDim.x, piv, b.dval, b.trace0, b.stop, rank);
}

}  // namespace

template <class T>
gp_status pivchol_run(const Prob& pb, const void* Xs_, int k, double tol, const int* piv_override,
                      void* L_, int64_t ldl, int* piv, int* rank, const PivBufs& b,
                      cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  T* L = static_cast<T*>(L_);
  if (k > 0) {
    if (ldl == pb.n) {
      GP_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(T) * (size_t)pb.n * k, st));
    } else {
      GP_CUDA_TRY(cudaMemset2DAsync(L, sizeof(T) * ldl, 0, sizeof(T) * pb.n, k, st));
    }
    GP_CUDA_TRY(cudaMemsetAsync(piv, 0xff, sizeof(int) * k, st));
  }
  GP_CUDA_TRY(cudaMemsetAsync(rank, 0, sizeof(int), st));
  if (k == 0) return GP_OK;
  const int blocks = (int)std::min<int64_t>(kPivBlocks, cdiv(pb.n, kThreads));
  const double floor_rel = (double)pb.n * (sizeof(T) == 4 ? 0x1p-24 : 0x1p-53);
  pivchol_init<T><<<blocks, kThreads, 0, st>>>(pb.n, pb.d, pb.kind, pb.D, pb.theta, k, tol,
                                                floor_rel, piv_override, b, piv, rank);
  GP_LAUNCH_CHECK();
  for (int m = 0; m < k; ++m) {
    size_t sm = sizeof(T) * (size_t)(m > 0 ? m : 1);
    pivchol_step<T><<<blocks, kThreads, sm, st>>>(pb.n, pb.d, pb.kind, pb.D, pb.theta, m, k,
                                                   tol, floor_rel, piv_override, Xs, L, ldl, b,
                                                   piv, rank);
    GP_LAUNCH_CHECK();
  }
  return GP_OK;
}

template gp_status pivchol_run<float>(const Prob&, const void*, int, double, const int*, void*,
                                      int64_t, int*, int*, const PivBufs&, cudaStream_t);
template gp_status pivchol_run<double>(const Prob&, const void*, int, double, const int*, void*,
                                       int64_t, int*, int*, const PivBufs&, cudaStream_t);

}  // namespace gp
