// CUDA-core (SIMT) kernel-matrix products: the FP64 path and the plain FP32 form.
//
//   kmvm:      W = (K + sigma^2 I) V                         (inner op of CG, Sec. 2.2)
//   kdmvm:     W = dK/dtheta_q V for one hyperparameter q     (eq. derivative_likelihood)
//   contract:  g_q = sum_ab dK_q[a,b] M[a,b], M = sum_c w_c A[:,c] B[:,c]^T
//              for every lengthscale and the output scale in one pass over K
//              (the kernel-derivative part of Alg. 2, see ops.h)
//
// One thread owns one row a; tiles of 64 columns b (scaled inputs and the
// right-hand sides) are staged in shared memory and broadcast to all threads.
// K is never stored.  Inputs are pre-scaled: Xs = (X - mean) / l.
#include "ops.h"

namespace gp {

namespace {

constexpr int kBM = 128;   // rows per CTA (one per thread)
constexpr int kBN = 64;    // columns staged per tile

template <class T>
__global__ void center_partial(int64_t n, int d, const T* __restrict__ X,
                               double* __restrict__ part, unsigned* counter,
                               double* __restrict__ mean) {
  __shared__ double sh[32];
  for (int j = 0; j < d; ++j) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      acc += (double)X[i * d + j];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x * d + j] = s;
  }
  if (last_block_arrived(counter)) {
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      double s = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) s += part[b * d + j];
      mean[j] = s / (double)n;
    }
  }
}

template <class T>
__global__ void scale_inputs(int64_t n, int d, int ard, const T* __restrict__ X,
                             const double* __restrict__ theta, const double* __restrict__ mean,
                             T* __restrict__ Xs) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * d) return;
  int j = (int)(e % d);
  double l = theta[ard ? j : 0];
  Xs[e] = (T)(((double)X[e] - mean[j]) / l);
}

// Rows per thread: two for FP32 (halves the shared-memory broadcasts per kernel
// entry), one for FP64 (register budget).
template <class T> struct Rpt { static constexpr int v = 2; };
template <> struct Rpt<double> { static constexpr int v = 1; };

template <class T, int DM, int TC>
__global__ void __launch_bounds__(kBM) kmvm_kernel(
    int64_t n, int d, int kind, int D, const double* __restrict__ theta,
    const T* __restrict__ Xs, const T* __restrict__ V, int64_t ldv, int tc,
    T* __restrict__ out, int64_t ldo, int64_t split_cols, int add_noise, const int* gate) {
  constexpr int R = Rpt<T>::v;
  if (gate && *gate == 0) return;
  __shared__ __align__(16) T sx[kBN][DM];
  __shared__ __align__(16) T sv[kBN][TC];
  const T s = (T)theta[D];
  int64_t i[R];
  T xi[R][DM];
  T acc[R][TC];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    i[r] = blockIdx.x * (int64_t)(kBM * R) + r * kBM + threadIdx.x;
#pragma unroll
    for (int q = 0; q < DM; ++q) xi[r][q] = (i[r] < n && q < d) ? Xs[i[r] * d + q] : T(0);
#pragma unroll
    for (int c = 0; c < TC; ++c) acc[r][c] = T(0);
  }
  const int64_t jb = blockIdx.y * split_cols;
  const int64_t je = min(n, jb + split_cols);
  for (int64_t j0 = jb; j0 < je; j0 += kBN) {
    const int jn = (int)min((int64_t)kBN, je - j0);
    for (int e = threadIdx.x; e < kBN * DM; e += kBM) {
      int jj = e / DM, q = e % DM;
      sx[jj][q] = (jj < jn && q < d) ? Xs[(j0 + jj) * d + q] : T(0);
    }
    for (int e = threadIdx.x; e < kBN * TC; e += kBM) {
      int c = e / kBN, jj = e % kBN;
      sv[jj][c] = (jj < jn && c < tc) ? V[(j0 + jj) + c * ldv] : T(0);
    }
    __syncthreads();
    for (int jj = 0; jj < jn; ++jj) {
      T kv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        T r2 = T(0);
#pragma unroll
        for (int q = 0; q < DM; ++q) {
          T df = xi[r][q] - sx[jj][q];
          r2 = fma(df, df, r2);
        }
        kv[r] = kval<T>(kind, r2, s);
      }
#pragma unroll
      for (int c = 0; c < TC; ++c) {
        const T v = sv[jj][c];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r][c] = fma(kv[r], v, acc[r][c]);
      }
    }
    __syncthreads();
  }
  const T s2 = (T)theta[D + 1];
  T* o = out + (int64_t)blockIdx.y * tc * ldo;   // split partial (blockIdx.y = 0 if none)
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (i[r] >= n) continue;
    for (int c = 0; c < tc; ++c) {
      T v = acc[r][c];
      if (add_noise) v = fma(s2, V[i[r] + c * ldv], v);
      o[i[r] + c * ldo] = v;
    }
  }
}

// W[:, c] = sum over splits of part + sigma^2 V[:, c]
template <class T>
__global__ void split_reduce(int64_t n, int tc, int splits, const T* __restrict__ part,
                             const T* __restrict__ V, int64_t ldv, const double* __restrict__ theta,
                             int D, T* __restrict__ W, int64_t ldw, int add_noise,
                             const int* gate) {
  if (gate && *gate == 0) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * tc) return;
  int c = (int)(e / n);
  int64_t i = e % n;
  T acc = T(0);
  for (int s = 0; s < splits; ++s) acc += part[((int64_t)s * tc + c) * n + i];
  if (add_noise) acc = fma((T)theta[D + 1], V[i + c * ldv], acc);
  W[i + c * ldw] = acc;
}

// dK/dtheta_q V, q < p - 1 (lengthscales then output scale).
template <class T, int DM, int TC>
__global__ void __launch_bounds__(kBM) kdmvm_kernel(
    int64_t n, int d, int kind, int ard, int D, int q, const double* __restrict__ theta,
    const T* __restrict__ Xs, const T* __restrict__ V, int64_t ldv, int tc,
    T* __restrict__ out, int64_t ldo, int64_t split_cols) {
  __shared__ T sx[kBN][DM];
  __shared__ T sv[kBN][TC];
  const T s = (T)theta[D];
  const int64_t i = blockIdx.x * (int64_t)kBM + threadIdx.x;
  T xi[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) xi[u] = (i < n && u < d) ? Xs[i * d + u] : T(0);
  const bool is_scale = (q == D);
  const int qd = (ard && !is_scale) ? q : 0;
  const T xq = (i < n && ard && !is_scale) ? Xs[i * d + qd] : T(0);
  T acc[TC];
#pragma unroll
  for (int c = 0; c < TC; ++c) acc[c] = T(0);
  const int64_t jb = blockIdx.y * split_cols;
  const int64_t je = min(n, jb + split_cols);
  for (int64_t j0 = jb; j0 < je; j0 += kBN) {
    const int jn = (int)min((int64_t)kBN, je - j0);
    for (int e = threadIdx.x; e < kBN * DM; e += kBM) {
      int jj = e / DM, u = e % DM;
      sx[jj][u] = (jj < jn && u < d) ? Xs[(j0 + jj) * d + u] : T(0);
    }
    for (int e = threadIdx.x; e < kBN * TC; e += kBM) {
      int c = e / kBN, jj = e % kBN;
      sv[jj][c] = (jj < jn && c < tc) ? V[(j0 + jj) + c * ldv] : T(0);
    }
    __syncthreads();
    for (int jj = 0; jj < jn; ++jj) {
      T r2 = T(0);
#pragma unroll
      for (int u = 0; u < DM; ++u) {
        T df = xi[u] - sx[jj][u];
        r2 = fma(df, df, r2);
      }
      T kv, fac;
      kval_fac<T>(kind, r2, s, kv, fac);
      T coef;
      if (is_scale) {
        coef = kv / s;
      } else if (ard) {
        T df = xq - sx[jj][qd];
        coef = fac * df * df;
      } else {
        coef = fac * r2;
      }
#pragma unroll
      for (int c = 0; c < TC; ++c) acc[c] = fma(coef, sv[jj][c], acc[c]);
    }
    __syncthreads();
  }
  if (i < n) {
    // lengthscale: sum (dx/l)^2 g / l_q  ==  sum dx^2 g / l_q^3
    T scale = is_scale ? T(1) : (T)(1.0 / theta[ard ? q : 0]);
    T* o = out + (int64_t)blockIdx.y * tc * ldo;
    for (int c = 0; c < tc; ++c) o[i + c * ldo] = acc[c] * scale;
  }
}

template <class T>
__global__ void copy_block(int64_t n, int tc, const T* __restrict__ V, int64_t ldv,
                           T* __restrict__ W, int64_t ldw) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * tc) return;
  int c = (int)(e / n);
  int64_t i = e % n;
  W[i + c * ldw] = V[i + c * ldv];
}

// Fused gradient contraction (see ops.h).  Per entry (a, b):
//   m = sum_c w_c A[a,c] B[b,c];  lengthscale u: acc_u += fac * m * (dxs_u)^2;
//   output scale: acc_s += k * m.
// Per-tile sums in T are folded into running Kahan-compensated sums, then into
// FP64 block partials; the last block adds the partials in a fixed order.
// 16-byte load from shared memory (4 floats or 2 doubles; p 16-byte aligned).
__device__ __forceinline__ void ld_shared16(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld_shared16(const double* p, double (&v)[2]) {
  const double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x; v[1] = q.y;
}

template <class T, int DM, int TC>
__global__ void __launch_bounds__(kBM) contract_kernel(
    int64_t n, int d, int kind, int ard, int D, const double* __restrict__ theta,
    const T* __restrict__ Xs, const T* __restrict__ A, int64_t lda,
    const T* __restrict__ B, int64_t ldb, const double* __restrict__ wts, int c0, int tc,
    int64_t split_cols, double* __restrict__ part, unsigned* counter,
    double* __restrict__ gout, int accumulate) {
  constexpr int NA = DM + 1;   // lengthscale accumulators (ARD: d, iso: 1) + scale
  constexpr int VW = 16 / (int)sizeof(T);   // elements per 16-byte shared-memory load
  static_assert(DM % VW == 0 && TC % VW == 0, "rows must be whole 16-byte vectors");
  __shared__ __align__(16) T sx[kBN][DM];
  __shared__ __align__(16) T sb[kBN][TC];
  __shared__ double sh[32];
  const T s = (T)theta[D];
  const int64_t i = blockIdx.x * (int64_t)kBM + threadIdx.x;
  T xi[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) xi[u] = (i < n && u < d) ? Xs[i * d + u] : T(0);
  T aw[TC];
#pragma unroll
  for (int c = 0; c < TC; ++c)
    aw[c] = (i < n && c < tc) ? (T)(wts[c0 + c] * (double)A[i + (int64_t)(c0 + c) * lda]) : T(0);
  T sum[NA], comp[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) { sum[u] = T(0); comp[u] = T(0); }

  const int64_t jb = blockIdx.y * split_cols;
  const int64_t je = min(n, jb + split_cols);
  for (int64_t j0 = jb; j0 < je; j0 += kBN) {
    const int jn = (int)min((int64_t)kBN, je - j0);
    for (int e = threadIdx.x; e < kBN * DM; e += kBM) {
      int jj = e / DM, u = e % DM;
      sx[jj][u] = (jj < jn && u < d) ? Xs[(j0 + jj) * d + u] : T(0);
    }
    for (int e = threadIdx.x; e < kBN * TC; e += kBM) {
      int c = e / kBN, jj = e % kBN;
      sb[jj][c] = (jj < jn && c < tc) ? B[(j0 + jj) + (int64_t)(c0 + c) * ldb] : T(0);
    }
    __syncthreads();
    T tacc[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) tacc[u] = T(0);
    for (int jj = 0; jj < jn; ++jj) {
      // every thread reads the same column jj: 16-byte broadcast loads
      T df[DM];
      T r2 = T(0);
#pragma unroll
      for (int u = 0; u < DM; u += VW) {
        T xv[VW];
        ld_shared16(&sx[jj][u], xv);
#pragma unroll
        for (int q = 0; q < VW; ++q) {
          df[u + q] = xi[u + q] - xv[q];
          r2 = fma(df[u + q], df[u + q], r2);
        }
      }
      T m = T(0);
#pragma unroll
      for (int c = 0; c < TC; c += VW) {
        T bv[VW];
        ld_shared16(&sb[jj][c], bv);
#pragma unroll
        for (int q = 0; q < VW; ++q) m = fma(aw[c + q], bv[q], m);
      }
      T kv, fac;
      kval_fac<T>(kind, r2, s, kv, fac);
      const T fm = fac * m;
      if (ard) {
#pragma unroll
        for (int u = 0; u < DM; ++u) tacc[u] = fma(fm, df[u] * df[u], tacc[u]);
      } else {
        tacc[0] = fma(fm, r2, tacc[0]);
      }
      tacc[DM] = fma(kv, m, tacc[DM]);
    }
#pragma unroll
    for (int u = 0; u < NA; ++u) {   // Kahan: sum += tacc
      T yv = tacc[u] - comp[u];
      T tv = sum[u] + yv;
      comp[u] = (tv - sum[u]) - yv;
      sum[u] = tv;
    }
    __syncthreads();
  }
  const int nblk = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  for (int u = 0; u < NA; ++u) {
    double v = block_sum((double)sum[u] - (double)comp[u], sh);
    if (threadIdx.x == 0) part[(int64_t)u * nblk + bid] = v;
  }
  if (last_block_arrived(counter)) {
    // outputs: D lengthscale entries then the scale
    for (int o = threadIdx.x; o < D + 1; o += blockDim.x) {
      int u = (o == D) ? DM : o;
      double acc = 0.0;
      for (int b = 0; b < nblk; ++b) acc += part[(int64_t)u * nblk + b];
      double scale = (o == D) ? 1.0 / theta[D] : 1.0 / theta[ard ? o : 0];
      gout[o] = (accumulate ? gout[o] : 0.0) + acc * scale;
    }
  }
}

// sum_a sum_c w_c A[a,c] B[a,c]  (the noise entry: dK_hat/dsigma^2 = I)
template <class T>
__global__ void diag_contract_kernel(int64_t n, const T* __restrict__ A, int64_t lda,
                                     const T* __restrict__ B, int64_t ldb,
                                     const double* __restrict__ wts, int t,
                                     double* __restrict__ part, unsigned* counter,
                                     double* __restrict__ gout) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < t; ++c) acc += wts[c] * (double)A[i + c * lda] * (double)B[i + c * ldb];
  double v = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  if (last_block_arrived(counter)) {
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) s += part[b];
      *gout = s;
    }
  }
}

int pick_dm(int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32; }
// column block of the gradient contraction: also 40 (t = 33 is the common l = 32 case)
int pick_tc_contract(int t) {
  return t <= 8 ? 8 : t <= 16 ? 16 : t <= 32 ? 32 : t <= 40 ? 40 : t <= 48 ? 48 : 64;
}
int pick_tc(int t) { return t <= 8 ? 8 : t <= 16 ? 16 : t <= 32 ? 32 : t <= 48 ? 48 : 64; }

int64_t split_cols_for(int64_t n, int64_t row_blocks, int* splits) {
  // aim for >= ~4 CTAs per SM; each split spans >= 256 columns
  int64_t want = cdiv(4 * 152, row_blocks);
  int64_t maxs = cdiv(n, 256);
  int64_t sp = want < 1 ? 1 : want;
  if (sp > maxs) sp = maxs;
  if (sp < 1) sp = 1;
  int64_t cols = cdiv(n, sp);
  cols = cdiv(cols, kBN) * kBN;
  *splits = (int)cdiv(n, cols);
  return cols;
}

#define GP_DISPATCH_CONTRACT(DMv, TCv, ...)                                        \
  switch (DMv * 100 + TCv) {                                                     \
    case 440: { constexpr int DM = 4, TC = 40; __VA_ARGS__; } break;               \
    case 840: { constexpr int DM = 8, TC = 40; __VA_ARGS__; } break;               \
    case 1640: { constexpr int DM = 16, TC = 40; __VA_ARGS__; } break;             \
    case 3240: { constexpr int DM = 32, TC = 40; __VA_ARGS__; } break;             \
    default: GP_DISPATCH_DM_TC(DMv, TCv, __VA_ARGS__);                             \
  }

#define GP_DISPATCH_DM_TC(DMv, TCv, ...)                                           \
  switch (DMv * 100 + TCv) {                                                     \
    case 408: { constexpr int DM = 4, TC = 8; __VA_ARGS__; } break;                \
    case 416: { constexpr int DM = 4, TC = 16; __VA_ARGS__; } break;               \
    case 432: { constexpr int DM = 4, TC = 32; __VA_ARGS__; } break;               \
    case 464: { constexpr int DM = 4, TC = 64; __VA_ARGS__; } break;               \
    case 808: { constexpr int DM = 8, TC = 8; __VA_ARGS__; } break;                \
    case 816: { constexpr int DM = 8, TC = 16; __VA_ARGS__; } break;               \
    case 832: { constexpr int DM = 8, TC = 32; __VA_ARGS__; } break;               \
    case 864: { constexpr int DM = 8, TC = 64; __VA_ARGS__; } break;               \
    case 1608: { constexpr int DM = 16, TC = 8; __VA_ARGS__; } break;              \
    case 1616: { constexpr int DM = 16, TC = 16; __VA_ARGS__; } break;             \
    case 1632: { constexpr int DM = 16, TC = 32; __VA_ARGS__; } break;             \
    case 1648: { constexpr int DM = 16, TC = 48; __VA_ARGS__; } break;             \
    case 1664: { constexpr int DM = 16, TC = 64; __VA_ARGS__; } break;             \
    case 3208: { constexpr int DM = 32, TC = 8; __VA_ARGS__; } break;              \
    case 3216: { constexpr int DM = 32, TC = 16; __VA_ARGS__; } break;             \
    case 3232: { constexpr int DM = 32, TC = 32; __VA_ARGS__; } break;             \
    case 3248: { constexpr int DM = 32, TC = 48; __VA_ARGS__; } break;             \
    case 3264: { constexpr int DM = 32, TC = 64; __VA_ARGS__; } break;             \
  }

}  // namespace

// ---------------------------------------------------------------------------
template <class T>
gp_status prep_inputs(const Prob& pb, const PrepBufs& pr, cudaStream_t st) {
  const T* X = static_cast<const T*>(pb.X);
  T* Xs = static_cast<T*>(pr.Xs);
  int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), kPrepBlocks);
  center_partial<T><<<blocks, 256, 0, st>>>(pb.n, pb.d, X, pr.part, pr.counter, pr.mean);
  GP_LAUNCH_CHECK();
  int64_t total = pb.n * pb.d;
  scale_inputs<T><<<(unsigned)cdiv(total, 256), 256, 0, st>>>(pb.n, pb.d, pb.ard, X, pb.theta,
                                                              pr.mean, Xs);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

size_t simt_scratch_elems(int64_t n, int t) {
  // the product with two rows per thread has the fewest row blocks, hence the
  // most column splits
  int splits;
  split_cols_for(n, cdiv(n, 2 * kBM), &splits);
  int tc = t < 64 ? t : 64;
  return (size_t)splits * tc * n;
}

template <class T>
gp_status kmvm_simt(const Prob& pb, const void* Xs_, const void* V_, int64_t ldv, int t,
                    void* W_, int64_t ldw, void* scratch, const int* gate, cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const T* V = static_cast<const T*>(V_);
  T* W = static_cast<T*>(W_);
  T* part = static_cast<T*>(scratch);
  const int64_t rb = cdiv(pb.n, kBM * Rpt<T>::v);
  int splits;
  const int64_t cols = split_cols_for(pb.n, rb, &splits);
  const int dm = pick_dm(pb.d);
  for (int c0 = 0; c0 < t; c0 += 64) {
    const int tc = std::min(64, t - c0);
    const int tcp = pick_tc(tc);
    dim3 grid((unsigned)rb, (unsigned)splits);
    T* dst = splits == 1 ? W + c0 * ldw : part;
    int64_t ldo = splits == 1 ? ldw : pb.n;
    GP_DISPATCH_DM_TC(dm, tcp,
        (kmvm_kernel<T, DM, TC><<<grid, kBM, 0, st>>>(pb.n, pb.d, pb.kind, pb.D, pb.theta, Xs,
                                                     V + c0 * ldv, ldv, tc, dst, ldo, cols,
                                                     splits == 1 ? 1 : 0, gate)));
    GP_LAUNCH_CHECK();
    if (splits > 1) {
      split_reduce<T><<<(unsigned)cdiv(pb.n * tc, 256), 256, 0, st>>>(
          pb.n, tc, splits, part, V + c0 * ldv, ldv, pb.theta, pb.D, W + c0 * ldw, ldw, 1, gate);
      GP_LAUNCH_CHECK();
    }
  }
  return GP_OK;
}

template <class T>
gp_status kdmvm_simt(const Prob& pb, const void* Xs_, const void* V_, int64_t ldv, int t,
                     void* dW_, int64_t ldw, void* scratch, cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const T* V = static_cast<const T*>(V_);
  T* dW = static_cast<T*>(dW_);
  T* part = static_cast<T*>(scratch);
  const int64_t rb = cdiv(pb.n, kBM);
  int splits;
  const int64_t cols = split_cols_for(pb.n, rb, &splits);
  const int dm = pick_dm(pb.d);
  for (int q = 0; q < pb.p; ++q) {
    T* blk = dW + (int64_t)q * ldw * t;
    if (q == pb.p - 1) {
      copy_block<T><<<(unsigned)cdiv(pb.n * t, 256), 256, 0, st>>>(pb.n, t, V, ldv, blk, ldw);
      GP_LAUNCH_CHECK();
      continue;
    }
    for (int c0 = 0; c0 < t; c0 += 64) {
      const int tc = std::min(64, t - c0);
      const int tcp = pick_tc(tc);
      dim3 grid((unsigned)rb, (unsigned)splits);
      T* dst = splits == 1 ? blk + c0 * ldw : part;
      int64_t ldo = splits == 1 ? ldw : pb.n;
      GP_DISPATCH_DM_TC(dm, tcp,
          (kdmvm_kernel<T, DM, TC><<<grid, kBM, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, q,
                                                        pb.theta, Xs, V + c0 * ldv, ldv, tc,
                                                        dst, ldo, cols)));
      GP_LAUNCH_CHECK();
      if (splits > 1) {
        split_reduce<T><<<(unsigned)cdiv(pb.n * tc, 256), 256, 0, st>>>(
            pb.n, tc, splits, part, V, ldv, pb.theta, pb.D, blk + c0 * ldw, ldw, 0, nullptr);
        GP_LAUNCH_CHECK();
      }
    }
  }
  return GP_OK;
}

size_t contract_part_elems(int64_t n) {
  int splits;
  split_cols_for(n, cdiv(n, kBM), &splits);
  return (size_t)(kMaxD + 1) * cdiv(n, kBM) * splits + 1024;
}

template <class T>
gp_status contract_simt(const Prob& pb, const void* Xs_, const void* A_, int64_t lda,
                        const void* B_, int64_t ldb, const double* wts, int t, double* part,
                        unsigned* counter, double* gout, cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const T* A = static_cast<const T*>(A_);
  const T* B = static_cast<const T*>(B_);
  const int64_t rb = cdiv(pb.n, kBM);
  int splits;
  const int64_t cols = split_cols_for(pb.n, rb, &splits);
  const int dm = pick_dm(pb.d);
  for (int c0 = 0; c0 < t; c0 += 64) {
    const int tc = std::min(64, t - c0);
    const int tcp = pick_tc_contract(tc);
    dim3 grid((unsigned)rb, (unsigned)splits);
    GP_DISPATCH_CONTRACT(dm, tcp,
        (contract_kernel<T, DM, TC><<<grid, kBM, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D,
                                                         pb.theta, Xs, A, lda, B, ldb, wts, c0,
                                                         tc, cols, part, counter, gout,
                                                         c0 > 0 ? 1 : 0)));
    GP_LAUNCH_CHECK();
  }
  int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), 256);
  diag_contract_kernel<T><<<blocks, 256, 0, st>>>(pb.n, A, lda, B, ldb, wts, t, part,
                                                  counter, gout + pb.D + 1);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template <class T>
gp_status contract_noise(const Prob& pb, const void* A_, int64_t lda, const void* B_, int64_t ldb,
                         const double* wts, int t, double* part, unsigned* counter, double* gout,
                         cudaStream_t st) {
  const T* A = static_cast<const T*>(A_);
  const T* B = static_cast<const T*>(B_);
  int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), 256);
  diag_contract_kernel<T><<<blocks, 256, 0, st>>>(pb.n, A, lda, B, ldb, wts, t, part, counter,
                                                  gout);
  GP_LAUNCH_CHECK();
  return GP_OK;
}
template gp_status contract_noise<float>(const Prob&, const void*, int64_t, const void*, int64_t,
                                         const double*, int, double*, unsigned*, double*,
                                         cudaStream_t);
template gp_status contract_noise<double>(const Prob&, const void*, int64_t, const void*, int64_t,
                                          const double*, int, double*, unsigned*, double*,
                                          cudaStream_t);

template gp_status prep_inputs<float>(const Prob&, const PrepBufs&, cudaStream_t);
template gp_status prep_inputs<double>(const Prob&, const PrepBufs&, cudaStream_t);
template gp_status kmvm_simt<float>(const Prob&, const void*, const void*, int64_t, int, void*,
                                    int64_t, void*, const int*, cudaStream_t);
template gp_status kmvm_simt<double>(const Prob&, const void*, const void*, int64_t, int, void*,
                                     int64_t, void*, const int*, cudaStream_t);
template gp_status kdmvm_simt<float>(const Prob&, const void*, const void*, int64_t, int, void*,
                                     int64_t, void*, cudaStream_t);
template gp_status kdmvm_simt<double>(const Prob&, const void*, const void*, int64_t, int, void*,
                                      int64_t, void*, cudaStream_t);
template gp_status contract_simt<float>(const Prob&, const void*, const void*, int64_t,
                                        const void*, int64_t, const double*, int, double*,
                                        unsigned*, double*, cudaStream_t);
template gp_status contract_simt<double>(const Prob&, const void*, const void*, int64_t,
                                         const void*, int64_t, const double*, int, double*,
                                         unsigned*, double*, cudaStream_t);

}  // namespace gp

namespace gp {
// The same product with the column split turned off, so it needs no scratch for
// split partials (used by the allocation-free entry point in noalloc.cu).
template <class T>
gp_status kmvm_simt_unsplit(const Prob& pb, const void* Xs_, const void* V_, int64_t ldv, int t,
                            void* W_, int64_t ldw, cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const T* V = static_cast<const T*>(V_);
  T* W = static_cast<T*>(W_);
  const int64_t rb = cdiv(pb.n, kBM * Rpt<T>::v);
  const int64_t cols = cdiv(pb.n, kBN) * kBN;
  const int dm = pick_dm(pb.d);
  for (int c0 = 0; c0 < t; c0 += 64) {
    const int tc = std::min(64, t - c0);
    const int tcp = pick_tc(tc);
    dim3 grid((unsigned)rb, 1u);
    GP_DISPATCH_DM_TC(dm, tcp,
        (kmvm_kernel<T, DM, TC><<<grid, kBM, 0, st>>>(pb.n, pb.d, pb.kind, pb.D, pb.theta, Xs,
                                                     V + c0 * ldv, ldv, tc, W + c0 * ldw, ldw,
                                                     cols, 1, nullptr)));
    GP_LAUNCH_CHECK();
  }
  return GP_OK;
}
template gp_status kmvm_simt_unsplit<float>(const Prob&, const void*, const void*, int64_t, int,
                                            void*, int64_t, cudaStream_t);
template gp_status kmvm_simt_unsplit<double>(const Prob&, const void*, const void*, int64_t, int,
                                             void*, int64_t, cudaStream_t);
}  // namespace gp
