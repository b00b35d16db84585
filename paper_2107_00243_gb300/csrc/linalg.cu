// Small dense FP64 linear algebra (k x k Woodbury core, triangular inverses,
// small GEMMs) and tall-skinny products A^T B reduced over n rows.
//
// GB300's FP64 pipe is narrow, so FP64 work here is O(k^2 t) or O(k^3) and spread
// over many CTAs; the O(n k t) products run in the problem precision with FP64
// chunk sums.
#include "ops.h"

namespace gp {
namespace {

constexpr int kTile = 32;

// part[ch][i][j] = sum over the chunk's rows r of A[r, i] * B[r, j].
template <class T>
__global__ void __launch_bounds__(256) atb_partial(int64_t n, const T* __restrict__ A, int64_t lda,
                                                   int ka, const T* __restrict__ B, int64_t ldb,
                                                   int kb, double* __restrict__ part) {
  __shared__ T sa[kTile][kTile + 1];
  __shared__ T sb[kTile][kTile + 1];
  const int i0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
  const int64_t r0 = (int64_t)blockIdx.z * kAtbRows;
  const int64_t r1 = min(n, r0 + kAtbRows);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t rb = r0; rb < r1; rb += kTile) {
    for (int e = threadIdx.x; e < kTile * kTile; e += 256) {
      int rr = e & 31, cc = e >> 5;
      int64_t r = rb + rr;
      sa[cc][rr] = (r < r1 && i0 + cc < ka) ? A[r + (int64_t)(i0 + cc) * lda] : T(0);
      sb[cc][rr] = (r < r1 && j0 + cc < kb) ? B[r + (int64_t)(j0 + cc) * ldb] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kTile; ++rr) {
      T bv = sb[tx][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(sa[ty + 8 * q][rr], bv, acc[q]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * ka * kb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < ka && j < kb) out[(int64_t)i * kb + j] = (double)acc[q];
  }
}

__global__ void sum_chunks(int64_t elems, int chunks, const double* __restrict__ part,
                           double* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= elems) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * elems + e];
  out[e] = s;
}

// C = s2 I + G ; in-place lower Cholesky (row-major) by one CTA, right-looking.
__global__ void __launch_bounds__(1024) core_cholesky(int k, const double* __restrict__ G,
                                                     const double* __restrict__ theta, int D,
                                                     int64_t n, double* __restrict__ C,
                                                     double* logdetP, int* status) {
  __shared__ int bad;
  __shared__ double ld;
  const double s2 = theta[D + 1];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nth = blockDim.x * blockDim.y;
  for (int e = tid; e < k * k; e += nth) {
    int i = e / k, j = e % k;
    double v = G[e] + (i == j ? s2 : 0.0);
    C[e] = (j <= i) ? v : 0.0;
  }
  if (tid == 0) { bad = 0; ld = 0.0; }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double p = C[j * k + j];
      if (!(p > 0.0)) { bad = 1; p = 1.0; }
      double r = sqrt(p);
      C[j * k + j] = r;
      ld += log(r);
    }
    __syncthreads();
    const double r = C[j * k + j];
    for (int i = j + 1 + tid; i < k; i += nth) C[i * k + j] /= r;
    __syncthreads();
    // trailing update of the lower triangle: C[i][l] -= C[i][j] C[l][j], j < l <= i
    for (int i = j + 1 + threadIdx.y; i < k; i += blockDim.y) {
      const double cij = C[i * k + j];
      for (int l = j + 1 + threadIdx.x; l <= i; l += blockDim.x) C[i * k + l] -= cij * C[l * k + j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    // log det P_hat = (n - k) log s2 + log det C   (determinant lemma)
    *logdetP = (double)(n - k) * log(s2) + 2.0 * ld;
    if (bad) raise_status(status, GP_ERR_NOT_SPD);
  }
}

// Linv = L^-1 for lower-triangular L (row-major); thread j forward-substitutes column j.
__global__ void tri_inv_kernel(int k, const double* __restrict__ Lm, double* __restrict__ Li) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  for (int i = 0; i < j; ++i) Li[i * k + j] = 0.0;
  Li[j * k + j] = 1.0 / Lm[j * k + j];
  for (int i = j + 1; i < k; ++i) {
    double a0 = 0.0, a1 = 0.0;
    int mm = j;
    for (; mm + 1 < i; mm += 2) {
      a0 += Lm[i * k + mm] * Li[mm * k + j];
      a1 += Lm[i * k + mm + 1] * Li[(mm + 1) * k + j];
    }
    if (mm < i) a0 += Lm[i * k + mm] * Li[mm * k + j];
    Li[i * k + j] = -(a0 + a1) / Lm[i * k + i];
  }
}

// C = alpha op(A) op(B) + beta C (row-major). op(A): m x kk, op(B): kk x nn.
__global__ void gemm64_kernel(int m, int nn, int kk, const double* __restrict__ A, int ta,
                              const double* __restrict__ B, int tb, double* __restrict__ C,
                              double alpha, double beta) {
  __shared__ double sa[16][17];
  __shared__ double sb[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < kk; k0 += 16) {
    int ak = k0 + tx, bk = k0 + ty;
    double av = 0.0, bv = 0.0;
    if (row < m && ak < kk) av = ta ? A[(int64_t)ak * m + row] : A[(int64_t)row * kk + ak];
    if (col < nn && bk < kk) bv = tb ? B[(int64_t)col * kk + bk] : B[(int64_t)bk * nn + col];
    sa[ty][tx] = av;
    sb[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc += sa[ty][q] * sb[q][tx];
    __syncthreads();
  }
  if (row < m && col < nn) {
    double prev = beta != 0.0 ? beta * C[(int64_t)row * nn + col] : 0.0;
    C[(int64_t)row * nn + col] = alpha * acc + prev;
  }
}

}  // namespace

int64_t atb_chunks(int64_t n) { return cdiv(n, kAtbRows); }

template <class T>
gp_status atb(int64_t n, const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb,
              double* part, double* out, cudaStream_t st) {
  if (ka == 0 || kb == 0) return GP_OK;
  const int64_t ch = atb_chunks(n);
  dim3 grid((unsigned)cdiv(ka, kTile), (unsigned)cdiv(kb, kTile), (unsigned)ch);
  atb_partial<T><<<grid, 256, 0, st>>>(n, static_cast<const T*>(A), lda, ka,
                                       static_cast<const T*>(B), ldb, kb, part);
  GP_LAUNCH_CHECK();
  const int64_t el = (int64_t)ka * kb;
  sum_chunks<<<(unsigned)cdiv(el, 256), 256, 0, st>>>(el, (int)ch, part, out);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template gp_status atb<float>(int64_t, const void*, int64_t, int, const void*, int64_t, int,
                              double*, double*, cudaStream_t);
template gp_status atb<double>(int64_t, const void*, int64_t, int, const void*, int64_t, int,
                               double*, double*, cudaStream_t);

gp_status tri_inv_lower(int k, const double* Lm, double* Linv, cudaStream_t st) {
  if (k == 0) return GP_OK;
  tri_inv_kernel<<<(unsigned)cdiv(k, 64), 64, 0, st>>>(k, Lm, Linv);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

gp_status gemm64(int m, int nn, int kk, const double* A, int ta, const double* B, int tb,
                 double* C, double alpha, double beta, cudaStream_t st) {
  if (m == 0 || nn == 0) return GP_OK;
  dim3 grid((unsigned)cdiv(nn, 16), (unsigned)cdiv(m, 16));
  gemm64_kernel<<<grid, dim3(16, 16), 0, st>>>(m, nn, kk, A, ta, B, tb, C, alpha, beta);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

// Woodbury core of P_hat = s2 I + L L^T:  C = s2 I + L^T L = Gc Gc^T (FP64),
// log det P_hat, and C^-1 = Gc^-T Gc^-1.  `work` holds k x k.
gp_status woodbury_core(int k, const double* G, const double* theta, int D, int64_t n,
                        double* C, double* Cinv, double* work, double* logdetP, int* status,
                        cudaStream_t st) {
  if (k == 0) {
    core_cholesky<<<1, dim3(32, 1), 0, st>>>(0, G, theta, D, n, C, logdetP, status);
    GP_LAUNCH_CHECK();
    return GP_OK;
  }
  core_cholesky<<<1, dim3(32, 32), 0, st>>>(k, G, theta, D, n, C, logdetP, status);
  GP_LAUNCH_CHECK();
  GP_TRY(tri_inv_lower(k, C, work, st));                         // work = Gc^-1
  GP_TRY(gemm64(k, k, k, work, 1, work, 0, Cinv, 1.0, 0.0, st));  // Gc^-T Gc^-1
  return GP_OK;
}

}  // namespace gp
