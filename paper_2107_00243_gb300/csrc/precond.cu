// Preconditioner terms of the gradient (Alg. 2 steps 3 and 7; eq. preconditioner_trace):
//   trP_q    = tr(P_hat^-1 dP_hat/dtheta_q)
//   probeP_q = (1/l) sum_i w_i^T dP_hat/dtheta_q w_i,   w_i = P_hat^-1 z_i
// with dP_hat taken at frozen pivots.  With the pivots fixed, the rank-k pivoted
// Cholesky factor satisfies L = Kc L_pi^-T (Kc = K[:, piv], L_pi = L[piv, :],
// lower triangular, L_pi L_pi^T = W = K[piv, piv]), so L L^T = Kc W^-1 Kc^T and
//   d(L L^T) = F L^T + L F^T - L S L^T,  F = Ddot L_pi^-T,  S = L_pi^-1 dW L_pi^-T,
// Ddot = dKc/dtheta_q, dW = Ddot[piv, :].  Substituting into the matrix inversion
// lemma with C = sigma^2 I + L^T L and C^-1 L^T L = I - sigma^2 C^-1 gives
//   trP_q    = 2 tr(C^-1 L^T F) - tr(C^-1 L^T L S) = 2 sum(A1 o Q_L) - sum(B1 o dW)
//     A1 = L_pi^-T C^-1,  B1 = L_pi^-T (I - sigma^2 C^-1) L_pi^-1,  Q_L = Ddot^T L
//   w^T dP w = 2 (Ddot^T w) . c - c^T dW c,   c = L_pi^-T L^T w
// and for the noise (dP/dsigma^2 = I): trP = sigma^-2 (n - k) + tr(C^-1),
// probeP = (1/l) sum_i ||w_i||^2.
// The O(n k (k + l)) products Ddot^T [L | W] are formed tile by tile, generating
// the kernel-derivative tile on the fly; everything k x k is FP64.
#include "ops.h"

namespace gp {
namespace {

constexpr int kTile = 32;

// part[ch][m][c] = sum over chunk rows a of Ddot_q[a, m] * Y[a, c],  Y = [L | W].
template <class T>
__global__ void __launch_bounds__(256) dk_atb_partial(
    int64_t n, int d, int kind, int ard, int D, int q, const double* __restrict__ theta,
    const T* __restrict__ Xs, const int* __restrict__ piv, int k,
    const T* __restrict__ L, int64_t ldl, const T* __restrict__ W, int64_t ldw, int nl,
    double* __restrict__ part) {
  __shared__ T sa[kTile][kTile + 1];   // [pivot m][row]
  __shared__ T sb[kTile][kTile + 1];   // [col c][row]
  __shared__ T xp[kTile][kMaxD];
  __shared__ int pv[kTile];
  const int kb = k + nl;
  const int m0 = blockIdx.x * kTile, j0 = blockIdx.y * kTile;
  const int64_t r0 = (int64_t)blockIdx.z * kAtbRows;
  const int64_t r1 = min(n, r0 + kAtbRows);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const T s = (T)theta[D];
  const bool is_scale = (q == D);
  const T qscale = is_scale ? (T)(1.0 / theta[D]) : (T)(1.0 / theta[ard ? q : 0]);
  for (int e = threadIdx.x; e < kTile; e += 256) pv[e] = (m0 + e < k) ? piv[m0 + e] : -1;
  __syncthreads();
  for (int e = threadIdx.x; e < kTile * d; e += 256) {
    int mm = e / d, u = e % d;
    xp[mm][u] = pv[mm] >= 0 ? Xs[(int64_t)pv[mm] * d + u] : T(0);
  }
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t rb = r0; rb < r1; rb += kTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTile * kTile; e += 256) {
      int rr = e & 31, cc = e >> 5;
      int64_t r = rb + rr;
      // derivative tile entry (row r, pivot m0 + cc)
      T v = T(0);
      if (r < r1 && pv[cc] >= 0) {
        T r2 = T(0), dq = T(0);
        for (int u = 0; u < d; ++u) {
          T df = Xs[r * d + u] - xp[cc][u];
          r2 = fma(df, df, r2);
          if (ard && u == q) dq = df * df;
        }
        T kv, fac;
        kval_fac<T>(kind, r2, s, kv, fac);
        v = is_scale ? kv : (ard ? fac * dq : fac * r2);
        v *= qscale;
      }
      sa[cc][rr] = v;
      T bv = T(0);
      int c = j0 + cc;
      if (r < r1 && c < kb) bv = (c < k) ? L[r + (int64_t)c * ldl] : W[r + (int64_t)(c - k) * ldw];
      sb[cc][rr] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kTile; ++rr) {
      T bv = sb[tx][rr];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(sa[ty + 8 * u][rr], bv, acc[u]);
    }
  }
  double* out = part + (int64_t)blockIdx.z * k * kb;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int m = m0 + ty + 8 * u, c = j0 + tx;
    if (m < k && c < kb) out[(int64_t)m * kb + c] = (double)acc[u];
  }
}

__global__ void sum_chunks_into(int64_t elems, int chunks, const double* __restrict__ part,
                                double* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= elems) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * elems + e];
  out[e] = s;
}

// dW[q][m1][m2] = dK/dtheta_q (x_{piv m1}, x_{piv m2}) for q < p - 1 (FP64).
template <class T>
__global__ void dw_kernel(int d, int kind, int ard, int D, const double* __restrict__ theta,
                          const T* __restrict__ Xs, const int* __restrict__ piv, int k,
                          double* __restrict__ dW) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  int m1 = (int)(e / k), m2 = (int)(e % k);
  int a = piv[m1], b = piv[m2];
  const int P1 = D + 1;
  if (a < 0 || b < 0) {
    for (int q = 0; q < P1; ++q) dW[(int64_t)q * k * k + e] = 0.0;
    return;
  }
  double r2 = 0.0;
  double df2[kMaxD];
  for (int u = 0; u < d; ++u) {
    double df = (double)Xs[(int64_t)a * d + u] - (double)Xs[(int64_t)b * d + u];
    df2[u] = df * df;
    r2 += df2[u];
  }
  double kv, fac;
  kval_fac<double>(kind, r2, theta[D], kv, fac);
  for (int q = 0; q < D; ++q) {
    double v = ard ? fac * df2[q] : fac * r2;
    dW[(int64_t)q * k * k + e] = v / theta[ard ? q : 0];
  }
  dW[(int64_t)D * k * k + e] = kv / theta[D];
}

// Lpi = L[piv, :] (k x k, row-major, FP64); rows past the rank are identity rows.
template <class T>
__global__ void gather_lpi(int k, const T* __restrict__ L, int64_t ldl,
                           const int* __restrict__ piv, const int* __restrict__ rank,
                           double* __restrict__ Lpi) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  int m = e / k, j = e % k;
  int r = *rank;
  double v;
  if (m < r) v = (j <= m) ? (double)L[piv[m] + (int64_t)j * ldl] : 0.0;
  else v = (m == j) ? 1.0 : 0.0;
  Lpi[e] = v;
}

// B1 = tmp - sigma^2 B1
__global__ void combine_b1(int64_t elems, const double* __restrict__ tmp,
                           const double* __restrict__ theta, int D, double* __restrict__ B1) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= elems) return;
  B1[e] = tmp[e] - theta[D + 1] * B1[e];
}

// One block per hyperparameter q: the FP64 contractions listed at the top.
__global__ void __launch_bounds__(256) terms_kernel(
    int k, int nl, int P, int64_t n, const double* __restrict__ theta, int D,
    const double* __restrict__ Q, const double* __restrict__ dW, const double* __restrict__ A1,
    const double* __restrict__ B1, const double* __restrict__ Cv, const double* __restrict__ Cinv,
    const double* __restrict__ wnorm2, double* __restrict__ trP, double* __restrict__ probeP) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  const double s2 = theta[D + 1];
  if (q == P - 1) {   // noise
    double acc = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) acc += Cinv[(int64_t)i * k + i];
    double tr = block_sum(acc, sh);
    if (threadIdx.x == 0) {
      trP[q] = (double)(n - k) / s2 + tr;
      probeP[q] = nl > 0 ? *wnorm2 / nl : 0.0;
    }
    return;
  }
  const int kb = k + nl;
  const double* Qq = Q + (int64_t)q * k * kb;
  const double* dWq = dW + (int64_t)q * k * k;
  double t1 = 0.0, t2 = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) {
    int i = (int)(e / k), j = (int)(e % k);
    t1 += A1[e] * Qq[(int64_t)i * kb + j];
    t2 += B1[e] * dWq[e];
  }
  // probe terms: sum_i [2 Q[:, k+i] . c_i - c_i^T dW c_i]
  double pr = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)k * nl; e += blockDim.x) {
    int m1 = (int)(e / nl), i = (int)(e % nl);
    const double c1 = Cv[(int64_t)m1 * nl + i];
    double row = 0.0;
    for (int m2 = 0; m2 < k; ++m2) row += dWq[(int64_t)m1 * k + m2] * Cv[(int64_t)m2 * nl + i];
    pr += 2.0 * Qq[(int64_t)m1 * kb + k + i] * c1 - c1 * row;
  }
  double T1 = block_sum(t1, sh);
  double T2 = block_sum(t2, sh);
  double PR = block_sum(pr, sh);
  if (threadIdx.x == 0) {
    trP[q] = 2.0 * T1 - T2;
    probeP[q] = nl > 0 ? PR / nl : 0.0;
  }
}

template <class T>
__global__ void sumsq_kernel(int64_t n, int nl, const T* __restrict__ W, int64_t ldw,
                             double* part, unsigned* counter, double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int c = 0; c < nl; ++c)
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
      double v = (double)W[a + c * ldw];
      acc += v * v;
    }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (last_block_arrived(counter)) {
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) r += part[b];
      *out = r;
    }
  }
}

}  // namespace

template <class T>
gp_status precond_terms(const Prob& pb, const void* Xs_, const T* L, int64_t ldl, int k,
                        const int* piv, const int* rank, const T* W, int64_t ldw, int nl,
                        const double* Cinv, const PrecBufs& b, double* trP, double* probeP,
                        cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const int P = pb.p;
  // ||w||^2 summed over probes (noise entry); reuse the tail of b.tmp for the partials
  double* wn = b.LtW + (int64_t)k * nl;         // 1 double after LtW
  unsigned* ctr = reinterpret_cast<unsigned*>(wn + 1);
  double* spart = wn + 2;
  {
    int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), 128);
    GP_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned), st));
    sumsq_kernel<T><<<blocks, 256, 0, st>>>(pb.n, nl, W, ldw, spart, ctr, wn);
    GP_LAUNCH_CHECK();
  }
  if (k > 0) {
    const int kb = k + nl;
    const int64_t ch = atb_chunks(pb.n);
    for (int q = 0; q < P - 1; ++q) {
      dim3 grid((unsigned)cdiv(k, kTile), (unsigned)cdiv(kb, kTile), (unsigned)ch);
      dk_atb_partial<T><<<grid, 256, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, q, pb.theta, Xs,
                                              piv, k, L, ldl, W, ldw, nl, b.part);
      GP_LAUNCH_CHECK();
      const int64_t el = (int64_t)k * kb;
      sum_chunks_into<<<(unsigned)cdiv(el, 256), 256, 0, st>>>(el, (int)ch, b.part,
                                                              b.Q + (int64_t)q * el);
      GP_LAUNCH_CHECK();
    }
    dw_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 128), 128, 0, st>>>(pb.d, pb.kind, pb.ard, pb.D,
                                                                       pb.theta, Xs, piv, k, b.dW);
    GP_LAUNCH_CHECK();
    gather_lpi<T><<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(k, L, ldl, piv, rank, b.Lpi);
    GP_LAUNCH_CHECK();
    GP_TRY(tri_inv_lower(k, b.Lpi, b.Lpinv, st));
    GP_TRY(gemm64(k, k, k, b.Lpinv, 1, Cinv, 0, b.A1, 1.0, 0.0, st));       // L_pi^-T C^-1
    GP_TRY(gemm64(k, k, k, b.Lpinv, 1, b.Lpinv, 0, b.tmp, 1.0, 0.0, st));  // W^-1
    GP_TRY(gemm64(k, k, k, b.A1, 0, b.Lpinv, 0, b.B1, 1.0, 0.0, st));      // L_pi^-T C^-1 L_pi^-1
    combine_b1<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>((int64_t)k * k, b.tmp,
                                                                   pb.theta, pb.D, b.B1);
    GP_LAUNCH_CHECK();
    if (nl > 0) {
      GP_TRY(atb<T>(pb.n, L, ldl, k, W, ldw, nl, b.part, b.LtW, st));      // L^T W
      GP_TRY(gemm64(k, nl, k, b.Lpinv, 1, b.LtW, 0, b.Cv, 1.0, 0.0, st));  // L_pi^-T L^T W
    }
  }
  terms_kernel<<<P, 256, 0, st>>>(k, nl, P, pb.n, pb.theta, pb.D, b.Q, b.dW, b.A1, b.B1, b.Cv,
                                  Cinv, wn, trP, probeP);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template gp_status precond_terms<float>(const Prob&, const void*, const float*, int64_t, int,
                                        const int*, const int*, const float*, int64_t, int,
                                        const double*, const PrecBufs&, double*, double*,
                                        cudaStream_t);
template gp_status precond_terms<double>(const Prob&, const void*, const double*, int64_t, int,
                                         const int*, const int*, const double*, int64_t, int,
                                         const double*, const PrecBufs&, double*, double*,
                                         cudaStream_t);

}  // namespace gp
