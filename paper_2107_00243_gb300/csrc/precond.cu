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
// Only contractions of Q = Ddot^T [L | W] with fixed matrices are needed:
//   sum(A1 o Q_L)                 = sum_{a,m} Ddot[a, m] Z1[a, m],  Z1 = L A1^T
//   sum_i Q_W[:, i] . c_i         = sum_{a,m} Ddot[a, m] Z2[a, m],  Z2 = W Cv^T
// so two tall GEMMs (n x k) and one fused pass over the n x k (point, pivot)
// pairs, which evaluates every hyperparameter's derivative of the kernel at once,
// replace p - 1 passes of an n x k x (k + l) product.  Everything k x k is FP64.
#include "ops.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gp {
namespace {

// Out (n x ncol, column-major) = Y (n x kk, column-major, ld ldy) Bt (kk x ncol, row-major).
// 128 x 64 output tile per block; thread (tr, tc) owns rows 4 tr .. + 3 and columns
// 8 tc .. + 7; Y and Bt are staged in shared memory 32 deep.
template <class T>
__global__ void __launch_bounds__(256) gemm_tall(int64_t n, int kk, int ncol,
                                                 const T* __restrict__ Y, int64_t ldy,
                                                 const T* __restrict__ Bt, T* __restrict__ Out) {
  __shared__ __align__(16) T sY[32][128];
  __shared__ __align__(16) T sB[32][64];
  const int tr = threadIdx.x & 31, tc = threadIdx.x >> 5;
  const int64_t a0 = blockIdx.x * (int64_t)128;
  const int c0 = blockIdx.y * 64;
  T acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = T(0);
  for (int j0 = 0; j0 < kk; j0 += 32) {
    const int jn = min(32, kk - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 128; e += 256) {
      const int rr = e % 128, jj = e / 128;
      const int64_t a = a0 + rr;
      sY[jj][rr] = (jj < jn && a < n) ? Y[a + (int64_t)(j0 + jj) * ldy] : T(0);
    }
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int cc = e % 64, jj = e / 64;
      sB[jj][cc] = (jj < jn && c0 + cc < ncol) ? Bt[(size_t)(j0 + jj) * ncol + c0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      T yv[4], bv[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) yv[a] = sY[jj][tr * 4 + a];
#pragma unroll
      for (int c = 0; c < 8; ++c) bv[c] = sB[jj][tc * 8 + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fma(yv[a], bv[c], acc[a][c]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t row = a0 + tr * 4 + a;
    if (row >= n) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = c0 + tc * 8 + c;
      if (col < ncol) Out[row + (int64_t)col * n] = acc[a][c];
    }
  }
}

// Bt[j][i] = M[i][j] in the problem precision (M row-major rows x cols, FP64).
template <class T>
__global__ void transpose_to(int rows, int cols, const double* __restrict__ M,
                             T* __restrict__ Bt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int i = e / cols, j = e % cols;
  Bt[(size_t)j * rows + i] = (T)M[e];
}

// E[q] = sum_{a,m} Ddot_q[a, m] Z1[a, m],  F[q] = sum_{a,m} Ddot_q[a, m] Z2[a, m] for every
// lengthscale and the output scale, Ddot_q[a, m] = d k(x_a, x_{piv m}) / d theta_q.
// One thread per point a, pivots staged in shared memory; per-block FP64 partials.
constexpr int kDkPiv = 64;
template <class T, int DM>
__global__ void __launch_bounds__(256) dk_contract(
    int64_t n, int d, int kind, int ard, int D, const double* __restrict__ theta,
    const T* __restrict__ Xs, const int* __restrict__ piv, const int* __restrict__ rank,
    const T* __restrict__ Z1, const T* __restrict__ Z2, double* __restrict__ part) {
  constexpr int NQ = DM + 1;                    // lengthscales (or 1) + output scale
  __shared__ T xp[kDkPiv][DM];
  __shared__ double sred[8][2 * NQ];
  const int64_t a = blockIdx.x * (int64_t)256 + threadIdx.x;
  const int r = *rank;
  const T s = (T)theta[D];
  T inv_l[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) inv_l[u] = (u < d) ? (T)(1.0 / theta[ard ? u : 0]) : T(0);
  const T inv_s = (T)(1.0 / theta[D]);
  T xa[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) xa[u] = (a < n && u < d) ? Xs[a * d + u] : T(0);
  double e1[NQ], e2[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { e1[q] = 0.0; e2[q] = 0.0; }
  for (int m0 = 0; m0 < r; m0 += kDkPiv) {
    const int mn = min(kDkPiv, r - m0);
    __syncthreads();
    for (int e = threadIdx.x; e < kDkPiv * DM; e += 256) {
      const int mm = e / DM, u = e % DM;
      xp[mm][u] = (mm < mn && u < d) ? Xs[(int64_t)piv[m0 + mm] * d + u] : T(0);
    }
    __syncthreads();
    if (a < n) {
      T f1[NQ], f2[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) { f1[q] = T(0); f2[q] = T(0); }
      for (int mm = 0; mm < mn; ++mm) {
        T df2[DM];
        T r2 = T(0);
#pragma unroll
        for (int u = 0; u < DM; ++u) {
          const T df = xa[u] - xp[mm][u];
          df2[u] = df * df;
          r2 += df2[u];
        }
        T kv, fac;
        kval_fac<T>(kind, r2, s, kv, fac);
        const T z1 = Z1[a + (int64_t)(m0 + mm) * n];
        const T z2 = Z2[a + (int64_t)(m0 + mm) * n];
        if (ard) {
#pragma unroll
          for (int u = 0; u < DM; ++u) {
            const T c = fac * df2[u];
            f1[u] = fma(c, z1, f1[u]);
            f2[u] = fma(c, z2, f2[u]);
          }
        } else {
          const T c = fac * r2;
          f1[0] = fma(c, z1, f1[0]);
          f2[0] = fma(c, z2, f2[0]);
        }
        f1[DM] = fma(kv, z1, f1[DM]);
        f2[DM] = fma(kv, z2, f2[DM]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        e1[q] += (double)f1[q];
        e2[q] += (double)f2[q];
      }
    }
  }
  // scale to the derivative: lengthscale q: / l_q ; output scale: / s
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double sc = (q == DM) ? (double)inv_s : (double)inv_l[q];
    const double v1 = warp_sum(e1[q] * sc), v2 = warp_sum(e2[q] * sc);
    if (lane == 0) { sred[warp][q] = v1; sred[warp][NQ + q] = v2; }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * NQ; e += 256) {
    double acc = 0.0;
    for (int w = 0; w < 8; ++w) acc += sred[w][e];
    part[(size_t)blockIdx.x * 2 * NQ + e] = acc;
  }
}

// EF[o] = sum over blocks (o < 2 NQ), fixed order.
__global__ void dk_combine(int nblk, int w, const double* __restrict__ part,
                           double* __restrict__ EF) {
  for (int o = threadIdx.x; o < w; o += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * w + o];
    EF[o] = acc;
  }
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

// E = I - sigma^2 C^-1 (= C^-1 L^T L, k x k row-major).  Both terms are O(1), so the
// difference is accurate to rounding of 1; B1 is then formed as L_pi^-T E L_pi^-1.
// The other order, W^-1 - sigma^2 L_pi^-T C^-1 L_pi^-1, subtracts two matrices whose
// entries grow like 1 / (smallest pivot residual) and loses every digit of B1 once the
// factor nears numerical rank deficiency.
__global__ void eye_minus_s2_cinv(int k, const double* __restrict__ Cinv,
                                  const double* __restrict__ theta, int D,
                                  double* __restrict__ E) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int i = (int)(e / k), j = (int)(e % k);
  E[e] = (i == j ? 1.0 : 0.0) - theta[D + 1] * Cinv[e];
}

// One block per hyperparameter q: the FP64 contractions listed at the top.
// EF holds E[0..NQ) then F[0..NQ) (NQ = DM + 1; entry DM is the output scale).
__global__ void __launch_bounds__(256) terms_kernel(
    int k, int nl, int P, int64_t n, const double* __restrict__ theta, int D, int NQ, int DM,
    const double* __restrict__ EF, const double* __restrict__ dW, const double* __restrict__ B1,
    const double* __restrict__ Cv, const double* __restrict__ Cinv,
    const double* __restrict__ wnorm2, double* __restrict__ trP, double* __restrict__ probeP,
    int nystrom) {
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
  const int slot = (q == D) ? DM : q;          // E/F index of this hyperparameter
  if (!nystrom) {
    // features: dP_hat = dPhi Phi^T + Phi dPhi^T has no pivot-block term
    if (threadIdx.x == 0) {
      trP[q] = 2.0 * EF[slot];
      probeP[q] = nl > 0 ? 2.0 * EF[NQ + slot] / nl : 0.0;
    }
    return;
  }
  const double* dWq = dW + (int64_t)q * k * k;
  double t2 = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) t2 += B1[e] * dWq[e];
  // probe terms: sum_i c_i^T dW c_i
  double pr = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)k * nl; e += blockDim.x) {
    int m1 = (int)(e / nl), i = (int)(e % nl);
    const double c1 = Cv[(int64_t)m1 * nl + i];
    double row = 0.0;
    for (int m2 = 0; m2 < k; ++m2) row += dWq[(int64_t)m1 * k + m2] * Cv[(int64_t)m2 * nl + i];
    pr += c1 * row;
  }
  double T2 = block_sum(t2, sh);
  double PR = block_sum(pr, sh);
  if (threadIdx.x == 0) {
    trP[q] = 2.0 * EF[slot] - T2;
    probeP[q] = nl > 0 ? (2.0 * EF[NQ + slot] - PR) / nl : 0.0;
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

// ---- random Fourier feature preconditioner (Tab. 2 "RFF") -----------------------------
// P_hat = sigma^2 I + Phi Phi^T with m frequencies u_j (in units of 1 / l), weights w_j
// (1/m for random features) and k = 2m features
//   Phi[a, j] = sqrt(s w_j) cos(u_j . x~_a),  Phi[a, m + j] = sqrt(s w_j) sin(u_j . x~_a)
// (x~ = (x - mean x) / l, the centred inputs of S1: a shift of the origin only turns each
// cos / sin pair, so Phi Phi^T is the same).  By Bochner's theorem E[Phi Phi^T] = K when
// u_j is drawn from the kernel's spectral density, written as a Gaussian scale mixture
// u_j = rho_j eps_j:
//   RBF rho = 1;  Matern-nu rho = sqrt(nu / g_j), g_j ~ Gamma(nu, 1) (a multivariate t
//   with 2 nu degrees of freedom);  rational quadratic (alpha = 1) rho = sqrt(g_j),
//   g_j ~ Gamma(1, 1) (1 / (1 + r^2/2) = E_g[exp(-g r^2 / 2)]).
// The draws eps_j, g_j are inputs.  Arguments and features are formed in FP64 (one pass
// each per evaluation) and stored in the problem precision.
constexpr int kFeatChunk = 32;    // frequencies staged in shared memory per step

__global__ void rff_freq_kernel(int kind, int m, int d, const double* __restrict__ eps,
                                const double* __restrict__ g, double* __restrict__ U,
                                double* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * d) return;
  const int j = e / d;
  if (e % d == 0) wt[j] = 1.0 / m;    // equal weights: E[Phi Phi^T] = K
  double rho = 1.0;
  if (kind == GP_RATQUAD) rho = sqrt(g[j]);
  else if (kind == GP_MATERN32) rho = sqrt(1.5 / g[j]);
  else if (kind == GP_MATERN52) rho = sqrt(2.5 / g[j]);
  U[e] = rho * eps[e];
}

// One thread per row a, a chunk of kFeatChunk frequencies per block (grid.y).
template <class T, int DM>
__global__ void __launch_bounds__(256) rff_build_kernel(int64_t n, int d, int m,
                                                        const T* __restrict__ Xs,
                                                        const double* __restrict__ U,
                                                        const double* __restrict__ wt,
                                                        const double* __restrict__ theta, int D,
                                                        T* __restrict__ Phi, int64_t ldp) {
  __shared__ double su[kFeatChunk][DM];
  const int j0 = blockIdx.y * kFeatChunk;
  const int jn = min(kFeatChunk, m - j0);
  for (int e = threadIdx.x; e < kFeatChunk * DM; e += blockDim.x) {
    const int jj = e / DM, u = e % DM;
    su[jj][u] = (jj < jn && u < d) ? U[(int64_t)(j0 + jj) * d + u] : 0.0;
  }
  __syncthreads();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= n) return;
  double xa[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) xa[u] = u < d ? (double)Xs[a * d + u] : 0.0;
  for (int jj = 0; jj < jn; ++jj) {
    const double amp = sqrt(theta[D] * wt[j0 + jj]);
    double arg = 0.0;
#pragma unroll
    for (int u = 0; u < DM; ++u) arg = fma(su[jj][u], xa[u], arg);
    double sn, c;
    sincos(arg, &sn, &c);
    Phi[a + (int64_t)(j0 + jj) * ldp] = (T)(amp * c);
    Phi[a + (int64_t)(m + j0 + jj) * ldp] = (T)(amp * sn);
  }
}

// E[q] = sum_{a, j} dPhi_q[a, j] Z1[a, j],  F[q] = sum_{a, j} dPhi_q[a, j] Z2[a, j] over the
// 2m feature columns, for every lengthscale and the output scale (frozen draws):
//   d cos / d l_i =  sin(arg) u_ji x~_i / l_i,  d sin / d l_i = -cos(arg) u_ji x~_i / l_i
//   (an isotropic l: the sum over i, i.e. arg / l),   d Phi / d s = Phi / (2 s).
// One thread per row a; per-block FP64 partials, as in dk_contract.
template <class T, int DM>
__global__ void __launch_bounds__(256) rff_contract(int64_t n, int d, int ard, int D, int m,
                                                    const double* __restrict__ theta,
                                                    const T* __restrict__ Xs,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ wt,
                                                    const T* __restrict__ Z1,
                                                    const T* __restrict__ Z2,
                                                    double* __restrict__ part) {
  constexpr int NQ = DM + 1;
  __shared__ double su[kFeatChunk][DM];
  __shared__ double sred[8][2 * NQ];
  const int64_t a = blockIdx.x * (int64_t)256 + threadIdx.x;
  double xa[DM];
#pragma unroll
  for (int u = 0; u < DM; ++u) xa[u] = (a < n && u < d) ? (double)Xs[a * d + u] : 0.0;
  double e1[NQ], e2[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) { e1[q] = 0.0; e2[q] = 0.0; }
  for (int j0 = 0; j0 < m; j0 += kFeatChunk) {
    const int jn = min(kFeatChunk, m - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < kFeatChunk * DM; e += 256) {
      const int jj = e / DM, u = e % DM;
      su[jj][u] = (jj < jn && u < d) ? U[(int64_t)(j0 + jj) * d + u] : 0.0;
    }
    __syncthreads();
    if (a >= n) continue;
    for (int jj = 0; jj < jn; ++jj) {
      const int j = j0 + jj;
      const double amp = sqrt(theta[D] * wt[j]);
      double arg = 0.0;
#pragma unroll
      for (int u = 0; u < DM; ++u) arg = fma(su[jj][u], xa[u], arg);
      double sn, c;
      sincos(arg, &sn, &c);
      const double z1c = (double)Z1[a + (int64_t)j * n], z1s = (double)Z1[a + (int64_t)(m + j) * n];
      const double z2c = (double)Z2[a + (int64_t)j * n], z2s = (double)Z2[a + (int64_t)(m + j) * n];
      const double g1 = amp * (sn * z1c - c * z1s), g2 = amp * (sn * z2c - c * z2s);
      if (ard) {
#pragma unroll
        for (int u = 0; u < DM; ++u) {
          const double w = su[jj][u] * xa[u];
          e1[u] = fma(g1, w, e1[u]);
          e2[u] = fma(g2, w, e2[u]);
        }
      } else {
        e1[0] = fma(g1, arg, e1[0]);
        e2[0] = fma(g2, arg, e2[0]);
      }
      e1[DM] += amp * (c * z1c + sn * z1s);
      e2[DM] += amp * (c * z2c + sn * z2s);
    }
  }
  // scale to the derivative: lengthscale q: / l_q ; output scale: / (2 s)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double sc = (q == DM) ? 0.5 / theta[D] : (q < D ? 1.0 / theta[q] : 0.0);
    const double v1 = warp_sum(e1[q] * sc), v2 = warp_sum(e2[q] * sc);
    if (lane == 0) { sred[warp][q] = v1; sred[warp][NQ + q] = v2; }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * NQ; e += 256) {
    double acc = 0.0;
    for (int w = 0; w < 8; ++w) acc += sred[w][e];
    part[(size_t)blockIdx.x * 2 * NQ + e] = acc;
  }
}

}  // namespace

int dm_of(int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32; }

template <class T>
gp_status precond_terms(const Prob& pb, const void* Xs_, const T* L, int64_t ldl, int k,
                        const int* piv, const int* rank, const T* W, int64_t ldw, int nl,
                        const double* Cinv, const PrecBufs& b, double* trP, double* probeP,
                        cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const int P = pb.p;
  // ||w||^2 summed over probes (noise entry); scratch after LtW
  double* wn = b.LtW + (int64_t)k * nl;
  unsigned* ctr = reinterpret_cast<unsigned*>(wn + 1);
  double* spart = wn + 2;
  {
    int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), 128);
    GP_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned), st));
    sumsq_kernel<T><<<blocks, 256, 0, st>>>(pb.n, nl, W, ldw, spart, ctr, wn);
    GP_LAUNCH_CHECK();
  }
  const int DM = dm_of(pb.d), NQ = DM + 1;
  double* EF = b.Cv + (size_t)std::max(k, 1) * std::max(nl, 1);   // 2 NQ doubles
  GP_CUDA_TRY(cudaMemsetAsync(EF, 0, sizeof(double) * 2 * NQ, st));
  if (k > 0) {
    dw_kernel<T><<<(unsigned)cdiv((int64_t)k * k, 128), 128, 0, st>>>(pb.d, pb.kind, pb.ard, pb.D,
                                                                       pb.theta, Xs, piv, k, b.dW);
    GP_LAUNCH_CHECK();
    gather_lpi<T><<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(k, L, ldl, piv, rank, b.Lpi);
    GP_LAUNCH_CHECK();
    GP_TRY(tri_inv_lower(k, b.Lpi, b.Lpinv, st));
    GP_TRY(gemm64(k, k, k, b.Lpinv, 1, Cinv, 0, b.A1, 1.0, 0.0, st));       // L_pi^-T C^-1
    eye_minus_s2_cinv<<<(unsigned)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, Cinv, pb.theta,
                                                                          pb.D, b.B1);
    GP_LAUNCH_CHECK();
    GP_TRY(gemm64(k, k, k, b.Lpinv, 1, b.B1, 0, b.tmp, 1.0, 0.0, st));     // L_pi^-T E
    GP_TRY(gemm64(k, k, k, b.tmp, 0, b.Lpinv, 0, b.B1, 1.0, 0.0, st));     // L_pi^-T E L_pi^-1
    T* Bt = reinterpret_cast<T*>(b.Q);                 // k x k then l x k, problem precision
    T* Z1 = reinterpret_cast<T*>(b.part);              // n x k
    T* Z2 = Z1 + (size_t)pb.n * k;                     // n x k
    // Z1 = L A1^T
    transpose_to<T><<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(k, k, b.A1, Bt);
    GP_LAUNCH_CHECK();
    dim3 gz((unsigned)cdiv(pb.n, 128), (unsigned)cdiv(k, 64));
    gemm_tall<T><<<gz, 256, 0, st>>>(pb.n, k, k, L, ldl, Bt, Z1);
    GP_LAUNCH_CHECK();
    if (nl > 0) {
      GP_TRY(atb<T>(pb.n, L, ldl, k, W, ldw, nl, b.dkpart, b.LtW, st));   // L^T W
      GP_TRY(gemm64(k, nl, k, b.Lpinv, 1, b.LtW, 0, b.Cv, 1.0, 0.0, st)); // c_i = L_pi^-T L^T w_i
      // Z2 = W Cv^T
      T* Bt2 = Bt + (size_t)k * k;
      transpose_to<T><<<(unsigned)cdiv(k * nl, 256), 256, 0, st>>>(k, nl, b.Cv, Bt2);
      GP_LAUNCH_CHECK();
      gemm_tall<T><<<gz, 256, 0, st>>>(pb.n, nl, k, W, ldw, Bt2, Z2);
      GP_LAUNCH_CHECK();
    } else {
      GP_CUDA_TRY(cudaMemsetAsync(Z2, 0, sizeof(T) * (size_t)pb.n * k, st));
    }
    const int nblk = (int)cdiv(pb.n, 256);
    switch (DM) {
      case 4: dk_contract<T, 4><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, pb.theta,
                                                      Xs, piv, rank, Z1, Z2, b.dkpart); break;
      case 8: dk_contract<T, 8><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, pb.theta,
                                                      Xs, piv, rank, Z1, Z2, b.dkpart); break;
      case 16: dk_contract<T, 16><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, pb.theta,
                                                        Xs, piv, rank, Z1, Z2, b.dkpart); break;
      default: dk_contract<T, 32><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.kind, pb.ard, pb.D, pb.theta,
                                                        Xs, piv, rank, Z1, Z2, b.dkpart); break;
    }
    GP_LAUNCH_CHECK();
    dk_combine<<<1, 128, 0, st>>>(nblk, 2 * NQ, b.dkpart, EF);
    GP_LAUNCH_CHECK();
  }
  terms_kernel<<<P, 256, 0, st>>>(k, nl, P, pb.n, pb.theta, pb.D, NQ, DM, EF, b.dW, b.B1, b.Cv,
                                  Cinv, wn, trP, probeP, 1);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

// ---- quadrature Fourier features (Tab. 2 "QFF", RBF kernel) -----------------------------
// E_w[cos(w . D)] with w ~ N(0, I_d) by the tensor-product Gauss-Hermite rule (weight
// exp(-t^2), w = sqrt(2) t, weights prod w_i / sqrt(pi)).  The mbar nodes are the
// eigenvalues of the Jacobi matrix of the Hermite recurrence (zero diagonal, off-diagonal
// sqrt(k / 2)), found by bisection on Sturm counts (the number of negative pivots of the
// LDL^T factorisation of J - x I is the number of eigenvalues below x).  The weights are
// Christoffel numbers 1 / sum_k psi_k(t)^2 of the orthonormal Hermite functions,
// psi_0 = pi^-1/4, psi_{k+1} = sqrt(2 / (k+1)) t psi_k - sqrt(k / (k+1)) psi_{k-1}.
namespace {
int sturm_below(int mbar, double x) {
  int cnt = 0;
  double q = -x;                                       // diagonal 0
  for (int i = 0; i < mbar; ++i) {
    if (i > 0) q = -x - (0.5 * i) / q;                 // off-diagonal^2 = i / 2
    if (q == 0.0) q = -1e-300;                         // on an eigenvalue: count it below
    if (q < 0.0) ++cnt;
  }
  return cnt;
}
}  // namespace

void hermite_rule(int mbar, std::vector<double>& t, std::vector<double>& w) {
  t.assign(mbar, 0.0);
  w.assign(mbar, 0.0);
  const double B = std::sqrt(2.0 * std::max(mbar - 1, 1)) + 1.0;   // Gershgorin bound
  for (int j = 0; j < mbar; ++j) {
    double lo = -B, hi = B;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo + hi)); ++it) {
      const double mid = 0.5 * (lo + hi);
      if (sturm_below(mbar, mid) > j) hi = mid;
      else lo = mid;
    }
    t[j] = 0.5 * (lo + hi);
    double p0 = std::pow(M_PI, -0.25), p1 = 0.0, s2 = p0 * p0;
    for (int k = 0; k + 1 < mbar; ++k) {
      const double p2 = std::sqrt(2.0 / (k + 1)) * t[j] * p0 - std::sqrt((double)k / (k + 1)) * p1;
      p1 = p0;
      p0 = p2;
      s2 += p0 * p0;
    }
    w[j] = 1.0 / s2;
  }
}

// The folded grid: m = mbar^d / 2 frequencies (units of 1 / l, row-major m x d) and
// weights summing to 1.  Multi-indices in row-major order (last index fastest) over the
// ascending nodes; of w and -w the one with a positive first coordinate is kept, with
// twice the weight (mbar even: no zero node).
void qff_table(int mbar, int d, std::vector<double>& U, std::vector<double>& W) {
  std::vector<double> t, w;
  hermite_rule(mbar, t, w);
  int64_t total = 1;
  for (int i = 0; i < d; ++i) total *= mbar;
  U.clear();
  W.clear();
  std::vector<int> q(d, 0);
  for (int64_t e = 0; e < total; ++e) {
    int64_t r = e;
    for (int i = d - 1; i >= 0; --i) {
      q[i] = (int)(r % mbar);
      r /= mbar;
    }
    if (!(t[q[0]] > 0.0)) continue;
    double wt = 2.0;
    for (int i = 0; i < d; ++i) {
      U.push_back(std::sqrt(2.0) * t[q[i]]);
      wt *= w[q[i]] / std::sqrt(M_PI);
    }
    W.push_back(wt);
  }
}

template <class T>
gp_status rff_build(const Prob& pb, const void* Xs_, const FeatSpec& f, double* U, double* wt,
                    T* Phi, int64_t ldp, cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const int m = f.m;
  if (f.hostU) {
    // a deterministic rule (quadrature features): frequencies and weights from the host
    GP_CUDA_TRY(cudaMemcpyAsync(U, f.hostU, sizeof(double) * (size_t)m * pb.d,
                                cudaMemcpyHostToDevice, st));
    GP_CUDA_TRY(cudaMemcpyAsync(wt, f.hostW, sizeof(double) * (size_t)m, cudaMemcpyHostToDevice,
                                st));
  } else {
    rff_freq_kernel<<<(unsigned)cdiv((int64_t)m * pb.d, 256), 256, 0, st>>>(pb.kind, m, pb.d,
                                                                             f.eps, f.g, U, wt);
    GP_LAUNCH_CHECK();
  }
  const dim3 grid((unsigned)cdiv(pb.n, 256), (unsigned)cdiv(m, kFeatChunk));
  switch (dm_of(pb.d)) {
    case 4: rff_build_kernel<T, 4><<<grid, 256, 0, st>>>(pb.n, pb.d, m, Xs, U, wt, pb.theta, pb.D,
                                                         Phi, ldp); break;
    case 8: rff_build_kernel<T, 8><<<grid, 256, 0, st>>>(pb.n, pb.d, m, Xs, U, wt, pb.theta, pb.D,
                                                         Phi, ldp); break;
    case 16: rff_build_kernel<T, 16><<<grid, 256, 0, st>>>(pb.n, pb.d, m, Xs, U, wt, pb.theta, pb.D,
                                                           Phi, ldp); break;
    default: rff_build_kernel<T, 32><<<grid, 256, 0, st>>>(pb.n, pb.d, m, Xs, U, wt, pb.theta, pb.D,
                                                           Phi, ldp); break;
  }
  GP_LAUNCH_CHECK();
  return GP_OK;
}

// The feature preconditioner's terms: trP_q = 2 sum(Z1 o dPhi_q) with Z1 = Phi C^-1 and
// probeP_q = (2 / l) sum(Z2 o dPhi_q) with Z2 = W (Phi^T W)^T, by the same identities
// as for the partial Cholesky factor (Phi^T P_hat^-1 = C^-1 Phi^T); the noise entries
// are the same as there.
template <class T>
gp_status feature_terms(const Prob& pb, const void* Xs_, const T* Phi, int64_t ldp, int m,
                        const double* U, const double* wt, const T* W, int64_t ldw, int nl,
                        const double* Cinv, const PrecBufs& b, double* trP, double* probeP,
                        cudaStream_t st) {
  const T* Xs = static_cast<const T*>(Xs_);
  const int P = pb.p, k = 2 * m;
  double* wn = b.LtW + (int64_t)k * nl;
  unsigned* ctr = reinterpret_cast<unsigned*>(wn + 1);
  double* spart = wn + 2;
  {
    int blocks = (int)std::min<int64_t>(cdiv(pb.n, 256), 128);
    GP_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned), st));
    sumsq_kernel<T><<<blocks, 256, 0, st>>>(pb.n, nl, W, ldw, spart, ctr, wn);
    GP_LAUNCH_CHECK();
  }
  const int DM = dm_of(pb.d), NQ = DM + 1;
  double* EF = b.Cv + (size_t)std::max(k, 1) * std::max(nl, 1);   // 2 NQ doubles
  T* Bt = reinterpret_cast<T*>(b.Q);                 // k x k then l x k, problem precision
  T* Z1 = reinterpret_cast<T*>(b.part);              // n x k
  T* Z2 = Z1 + (size_t)pb.n * k;                     // n x k
  // Z1 = Phi C^-1 (C^-1 is symmetric)
  transpose_to<T><<<(unsigned)cdiv(k * k, 256), 256, 0, st>>>(k, k, Cinv, Bt);
  GP_LAUNCH_CHECK();
  const dim3 gz((unsigned)cdiv(pb.n, 128), (unsigned)cdiv(k, 64));
  gemm_tall<T><<<gz, 256, 0, st>>>(pb.n, k, k, Phi, ldp, Bt, Z1);
  GP_LAUNCH_CHECK();
  if (nl > 0) {
    GP_TRY(atb<T>(pb.n, Phi, ldp, k, W, ldw, nl, b.dkpart, b.LtW, st));   // Phi^T W
    T* Bt2 = Bt + (size_t)k * k;
    transpose_to<T><<<(unsigned)cdiv(k * nl, 256), 256, 0, st>>>(k, nl, b.LtW, Bt2);
    GP_LAUNCH_CHECK();
    gemm_tall<T><<<gz, 256, 0, st>>>(pb.n, nl, k, W, ldw, Bt2, Z2);      // W (Phi^T W)^T
    GP_LAUNCH_CHECK();
  } else {
    GP_CUDA_TRY(cudaMemsetAsync(Z2, 0, sizeof(T) * (size_t)pb.n * k, st));
  }
  const int nblk = (int)cdiv(pb.n, 256);
  switch (DM) {
    case 4: rff_contract<T, 4><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.ard, pb.D, m, pb.theta, Xs, U,
                                                     wt, Z1, Z2, b.dkpart); break;
    case 8: rff_contract<T, 8><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.ard, pb.D, m, pb.theta, Xs, U,
                                                     wt, Z1, Z2, b.dkpart); break;
    case 16: rff_contract<T, 16><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.ard, pb.D, m, pb.theta, Xs,
                                                       U, wt, Z1, Z2, b.dkpart); break;
    default: rff_contract<T, 32><<<nblk, 256, 0, st>>>(pb.n, pb.d, pb.ard, pb.D, m, pb.theta, Xs,
                                                       U, wt, Z1, Z2, b.dkpart); break;
  }
  GP_LAUNCH_CHECK();
  dk_combine<<<1, 128, 0, st>>>(nblk, 2 * NQ, b.dkpart, EF);
  GP_LAUNCH_CHECK();
  terms_kernel<<<P, 256, 0, st>>>(k, nl, P, pb.n, pb.theta, pb.D, NQ, DM, EF, b.dW, b.B1, b.Cv,
                                  Cinv, wn, trP, probeP, 0);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

#define GP_FEAT_INST(T)                                                                        \
  template gp_status rff_build<T>(const Prob&, const void*, const FeatSpec&, double*, double*, \
                                  T*, int64_t, cudaStream_t);                                  \
  template gp_status feature_terms<T>(const Prob&, const void*, const T*, int64_t, int,        \
                                      const double*, const double*, const T*, int64_t, int,    \
                                      const double*, const PrecBufs&, double*, double*,        \
                                      cudaStream_t);
GP_FEAT_INST(float)
GP_FEAT_INST(double)
#undef GP_FEAT_INST

template gp_status precond_terms<float>(const Prob&, const void*, const float*, int64_t, int,
                                        const int*, const int*, const float*, int64_t, int,
                                        const double*, const PrecBufs&, double*, double*,
                                        cudaStream_t);
template gp_status precond_terms<double>(const Prob&, const void*, const double*, int64_t, int,
                                         const int*, const int*, const double*, int64_t, int,
                                         const double*, const PrecBufs&, double*, double*,
                                         cudaStream_t);

}  // namespace gp
