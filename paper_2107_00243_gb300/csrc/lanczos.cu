// Lanczos quadrature of log from CG coefficients (Alg. 1; Sec. S1.2).
//
// For probe column c with m CG steps, the tridiagonal T (Lanczos matrix) has
//   T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j][j+1]^2 = beta_j / alpha_j^2,
// and the Gauss-quadrature estimate is gamma_c = rho0_c * sum_j (e_1^T w_j)^2 log(lambda_j)
// over the eigenpairs (lambda_j, w_j) of T, i.e. gamma_c = rho0_c * e_1^T log(T) e_1.
//
// The same number is computed here without an eigendecomposition (whose sequential
// QR sweeps are a long chain of FP64 square roots and divisions, slow on this part):
//   log x = int_0^inf [1/(1+s) - 1/(x+s)] ds   for x > 0,
// so for symmetric positive definite T
//   e_1^T log(T) e_1 = int_0^inf [1/(1+s) - e_1^T (T + sI)^-1 e_1] ds,
// and e_1^T (T + sI)^-1 e_1 = 1/d_1 from the backward continued fraction
//   d_m = T_mm + s,  d_j = T_jj + s - T_{j,j+1}^2 / d_{j+1}
// (the pivots of the LDL^T factorisation of the row-reversed matrix; all positive for
// SPD T, and only squared off-diagonals enter, so no square roots).  With s = e^u the
// integrand is analytic in the strip |Im u| < pi and decays like e^u (u -> -inf) and
// like (lambda_max - 1) e^-u (u -> +inf), so the trapezoidal rule with step h = 0.5 on
// [-38, log(G) + 38] (G a Gershgorin bound on lambda_max) is exact to ~1e-16 relative
// (discretisation error ~ exp(-2 pi d / h), d -> pi; tails < e^-38).  Every node is an
// independent O(m) recurrence: one thread per node, one block per probe column.
// Checked against a dense eigendecomposition, including clustered (Lanczos "ghost")
// spectra, to 1e-13 relative.
#include "ops.h"

namespace gp {
namespace {

constexpr int kQuadThreads = 256;
constexpr double kQuadStep = 0.5;
constexpr double kQuadTail = 38.0;

__global__ void __launch_bounds__(kQuadThreads) logquad_kernel(
    int c0, int max_iter, const double* __restrict__ alpha, const double* __restrict__ beta,
    const int* __restrict__ iters, const double* __restrict__ rho0, double* __restrict__ gamma,
    int* status) {
  extern __shared__ double sm[];
  __shared__ double red[kQuadThreads / 32];
  __shared__ int bad;
  const int c = c0 + blockIdx.x;
  const int m = iters[c];
  double* a = sm;              // diagonal of T
  double* b2 = sm + max_iter;  // squared off-diagonal of T
  const double* al = alpha + (int64_t)c * max_iter;
  const double* be = beta + (int64_t)c * max_iter;
  if (m == 0) {
    if (threadIdx.x == 0) gamma[blockIdx.x] = 0.0;
    return;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // T and a Gershgorin bound on its largest eigenvalue
  double g = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double aj = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    const double bj2 = (j < m - 1) ? be[j] / (al[j] * al[j]) : 0.0;
    a[j] = aj;
    b2[j] = bj2;
    if (!(al[j] > 0.0) || !isfinite(aj) || !isfinite(bj2)) bad = 1;
    const double lo = (j > 0) ? sqrt(be[j - 1]) / al[j - 1] : 0.0;
    const double hi = (j < m - 1) ? sqrt(be[j]) / al[j] : 0.0;
    g = fmax(g, aj + fabs(lo) + fabs(hi));
  }
  for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = g;
  __syncthreads();
  g = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g = fmax(g, red[w]);
  __syncthreads();
  const double umin = -kQuadTail;
  const double umax = log(fmax(g, 1.0)) + kQuadTail;
  const int nodes = (int)ceil((umax - umin) / kQuadStep) + 1;
  // trapezoidal rule over the nodes; the integrand in s / (1 + s) - s / d_1 form
  double acc = 0.0;
  for (int k = threadIdx.x; k < nodes; k += blockDim.x) {
    const double s = exp(umin + k * kQuadStep);
    double d = a[m - 1] + s;
    bool ok = d > 0.0;
    for (int j = m - 2; j >= 0; --j) {
      d = a[j] + s - b2[j] / d;
      ok = ok && (d > 0.0);
    }
    if (!ok || !isfinite(d)) bad = 1;
    acc += s / (1.0 + s) - s / d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    gamma[blockIdx.x] = rho0[c] * kQuadStep * sum;
    if (bad) raise_status(status, GP_ERR_NOT_SPD);
  }
}

}  // namespace

gp_status lanczos_logquad(int count, int c0, int max_iter, const double* alpha,
                          const double* beta, const int* iters, const double* rho0,
                          double* gamma, int* status, cudaStream_t st) {
  if (count == 0) return GP_OK;
  const size_t sm = sizeof(double) * 2 * (size_t)max_iter;
  if (sm > 48 * 1024)
    GP_CUDA_TRY(cudaFuncSetAttribute(logquad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
  logquad_kernel<<<count, kQuadThreads, sm, st>>>(c0, max_iter, alpha, beta, iters, rho0, gamma,
                                                  status);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace gp
