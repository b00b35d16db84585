// Lanczos quadrature of log from CG coefficients (Alg. 1 steps 6-8; Sec. S1.2).
//
// For probe column c with m CG steps, the tridiagonal
//   T[j][j] = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T[j][j+1] = sqrt(beta_j)/alpha_j
// has eigenpairs (lambda_j, w_j); the Gauss-quadrature estimate is
//   gamma_c = rho0_c * sum_j (e_1^T w_j)^2 log(lambda_j).
// Eigenvalues come from implicit symmetric QR steps with a Wilkinson shift
// (Golub & Van Loan, "Matrix Computations", Sec. 8.3), chasing the bulge with
// Givens rotations; only the first row of the accumulated rotation matrix is
// kept, which is all the weights need (O(m^2) work per column, FP64).
#include "ops.h"

namespace gp {
namespace {

__global__ void logquad_kernel(int c0, int max_iter, const double* __restrict__ alpha,
                               const double* __restrict__ beta, const int* __restrict__ iters,
                               const double* __restrict__ rho0, double* __restrict__ gamma,
                               int* status) {
  extern __shared__ double sm[];
  if (threadIdx.x != 0) return;
  const int c = c0 + blockIdx.x;
  const int m = iters[c];
  double* a = sm;
  double* b = sm + max_iter;
  double* q = sm + 2 * max_iter;
  const double* al = alpha + (int64_t)c * max_iter;
  const double* be = beta + (int64_t)c * max_iter;
  if (m == 0) {
    gamma[blockIdx.x] = 0.0;
    return;
  }
  for (int j = 0; j < m; ++j) {
    a[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    b[j] = (j < m - 1) ? sqrt(be[j]) / al[j] : 0.0;
    q[j] = (j == 0) ? 1.0 : 0.0;
  }
  const double eps = 4.0 * 2.220446049250313e-16;
  int hi = m - 1;
  long sweeps = 0;
  const long cap = 60L * m + 100;
  bool timeout = false;
  while (hi > 0) {
    if (fabs(b[hi - 1]) <= eps * (fabs(a[hi - 1]) + fabs(a[hi]))) {
      b[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(b[lo - 1]) > eps * (fabs(a[lo - 1]) + fabs(a[lo]))) --lo;
    if (lo > 0) b[lo - 1] = 0.0;
    if (++sweeps > cap) {
      timeout = true;
      break;
    }
    // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to a[hi]
    const double dd = 0.5 * (a[hi - 1] - a[hi]);
    const double bb = b[hi - 1];
    const double mu = a[hi] - bb * bb / (dd + copysign(hypot(dd, bb), dd));
    double x = a[lo] - mu, z = b[lo];
    for (int kk = lo; kk < hi; ++kk) {
      // entries here stay far from the overflow range, so r = sqrt(x^2 + z^2) directly
      const double r2 = x * x + z * z;
      double r = 0.0, cs = 1.0, sn = 0.0;
      if (r2 > 0.0) {
        r = sqrt(r2);
        const double ir = 1.0 / r;
        cs = x * ir;
        sn = z * ir;
      }
      if (kk > lo) b[kk - 1] = r;
      const double akk = a[kk], ak1 = a[kk + 1], bk = b[kk];
      a[kk] = cs * cs * akk + 2.0 * cs * sn * bk + sn * sn * ak1;
      a[kk + 1] = sn * sn * akk - 2.0 * cs * sn * bk + cs * cs * ak1;
      b[kk] = cs * sn * (ak1 - akk) + (cs * cs - sn * sn) * bk;
      if (kk + 1 < hi) {
        x = b[kk];
        z = sn * b[kk + 1];
        b[kk + 1] = cs * b[kk + 1];
      }
      const double q0 = q[kk], q1 = q[kk + 1];
      q[kk] = cs * q0 + sn * q1;
      q[kk + 1] = -sn * q0 + cs * q1;
    }
  }
  double acc = 0.0;
  bool bad = false;
  for (int j = 0; j < m; ++j) {
    if (!(a[j] > 0.0)) bad = true;
    acc += q[j] * q[j] * log(a[j]);
  }
  gamma[blockIdx.x] = rho0[c] * acc;
  if (timeout) atomicExch(status, GP_ERR_DEVICE_TIMEOUT);
  else if (bad) atomicExch(status, GP_ERR_NOT_SPD);
}

}  // namespace

gp_status lanczos_logquad(int count, int c0, int max_iter, const double* alpha,
                          const double* beta, const int* iters, const double* rho0,
                          double* gamma, int* status, cudaStream_t st) {
  if (count == 0) return GP_OK;
  size_t sm = sizeof(double) * 3 * (size_t)max_iter;
  if (sm > 48 * 1024)
    GP_CUDA_TRY(cudaFuncSetAttribute(logquad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
  logquad_kernel<<<count, 32, sm, st>>>(c0, max_iter, alpha, beta, iters, rho0, gamma, status);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

}  // namespace gp
