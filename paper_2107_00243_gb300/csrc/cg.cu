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
  return d;
}

// x = 0, r = b, ||b||^2, caps, active set.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_init(int64_t n, int t, int max_iter,
                                                   const int* __restrict__ iters_override,
                                                   Dev<T> g) {
  __shared__ double sh[32];
  const int nb = gridDim.x;
  for (int c = 0; c < t; ++c) {
    double acc = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x; a < n;
         a += (int64_t)nb * kThreads) {
      T b = g.B[a + c * g.ldb];
      g.X[a + c * n] = T(0);
      g.R[a + c * n] = b;
      acc += (double)b * (double)b;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) g.part[c * nb + blockIdx.x] = s;
  }
  if (last_block_arrived(g.counter)) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < t; c += blockDim.x) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += g.part[c * nb + b];
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

// Sp[i][c] = sum_m Cinv[i][m] S[m][c] for active columns (FP64 product, stored in T).
template <class T>
__global__ void apply_cinv(int k, int t, const double* __restrict__ Cinv, Dev<T> g) {
  if (*g.n_active == 0) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * t) return;
  int i = e / t, c = e % t;
  if (!g.active[c]) return;
  const double* crow = Cinv + (int64_t)i * k;
  double a0 = 0.0, a1 = 0.0;
  int m = 0;
  for (; m + 1 < k; m += 2) {
    a0 += crow[m] * g.S[(int64_t)m * t + c];
    a1 += crow[m + 1] * g.S[(int64_t)(m + 1) * t + c];
  }
  if (m < k) a0 += crow[m] * g.S[(int64_t)m * t + c];
  g.Sp[(int64_t)i * t + c] = (T)(a0 + a1);
}

// z = sigma^-2 (r - L Sp) and rho' = r^T z for active columns.
//   mode 0 (start): rho = rho0 = rho'
//   mode 1 (step j): beta_j = rho' / rho, rho = rho'
constexpr int kPc = 32;   // columns per pass
constexpr int kPm = 64;   // rows of Sp staged per tile
template <class T>
__global__ void __launch_bounds__(kThreads) precond_rho(int64_t n, int t, const T* __restrict__ L,
                                                       int64_t ldl, int k,
                                                       const double* __restrict__ theta, int D,
                                                       int mode, int j, int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  __shared__ T ssp[kPm][kPc];
  __shared__ double sh[32];
  const int nb = gridDim.x;
  const T inv_s2 = (T)(1.0 / theta[D + 1]);
  for (int c0 = 0; c0 < t; c0 += kPc) {
    const int tc = min(kPc, t - c0);
    double rz[kPc];
#pragma unroll
    for (int c = 0; c < kPc; ++c) rz[c] = 0.0;
    for (int64_t a0 = blockIdx.x * (int64_t)kThreads; a0 < n; a0 += (int64_t)nb * kThreads) {
      const int64_t a = a0 + threadIdx.x;
      T acc[kPc];
#pragma unroll
      for (int c = 0; c < kPc; ++c) acc[c] = T(0);
      for (int m0 = 0; m0 < k; m0 += kPm) {
        const int mn = min(kPm, k - m0);
        __syncthreads();
        for (int e = threadIdx.x; e < kPm * kPc; e += kThreads) {
          int mm = e / kPc, c = e % kPc;
          ssp[mm][c] = (mm < mn && c < tc) ? g.Sp[(int64_t)(m0 + mm) * t + c0 + c] : T(0);
        }
        __syncthreads();
        if (a < n) {
          for (int mm = 0; mm < mn; ++mm) {
            const T l = L[a + (int64_t)(m0 + mm) * ldl];
#pragma unroll
            for (int c = 0; c < kPc; ++c) acc[c] = fma(l, ssp[mm][c], acc[c]);
          }
        }
      }
      if (a < n) {
#pragma unroll
        for (int c = 0; c < kPc; ++c) {
          if (c < tc && g.active[c0 + c]) {
            const int64_t off = a + (int64_t)(c0 + c) * n;
            const T r = g.R[off];
            const T z = (r - acc[c]) * inv_s2;
            g.Z[off] = z;
            rz[c] += (double)r * (double)z;
          }
        }
      }
    }
    for (int c = 0; c < tc; ++c) {
      if (!g.active[c0 + c]) continue;
      double s = block_sum(rz[c], sh);
      if (threadIdx.x == 0) g.part[(c0 + c) * nb + blockIdx.x] = s;
    }
  }
  if (last_block_arrived(g.counter)) {
    for (int c = threadIdx.x; c < t; c += blockDim.x) {
      if (!g.active[c]) continue;
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += g.part[c * nb + b];
      if (mode == 0) {
        g.rho[c] = s;
        g.rho0[c] = s;
      } else {
        double be = s / g.rho[c];
        if (!isfinite(be)) { *g.status = GP_ERR_NUMERIC; be = 0.0; }
        g.beta[(int64_t)c * max_iter + j] = be;
        g.rho[c] = s;
      }
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
  __shared__ double sh[32];
  const int nb = gridDim.x;
  for (int c = 0; c < t; ++c) {
    if (!g.active[c]) continue;
    double acc = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x; a < n;
         a += (int64_t)nb * kThreads)
      acc += (double)g.P[a + c * n] * (double)g.Q[a + c * n];
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) g.part[c * nb + blockIdx.x] = s;
  }
  if (last_block_arrived(g.counter)) {
    for (int c = threadIdx.x; c < t; c += blockDim.x) {
      if (!g.active[c]) continue;
      double pq = 0.0;
      for (int b = 0; b < nb; ++b) pq += g.part[c * nb + b];
      double al = g.rho[c] / pq;
      if (!(pq > 0.0) || !isfinite(al)) {
        *g.status = GP_ERR_NUMERIC;
        al = 0.0;
      }
      g.alpha[(int64_t)c * max_iter + j] = al;
    }
  }
}

__device__ void decide(int t, int j, const double* rnorm2_part, int nb, double tol2,
                       int use_caps, int max_iter, int* active, const int* caps, int* iters,
                       const double* bnorm2, int* n_active) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < t; c += blockDim.x) {
    if (!active[c]) continue;
    bool stop;
    if (use_caps) {
      stop = (j + 1) >= caps[c];
    } else {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += rnorm2_part[c * nb + b];
      stop = (s <= tol2 * bnorm2[c]) || (j + 1 >= max_iter);
    }
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
  __shared__ double sh[32];
  const int nb = gridDim.x;
  for (int c = 0; c < t; ++c) {
    if (!g.active[c]) continue;
    const T al = (T)g.alpha[(int64_t)c * max_iter + j];
    double acc = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x; a < n;
         a += (int64_t)nb * kThreads) {
      const int64_t off = a + c * n;
      g.X[off] = fma(al, g.P[off], g.X[off]);
      T r = fma(-al, g.Q[off], g.R[off]);
      g.R[off] = r;
      acc += (double)r * (double)r;
    }
    if (!recompute) {
      double s = block_sum(acc, sh);
      if (threadIdx.x == 0) g.part[c * nb + blockIdx.x] = s;
    }
  }
  if (recompute) return;
  if (last_block_arrived(g.counter))
    decide(t, j, g.part, nb, tol2, use_caps, max_iter, g.active, g.caps, g.iters, g.bnorm2,
           g.n_active);
}

// r = b - K_hat x (Q holds K_hat x), ||r||^2, stopping decision.
template <class T>
__global__ void __launch_bounds__(kThreads) cg_resid(int64_t n, int t, int j, int max_iter,
                                                    double tol2, int use_caps, Dev<T> g) {
  if (*g.n_active == 0) return;
  __shared__ double sh[32];
  const int nb = gridDim.x;
  for (int c = 0; c < t; ++c) {
    if (!g.active[c]) continue;
    double acc = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x; a < n;
         a += (int64_t)nb * kThreads) {
      const int64_t off = a + c * n;
      T r = g.B[a + c * g.ldb] - g.Q[off];
      g.R[off] = r;
      acc += (double)r * (double)r;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) g.part[c * nb + blockIdx.x] = s;
  }
  if (last_block_arrived(g.counter))
    decide(t, j, g.part, nb, tol2, use_caps, max_iter, g.active, g.caps, g.iters, g.bnorm2,
           g.n_active);
}

// p = z + beta_j p for active columns.
template <class T>
__global__ void cg_pupdate(int64_t n, int t, int j, int max_iter, Dev<T> g) {
  if (*g.n_active == 0) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * t) return;
  int c = (int)(e / n);
  if (!g.active[c]) return;
  const T be = (T)g.beta[(int64_t)c * max_iter + j];
  g.P[e] = fma(be, g.P[e], g.Z[e]);
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

template <class T>
gp_status precond_apply(int64_t n, int t, const T* L, int64_t ldl, int k, const double* Cinv,
                        const double* theta, int D, int mode, int j, int max_iter,
                        const CgBufs<T>& cb, Dev<T>& g, int nb, cudaStream_t st) {
  if (k > 0) {
    GP_TRY(atb<T>(n, L, ldl, k, g.R, n, t, cb.atb_part, cb.S, st));
    apply_cinv<T><<<(unsigned)cdiv((int64_t)k * t, 256), 256, 0, st>>>(k, t, Cinv, g);
    GP_LAUNCH_CHECK();
  }
  precond_rho<T><<<nb, kThreads, 0, st>>>(n, t, L, ldl, k, theta, D, mode, j, max_iter, g);
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
