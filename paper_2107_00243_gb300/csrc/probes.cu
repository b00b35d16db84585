// Right-hand sides of the CG call: B = [y, z_1 .. z_l] with probes of covariance
// P_hat,  z_i = L eps1_i + sigma eps2_i  (eps +-1 Rademacher, Sec. 2.2 "Stochastic
// Trace Estimation").  Signs come from the counter-based SplitMix64 hash in
// common.cuh, or from a caller-supplied int8 array.
#include "ops.h"

namespace gp {
namespace {

constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) rhs_kernel(
    int64_t n, const T* __restrict__ y, const T* __restrict__ L, int64_t ldl, int k,
    const double* __restrict__ theta, int D, uint64_t seed, const int8_t* __restrict__ eps,
    T* __restrict__ B, int64_t ldb) {
  extern __shared__ unsigned char raw[];
  T* e1 = reinterpret_cast<T*>(raw);
  const int i = blockIdx.y;              // probe index
  const int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const uint64_t key1 = probe_key(seed, 1), key2 = probe_key(seed, 2);
  const int64_t lde = (int64_t)k + n;
  for (int m = threadIdx.x; m < k; m += kThreads)
    e1[m] = eps ? (T)eps[m + i * lde] : (T)probe_sign(key1, (uint64_t)m, (uint64_t)i);
  __syncthreads();
  if (a >= n) return;
  if (i == 0) B[a] = y[a];
  T acc = T(0);
  for (int m = 0; m < k; ++m) acc = fma(L[a + (int64_t)m * ldl], e1[m], acc);
  const T e2 = eps ? (T)eps[k + a + i * lde] : (T)probe_sign(key2, (uint64_t)a, (uint64_t)i);
  const T sigma = (T)sqrt(theta[D + 1]);
  B[a + (int64_t)(i + 1) * ldb] = fma(sigma, e2, acc);
}

__global__ void sign_kernel(uint64_t key, int64_t rows, int cols, int8_t* out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  int64_t r = e % rows;
  int c = (int)(e / rows);
  out[e] = (int8_t)probe_sign(key, (uint64_t)r, (uint64_t)c);
}

}  // namespace

template <class T>
gp_status make_rhs(const Prob& pb, const T* y, const T* L, int64_t ldl, int k, int n_probes,
                   uint64_t seed, const int8_t* eps_override, T* B, int64_t ldb,
                   cudaStream_t st) {
  dim3 grid((unsigned)cdiv(pb.n, kThreads), (unsigned)std::max(n_probes, 1));
  size_t sm = sizeof(T) * (size_t)std::max(k, 1);
  if (n_probes == 0) {
    GP_CUDA_TRY(cudaMemcpyAsync(B, y, sizeof(T) * pb.n, cudaMemcpyDeviceToDevice, st));
    return GP_OK;
  }
  if (sm > 48 * 1024)
    GP_CUDA_TRY(cudaFuncSetAttribute(rhs_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
  rhs_kernel<T><<<grid, kThreads, sm, st>>>(pb.n, y, L, ldl, k, pb.theta, pb.D, seed,
                                            eps_override, B, ldb);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

gp_status rademacher_fill(uint64_t seed, int stream_id, int64_t rows, int cols, int8_t* out,
                          cudaStream_t st) {
  int64_t total = rows * cols;
  if (total == 0) return GP_OK;
  sign_kernel<<<(unsigned)cdiv(total, 256), 256, 0, st>>>(probe_key(seed, (uint64_t)stream_id),
                                                          rows, cols, out);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

template gp_status make_rhs<float>(const Prob&, const float*, const float*, int64_t, int, int,
                                   uint64_t, const int8_t*, float*, int64_t, cudaStream_t);
template gp_status make_rhs<double>(const Prob&, const double*, const double*, int64_t, int, int,
                                    uint64_t, const int8_t*, double*, int64_t, cudaStream_t);

}  // namespace gp
