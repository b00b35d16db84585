// Shared device/host helpers of the GP estimator library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <cmath>

#include "../../include/gp.h"

namespace gp {

constexpr int kMaxD = 32;      // input dimension limit (kept in registers)
constexpr int kMaxK = 2048;    // preconditioner rank limit
constexpr int kMaxT = 1024;    // right-hand-side column limit

// ---------------------------------------------------------------------------
// Host-side error reporting
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
const char* last_error();

#define GP_CUDA_TRY(expr)                                                       \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::gp::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr,                \
                      cudaGetErrorString(e_));                                  \
      return GP_ERR_CUDA;                                                       \
    }                                                                           \
  } while (0)

void count_launch();
#define GP_LAUNCH_CHECK()          \
  do {                             \
    ::gp::count_launch();          \
    GP_CUDA_TRY(cudaGetLastError()); \
  } while (0)

#define GP_REQUIRE(cond, ...)                                                   \
  do {                                                                          \
    if (!(cond)) {                                                              \
      ::gp::set_error(__VA_ARGS__);                                             \
      return GP_ERR_INVALID_ARG;                                                \
    }                                                                           \
  } while (0)

#define GP_TRY(expr)                                                            \
  do {                                                                          \
    gp_status s_ = (expr);                                                      \
    if (s_ < 0) return s_;                                                      \
  } while (0)

// ---------------------------------------------------------------------------
// Workspace carving: the same plan runs once without a base (size query) and
// once with the caller's buffer.
// ---------------------------------------------------------------------------
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class U>
  U* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
    off += count * sizeof(U);
    return p;
  }
};

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Problem description shared by kernels.
// ---------------------------------------------------------------------------
struct Prob {
  int64_t n;
  int d, kind, ard, D, p, prec;
  const void* X;
  const double* theta;
};

// Device-side scalars derived from theta: 1/l_j per dimension, s, sigma^2.
struct Hyper {
  double inv_l[kMaxD];
  double l[kMaxD];
  double s, s2;
};

// ---------------------------------------------------------------------------
// Kernel functions of the scaled squared distance r^2 (Sec. 5 kernels).
//   kval:  k(r^2)
//   kfac:  -2 dk/dr^2, the factor shared by every lengthscale derivative
// ---------------------------------------------------------------------------
template <class T> struct M;
template <> struct M<float> {
  static __device__ __forceinline__ float ex(float x) { return expf(x); }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
};
template <> struct M<double> {
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
};

template <class T>
__device__ __forceinline__ T kval(int kind, T r2, T s) {
  r2 = r2 > T(0) ? r2 : T(0);
  if (kind == GP_RBF) return s * M<T>::ex(T(-0.5) * r2);
  if (kind == GP_RATQUAD) return s / (T(1) + T(0.5) * r2);
  T r = M<T>::sq(r2);
  if (kind == GP_MATERN32) {
    T ar = T(1.7320508075688772) * r;
    return s * (T(1) + ar) * M<T>::ex(-ar);
  }
  T ar = T(2.23606797749979) * r;
  return s * (T(1) + ar + T(5.0 / 3.0) * r2) * M<T>::ex(-ar);
}

// k and -2 dk/dr^2 together.
template <class T>
__device__ __forceinline__ void kval_fac(int kind, T r2, T s, T& k, T& fac) {
  r2 = r2 > T(0) ? r2 : T(0);
  if (kind == GP_RBF) {
    k = s * M<T>::ex(T(-0.5) * r2);
    fac = k;
    return;
  }
  if (kind == GP_RATQUAD) {
    const T q = T(1) / (T(1) + T(0.5) * r2);
    k = s * q;
    fac = k * q;
    return;
  }
  T r = M<T>::sq(r2);
  if (kind == GP_MATERN32) {
    T ar = T(1.7320508075688772) * r;
    T e = s * M<T>::ex(-ar);
    k = (T(1) + ar) * e;
    fac = T(3) * e;
    return;
  }
  T ar = T(2.23606797749979) * r;
  T e = s * M<T>::ex(-ar);
  k = (T(1) + ar + T(5.0 / 3.0) * r2) * e;
  fac = T(5.0 / 3.0) * (T(1) + ar) * e;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output from state x is the finaliser
// applied to x + golden-ratio increment.  Probe sign of (row, col) in a stream:
//   h = mix(mix(mix(seed) ^ stream) ^ ((col << 32) | row)), sign = top bit ? -1 : +1
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t probe_key(uint64_t seed, uint64_t stream) {
  return splitmix_out(splitmix_out(seed) ^ stream);
}
__device__ __forceinline__ int probe_sign(uint64_t key, uint64_t row, uint64_t col) {
  uint64_t h = splitmix_out(key ^ ((col << 32) | row));
  return (h >> 63) ? -1 : 1;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <class U>
__device__ __forceinline__ U warp_sum(U v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one value per thread; result valid in thread 0.  `sh` needs
// blockDim.x / 32 entries.
template <class U>
__device__ __forceinline__ U block_sum(U v, U* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  U r = U(0);
  if (w == 0) {
    int nw = blockDim.x >> 5;
    r = lane < nw ? sh[lane] : U(0);
    r = warp_sum(r);
  }
  return r;
}

// "Last block" protocol: every block writes its partial results, then calls
// this; exactly one block (the last to arrive) gets true and may reduce the
// partials.  The counter is reset by that block for the next launch.
__device__ __forceinline__ bool last_block_arrived(unsigned int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x * gridDim.y * gridDim.z - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Device status word: 0 = fine, > 0 a warning, < 0 an error.  An error replaces 0 or a
// warning, and the first error stays (a later failure is usually a consequence of it);
// a warning replaces only 0.
__device__ __forceinline__ void raise_status(int* status, int code) {
  int old = *reinterpret_cast<volatile int*>(status);
  while (old >= 0 && (code < 0 || old == 0) && old != code) {
    const int prev = atomicCAS(status, old, code);
    if (prev == old) break;
    old = prev;
  }
}

__device__ __forceinline__ void load_hyper(const double* theta, int d, int ard, Hyper& h) {
  int D = ard ? d : 1;
  for (int j = 0; j < d; ++j) {
    double l = theta[ard ? j : 0];
    h.l[j] = l;
    h.inv_l[j] = 1.0 / l;
  }
  h.s = theta[D];
  h.s2 = theta[D + 1];
}

}  // namespace gp
