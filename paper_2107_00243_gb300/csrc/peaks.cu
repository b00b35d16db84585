// Throughput microbenchmarks of the arithmetic units on the estimator's path, for the
// roofline denominators that the HBM-copy and BF16-GEMM measurements do not give:
//   FP32 FMA (the FP32 kernel product and the CG vector kernels),
//   ex2.approx.f32 on the MUFU pipe (one per kernel entry in the tensor-core product),
//   ex2.approx.f16x2 (two results per instruction),
//   FP64 FMA (the Woodbury core, Lanczos and the reductions).
// Each kernel keeps eight independent dependency chains per thread and runs 8 CTAs of 256
// threads per SM, so the unit, not latency, is the limit.  Every thread writes one value
// (its chains' sum) to scratch[global thread index], so nothing is optimised away and
// every store is in bounds.
#include "ops.h"

#include <cuda_fp16.h>

namespace gp {
namespace {

constexpr int kPkThreads = 256;
constexpr int kPkCtasPerSm = 8;
constexpr int kPkChains = 8;

__global__ void __launch_bounds__(kPkThreads) pk_ffma(int iters, float* out) {
  float a[kPkChains];
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) a[q] = 1e-3f * (float)(threadIdx.x & 15) + (float)q;
  const float m = 0.9999999f, c = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int q = 0; q < kPkChains; ++q) a[q] = fmaf(a[q], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPkThreads) pk_dfma(int iters, float* out) {
  double a[kPkChains];
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) a[q] = 1e-3 * (double)(threadIdx.x & 15) + (double)q;
  const double m = 0.9999999, c = 1e-7;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int q = 0; q < kPkChains; ++q) a[q] = fma(a[q], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = (float)s;
}

// x <- 2^-x stays in (1/2, 1) for x in (0, 1]
__global__ void __launch_bounds__(kPkThreads) pk_ex2(int iters, float* out) {
  float a[kPkChains];
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) a[q] = 0.5f + 0.01f * (float)q + 1e-3f * (float)(threadIdx.x & 15);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int q = 0; q < kPkChains; ++q)
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[q]) : "f"(-a[q]));
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

// the same map on two FP16 lanes per instruction (sign flip by xor of the sign bits)
__global__ void __launch_bounds__(kPkThreads) pk_ex2h2(int iters, float* out) {
  uint32_t a[kPkChains];
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) {
    const __half2 h = __floats2half2_rn(0.5f + 0.01f * (float)q, 0.75f - 0.01f * (float)q);
    a[q] = *reinterpret_cast<const uint32_t*>(&h);
  }
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int q = 0; q < kPkChains; ++q)
        asm volatile("ex2.approx.f16x2 %0, %1;" : "=r"(a[q]) : "r"(a[q] ^ 0x80008000u));
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPkChains; ++q) {
    const __half2 h = *reinterpret_cast<const __half2*>(&a[q]);
    s += __low2float(h) + __high2float(h);
  }
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

int pk_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// best of three timed launches (after one warm-up) in seconds
template <class K>
gp_status pk_time(K kernel, int grid, int iters, float* scratch, cudaStream_t st, double* best) {
  cudaEvent_t e0, e1;
  GP_CUDA_TRY(cudaEventCreate(&e0));
  GP_CUDA_TRY(cudaEventCreate(&e1));
  *best = 1e30;
  for (int r = 0; r < 4; ++r) {
    GP_CUDA_TRY(cudaEventRecord(e0, st));
    kernel<<<grid, kPkThreads, 0, st>>>(iters, scratch);
    GP_LAUNCH_CHECK();
    GP_CUDA_TRY(cudaEventRecord(e1, st));
    GP_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    GP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (r > 0 && ms * 1e-3 < *best) *best = ms * 1e-3;
  }
  GP_CUDA_TRY(cudaEventDestroy(e0));
  GP_CUDA_TRY(cudaEventDestroy(e1));
  return GP_OK;
}

}  // namespace
}  // namespace gp

extern "C" size_t gp_peaks_scratch_elems(void) {
  const int sms = gp::pk_sms();
  return (size_t)(sms > 0 ? sms : 1) * gp::kPkCtasPerSm * gp::kPkThreads;
}

extern "C" gp_status gp_measure_peaks(float* scratch, double* out, gp_stream_t stream) {
  using namespace gp;
  GP_REQUIRE(scratch && out, "scratch or out is NULL");
  const int sms = pk_sms();
  GP_REQUIRE(sms > 0, "no CUDA device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int grid = sms * kPkCtasPerSm;
  const double threads = (double)grid * kPkThreads;
  const double per_iter = 16.0 * kPkChains * threads;   // operations per loop iteration
  double t;
  const int it_ffma = 8192, it_ex2 = 4096, it_dfma = 256;
  GP_TRY(pk_time(pk_ffma, grid, it_ffma, scratch, st, &t));
  out[0] = 2.0 * per_iter * it_ffma / t;
  GP_TRY(pk_time(pk_ex2, grid, it_ex2, scratch, st, &t));
  out[1] = per_iter * it_ex2 / t;
  GP_TRY(pk_time(pk_ex2h2, grid, it_ex2, scratch, st, &t));
  out[2] = 2.0 * per_iter * it_ex2 / t;
  GP_TRY(pk_time(pk_dfma, grid, it_dfma, scratch, st, &t));
  out[3] = 2.0 * per_iter * it_dfma / t;
  return GP_OK;
}
