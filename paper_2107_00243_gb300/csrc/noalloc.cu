// gp_kernel_mvm_noalloc: the kernel-matrix product W = (K + sigma^2 I) V for callers
// that cannot allocate device memory.  Its scratch lives in one file-scope device
// array (below) that every GPU loading the library holds until the process exits.
// This entry point has no counterpart in the paper; it repackages gp_kernel_mvm.
#include <mutex>

#include "ops.h"

namespace gp {
namespace {

// Scratch: scaled inputs Xs (n * d reals) followed by the centring sums.
constexpr size_t kNoAllocXsBytes = size_t(16) << 20;            // 16 MiB of Xs
constexpr size_t kNoAllocTailBytes = size_t(80) << 10;          // mean, partials, counter
constexpr size_t kNoAllocBytes = kNoAllocXsBytes + kNoAllocTailBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host code the
// array's name is only a host-side stand-in, so the address must be looked up once
// per device with that device current.
gp_status scratch_for_current_device(void** out) {
  int dev = 0;
  GP_CUDA_TRY(cudaGetDevice(&dev));
  GP_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    GP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return GP_OK;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" gp_status gp_kernel_mvm_noalloc(const gp_problem* prob, const void* V, int64_t ldv,
                                           int32_t t, void* W, int64_t ldw,
                                           gp_stream_t stream) {
  GP_REQUIRE(prob != nullptr, "problem is NULL");
  GP_REQUIRE(prob->n >= 1 && prob->n < (int64_t(1) << 31), "n out of range");
  GP_REQUIRE(prob->d >= 1 && prob->d <= kMaxD, "d=%d out of range [1, %d]", prob->d, kMaxD);
  GP_REQUIRE(prob->kind == GP_RBF || prob->kind == GP_MATERN32 || prob->kind == GP_MATERN52 ||
                 prob->kind == GP_RATQUAD,
             "unknown kernel kind %d", prob->kind);
  GP_REQUIRE(prob->precision == GP_FP64 || prob->precision == GP_FP32,
             "gp_kernel_mvm_noalloc supports GP_FP64 and GP_FP32 only");
  GP_REQUIRE(prob->X && prob->theta && V && W, "NULL pointer");
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(ldv >= prob->n && ldw >= prob->n, "leading dimensions must be >= n");
  GP_REQUIRE(V != W, "W must not alias V");
  const size_t elem = prob->precision == GP_FP64 ? sizeof(double) : sizeof(float);
  const size_t need = (size_t)prob->n * prob->d * elem;
  GP_REQUIRE(need <= kNoAllocXsBytes,
             "n * d * %zu = %zu bytes exceeds the %zu-byte scratch of gp_kernel_mvm_noalloc",
             elem, need, kNoAllocXsBytes);
  void* base = nullptr;
  GP_TRY(scratch_for_current_device(&base));

  Prob pb;
  pb.n = prob->n;
  pb.d = prob->d;
  pb.kind = prob->kind;
  pb.ard = prob->ard ? 1 : 0;
  pb.D = pb.ard ? pb.d : 1;
  pb.p = pb.D + 2;
  pb.prec = prob->precision;
  pb.X = prob->X;
  pb.theta = prob->theta;

  char* b = static_cast<char*>(base);
  PrepBufs pr;
  pr.Xs = b;
  pr.mean = reinterpret_cast<double*>(b + kNoAllocXsBytes);
  pr.part = pr.mean + kMaxD;                                   // kPrepBlocks * kMaxD doubles
  pr.counter = reinterpret_cast<unsigned*>(pr.part + (size_t)kPrepBlocks * kMaxD);
  static_assert((kMaxD + (size_t)kPrepBlocks * kMaxD) * sizeof(double) + 16 <= kNoAllocTailBytes,
                "scratch tail too small");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the centring kernel's arrival counter must start at zero on every call
  GP_CUDA_TRY(cudaMemsetAsync(pr.counter, 0, 4 * sizeof(unsigned), st));
  if (pb.prec == GP_FP64) {
    GP_TRY(prep_inputs<double>(pb, pr, st));
    return kmvm_simt_unsplit<double>(pb, pr.Xs, V, ldv, t, W, ldw, st);
  }
  GP_TRY(prep_inputs<float>(pb, pr, st));
  return kmvm_simt_unsplit<float>(pb, pr.Xs, V, ldv, t, W, ldw, st);
}
