// C ABI entry points (include/gp.h): argument validation, workspace planning and
// the order of the estimator's steps (Alg. 1 and Alg. 2 fused into one CG call).
#include <cstdarg>
#include <algorithm>
#include <cstring>
#include <vector>

#include "ops.h"

namespace gp {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

namespace {

size_t elem_size(int prec) { return prec == GP_FP64 ? sizeof(double) : sizeof(float); }

gp_status check_problem(const gp_problem* prob, bool need_data = true) {
  GP_REQUIRE(prob != nullptr, "problem is NULL");
  GP_REQUIRE(prob->n >= 1 && prob->n < (int64_t(1) << 31), "n=%lld out of range [1, 2^31)",
             (long long)prob->n);
  GP_REQUIRE(prob->d >= 1 && prob->d <= kMaxD, "d=%d out of range [1, %d]", prob->d, kMaxD);
  GP_REQUIRE(prob->kind == GP_RBF || prob->kind == GP_MATERN32 || prob->kind == GP_MATERN52 ||
                 prob->kind == GP_RATQUAD,
             "unknown kernel kind %d", prob->kind);
  GP_REQUIRE(prob->precision >= GP_FP64 && prob->precision <= GP_BF16, "unknown precision %d",
             prob->precision);
  if (need_data) {
    GP_REQUIRE(prob->X != nullptr, "X is NULL");
    GP_REQUIRE(prob->theta != nullptr, "theta is NULL");
  }
  return GP_OK;
}

Prob make_prob(const gp_problem* p) {
  Prob pb;
  pb.n = p->n;
  pb.d = p->d;
  pb.kind = p->kind;
  pb.ard = p->ard ? 1 : 0;
  pb.D = pb.ard ? pb.d : 1;
  pb.p = pb.D + 2;
  pb.prec = p->precision;
  pb.X = p->X;
  pb.theta = p->theta;
  return pb;
}

// ---- workspace plans ---------------------------------------------------------------
struct PrepPlan {
  PrepBufs pr;
};
void plan_prep(Arena& A, const Prob& pb, PrepPlan& P) {
  P.pr.Xs = A.take<char>(elem_size(pb.prec) * (size_t)pb.n * pb.d);
  P.pr.mean = A.take<double>(kMaxD);
  P.pr.part = A.take<double>((size_t)kPrepBlocks * kMaxD);
  P.pr.counter = A.take<unsigned>(4);
}

struct MvmPlan {
  PrepPlan prep;
  void* scratch;     // SIMT split partials
  TcBufs tc;
  bool use_tc;
};
void plan_mvm(Arena& A, const Prob& pb, int t, MvmPlan& P) {
  plan_prep(A, pb, P.prep);
  P.use_tc = (pb.prec == GP_BF16 || pb.prec == GP_TF32);
  P.scratch = nullptr;
  P.tc = TcBufs{};
  if (P.use_tc) {
    P.tc.xpack = A.take<char>(tc_xpack_bytes(pb.n, pb.d, pb.prec));
    P.tc.norms = A.take<float>((size_t)pb.n);
    P.tc.vpack = A.take<char>(tc_vpack_bytes(pb.n, t, pb.prec));
    P.tc.vscale = A.take<float>(kTcVscaleElems);
    P.tc.part = A.take<float>(tc_part_elems(pb.n, t));
    P.tc.err = A.take<int>(kTcErrInts);
  } else {
    P.scratch = A.take<char>(elem_size(pb.prec) * simt_scratch_elems(pb.n, t));
  }
}

struct PivPlan {
  PivBufs b;
};
void plan_piv(Arena& A, const Prob& pb, int k, PivPlan& P) {
  P.b.dres = A.take<double>((size_t)pb.n);
  P.b.pval = A.take<double>(kPivBlocks);
  P.b.pidx = A.take<int>(kPivBlocks);
  P.b.psum = A.take<double>(kPivBlocks);
  P.b.dval = A.take<double>((size_t)k + 2);
  P.b.trace0 = A.take<double>(2);
  P.b.stop = A.take<int>(1);
  P.b.counter = A.take<unsigned>(4);
}

template <class T>
void plan_cg(Arena& A, const Prob& pb, int k, int t, int max_iter, CgBufs<T>& c) {
  const size_t nt = (size_t)pb.n * t;
  c.X = A.take<T>(nt);
  c.R = A.take<T>(nt);
  c.Z = A.take<T>(nt);
  c.P = A.take<T>(nt);
  c.Q = A.take<T>(nt);
  c.Sp = A.take<T>((size_t)std::max(k, 1) * t);
  c.atb_part = A.take<double>(cg_atb_part_elems(pb.n, k, t));
  c.S = A.take<double>((size_t)std::max(k, 1) * t);
  c.rho = A.take<double>(t);
  c.rho0 = A.take<double>(t);
  c.bnorm2 = A.take<double>(t);
  c.alpha = A.take<double>((size_t)t * max_iter);
  c.beta = A.take<double>((size_t)t * max_iter);
  c.part = A.take<double>(cg_part_elems(pb.n, t));
  c.active = A.take<int>(t);
  c.caps = A.take<int>(t);
  c.iters = A.take<int>(t);
  c.n_active = A.take<int>(1);
  c.status = A.take<int>(1);
  c.counter = A.take<unsigned>(4);
  c.ctl = A.take<int>(4);
}

struct CorePlan {
  double *G, *Cfac, *Cinv, *work, *atb_part, *logdet;
};
void plan_core(Arena& A, const Prob& pb, int k, CorePlan& P) {
  size_t kk = (size_t)std::max(k, 1) * std::max(k, 1);
  P.G = A.take<double>(kk);
  P.Cfac = A.take<double>(kk);
  P.Cinv = A.take<double>(kk);
  P.work = A.take<double>(kk);
  P.atb_part = A.take<double>((size_t)atb_chunks(pb.n) * kk);
  P.logdet = A.take<double>(1);
}

void plan_prec(Arena& A, const Prob& pb, int k, int nl, PrecBufs& b) {
  size_t K = std::max(k, 1), NL = std::max(nl, 1);
  b.Q = A.take<double>(K * K + NL * K);
  b.dW = A.take<double>((size_t)(pb.p - 1) * K * K);
  b.Lpi = A.take<double>(K * K);
  b.Lpinv = A.take<double>(K * K);
  b.A1 = A.take<double>(K * K);
  b.B1 = A.take<double>(K * K);
  b.tmp = A.take<double>(K * K);
  b.LtW = A.take<double>(K * NL + 512);
  b.Cv = A.take<double>(K * NL + 2 * (kMaxD + 1));
  b.part = reinterpret_cast<double*>(A.take<char>(2 * (size_t)pb.n * K * elem_size(pb.prec)));
  b.dkpart = A.take<double>(std::max<size_t>((size_t)atb_chunks(pb.n) * K * NL,
                                              (size_t)cdiv(pb.n, 256) * 2 * (kMaxD + 1)));
}

// ---- matrix-vector products used by CG ----------------------------------------------
template <class T>
struct SimtMvm : MvmOp {
  Prob pb;
  const void* Xs;
  void* scratch;
  gp_status apply(const void* V, int64_t ldv, int t, void* W, int64_t ldw, const int* gate,
                  cudaStream_t st) override {
    return kmvm_simt<T>(pb, Xs, V, ldv, t, W, ldw, scratch, gate, st);
  }
};

struct TcMvm : MvmOp {
  Prob pb;
  TcBufs tb;
  int mode = 0;   // 0 fast, 1 split, 2 the device's split flag decides (kmvm_tc)
  gp_status apply(const void* V, int64_t ldv, int t, void* W, int64_t ldw, const int* gate,
                  cudaStream_t st) override {
    return kmvm_tc(pb, tb, static_cast<const float*>(V), ldv, t, static_cast<float*>(W), ldw,
                   gate, mode, st);
  }
};

template <class T>
gp_status run_prep(const Prob& pb, const PrepPlan& P, cudaStream_t st) {
  GP_CUDA_TRY(cudaMemsetAsync(P.pr.counter, 0, 4 * sizeof(unsigned), st));
  return prep_inputs<T>(pb, P.pr, st);
}

template <class T>
gp_status run_kernel_mvm(const Prob& pb, const void* V, int64_t ldv, int t, void* W, int64_t ldw,
                         MvmPlan& P, cudaStream_t st) {
  GP_TRY(run_prep<T>(pb, P.prep, st));
  if (P.use_tc) {
    GP_CUDA_TRY(cudaMemsetAsync(P.tc.err, 0, kTcErrInts * sizeof(int), st));
    GP_TRY(tc_prepare_inputs(pb, P.prep.pr.Xs, P.tc, st));
    TcMvm op;
    op.pb = pb;
    op.tb = P.tc;
    return op.apply(V, ldv, t, W, ldw, nullptr, st);
  }
  SimtMvm<T> op;
  op.pb = pb;
  op.Xs = P.prep.pr.Xs;
  op.scratch = P.scratch;
  return op.apply(V, ldv, t, W, ldw, nullptr, st);
}

// ---- small kernels for the assembly ---------------------------------------------------
__global__ void fill_weights(int t, double* w) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= t) return;
  // column 0: (u, u) with 1/2; probe columns: (K^-1 z_i, P^-1 z_i) with -1/(2l)
  w[c] = (c == 0) ? 0.5 : -0.5 / (double)(t - 1);
}

__global__ void assemble(int64_t n, int P, int nl, int k, const int* rank, const int* iters,
                         const int* piv, const int* dev_status, const int* tc_err,
                         double* out, int* iout) {
  if (threadIdx.x != 0) return;
  const double LOG2PI = 1.8378770664093453;
  double stoch = 0.0;
  for (int i = 0; i < nl; ++i) stoch += out[GP_OUT_GAMMA(P) + i];
  stoch = nl > 0 ? stoch / nl : 0.0;
  out[GP_OUT_STOCH] = stoch;
  out[GP_OUT_LOGDET] = out[GP_OUT_LOGDETP] + stoch;
  out[GP_OUT_MLL] = -0.5 * (out[GP_OUT_QUAD] + out[GP_OUT_LOGDET] + (double)n * LOG2PI);
  for (int q = 0; q < P; ++q)
    out[GP_OUT_GRAD(P) + q] = out[GP_OUT_GK(P) + q] + 0.5 * out[GP_OUT_PROBEP(P) + q] -
                              0.5 * out[GP_OUT_TRP(P) + q];
  for (int h = 5; h < GP_OUT_HEAD; ++h) out[h] = 0.0;
  const int t = nl + 1;
  // a tensor-core product that gave up waiting (its outputs are NaN) outranks the
  // CG status
  iout[GP_IOUT_STATUS] = (tc_err && tc_err[0] < 0) ? tc_err[0] : *dev_status;
  iout[GP_IOUT_RANK] = *rank;
  for (int c = 0; c < t; ++c) iout[GP_IOUT_ITERS + c] = iters[c];
  for (int m = 0; m < k; ++m) iout[GP_IOUT_PIV(t) + m] = piv[m];
}

template <class T>
__global__ void copy_col(int64_t n, const T* src, T* dst) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a < n) dst[a] = src[a];
}

// Non-blocking side streams with two events each, per host thread and device: index
// 0 serves single calls, 1 .. kBatchStreams the worker streams of a batched call.
constexpr int kBatchStreams = 8;
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int device = -1;
  bool ok = false;
};
SideStream& side_stream(int i = 0) {
  static thread_local SideStream ss[kBatchStreams + 1];
  SideStream& s = ss[i];
  int dev = 0;
  cudaGetDevice(&dev);
  if (!s.ok || s.device != dev) {
    s.ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming) == cudaSuccess;
    s.device = dev;
  }
  return s;
}

// Hyperparameters must be finite and positive (lengthscales, output scale, noise).
__global__ void theta_check(const double* theta, int p, int* status) {
  const int q = threadIdx.x;
  if (q >= p) return;
  const double v = theta[q];
  if (!(v > 0.0) || !isfinite(v)) raise_status(status, GP_ERR_INVALID_ARG);
}

// Runs theta_check on `status` (zeroed first).  Outside stream capture the result is
// read back: an invalid theta returns GP_ERR_INVALID_ARG (also stored in *iout, when
// given) before anything else runs.  Under capture the check stays on the device and
// the evaluation's status word carries the error.
gp_status check_theta(const Prob& pb, int* status, int* iout, cudaStream_t st) {
  GP_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  theta_check<<<1, 64, 0, st>>>(pb.theta, pb.p, status);
  GP_LAUNCH_CHECK();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive) return GP_OK;
  int h = 0;
  GP_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  if (h < 0) {
    if (iout) GP_CUDA_TRY(cudaMemcpyAsync(iout + GP_IOUT_STATUS, status, sizeof(int),
                                          cudaMemcpyDeviceToDevice, st));
    set_error("theta must be finite and positive (lengthscales, output scale, noise)");
    return GP_ERR_INVALID_ARG;
  }
  return GP_OK;
}

// ---- split mode of the tensor-core product (GP_OPT_*) ----------------------------------
__global__ void set_int_kernel(int* p, int v) { *p = v; }

template <class T>
__global__ void fill_ones(int64_t n, T* x) {
  int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a < n) x[a] = T(1);
}

// flag = 1 when 2^-11 max_i (K_hat 1)_i > 8 sigma^2 (Gershgorin bound on lambda_max).
template <class T>
__global__ void split_decide(int64_t n, const T* __restrict__ rowsum,
                             const double* __restrict__ theta, int D, int* flag) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int64_t a = threadIdx.x; a < n; a += blockDim.x) m = fmax(m, (double)rowsum[a]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    const double s2 = theta[D + 1];
    *flag = (m * 0.00048828125 > 8.0 * s2) ? 1 : 0;
  }
}

// Sets the split flag (err[2]) of the TC product before CG: forced, or from the
// Gershgorin bound (one product of K_hat with a vector of ones, into scratch
// columns that CG overwrites afterwards).
template <class T>
gp_status tc_split_setup(const Prob& pb, MvmOp& op, const TcBufs& tb, T* ones, T* rowsum,
                         const gp_opts& o, cudaStream_t st) {
  if (o.flags & GP_OPT_SPLIT_P) {
    set_int_kernel<<<1, 1, 0, st>>>(tb.err + 2, 1);
    GP_LAUNCH_CHECK();
  } else if (o.flags & GP_OPT_AUTO_SPLIT) {
    fill_ones<T><<<(unsigned)cdiv(pb.n, 256), 256, 0, st>>>(pb.n, ones);
    GP_LAUNCH_CHECK();
    GP_TRY(op.apply(ones, pb.n, 1, rowsum, pb.n, nullptr, st));
    split_decide<T><<<1, 1024, 0, st>>>(pb.n, rowsum, pb.theta, pb.D, tb.err + 2);
    GP_LAUNCH_CHECK();
  }
  return GP_OK;
}

// The product's operand form for CG under these options (TcMvm::mode).
inline int split_mode_of(const gp_opts& o) {
  if (o.flags & GP_OPT_SPLIT_P) return 1;
  if (o.flags & GP_OPT_AUTO_SPLIT) return 2;
  return 0;
}

// After an eager CG call that broke down in fast mode: true (and split mode set)
// when CG should run again.
inline bool tc_retry_split(const TcBufs& tb, int host_status, cudaStream_t st) {
  if (host_status != GP_ERR_NUMERIC) return false;
  int flag = 1;
  if (cudaMemcpyAsync(&flag, tb.err + 2, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || flag != 0)
    return false;
  set_int_kernel<<<1, 1, 0, st>>>(tb.err + 2, 1);
  return cudaGetLastError() == cudaSuccess;
}

// First-order change of the estimator when the kernel product switches from fast to
// split mode: with D = (K_split - K_fast) X (X the CG solutions [u, K^-1 z_i]),
//   d quad   ~ -u^T D_0            (u = K_hat^-1 y),
//   d logdet ~ (1/l) sum_i (P^-1 z_i)^T D_i
// (the unbiased trace estimator of tr(K_hat^-1 D), as in the gradient).  Columns are
// reduced per block in FP64 and combined by the last block: out = {u^T D_0,
// sum_i (P^-1 z_i)^T D_i}.
template <class T>
__global__ void split_drift(int64_t n, int t, const T* __restrict__ X, const T* __restrict__ PinvB,
                            const T* __restrict__ Wf, const T* __restrict__ Ws,
                            double* __restrict__ part, unsigned* counter, double* out) {
  const int nb = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t per = (n + nb - 1) / nb, r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (int c = warp; c < t; c += blockDim.x >> 5) {
    const T* a = (c == 0 ? X : PinvB) + (int64_t)c * n;
    double acc = 0.0;
    for (int64_t i = r0 + lane; i < r1; i += 32)
      acc += (double)a[i] * ((double)Ws[i + (int64_t)c * n] - (double)Wf[i + (int64_t)c * n]);
    acc = warp_sum(acc);
    if (lane == 0) part[(size_t)c * nb + blockIdx.x] = acc;
  }
  if (last_block_arrived(counter) && threadIdx.x == 0) {
    double q = 0.0, tr = 0.0;
    for (int c = 0; c < t; ++c) {
      double s = 0.0;
      for (int b = 0; b < nb; ++b) s += part[(size_t)c * nb + b];
      if (c == 0) q = s;
      else tr += s;
    }
    out[0] = q;
    out[1] = tr;
  }
}

// ---- gp_mll_and_grad plan -----------------------------------------------------------
template <class T>
struct MllPlan {
  MvmPlan mvm;
  PivPlan piv;
  CorePlan core;
  CgBufs<T> cg;
  PrecBufs prec;
  TcGradBufs tg;     // tensor-core gradient contraction (use_tg)
  bool use_tg;
  T* L;
  int* pivots;
  int* rank;
  double* featU;     // Fourier features: m x d frequencies (m <= k / 2)
  double* featW;     // and their m weights
  T* B;
  T* PinvB;
  double* wts;
  double* part;
  unsigned* counter;
  int* status;
};
template <class T>
void plan_mll(Arena& A, const Prob& pb, int k, int nl, int max_iter, MllPlan<T>& P) {
  const int t = nl + 1;
  plan_mvm(A, pb, t, P.mvm);
  plan_piv(A, pb, k, P.piv);
  plan_core(A, pb, k, P.core);
  plan_cg<T>(A, pb, k, t, max_iter, P.cg);
  plan_prec(A, pb, k, nl, P.prec);
  P.featU = A.take<double>((size_t)std::max(k / 2, 1) * pb.d);
  P.featW = A.take<double>((size_t)std::max(k / 2, 1));
  P.use_tg = P.mvm.use_tc && tc_grad_supported(pb, t);
  P.tg = TcGradBufs{};
  if (P.use_tg) {
    P.tg.pack = A.take<char>(tc_grad_bytes(pb.n, pb.d, t));
    P.tg.part = A.take<double>(tc_grad_part_elems());
    P.tg.cmax = A.take<int>(128);
    P.tg.mscale = A.take<float>(128);
    P.tg.inv2E = A.take<double>(1);
  }
  P.L = A.take<T>((size_t)pb.n * std::max(k, 1));
  P.pivots = A.take<int>(std::max(k, 1));
  P.rank = A.take<int>(1);
  P.B = A.take<T>((size_t)pb.n * t);
  P.PinvB = A.take<T>((size_t)pb.n * t);
  P.wts = A.take<double>(t);
  // block partials of the contraction, dot_into (one per block) and split_drift
  // (t columns x one per block)
  const size_t drift = (size_t)t * (size_t)std::min<int64_t>(kCgBlocks, cdiv(pb.n, 256));
  P.part = A.take<double>(std::max({contract_part_elems(pb.n), (size_t)4 * kCgBlocks, drift}));
  P.counter = A.take<unsigned>(4);
  P.status = A.take<int>(1);
}

template <class T>
gp_status mll_impl(const Prob& pb, const T* y, int k, int nl, const int8_t* eps,
                   const int* piv_override, const int* iters_override, double* out, int* iout,
                   const gp_opts& o, void* ws, size_t ws_bytes, cudaStream_t st,
                   int side_index = 0, const FeatSpec* feat = nullptr) {
  const int t = nl + 1;
  MllPlan<T> P;
  {
    Arena dry;
    plan_mll<T>(dry, pb, k, nl, o.max_iter, P);
    if (dry.off > ws_bytes) {
      set_error("workspace too small: need %zu bytes, got %zu", dry.off, ws_bytes);
      return GP_ERR_WORKSPACE;
    }
  }
  Arena A;
  A.base = static_cast<char*>(ws);
  plan_mll<T>(A, pb, k, nl, o.max_iter, P);

  GP_CUDA_TRY(cudaMemsetAsync(P.counter, 0, 4 * sizeof(unsigned), st));
  GP_CUDA_TRY(cudaMemsetAsync(P.piv.b.counter, 0, 4 * sizeof(unsigned), st));
  GP_CUDA_TRY(cudaMemsetAsync(P.cg.counter, 0, 4 * sizeof(unsigned), st));
  GP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * GP_OUT_LEN(pb.p, nl), st));
  GP_TRY(check_theta(pb, P.cg.status, iout, st));

  // S1: scaled inputs
  GP_TRY(run_prep<T>(pb, P.mvm.prep, st));
  const void* Xs = P.mvm.prep.pr.Xs;
  if (feat) {
    // S2': Fourier features (Tab. 2) as the low-rank factor: rank k = 2m, no pivots
    GP_TRY(rff_build<T>(pb, Xs, *feat, P.featU, P.featW, P.L, pb.n, st));
    GP_CUDA_TRY(cudaMemsetAsync(P.pivots, 0xff, sizeof(int) * (size_t)k, st));
    set_int_kernel<<<1, 1, 0, st>>>(P.rank, k);
    GP_LAUNCH_CHECK();
  } else {
    // S2: pivoted Cholesky
    GP_TRY(pivchol_run<T>(pb, Xs, k, o.pivchol_tol, piv_override, P.L, pb.n, P.pivots, P.rank,
                          P.piv.b, st));
  }
  // S3: Woodbury core and log det P_hat
  if (k > 0) GP_TRY(atb<T>(pb.n, P.L, pb.n, k, P.L, pb.n, k, P.core.atb_part, P.core.G, st));
  GP_TRY(woodbury_core(k, P.core.G, pb.theta, pb.D, pb.n, P.core.Cfac, P.core.Cinv, P.core.work,
                       out + GP_OUT_LOGDETP, P.cg.status, st));
  // S4: probes, B = [y, z_1..z_l]
  GP_TRY(make_rhs<T>(pb, y, P.L, pb.n, k, nl, o.seed, eps, P.B, pb.n, st));
  // S5-S7: mBCG
  int host_status = 0;
  if (P.mvm.use_tc) {
    GP_CUDA_TRY(cudaMemsetAsync(P.mvm.tc.err, 0, kTcErrInts * sizeof(int), st));
    GP_TRY(tc_prepare_inputs(pb, Xs, P.mvm.tc, st));
    TcMvm op;
    op.pb = pb;
    op.tb = P.mvm.tc;
    GP_TRY(tc_split_setup<T>(pb, op, P.mvm.tc, P.cg.Q, P.cg.R, o, st));
    op.mode = split_mode_of(o);
    GP_TRY(cg_solve<T>(pb, op, P.L, pb.n, k, P.core.Cinv, P.B, pb.n, t, iters_override, o, P.cg,
                       P.PinvB, pb.n, &host_status, st));
    if (!(o.flags & GP_OPT_FAST_ONLY) && tc_retry_split(P.mvm.tc, host_status, st)) {
      op.mode = 1;
      GP_CUDA_TRY(cudaMemsetAsync(P.cg.status, 0, sizeof(int), st));
      GP_TRY(cg_solve<T>(pb, op, P.L, pb.n, k, P.core.Cinv, P.B, pb.n, t, iters_override, o,
                         P.cg, P.PinvB, pb.n, &host_status, st));
    }
  } else {
    SimtMvm<T> op;
    op.pb = pb;
    op.Xs = Xs;
    op.scratch = P.mvm.scratch;
    GP_TRY(cg_solve<T>(pb, op, P.L, pb.n, k, P.core.Cinv, P.B, pb.n, t, iters_override, o, P.cg,
                       P.PinvB, pb.n, &host_status, st));
  }
  // S8: Lanczos quadrature per probe.  It needs only the CG coefficients, uses one
  // block per probe, and runs on a side stream next to S9 and S10.
  SideStream& side = side_stream(side_index);
  if (!side.ok) {
    set_error("could not create the side stream");
    return GP_ERR_CUDA;
  }
  GP_CUDA_TRY(cudaEventRecord(side.fork, st));
  GP_CUDA_TRY(cudaStreamWaitEvent(side.stream, side.fork, 0));
  GP_TRY(lanczos_logquad(nl, 1, o.max_iter, P.cg.alpha, P.cg.beta, P.cg.iters, P.cg.rho0,
                         out + GP_OUT_GAMMA(pb.p), P.cg.status, side.stream));
  GP_CUDA_TRY(cudaEventRecord(side.join, side.stream));
  // quadratic term y^T u
  GP_TRY(dot_into<T>(pb.n, y, P.cg.X, P.part, P.counter, out + GP_OUT_QUAD, st));
  // S9: gradient contraction with A = [u, K^-1 z_i], B = [u, P^-1 z_i]
  copy_col<T><<<(unsigned)cdiv(pb.n, 256), 256, 0, st>>>(pb.n, P.cg.X, P.PinvB);
  GP_LAUNCH_CHECK();
  fill_weights<<<(unsigned)cdiv(t, 128), 128, 0, st>>>(t, P.wts);
  GP_LAUNCH_CHECK();
  const bool timed = mvm_timing_enabled();
  if (timed) mvm_timing_begin(st, 1);
  if (P.use_tg && !(o.flags & GP_OPT_SIMT_GRAD)) {
    GP_TRY(tc_grad_prepare(pb, Xs, P.tg, t, st));
    GP_TRY(contract_tc(pb, Xs, P.mvm.tc, P.tg, reinterpret_cast<const float*>(P.cg.X), pb.n,
                       reinterpret_cast<const float*>(P.PinvB), pb.n, P.wts, t,
                       out + GP_OUT_GK(pb.p), st));
    GP_TRY(contract_noise<T>(pb, P.cg.X, pb.n, P.PinvB, pb.n, P.wts, t, P.part, P.counter,
                             out + GP_OUT_GK(pb.p) + pb.D + 1, st));
  } else {
    GP_TRY(contract_simt<T>(pb, Xs, P.cg.X, pb.n, P.PinvB, pb.n, P.wts, t, P.part, P.counter,
                            out + GP_OUT_GK(pb.p), st));
  }
  if (timed) mvm_timing_end(st, 1);
  // S10: preconditioner terms with W = P^-1 z_i (columns 1..l of PinvB)
  if (feat) {
    GP_TRY(feature_terms<T>(pb, Xs, P.L, pb.n, feat->m, P.featU, P.featW, P.PinvB + pb.n,
                            pb.n, nl, P.core.Cinv, P.prec, out + GP_OUT_TRP(pb.p),
                            out + GP_OUT_PROBEP(pb.p), st));
  } else {
    GP_TRY(precond_terms<T>(pb, Xs, P.L, pb.n, k, P.pivots, P.rank, P.PinvB + pb.n, pb.n, nl,
                            P.core.Cinv, P.prec, out + GP_OUT_TRP(pb.p),
                            out + GP_OUT_PROBEP(pb.p), st));
  }
  // S11: assembly
  GP_CUDA_TRY(cudaStreamWaitEvent(st, side.join, 0));
  assemble<<<1, 32, 0, st>>>(pb.n, pb.p, nl, k, P.rank, P.cg.iters, P.pivots, P.cg.status,
                             P.mvm.use_tc ? P.mvm.tc.err : nullptr, out, iout);
  GP_LAUNCH_CHECK();

  // under stream capture nothing is read back: the statuses are in iout once the
  // graph has run
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive) return GP_OK;

  int hstat = 0, hrank = 0, herr[2] = {0, 0};
  GP_CUDA_TRY(cudaMemcpyAsync(&hstat, P.cg.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaMemcpyAsync(&hrank, P.rank, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (P.mvm.use_tc)
    GP_CUDA_TRY(cudaMemcpyAsync(herr, P.mvm.tc.err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  GP_CUDA_TRY(cudaGetLastError());
  if (herr[0] < 0) {
    set_error("tensor-core product gave up waiting (site %d)", herr[1]);
    return (gp_status)herr[0];
  }
  if (hstat < 0) return (gp_status)hstat;
  const gp_status warn = hstat > 0 ? (gp_status)hstat
                                   : (hrank < k ? GP_WARN_RANK_DEFICIENT : GP_OK);
  // Mixed precision in fast mode: estimate the first-order change of the MLL had the
  // product carried k(r)/s to 22 bits (split mode) instead of 11; beyond the 5e-3
  // mixed-precision bound, evaluate again in split mode.  Where the change matters,
  // the first-order estimate overstates it about twofold (measured: n = 1e5 RBF
  // workload, estimate 3.0e-3 vs. actual 1.5e-3 of |MLL|; a smooth low-noise
  // problem, 2.9e-2 vs. 1.6e-2), so the bound on the estimate keeps a margin.
  if (P.mvm.use_tc && !(o.flags & (GP_OPT_SPLIT_P | GP_OPT_AUTO_SPLIT | GP_OPT_FAST_ONLY)) &&
      nl > 0) {
    int hsplit = 1;
    GP_CUDA_TRY(cudaMemcpyAsync(&hsplit, P.mvm.tc.err + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    GP_CUDA_TRY(cudaStreamSynchronize(st));
    if (hsplit == 0) {
      TcMvm op;
      op.pb = pb;
      op.tb = P.mvm.tc;
      GP_TRY(op.apply(P.cg.X, pb.n, t, P.cg.Q, pb.n, nullptr, st));           // fast
      set_int_kernel<<<1, 1, 0, st>>>(P.mvm.tc.err + 2, 1);
      op.mode = 1;
      GP_LAUNCH_CHECK();
      GP_TRY(op.apply(P.cg.X, pb.n, t, P.cg.R, pb.n, nullptr, st));           // split
      set_int_kernel<<<1, 1, 0, st>>>(P.mvm.tc.err + 2, 0);
      GP_LAUNCH_CHECK();
      const int nb = (int)std::min<int64_t>(kCgBlocks, cdiv(pb.n, 256));
      split_drift<T><<<nb, 256, 0, st>>>(pb.n, t, P.cg.X, P.PinvB, P.cg.Q, P.cg.R, P.part,
                                         P.counter, P.wts);
      GP_LAUNCH_CHECK();
      double hd[2] = {0.0, 0.0}, hmll = 0.0;
      GP_CUDA_TRY(cudaMemcpyAsync(hd, P.wts, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaMemcpyAsync(&hmll, out + GP_OUT_MLL, sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      const double dd[2] = {-hd[0], hd[1] / nl};   // d quad, d logdet
      const double dmll = -0.5 * (dd[0] + dd[1]);
      gp_status r = GP_OK;
      if (!(fabs(dmll) <= 5e-3 * fabs(hmll))) {
        gp_opts o2 = o;
        o2.flags |= GP_OPT_SPLIT_P;
        r = mll_impl<T>(pb, y, k, nl, eps, piv_override, iters_override, out, iout, o2, ws,
                        ws_bytes, st, side_index, feat);
        if (r < 0) return r;
      }
      // report the estimates in the output head (GP_OUT_DRIFT_QUAD / _LOGDET)
      GP_CUDA_TRY(cudaMemcpyAsync(out + GP_OUT_DRIFT_QUAD, dd, 2 * sizeof(double),
                                  cudaMemcpyHostToDevice, st));
      GP_CUDA_TRY(cudaStreamSynchronize(st));
      if (r != GP_OK) return r;
    }
  }
  return warn;
}

template <class T>
gp_status mbcg_impl(const Prob& pb, const T* L, int64_t ldl, int k, const T* B, int64_t ldb,
                    int t, const int* iters_override, T* Xsol, int64_t ldx, T* PinvB,
                    double* T_diag, double* T_off, double* rho0, int* iters, int* status,
                    const gp_opts& o, void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace
}  // namespace gp

using namespace gp;

// ---- workspace sizes --------------------------------------------------------------------
extern "C" size_t gp_workspace_size(int32_t fn, int64_t n, int32_t d, int32_t k, int32_t t,
                                    int32_t precision, int32_t max_iter) {
  Prob pb{};
  pb.n = n;
  pb.d = d;
  pb.ard = 1;
  pb.D = d;
  pb.p = d + 2;
  pb.prec = precision;
  if (n < 1 || d < 1 || d > kMaxD || t < 0 || k < 0 || max_iter < 0) return 0;
  Arena A;
  switch (fn) {
    case GP_FN_KERNEL_MVM:
    case GP_FN_KERNEL_GRAD_MVM: {
      MvmPlan P;
      plan_mvm(A, pb, std::max(t, 1), P);
      if (fn == GP_FN_KERNEL_GRAD_MVM) {
        PrepPlan pp;
        (void)pp;
        // the derivative products always run on CUDA cores
        A.take<char>(elem_size(precision) * simt_scratch_elems(n, std::max(t, 1)));
      }
      break;
    }
    case GP_FN_PIVCHOL: {
      PrepPlan pp;
      plan_prep(A, pb, pp);
      PivPlan P;
      plan_piv(A, pb, k, P);
      break;
    }
    case GP_FN_MBCG: {
      MvmPlan mp;
      plan_mvm(A, pb, std::max(t, 1), mp);
      CorePlan cp;
      plan_core(A, pb, k, cp);
      if (precision == GP_FP64) {
        CgBufs<double> c;
        plan_cg<double>(A, pb, k, std::max(t, 1), std::max(max_iter, 1), c);
      } else {
        CgBufs<float> c;
        plan_cg<float>(A, pb, k, std::max(t, 1), std::max(max_iter, 1), c);
      }
      break;
    }
    case GP_FN_MLL_AND_GRAD: {
      int nl = std::max(t - 1, 0);
      if (precision == GP_FP64) {
        MllPlan<double> P;
        plan_mll<double>(A, pb, k, nl, std::max(max_iter, 1), P);
      } else {
        MllPlan<float> P;
        plan_mll<float>(A, pb, k, nl, std::max(max_iter, 1), P);
      }
      break;
    }
    default:
      return 0;
  }
  return A.off + 256;
}

extern "C" const char* gp_status_string(int32_t s) {
  switch (s) {
    case GP_OK: return "GP_OK";
    case GP_WARN_NOT_CONVERGED: return "GP_WARN_NOT_CONVERGED";
    case GP_WARN_RANK_DEFICIENT: return "GP_WARN_RANK_DEFICIENT";
    case GP_ERR_INVALID_ARG: return "GP_ERR_INVALID_ARG";
    case GP_ERR_CUDA: return "GP_ERR_CUDA";
    case GP_ERR_NOT_SPD: return "GP_ERR_NOT_SPD";
    case GP_ERR_WORKSPACE: return "GP_ERR_WORKSPACE";
    case GP_ERR_DEVICE_TIMEOUT: return "GP_ERR_DEVICE_TIMEOUT";
    case GP_ERR_NUMERIC: return "GP_ERR_NUMERIC";
    default: return "GP_UNKNOWN_STATUS";
  }
}

extern "C" const char* gp_last_error_message(void) { return last_error(); }

static gp_status check_ws(void* ws, size_t have, size_t need) {
  if (have < need || (need > 256 && ws == nullptr)) {
    set_error("workspace too small: need %zu bytes, got %zu", need, have);
    return GP_ERR_WORKSPACE;
  }
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
    set_error("workspace must be 256-byte aligned");
    return GP_ERR_WORKSPACE;
  }
  return GP_OK;
}

extern "C" gp_status gp_kernel_mvm(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                                   void* W, int64_t ldw, void* ws, size_t ws_bytes,
                                   gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(V && W, "V or W is NULL");
  GP_REQUIRE(ldv >= prob->n && ldw >= prob->n, "leading dimensions must be >= n");
  GP_REQUIRE(V != W, "W must not alias V");
  Prob pb = make_prob(prob);
  GP_TRY(check_ws(ws, ws_bytes, gp_workspace_size(GP_FN_KERNEL_MVM, pb.n, pb.d, 0, t, pb.prec, 1)));
  GP_REQUIRE(!((pb.prec == GP_BF16 || pb.prec == GP_TF32) && !tc_supported(pb, t)),
             "tensor-core precision does not support this shape");
  Arena A;
  A.base = static_cast<char*>(ws);
  MvmPlan P;
  plan_mvm(A, pb, t, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pb.prec == GP_FP64) return run_kernel_mvm<double>(pb, V, ldv, t, W, ldw, P, st);
  return run_kernel_mvm<float>(pb, V, ldv, t, W, ldw, P, st);
}

extern "C" gp_status gp_autotune(const gp_problem* prob, const void* V, int64_t ldv, int32_t t,
                                 void* W, int64_t ldw, void* ws, size_t ws_bytes,
                                 gp_stream_t stream, int32_t* best) {
  GP_TRY(check_problem(prob));
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(V && W, "V or W is NULL");
  GP_REQUIRE(ldv >= prob->n && ldw >= prob->n, "leading dimensions must be >= n");
  GP_REQUIRE(V != W, "W must not alias V");
  Prob pb = make_prob(prob);
  GP_REQUIRE(pb.prec == GP_BF16 && tc_supported(pb, t),
             "autotuning applies to the tensor-core product (GP_BF16, t <= 64)");
  GP_TRY(check_ws(ws, ws_bytes, gp_workspace_size(GP_FN_KERNEL_MVM, pb.n, pb.d, 0, t, pb.prec, 1)));
  Arena A;
  A.base = static_cast<char*>(ws);
  MvmPlan P;
  plan_mvm(A, pb, t, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GP_TRY(run_prep<float>(pb, P.prep, st));
  GP_CUDA_TRY(cudaMemsetAsync(P.tc.err, 0, kTcErrInts * sizeof(int), st));
  GP_TRY(tc_prepare_inputs(pb, P.prep.pr.Xs, P.tc, st));
  int b4[4] = {0, 0, 0, 0};
  GP_TRY(tc_autotune(pb, P.tc, static_cast<const float*>(V), ldv, t, static_cast<float*>(W), ldw,
                     st, b4));
  if (best)
    for (int i = 0; i < 4; ++i) best[i] = b4[i];
  return GP_OK;
}

extern "C" gp_status gp_tc_config(const gp_problem* prob, int32_t t, int32_t* config) {
  GP_TRY(check_problem(prob, false));
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(config, "config is NULL");
  Prob pb = make_prob(prob);
  int c4[4];
  tc_config(pb, t, c4);
  for (int i = 0; i < 4; ++i) config[i] = c4[i];
  return GP_OK;
}

extern "C" gp_status gp_kernel_grad_mvm(const gp_problem* prob, const void* V, int64_t ldv,
                                        int32_t t, void* dW, int64_t ldw, void* ws,
                                        size_t ws_bytes, gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(V && dW, "V or dW is NULL");
  GP_REQUIRE(ldv >= prob->n && ldw >= prob->n, "leading dimensions must be >= n");
  Prob pb = make_prob(prob);
  GP_TRY(check_ws(ws, ws_bytes,
                  gp_workspace_size(GP_FN_KERNEL_GRAD_MVM, pb.n, pb.d, 0, t, pb.prec, 1)));
  Arena A;
  A.base = static_cast<char*>(ws);
  MvmPlan P;
  plan_mvm(A, pb, t, P);
  void* scratch = A.take<char>(elem_size(pb.prec) * simt_scratch_elems(pb.n, t));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pb.prec == GP_FP64) {
    GP_TRY(run_prep<double>(pb, P.prep, st));
    return kdmvm_simt<double>(pb, P.prep.pr.Xs, V, ldv, t, dW, ldw, scratch, st);
  }
  GP_TRY(run_prep<float>(pb, P.prep, st));
  return kdmvm_simt<float>(pb, P.prep.pr.Xs, V, ldv, t, dW, ldw, scratch, st);
}

extern "C" gp_status gp_pivchol(const gp_problem* prob, int32_t k, double tol,
                                const int32_t* piv_override, void* L, int64_t ldl, int32_t* piv,
                                int32_t* rank_out, void* ws, size_t ws_bytes,
                                gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_REQUIRE(k >= 0 && k <= kMaxK && k <= prob->n, "k=%d out of range [0, min(n, %d)]", k,
             kMaxK);
  GP_REQUIRE(tol >= 0.0, "tol must be >= 0");
  GP_REQUIRE(k == 0 || (L && piv), "L or piv is NULL");
  GP_REQUIRE(rank_out, "rank_out is NULL");
  GP_REQUIRE(ldl >= prob->n, "ldl must be >= n");
  Prob pb = make_prob(prob);
  GP_TRY(check_ws(ws, ws_bytes, gp_workspace_size(GP_FN_PIVCHOL, pb.n, pb.d, k, 1, pb.prec, 1)));
  Arena A;
  A.base = static_cast<char*>(ws);
  PrepPlan pp;
  plan_prep(A, pb, pp);
  PivPlan P;
  plan_piv(A, pb, k, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GP_CUDA_TRY(cudaMemsetAsync(P.b.counter, 0, 4 * sizeof(unsigned), st));
  if (pb.prec == GP_FP64) {
    GP_TRY(run_prep<double>(pb, pp, st));
    return pivchol_run<double>(pb, pp.pr.Xs, k, tol, piv_override, L, ldl, piv, rank_out, P.b, st);
  }
  GP_TRY(run_prep<float>(pb, pp, st));
  return pivchol_run<float>(pb, pp.pr.Xs, k, tol, piv_override, L, ldl, piv, rank_out, P.b, st);
}

static gp_status check_opts(const gp_opts* o) {
  GP_REQUIRE(o != nullptr, "opts is NULL");
  GP_REQUIRE(o->max_iter >= 1 && o->max_iter <= 8192, "max_iter=%d out of range [1, 8192]",
             o->max_iter);
  GP_REQUIRE(o->cg_tol >= 0.0, "cg_tol must be >= 0");
  GP_REQUIRE(o->recompute_every >= 0, "recompute_every must be >= 0");
  GP_REQUIRE(o->pivchol_tol >= 0.0, "pivchol_tol must be >= 0");
  return GP_OK;
}

namespace gp {
namespace {
template <class T>
gp_status mbcg_impl(const Prob& pb, const T* L, int64_t ldl, int k, const T* B, int64_t ldb,
                    int t, const int* iters_override, T* Xsol, int64_t ldx, T* PinvB,
                    double* T_diag, double* T_off, double* rho0, int* iters, int* status,
                    const gp_opts& o, void* ws, size_t ws_bytes, cudaStream_t st) {
  Arena A;
  A.base = static_cast<char*>(ws);
  MvmPlan mp;
  plan_mvm(A, pb, t, mp);
  CorePlan cp;
  plan_core(A, pb, k, cp);
  CgBufs<T> cb;
  plan_cg<T>(A, pb, k, t, o.max_iter, cb);
  (void)ws_bytes;
  GP_CUDA_TRY(cudaMemsetAsync(cb.counter, 0, 4 * sizeof(unsigned), st));
  GP_TRY(check_theta(pb, cb.status, nullptr, st));
  GP_CUDA_TRY(cudaMemsetAsync(cb.alpha, 0, sizeof(double) * (size_t)t * o.max_iter, st));
  GP_CUDA_TRY(cudaMemsetAsync(cb.beta, 0, sizeof(double) * (size_t)t * o.max_iter, st));
  GP_TRY(run_prep<T>(pb, mp.prep, st));
  if (k > 0) GP_TRY(atb<T>(pb.n, L, ldl, k, L, ldl, k, cp.atb_part, cp.G, st));
  GP_TRY(woodbury_core(k, cp.G, pb.theta, pb.D, pb.n, cp.Cfac, cp.Cinv, cp.work, cp.logdet,
                       cb.status, st));
  int host_status = 0;
  if (mp.use_tc) {
    GP_CUDA_TRY(cudaMemsetAsync(mp.tc.err, 0, kTcErrInts * sizeof(int), st));
    GP_TRY(tc_prepare_inputs(pb, mp.prep.pr.Xs, mp.tc, st));
    TcMvm op;
    op.pb = pb;
    op.tb = mp.tc;
    GP_TRY(tc_split_setup<T>(pb, op, mp.tc, cb.Q, cb.R, o, st));
    op.mode = split_mode_of(o);
    GP_TRY(cg_solve<T>(pb, op, L, ldl, k, cp.Cinv, B, ldb, t, iters_override, o, cb, PinvB, ldx,
                       &host_status, st));
    if (!(o.flags & GP_OPT_FAST_ONLY) && tc_retry_split(mp.tc, host_status, st)) {
      op.mode = 1;
      GP_CUDA_TRY(cudaMemsetAsync(cb.status, 0, sizeof(int), st));
      GP_TRY(cg_solve<T>(pb, op, L, ldl, k, cp.Cinv, B, ldb, t, iters_override, o, cb, PinvB,
                         ldx, &host_status, st));
    }
  } else {
    SimtMvm<T> op;
    op.pb = pb;
    op.Xs = mp.prep.pr.Xs;
    op.scratch = mp.scratch;
    GP_TRY(cg_solve<T>(pb, op, L, ldl, k, cp.Cinv, B, ldb, t, iters_override, o, cb, PinvB, ldx,
                       &host_status, st));
  }
  // outputs
  GP_CUDA_TRY(cudaMemcpy2DAsync(Xsol, sizeof(T) * ldx, cb.X, sizeof(T) * pb.n, sizeof(T) * pb.n,
                                t, cudaMemcpyDeviceToDevice, st));
  GP_TRY(cg_tridiag<T>(t, o.max_iter, cb, T_diag, T_off, st));
  GP_CUDA_TRY(cudaMemcpyAsync(rho0, cb.rho0, sizeof(double) * t, cudaMemcpyDeviceToDevice, st));
  GP_CUDA_TRY(cudaMemcpyAsync(iters, cb.iters, sizeof(int) * t, cudaMemcpyDeviceToDevice, st));
  GP_CUDA_TRY(cudaMemcpyAsync(status, cb.status, sizeof(int), cudaMemcpyDeviceToDevice, st));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive) return GP_OK;   // status read after the graph runs
  int hs = 0, herr[2] = {0, 0};
  GP_CUDA_TRY(cudaMemcpyAsync(&hs, cb.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (mp.use_tc)
    GP_CUDA_TRY(cudaMemcpyAsync(herr, mp.tc.err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr[0] < 0) {
    set_error("tensor-core product gave up waiting (site %d)", herr[1]);
    return (gp_status)herr[0];
  }
  return (gp_status)hs;   // 0, a warning (> 0) or an error (< 0)
}
}  // namespace
}  // namespace gp

extern "C" gp_status gp_mbcg(const gp_problem* prob, const void* L, int64_t ldl, int32_t k,
                             const void* B, int64_t ldb, int32_t t,
                             const int32_t* iters_override, void* Xsol, int64_t ldx, void* PinvB,
                             double* T_diag, double* T_off, double* rho0, int32_t* iters,
                             int32_t* status, const gp_opts* opts, void* ws, size_t ws_bytes,
                             gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_TRY(check_opts(opts));
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range [1, %d]", t, kMaxT);
  GP_REQUIRE(k >= 0 && k <= kMaxK && k <= prob->n, "k out of range");
  GP_REQUIRE(k == 0 || L, "L is NULL");
  GP_REQUIRE(B && Xsol && T_diag && T_off && rho0 && iters && status, "NULL output");
  GP_REQUIRE(ldl >= prob->n && ldb >= prob->n && ldx >= prob->n, "leading dimensions must be >= n");
  Prob pb = make_prob(prob);
  GP_REQUIRE(!((pb.prec == GP_BF16 || pb.prec == GP_TF32) && !tc_supported(pb, t)),
             "tensor-core precision does not support this shape");
  GP_TRY(check_ws(ws, ws_bytes,
                  gp_workspace_size(GP_FN_MBCG, pb.n, pb.d, k, t, pb.prec, opts->max_iter)));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pb.prec == GP_FP64)
    return mbcg_impl<double>(pb, (const double*)L, ldl, k, (const double*)B, ldb, t,
                             iters_override, (double*)Xsol, ldx, (double*)PinvB, T_diag, T_off,
                             rho0, iters, status, *opts, ws, ws_bytes, st);
  return mbcg_impl<float>(pb, (const float*)L, ldl, k, (const float*)B, ldb, t, iters_override,
                          (float*)Xsol, ldx, (float*)PinvB, T_diag, T_off, rho0, iters, status,
                          *opts, ws, ws_bytes, st);
}

extern "C" gp_status gp_mll_and_grad(const gp_problem* prob, const void* y, int32_t k,
                                     int32_t n_probes, const int8_t* eps_override,
                                     const int32_t* piv_override, const int32_t* iters_override,
                                     double* out, int32_t* iout, const gp_opts* opts, void* ws,
                                     size_t ws_bytes, gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_TRY(check_opts(opts));
  GP_REQUIRE(y && out && iout, "y, out or iout is NULL");
  GP_REQUIRE(k >= 0 && k <= kMaxK && k <= prob->n, "k=%d out of range [0, min(n, %d)]", k, kMaxK);
  GP_REQUIRE(n_probes >= 0 && n_probes + 1 <= kMaxT, "n_probes=%d out of range", n_probes);
  Prob pb = make_prob(prob);
  const int t = n_probes + 1;
  GP_REQUIRE(!((pb.prec == GP_BF16 || pb.prec == GP_TF32) && !tc_supported(pb, t)),
             "tensor-core precision does not support this shape");
  GP_TRY(check_ws(ws, ws_bytes,
                  gp_workspace_size(GP_FN_MLL_AND_GRAD, pb.n, pb.d, k, t, pb.prec, opts->max_iter)));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (pb.prec == GP_FP64)
    return mll_impl<double>(pb, (const double*)y, k, n_probes, eps_override, piv_override,
                            iters_override, out, iout, *opts, ws, ws_bytes, st);
  return mll_impl<float>(pb, (const float*)y, k, n_probes, eps_override, piv_override,
                         iters_override, out, iout, *opts, ws, ws_bytes, st);
}

extern "C" gp_status gp_mll_and_grad_rff(const gp_problem* prob, const void* y, int32_t m,
                                         int32_t n_probes, const double* eps, const double* g,
                                         const int8_t* eps_override,
                                         const int32_t* iters_override, double* out,
                                         int32_t* iout, const gp_opts* opts, void* ws,
                                         size_t ws_bytes, gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_TRY(check_opts(opts));
  GP_REQUIRE(y && out && iout, "y, out or iout is NULL");
  GP_REQUIRE(m >= 1 && 2 * (int64_t)m <= kMaxK && 2 * (int64_t)m <= prob->n,
             "m=%d out of range [1, min(n, %d) / 2]", m, kMaxK);
  GP_REQUIRE(eps, "eps is NULL");
  GP_REQUIRE(g || prob->kind == GP_RBF, "g is NULL (every kernel but the RBF needs it)");
  GP_REQUIRE(n_probes >= 0 && n_probes + 1 <= kMaxT, "n_probes=%d out of range", n_probes);
  Prob pb = make_prob(prob);
  const int t = n_probes + 1, k = 2 * m;
  GP_REQUIRE(!((pb.prec == GP_BF16 || pb.prec == GP_TF32) && !tc_supported(pb, t)),
             "tensor-core precision does not support this shape");
  GP_TRY(check_ws(ws, ws_bytes,
                  gp_workspace_size(GP_FN_MLL_AND_GRAD, pb.n, pb.d, k, t, pb.prec, opts->max_iter)));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const FeatSpec feat{m, eps, g, nullptr, nullptr};
  if (pb.prec == GP_FP64)
    return mll_impl<double>(pb, (const double*)y, k, n_probes, eps_override, nullptr,
                            iters_override, out, iout, *opts, ws, ws_bytes, st, 0, &feat);
  return mll_impl<float>(pb, (const float*)y, k, n_probes, eps_override, nullptr,
                         iters_override, out, iout, *opts, ws, ws_bytes, st, 0, &feat);
}

extern "C" int32_t gp_qff_rule(int32_t mbar, int32_t d, double* U, double* W) {
  GP_REQUIRE(mbar >= 2 && mbar % 2 == 0, "mbar=%d must be even and >= 2", mbar);
  GP_REQUIRE(d >= 1 && d <= kMaxD, "d=%d out of range [1, %d]", d, kMaxD);
  int64_t total = 1;
  for (int i = 0; i < d && total <= 2 * (int64_t)kMaxK; ++i) total *= mbar;
  GP_REQUIRE(total <= 2 * (int64_t)kMaxK, "mbar^d exceeds %d", 2 * kMaxK);
  std::vector<double> u, w;
  qff_table(mbar, d, u, w);
  if (U) std::copy(u.begin(), u.end(), U);
  if (W) std::copy(w.begin(), w.end(), W);
  return (int32_t)w.size();
}

extern "C" gp_status gp_mll_and_grad_qff(const gp_problem* prob, const void* y, int32_t mbar,
                                         int32_t n_probes, const int8_t* eps_override,
                                         const int32_t* iters_override, double* out,
                                         int32_t* iout, const gp_opts* opts, void* ws,
                                         size_t ws_bytes, gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_TRY(check_opts(opts));
  GP_REQUIRE(y && out && iout, "y, out or iout is NULL");
  GP_REQUIRE(prob->kind == GP_RBF, "quadrature Fourier features need the RBF kernel");
  GP_REQUIRE(mbar >= 2 && mbar % 2 == 0, "mbar=%d must be even and >= 2", mbar);
  int64_t k = 1;
  for (int i = 0; i < prob->d && k <= kMaxK; ++i) k *= mbar;
  GP_REQUIRE(k <= kMaxK && k <= prob->n, "mbar^d = %lld features exceed min(n, %d)",
             (long long)k, kMaxK);
  GP_REQUIRE(n_probes >= 0 && n_probes + 1 <= kMaxT, "n_probes=%d out of range", n_probes);
  Prob pb = make_prob(prob);
  const int t = n_probes + 1;
  GP_REQUIRE(!((pb.prec == GP_BF16 || pb.prec == GP_TF32) && !tc_supported(pb, t)),
             "tensor-core precision does not support this shape");
  GP_TRY(check_ws(ws, ws_bytes, gp_workspace_size(GP_FN_MLL_AND_GRAD, pb.n, pb.d, (int)k, t,
                                                  pb.prec, opts->max_iter)));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  GP_REQUIRE(cap == cudaStreamCaptureStatusNone,
             "gp_mll_and_grad_qff copies its quadrature table from the host: not capturable");
  std::vector<double> U, W;
  qff_table(mbar, pb.d, U, W);
  const int m = (int)W.size();
  GP_REQUIRE(2 * m == (int)k, "internal: %d frequencies for %lld features", m, (long long)k);
  const FeatSpec feat{m, nullptr, nullptr, U.data(), W.data()};
  gp_status r;
  if (pb.prec == GP_FP64)
    r = mll_impl<double>(pb, (const double*)y, (int)k, n_probes, eps_override, nullptr,
                         iters_override, out, iout, *opts, ws, ws_bytes, st, 0, &feat);
  else
    r = mll_impl<float>(pb, (const float*)y, (int)k, n_probes, eps_override, nullptr,
                        iters_override, out, iout, *opts, ws, ws_bytes, st, 0, &feat);
  // the host table must outlive its copies
  GP_CUDA_TRY(cudaStreamSynchronize(st));
  return r;
}

// ---- batched evaluation --------------------------------------------------------------
// Independent problems run concurrently on a pool of worker streams (each problem's
// own steps stay in order on one stream; its Lanczos quadrature forks to a side
// stream of that worker).  The whole batch is recorded as one CUDA graph: mBCG's
// iteration loops become conditional WHILE nodes (no host round trips), and the
// instantiated graph is cached per argument set, so a repeated call (for example an
// optimiser step with new hyperparameter values in the same device buffers) is a
// single graph launch.  When the caller's stream is itself being captured, the batch
// is recorded into the caller's graph instead.
namespace gp {
namespace {

struct StreamPool {
  cudaStream_t s[kBatchStreams] = {};
  cudaStream_t capture = nullptr;
  cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
  int device = -1;
  bool ok = false;
};
StreamPool& stream_pool() {
  static thread_local StreamPool p;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!p.ok || p.device != dev) {
    bool ok = cudaStreamCreateWithFlags(&p.capture, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int w = 0; w < kBatchStreams && ok; ++w)
      ok = cudaStreamCreateWithFlags(&p.s[w], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&p.join[w], cudaEventDisableTiming) == cudaSuccess;
    p.ok = ok;
    p.device = dev;
  }
  return p;
}

constexpr size_t kBatchAlign = 256;
size_t batch_layout(int np, const Prob* pbs, int k, int t, int max_iter, size_t* offs,
                    size_t* sizes) {
  size_t off = 0;
  for (int i = 0; i < np; ++i) {
    const size_t sz = gp_workspace_size(GP_FN_MLL_AND_GRAD, pbs[i].n, pbs[i].d, k, t, pbs[i].prec,
                                        max_iter);
    if (offs) offs[i] = off;
    if (sizes) sizes[i] = sz;
    off += (sz + kBatchAlign - 1) / kBatchAlign * kBatchAlign;
  }
  return off;
}

// Issue every problem of the batch on the worker streams, forked from and joined back
// into `origin` (which is being captured).  Largest problems first, each to the
// worker with the least work so far (work ~ n^2).
gp_status issue_batch(int np, const Prob* pbs, const void* const* ys, int k, int nl,
                      double* const* outs, int* const* iouts, const gp_opts& o, char* ws,
                      const size_t* offs, const size_t* sizes, cudaStream_t origin) {
  StreamPool& P = stream_pool();
  if (!P.ok) {
    set_error("could not create the batch streams");
    return GP_ERR_CUDA;
  }
  const int nw = std::min(np, kBatchStreams);
  std::vector<int> order(np);
  for (int i = 0; i < np; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return pbs[a].n > pbs[b].n; });
  std::vector<double> load(nw, 0.0);
  GP_CUDA_TRY(cudaEventRecord(P.fork, origin));
  for (int w = 0; w < nw; ++w) GP_CUDA_TRY(cudaStreamWaitEvent(P.s[w], P.fork, 0));
  for (int i : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += (double)pbs[i].n * (double)pbs[i].n;
    gp_opts oi = o;
    oi.seed = o.seed + (uint64_t)i;   // problem i draws its probes from seed + i
    gp_status r;
    if (pbs[i].prec == GP_FP64)
      r = mll_impl<double>(pbs[i], (const double*)ys[i], k, nl, nullptr, nullptr, nullptr,
                           outs[i], iouts[i], oi, ws + offs[i], sizes[i], P.s[w], 1 + w);
    else
      r = mll_impl<float>(pbs[i], (const float*)ys[i], k, nl, nullptr, nullptr, nullptr, outs[i],
                          iouts[i], oi, ws + offs[i], sizes[i], P.s[w], 1 + w);
    if (r != GP_OK) return r;
  }
  for (int w = 0; w < nw; ++w) {
    GP_CUDA_TRY(cudaEventRecord(P.join[w], P.s[w]));
    GP_CUDA_TRY(cudaStreamWaitEvent(origin, P.join[w], 0));
  }
  return GP_OK;
}

// Instantiated batch graphs of this host thread, keyed by every argument that the
// recorded work depends on (pointers, sizes, options).
struct BatchGraph {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
};
std::vector<BatchGraph>& batch_graphs() {
  static thread_local std::vector<BatchGraph> cache;
  return cache;
}
constexpr size_t kBatchGraphCache = 4;

}  // namespace
}  // namespace gp

extern "C" size_t gp_workspace_size_batched(int32_t n_problems, const gp_problem* probs,
                                            int32_t k, int32_t n_probes, int32_t max_iter) {
  if (n_problems < 1 || !probs || n_probes < 0 || n_probes + 1 > kMaxT || max_iter < 1) return 0;
  std::vector<Prob> pbs(n_problems);
  for (int i = 0; i < n_problems; ++i) {
    if (check_problem(&probs[i], false) != GP_OK) return 0;
    pbs[i] = make_prob(&probs[i]);
  }
  return batch_layout(n_problems, pbs.data(), k, n_probes + 1, max_iter, nullptr, nullptr);
}

extern "C" gp_status gp_mll_and_grad_batched(int32_t n_problems, const gp_problem* probs,
                                             const void* const* ys, int32_t k, int32_t n_probes,
                                             double* const* outs, int32_t* const* iouts,
                                             const gp_opts* opts, void* ws, size_t ws_bytes,
                                             gp_stream_t stream) {
  GP_REQUIRE(n_problems >= 1 && n_problems <= 4096, "n_problems=%d out of range [1, 4096]",
             n_problems);
  GP_REQUIRE(probs && ys && outs && iouts, "probs, ys, outs or iouts is NULL");
  GP_TRY(check_opts(opts));
  GP_REQUIRE(n_probes >= 0 && n_probes + 1 <= kMaxT, "n_probes=%d out of range", n_probes);
  const int t = n_probes + 1;
  std::vector<Prob> pbs(n_problems);
  for (int i = 0; i < n_problems; ++i) {
    gp_status r = check_problem(&probs[i]);
    if (r != GP_OK) {
      char msg[512];
      snprintf(msg, sizeof(msg), "%s", last_error());
      set_error("problem %d: %s", i, msg);
      return r;
    }
    GP_REQUIRE(ys[i] && outs[i] && iouts[i], "problem %d: y, out or iout is NULL", i);
    GP_REQUIRE(k >= 0 && k <= kMaxK && k <= probs[i].n,
               "problem %d: k=%d out of range [0, min(n, %d)]", i, k, kMaxK);
    pbs[i] = make_prob(&probs[i]);
    GP_REQUIRE(!((pbs[i].prec == GP_BF16 || pbs[i].prec == GP_TF32) && !tc_supported(pbs[i], t)),
               "problem %d: tensor-core precision does not support this shape", i);
  }
  std::vector<size_t> offs(n_problems), sizes(n_problems);
  const size_t need = batch_layout(n_problems, pbs.data(), k, t, opts->max_iter, offs.data(),
                                   sizes.data());
  GP_TRY(check_ws(ws, ws_bytes, need));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GP_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap == cudaStreamCaptureStatusActive)
    return issue_batch(n_problems, pbs.data(), ys, k, n_probes, outs, iouts, *opts, wsb,
                       offs.data(), sizes.data(), st);

  // key of the recorded work
  std::vector<uint64_t> key;
  int dev = 0;
  GP_CUDA_TRY(cudaGetDevice(&dev));
  key.push_back((uint64_t)dev);
  key.push_back((uint64_t)n_problems);
  key.push_back((uint64_t)k);
  key.push_back((uint64_t)n_probes);
  key.push_back((uint64_t)reinterpret_cast<uintptr_t>(ws));
  key.push_back((uint64_t)ws_bytes);
  {
    uint64_t ob[sizeof(gp_opts) / 8 + 1] = {};
    memcpy(ob, opts, sizeof(gp_opts));
    for (uint64_t v : ob) key.push_back(v);
  }
  for (int i = 0; i < n_problems; ++i) {
    key.push_back((uint64_t)probs[i].n);
    key.push_back(((uint64_t)(uint32_t)probs[i].d << 32) | (uint32_t)probs[i].kind);
    key.push_back(((uint64_t)(uint32_t)probs[i].ard << 32) | (uint32_t)probs[i].precision);
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(probs[i].X));
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(probs[i].theta));
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(ys[i]));
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(outs[i]));
    key.push_back((uint64_t)reinterpret_cast<uintptr_t>(iouts[i]));
  }
  std::vector<BatchGraph>& cache = batch_graphs();
  for (BatchGraph& bg : cache)
    if (bg.key == key) {
      GP_CUDA_TRY(cudaGraphLaunch(bg.exec, st));
      return GP_OK;
    }

  StreamPool& P = stream_pool();
  if (!P.ok) {
    set_error("could not create the batch streams");
    return GP_ERR_CUDA;
  }
  GP_CUDA_TRY(cudaStreamBeginCapture(P.capture, cudaStreamCaptureModeRelaxed));
  const gp_status r = issue_batch(n_problems, pbs.data(), ys, k, n_probes, outs, iouts, *opts,
                                  wsb, offs.data(), sizes.data(), P.capture);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(P.capture, &graph);
  if (r != GP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  GP_CUDA_TRY(ec);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  GP_CUDA_TRY(ei);
  if (cache.size() >= kBatchGraphCache) {
    cudaGraphExecDestroy(cache.front().exec);
    cache.erase(cache.begin());
  }
  cache.push_back(BatchGraph{key, exec});
  GP_CUDA_TRY(cudaGraphLaunch(exec, st));
  return GP_OK;
}

extern "C" gp_status gp_rademacher(uint64_t seed, int32_t stream_id, int64_t rows, int32_t cols,
                                   int8_t* out, gp_stream_t stream) {
  GP_REQUIRE(rows >= 0 && cols >= 0, "negative size");
  GP_REQUIRE(rows * cols == 0 || out, "out is NULL");
  GP_REQUIRE(stream_id == 1 || stream_id == 2, "stream_id must be 1 or 2");
  return rademacher_fill(seed, stream_id, rows, cols, out, reinterpret_cast<cudaStream_t>(stream));
}

// ---- instrumentation ---------------------------------------------------------------------
#include <atomic>
#include <mutex>
#include <vector>

namespace gp {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_tmu;
std::vector<cudaEvent_t> g_free_events;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pairs[3];   // per phase
cudaEvent_t g_open[3] = {nullptr, nullptr, nullptr};
cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
bool mvm_timing_enabled() { return g_timing.load() != 0; }
void mvm_timing_begin(cudaStream_t st, int phase) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_open[phase] = take_event();
  if (g_open[phase]) cudaEventRecord(g_open[phase], st);
}
void mvm_timing_end(cudaStream_t st, int phase) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (!g_open[phase]) return;
  cudaEvent_t e = take_event();
  if (!e) return;
  cudaEventRecord(e, st);
  g_pairs[phase].emplace_back(g_open[phase], e);
  g_open[phase] = nullptr;
}
gp_status phase_timing_read(int phase, double* total_ms, int64_t* count) {
  std::lock_guard<std::mutex> lk(g_tmu);
  double tot = 0.0;
  int64_t cnt = 0;
  for (auto& pr : g_pairs[phase]) {
    GP_CUDA_TRY(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    GP_CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
    ++cnt;
    g_free_events.push_back(pr.first);
    g_free_events.push_back(pr.second);
  }
  g_pairs[phase].clear();
  if (total_ms) *total_ms = tot;
  if (count) *count = cnt;
  return GP_OK;
}
}  // namespace gp

extern "C" int64_t gp_launch_count(void) { return (int64_t)gp::g_launches.load(); }

extern "C" void gp_mvm_timing(int32_t enable) { gp::g_timing.store(enable ? 1 : 0); }

extern "C" gp_status gp_mvm_timing_read(double* total_ms, int64_t* products) {
  return gp::phase_timing_read(0, total_ms, products);
}

extern "C" gp_status gp_phase_timing_read(int32_t phase, double* total_ms, int64_t* count) {
  GP_REQUIRE(phase >= 0 && phase <= 2, "phase must be 0, 1 or 2");
  return gp::phase_timing_read(phase, total_ms, count);
}

extern "C" gp_status gp_tc_exponent_tile(const gp_problem* prob, const void* V, int64_t ldv,
                                         int32_t t, void* W, int64_t ldw, float* S_out, void* ws,
                                         size_t ws_bytes, gp_stream_t stream) {
  GP_TRY(check_problem(prob));
  GP_REQUIRE(prob->precision == GP_BF16, "gp_tc_exponent_tile needs precision GP_BF16");
  GP_REQUIRE(t >= 1 && t <= kMaxT, "t=%d out of range", t);
  GP_REQUIRE(V && W && S_out, "NULL pointer");
  GP_REQUIRE(ldv >= prob->n && ldw >= prob->n, "leading dimensions must be >= n");
  Prob pb = make_prob(prob);
  GP_REQUIRE(tc_supported(pb, t), "tensor-core precision does not support this shape");
  GP_TRY(check_ws(ws, ws_bytes, gp_workspace_size(GP_FN_KERNEL_MVM, pb.n, pb.d, 0, t, pb.prec, 1)));
  Arena A;
  A.base = static_cast<char*>(ws);
  MvmPlan P;
  plan_mvm(A, pb, t, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GP_TRY(run_prep<float>(pb, P.prep, st));
  GP_CUDA_TRY(cudaMemsetAsync(P.tc.err, 0, kTcErrInts * sizeof(int), st));
  GP_TRY(tc_prepare_inputs(pb, P.prep.pr.Xs, P.tc, st));
  return kmvm_tc_debug(pb, P.tc, static_cast<const float*>(V), ldv, t, static_cast<float*>(W),
                       ldw, nullptr, S_out, 0, st);
}
