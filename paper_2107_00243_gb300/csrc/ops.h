// Internal interfaces between the translation units of the library.
#pragma once

#include "common.cuh"

#include <vector>

namespace gp {

constexpr int kPrepBlocks = 256;

// ---- inputs: Xs = (X - mean(X)) / l, per dimension --------------------------
struct PrepBufs {
  void* Xs;          // n x d, problem precision
  double* mean;      // d
  double* part;      // kPrepBlocks * d
  unsigned* counter; // 1
};
template <class T> gp_status prep_inputs(const Prob& pb, const PrepBufs& pr, cudaStream_t st);

// ---- SIMT kernel products (kmvm_simt.cu) ---------------------------------------
size_t simt_scratch_elems(int64_t n, int t);
template <class T>
gp_status kmvm_simt(const Prob& pb, const void* Xs, const void* V, int64_t ldv, int t,
                    void* W, int64_t ldw, void* scratch, const int* gate, cudaStream_t st);
template <class T>
gp_status kmvm_simt_unsplit(const Prob& pb, const void* Xs, const void* V, int64_t ldv, int t,
                            void* W, int64_t ldw, cudaStream_t st);
template <class T>
gp_status kdmvm_simt(const Prob& pb, const void* Xs, const void* V, int64_t ldv, int t,
                     void* dW, int64_t ldw, void* scratch, cudaStream_t st);
// Gradient contraction, hot path of Alg. 2:
//   gout[q] = sum_ab dK/dtheta_q[a,b] sum_c wts[c] A[a,c] B[b,c]   (q < D: lengthscales,
//   q = D: output scale),  gout[D + 1] = sum_a sum_c wts[c] A[a,c] B[a,c]  (noise).
size_t contract_part_elems(int64_t n);
template <class T>
gp_status contract_simt(const Prob& pb, const void* Xs, const void* A, int64_t lda,
                        const void* B, int64_t ldb, const double* wts, int t, double* part,
                        unsigned* counter, double* gout, cudaStream_t st);

// ---- tensor-core kernel products (kmvm_tc.cu) -----------------------------------
struct TcBufs {
  void* xpack;       // packed exponent operand tiles: two-part (A, B), three-part (A, B)
  float* norms;      // n
  void* vpack;       // packed right-hand-side tiles
  float* vscale;     // kTcVscaleElems: column scales of V, their inverses, partial maxima
  float* part;       // split partial sums
  int* err;          // kTcErrInts: device-side status, the wait that gave up, counters
};
constexpr int kTcErrCounters = 4;               // err[4 ..]: per-column block counters
constexpr int kTcErrInts = kTcErrCounters + 64;
constexpr int kTcVscaleElems = 2 * 64 + 64 * 16;
size_t tc_xpack_bytes(int64_t n, int d, int prec);
size_t tc_vpack_bytes(int64_t n, int t, int prec);
size_t tc_part_elems(int64_t n, int t);
bool tc_supported(const Prob& pb, int t);
gp_status tc_prepare_inputs(const Prob& pb, const void* Xs, const TcBufs& tb, cudaStream_t st);
// mode: 0 fast, 1 split (three-part exponent operands, FP16 hi + lo k(r)/s), 2 chosen
// on the device by the split flag (err[2]) at launch.
gp_status kmvm_tc(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                  float* W, int64_t ldw, const int* gate, int mode, cudaStream_t st);
// Same, and (dbg != null) the exponent tile S of the first tile pair -> dbg (128 x 128).
// Autotuner of the TC launch configuration (column chunks, ring depths) for this
// shape; best_out (may be null) = {nchunks, nsb, nsv, candidates timed}.
gp_status tc_autotune(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                      float* W, int64_t ldw, cudaStream_t st, int* best_out);
void tc_config(const Prob& pb, int t, int* out4);
gp_status kmvm_tc_debug(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                        float* W, int64_t ldw, const int* gate, float* dbg, int mode,
                        cudaStream_t st);

// ---- tensor-core gradient contraction (grad_tc.cu) ---------------------------------
// The contraction of contract_simt (lengthscale and output-scale entries) for the
// mixed precision on tcgen05 tensor cores; the noise entry comes from contract_noise.
struct TcGradBufs {
  void* pack;        // tc_grad_bytes(n, d, t): M operand tiles A', B' and coordinate tiles
  double* part;      // tc_grad_part_elems(): per-CTA partial sums
  int* cmax;         // 2 x 64: column maxima of |A| and |B|
  float* mscale;     // 2 x 64: power-of-two column scales of A' and B'
  double* inv2E;     // 1
};
bool tc_grad_supported(const Prob& pb, int t);
size_t tc_grad_bytes(int64_t n, int d, int t);
size_t tc_grad_part_elems();
// coordinate tiles of the scaled inputs (once per evaluation)
gp_status tc_grad_prepare(const Prob& pb, const void* Xs, const TcGradBufs& gb, int t,
                          cudaStream_t st);
// gout[0 .. D] (lengthscales, output scale); tb holds the packed exponent operands
gp_status contract_tc(const Prob& pb, const void* Xs, const TcBufs& tb, const TcGradBufs& gb,
                      const float* A, int64_t lda, const float* B, int64_t ldb,
                      const double* wts, int t, double* gout, cudaStream_t st);
// gout = sum_a sum_c w_c A[a,c] B[a,c]  (the noise entry: dK_hat/dsigma^2 = I)
template <class T>
gp_status contract_noise(const Prob& pb, const void* A, int64_t lda, const void* B, int64_t ldb,
                         const double* wts, int t, double* part, unsigned* counter, double* gout,
                         cudaStream_t st);

// ---- pivoted Cholesky (pivchol.cu) ----------------------------------------------
struct PivBufs {
  double* dres;      // n: residual diagonal, -1 marks chosen rows
  double* pval;      // per block best value
  int* pidx;         // per block best index
  double* psum;      // per block residual sum
  double* dval;      // k + 1: residual diagonal of each pivot
  double* trace0;    // 2: tr K and max_i K_ii of the initial diagonal
  int* stop;         // 1
  unsigned* counter; // 1
};
constexpr int kPivBlocks = 304;
template <class T>
gp_status pivchol_run(const Prob& pb, const void* Xs, int k, double tol, const int* piv_override,
                      void* L, int64_t ldl, int* piv, int* rank, const PivBufs& b, cudaStream_t st);

// ---- small dense FP64 linear algebra and tall-skinny products (linalg.cu) ----------
constexpr int kAtbRows = 1024;   // rows per chunk of a tall-skinny A^T B
int64_t atb_chunks(int64_t n);
// part[ch][i][j] = sum_{rows in chunk ch} A[r, i] B[r, j]  (A, B column-major);
// out[i][j] = sum_ch part (row-major ka x kb, double).
template <class T>
gp_status atb(int64_t n, const void* A, int64_t lda, int ka, const void* B, int64_t ldb, int kb,
              double* part, double* out, cudaStream_t st);
// C = s2 I + G (k x k), Cholesky in place (lower, row-major), logdet -> *logdet_out
// (adds (n - k) log s2 when n_for_logdet > 0), status word set to GP_ERR_NOT_SPD on failure.
gp_status woodbury_core(int k, const double* G, const double* theta, int D, int64_t n,
                        double* C, double* Cinv, double* work, double* logdetP, int* status,
                        cudaStream_t st);
gp_status tri_inv_lower(int k, const double* Lm, double* Linv, cudaStream_t st);
// C = op(A) op(B), row-major; ta/tb transpose flags; A is (ta ? kk x m : m x kk) etc.
gp_status gemm64(int m, int nn, int kk, const double* A, int ta, const double* B, int tb,
                 double* C, double alpha, double beta, cudaStream_t st);

// ---- CG (cg.cu) ----------------------------------------------------------------------
template <class T>
struct CgBufs {
  T *X, *R, *Z, *P, *Q;      // n x t, ld n
  T* Sp;                     // k x t: C^-1 L^T R
  double* atb_part;          // cg_atb_part_elems(n, k, t): block partials of L^T R
  double* S;                 // k x t
  double* rho;               // t
  double* rho0;              // t
  double* bnorm2;            // t
  double* alpha;             // t x max_iter
  double* beta;              // t x max_iter
  double* part;              // cg_part_elems(n, t): per-block column partials
  int* active;               // t
  int* caps;                 // t
  int* iters;                // t
  int* n_active;             // 1
  int* status;               // 1
  unsigned* counter;         // 1
  int* ctl;                  // 4: device loop control (iteration j, recompute flag and gate)
};
constexpr int kCgBlocks = 1216;   // 8 per SM: short per-lane loops in the column reductions
size_t cg_atb_part_elems(int64_t n, int k, int t);
size_t cg_part_elems(int64_t n, int t);
// Matrix-vector product used by CG: W = K_hat V on all t columns; `gate` (device
// int, may be null) lets the product return immediately when it reads 0.
struct MvmOp {
  virtual gp_status apply(const void* V, int64_t ldv, int t, void* W, int64_t ldw,
                          const int* gate, cudaStream_t st) = 0;
  virtual ~MvmOp() {}
};
// Optional CUDA-event timing of the products issued by cg_solve.
// Phase 0: kernel-matrix products; phase 1: the gradient contraction.
bool mvm_timing_enabled();
void mvm_timing_begin(cudaStream_t st, int phase = 0);
void mvm_timing_end(cudaStream_t st, int phase = 0);
template <class T>
gp_status cg_solve(const Prob& pb, MvmOp& mvm, const T* L, int64_t ldl, int k,
                   const double* Cinv, const T* B, int64_t ldb, int t,
                   const int* iters_override, const gp_opts& o, const CgBufs<T>& cb,
                   T* PinvB, int64_t ldpb, int* host_status, cudaStream_t st);
template <class T>
gp_status cg_tridiag(int t, int max_iter, const CgBufs<T>& cb, double* T_diag, double* T_off,
                     cudaStream_t st);

// ---- Lanczos quadrature (lanczos.cu) ----------------------------------------------
// gamma[i] = rho0[c] e1^T log(T_c) e1 for columns c = c0 + i, i < count.
gp_status lanczos_logquad(int count, int c0, int max_iter, const double* alpha,
                          const double* beta, const int* iters, const double* rho0,
                          double* gamma, int* status, cudaStream_t st);

// ---- probes (probes.cu) --------------------------------------------------------------
template <class T>
gp_status make_rhs(const Prob& pb, const T* y, const T* L, int64_t ldl, int k, int n_probes,
                   uint64_t seed, const int8_t* eps_override, T* B, int64_t ldb, cudaStream_t st);
gp_status rademacher_fill(uint64_t seed, int stream_id, int64_t rows, int cols, int8_t* out,
                          cudaStream_t st);

// ---- preconditioner derivative terms (precond.cu) ---------------------------------------
struct PrecBufs {
  double* Q;        // k x k + l x k reals in the problem precision (transposed A1, Cv)
  double* dW;       // (p-1) x k x k: dK/dtheta_q at pivot pairs
  double* Lpi;      // k x k
  double* Lpinv;    // k x k
  double* A1;       // k x k
  double* B1;       // k x k
  double* tmp;      // k x k
  double* LtW;      // k x l (+ scratch for ||w||^2)
  double* Cv;       // k x l (+ 2 (kMaxD + 1) for the E / F sums)
  double* part;     // 2 n k reals in the problem precision: Z1 = L A1^T, Z2 = W Cv^T
  double* dkpart;   // max(atb partials of L^T W, per-block E / F partials)
};
// Random Fourier feature preconditioner: m frequencies u_j = rho_j eps_j (U, m x d FP64)
// from the standard-normal draws eps (m x d, row-major) and the Gamma draws g (m; unused
// for the RBF), and the n x 2m feature matrix Phi (ld ldp) in the problem precision.
// Or a deterministic weighted set (hostU: m x d frequencies, hostW: m weights, host
// memory; the quadrature features of qff_table), copied to the device.
struct FeatSpec {
  int m;
  const double* eps;
  const double* g;
  const double* hostU;
  const double* hostW;
};
template <class T>
gp_status rff_build(const Prob& pb, const void* Xs, const FeatSpec& f, double* U, double* wt,
                    T* Phi, int64_t ldp, cudaStream_t st);
// trP and probeP of P_hat = sigma^2 I + Phi Phi^T (dP_hat at frozen frequencies).
template <class T>
gp_status feature_terms(const Prob& pb, const void* Xs, const T* Phi, int64_t ldp, int m,
                        const double* U, const double* wt, const T* W, int64_t ldw,
                        int n_probes, const double* Cinv, const PrecBufs& b, double* trP,
                        double* probeP, cudaStream_t st);
// Gauss-Hermite rule (weight exp(-t^2)) of mbar nodes, and the folded d-dimensional grid
// of the quadrature Fourier features (m = mbar^d / 2 frequencies, weights summing to 1).
void hermite_rule(int mbar, std::vector<double>& t, std::vector<double>& w);
void qff_table(int mbar, int d, std::vector<double>& U, std::vector<double>& W);
template <class T>
gp_status precond_terms(const Prob& pb, const void* Xs, const T* L, int64_t ldl, int k,
                        const int* piv, const int* rank, const T* W, int64_t ldw, int n_probes,
                        const double* Cinv, const PrecBufs& b, double* trP, double* probeP,
                        cudaStream_t st);

// ---- small reductions (cg.cu) -------------------------------------------------------
template <class T>
gp_status dot_into(int64_t n, const T* a, const T* b, double* part, unsigned* counter,
                   double* out, cudaStream_t st);

}  // namespace gp
