// Tensor-core (tcgen05 / TMEM) kernel-matrix product for the BF16 precision:
//   W = (K + sigma^2 I) V,  computed tile by tile like fused attention without the
//   softmax normalisation (K is never stored):
//
//   GEMM1  S = A_I B_J^T          (128 x 128 per tile, FP32 in TMEM)
//          A_i = [c x_i, 1, -c |x_i|^2 / 2],  B_j = [x_j, -c |x_j|^2 / 2, 1]
//          so S_ij = c (x_i . x_j - |x_i|^2/2 - |x_j|^2/2) = -c r_ij^2 / 2.
//          RBF: c = log2(e)  ->  k_ij / s = 2^S_ij.
//          Matern: c = 1     ->  r = sqrt(-2 S), k / s = poly(r) e^{-a r}.
//          Each operand is split into BF16 hi + lo parts and the product is formed as
//          hi.hi + hi.lo + lo.hi, which keeps ~16 significant bits in S despite the
//          cancellation between the norms and the dot product.  Split mode (below) uses
//          a three-part split hi + mid + lo and the six products of total order <= 2
//          (~24 bits): on inputs with large norms (|x|^2 ~ 30) the 16-bit form
//          perturbs K by |dK|_2 ~ 1e-6 n, which exceeds sigma^2 = 0.1 at n = 5e5.
//   epilogue  P = k(S) / s in [0, 1], FP32 in registers, rounded to FP16 (11
//          significant bits) and written to one of two 64-column TMEM P buffers (two
//          FP16 values per column), so the S buffer is free for the next GEMM1 as soon
//          as it has been read; tcgen05.ld / tcgen05.st, one thread per row.
//   GEMM2  O_I += P [V_hi | V_lo]   (A = P from TMEM, B = the FP16 hi and lo parts of
//          the V tile in shared memory, N = 2 tp).  Each column c of V is scaled by a
//          power of two 2^e_c that puts max |V_c| in [2^13, 2^14), so both parts stay
//          in FP16's normal range; W = s 2^-e_c (O_hi + O_lo) + sigma^2 V.
//          Accuracy: the FP16 rounding of P perturbs K by E with |E_ij| <= 2^-11 K_ij;
//          for the n = 1e5 RBF workload |E|_2 is a fraction of sigma^2, so CG stays on a
//          positive-definite operator.  BF16 P (2^-8) is not enough: |E|_2 exceeds
//          sigma^2 and CG breaks down (p^T K p <= 0).
//   split mode (a device flag, read at launch): for smooth, ill-conditioned kernels
//          (lambda_max(K) / sigma^2 large) even FP16 P can make K + sigma^2 I
//          indefinite.  Then P is carried as FP16 P_hi + P_lo (22 bits) and GEMM2 also
//          adds P_lo [V_hi | V_lo] into O (so O_hi + O_lo = (P_hi + P_lo)(V_hi + V_lo)):
//          16 MMAs per tile, one 128-column P buffer instead of two of 64.
//   tp = t rounded up to a multiple of 8 (N = 2 tp is then a multiple of 16, as an
//          M = 128 MMA requires): t = 33 gives N = 80.
//
// Roles of a CTA (persistent over (row tile, column chunk) work units):
//   warp 0      producer: bulk TMA copies (cp.async.bulk) of the pre-tiled A and B tiles
//   warp 1      producer of the V tiles for GEMM2 (warp 0 loads A and the B tiles)
//   warp 2      issues GEMM2 of every tile
//   warp 19     TMEM allocator; issues GEMM1 of every tile (two issuing warps, so the
//               wait / fence / commit latencies of the two GEMMs overlap instead of
//               adding up; placing the GEMM1 issuer on the fourth scheduler, next to
//               the epilogue warps of TMEM lanes 96-127, measured 3-4% faster than
//               on the second)
//   warps 3-18  epilogue: two teams of eight warps on alternate tiles; warp w reads
//               TMEM lanes 32 (w % 4) .. + 31 and 64 S columns of its team's tiles
// Synchronisation uses mbarriers; every wait gives up after a time limit, sets an
// abort flag and an error code, and the CTA drains its own copies and MMAs (again
// with a limit) before freeing TMEM and returning.
//
// Operands are laid out in HBM by the pack kernels below in the canonical
// no-swizzle K-major UMMA layout: 8-row x 16-byte core matrices, core matrices
// adjacent along K 128 bytes apart (leading byte offset), 8-row groups
// (K/8) * 128 bytes apart (stride byte offset).  Each 128-row tile is one
// contiguous block, so one bulk copy moves it.
#include "ops.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <map>
#include <mutex>
#include <vector>

namespace gp {
namespace {

using namespace tcx;

constexpr int BM = 128;        // rows per tile (MMA M)
constexpr int BN = 128;        // columns per tile (GEMM1 N, GEMM2 K)
constexpr int kMaxStages = 4;   // per operand ring (B tiles for GEMM1, V tiles for GEMM2)
constexpr int kThreads = 640;  // 20 warps
constexpr int kEpiWarp0 = 3;   // first epilogue warp (warps 3 .. 18)
constexpr int kVWarp = 1;      // producer of the V ring
constexpr int kG1Warp = 19;    // GEMM1 issuer (and TMEM allocator)
constexpr int kSBuf = 2;       // FP32 S buffers in TMEM (128 columns each)
constexpr int kPBuf = 2;       // FP16 P buffers in TMEM (64 columns each; split mode: one
                               // buffer of 128, P_hi then P_lo)
constexpr int kEpiWarps = 16;

struct TcArgs {
  const __nv_bfloat16* xa;   // ntiles tiles of BM x kx (A form, two-part split)
  const __nv_bfloat16* xb;   // ntiles tiles of BN x kx (B form)
  const __nv_bfloat16* xa3;  // the same with the three-part split (split mode), kx3 wide
  const __nv_bfloat16* xb3;
  const __half* vp;          // ntiles tiles of 2 tp x BN (FP16 hi and lo parts)
  float* part;               // nchunks x tp x npad
  int n, npad, ntiles, nchunks, tiles_per_chunk, kx, kx3, tp, t, kind, D;
  int kx3_ok;                // shared memory fits the three-part operands
  int nsb, nsv;              // shared-memory stages of the B and V rings (2 .. 4)
  const int* gate;
  int* err;                  // err[0] = status, err[1] = where a wait gave up,
                             // err[2] = split mode (P as FP16 hi + lo) when nonzero
  float* dbg;                // optional: S of the first tile of unit 0
};

struct __align__(8) Bars {
  unsigned long long fullB[kMaxStages], emptyB[kMaxStages], fullV[kMaxStages], emptyV[kMaxStages];
  unsigned long long a_full, a_free, s_full[kSBuf], s_free[kSBuf], p_ready[kPBuf], p_free[kPBuf],
      o_full, o_free,
      drain1, drain2;
  unsigned int tmem_base;
  int abort;
};

// k(r) / s from the exponent tile value S (see the header).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KIND>
__device__ __forceinline__ float kernel_from_s(float sv) {
  if (KIND == GP_RBF) return ex2(sv);
  // rational quadratic (alpha = 1): 1 / (1 + r^2/2) = 1 / (1 - S), S <= 0
  if (KIND == GP_RATQUAD) return rcp_approx(1.0f - fminf(sv, 0.0f));
  const float r2 = fmaxf(-2.0f * sv, 0.0f);
  const float r = sqrtf(r2);
  const float L2E = 1.4426950408889634f;
  if (KIND == GP_MATERN32) {
    const float ar = 1.7320508075688772f * r;
    return (1.0f + ar) * ex2(-ar * L2E);
  }
  const float ar = 2.23606797749979f * r;
  return (1.0f + ar + 1.6666666666666667f * r2) * ex2(-ar * L2E);
}

// P = k(S)/s for this thread's 32 S values, packed as 16 FP16 pairs; in split mode
// also the FP16 residuals P - P_hi.
template <int KIND>
__device__ __forceinline__ void p_from_s(const uint32_t (&v)[32], uint32_t (&pk)[16],
                                         uint32_t (&pl)[16], bool split) {
  if (!split) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      pk[q] = pack_f16(kernel_from_s<KIND>(__uint_as_float(v[2 * q])),
                       kernel_from_s<KIND>(__uint_as_float(v[2 * q + 1])));
    return;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float p0 = kernel_from_s<KIND>(__uint_as_float(v[2 * q]));
    const float p1 = kernel_from_s<KIND>(__uint_as_float(v[2 * q + 1]));
    const uint32_t h = pack_f16(p0, p1);
    pk[q] = h;
    const __half2 hh = *reinterpret_cast<const __half2*>(&h);
    pl[q] = pack_f16(p0 - __low2float(hh), p1 - __high2float(hh));
  }
}


// kMaySplit = false: the split flag is known to be off (mode 0), and split mode's code
// is compiled out, which keeps the fast form's registers free of it.
template <bool kMaySplit>
__global__ void __launch_bounds__(kThreads, 1) kmvm_tc_kernel(TcArgs g) {
  if (g.gate && *g.gate == 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool split = kMaySplit && g.err[2] != 0;
  // split mode: the three-part exponent operands, when the launch's shared memory was
  // sized for them (always, unless the host knew the flag was off or the shape is too
  // wide for them)
  const bool wide = split && g.kx3_ok;
  const int kx = wide ? g.kx3 : g.kx, tp = g.tp, nsb = g.nsb, nsv = g.nsv;
  const __nv_bfloat16* xa = wide ? g.xa3 : g.xa;
  const __nv_bfloat16* xb = wide ? g.xb3 : g.xb;
  const uint32_t npb = split ? 1u : (uint32_t)kPBuf;   // P buffers in the ring
  const uint32_t a_bytes = BM * kx * 2, b_bytes = BN * kx * 2;
  const uint32_t v_bytes = 2u * tp * BN * 2;   // FP16 hi and lo parts of V
  unsigned char* sA = smem;
  unsigned char* sB = sA + a_bytes;
  unsigned char* sV = sB + nsb * b_bytes;
  Bars* bars = reinterpret_cast<Bars*>(sV + nsv * v_bytes);
  volatile int* abort = &bars->abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(smem_u32(&bars->fullB[s]), 1);
      mbar_init(smem_u32(&bars->emptyB[s]), 1);
      mbar_init(smem_u32(&bars->fullV[s]), 1);
      mbar_init(smem_u32(&bars->emptyV[s]), 1);
    }
    mbar_init(smem_u32(&bars->a_full), 1);
    mbar_init(smem_u32(&bars->a_free), 1);
    for (int b = 0; b < kSBuf; ++b) {
      mbar_init(smem_u32(&bars->s_full[b]), 1);            // GEMM1 commit
      mbar_init(smem_u32(&bars->s_free[b]), kEpiWarps / 2);   // each warp of the team read S
    }
    for (int b = 0; b < kPBuf; ++b) {
      mbar_init(smem_u32(&bars->p_ready[b]), kEpiWarps / 2);  // each warp of the team wrote P
      mbar_init(smem_u32(&bars->p_free[b]), 1);            // GEMM2 commit
    }
    mbar_init(smem_u32(&bars->o_full), 1);
    mbar_init(smem_u32(&bars->o_free), BM);
    mbar_init(smem_u32(&bars->drain1), 1);
    mbar_init(smem_u32(&bars->drain2), 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kG1Warp) {
    tmem_alloc(smem_u32(&bars->tmem_base), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  // TMEM columns: FP32 S buffers b at 128 b (b < 2), FP16 P buffers b at 256 + 64 b
  // (b < 2; epilogue group g writes columns 16 g .. 16 g + 15, the packed pairs of
  // its 32 S columns), O accumulator at 384 (2 tp <= 128 columns).  S is released as
  // soon as the epilogue has read it, P once GEMM2 has consumed it.
  const uint32_t t_o = tmem + 384;
  const int nunits = g.ntiles * g.nchunks;

  if (warp == 0 || warp == kVWarp) {
    // ------------------------------------------------------------ producers
    // warp 0: the row tile A of each unit and the B ring (freed by GEMM1);
    // warp 1: the V ring (freed by GEMM2).  Separate warps, so neither producer's
    // wait holds up the other, and B tiles are fetched as early as GEMM1 allows.
    if (lane == 0) {
      const bool is_b = warp == 0;
      const int ns = is_b ? nsb : nsv;
      const uint32_t bytes = is_b ? b_bytes : v_bytes;
      unsigned char* sbase = is_b ? sB : sV;
      const unsigned char* gsrc = is_b ? reinterpret_cast<const unsigned char*>(xb)
                                       : reinterpret_cast<const unsigned char*>(g.vp);
      unsigned long long* fullr = is_b ? bars->fullB : bars->fullV;
      unsigned long long* emptyr = is_b ? bars->emptyB : bars->emptyV;
      uint32_t a_par = 0, a_arms = 0;
      Ring sr{0, 0};
      int armed[kMaxStages] = {0, 0, 0, 0};
      uint32_t arm_par[kMaxStages] = {0, 0, 0, 0};
      bool first = true;
      for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x) {
        const int rt = u / g.nchunks, ch = u % g.nchunks;
        const int j0 = ch * g.tiles_per_chunk;
        const int j1 = min(g.ntiles, j0 + g.tiles_per_chunk);
        if (is_b) {
          if (!first && !mbar_wait(smem_u32(&bars->a_free), a_par, abort, g.err, 11)) break;
          if (!first) a_par ^= 1;
          first = false;
          mbar_expect_tx(smem_u32(&bars->a_full), a_bytes);
          bulk_g2s(smem_u32(sA),
                   reinterpret_cast<const unsigned char*>(xa) + (size_t)rt * a_bytes, a_bytes,
                   smem_u32(&bars->a_full));
          ++a_arms;
        }
        bool ok = true;
        for (int j = j0; j < j1; ++j) {
          const uint32_t st = sr.idx, ph = sr.phase;
          if (!mbar_wait(smem_u32(&emptyr[st]), ph ^ 1, abort, g.err, 12)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&fullr[st]);
          mbar_expect_tx(fb, bytes);
          bulk_g2s(smem_u32(sbase + st * bytes), gsrc + (size_t)j * bytes, bytes, fb);
          armed[st] = 1;
          arm_par[st] = ph;
          sr.next(ns);
        }
        if (!ok) break;
      }
      if (*abort) {
        // drain: every copy this thread issued must land before the CTA exits
        for (int st = 0; st < ns; ++st) {
          if (!armed[st]) continue;
          const unsigned long long t0 = gtime();
          while (!mbar_try_wait(smem_u32(&fullr[st]), arm_par[st]) &&
                 gtime() - t0 < (unsigned long long)kWaitNs) {
          }
        }
        if (a_arms > 0) {
          const unsigned long long t0 = gtime();
          while (!mbar_try_wait(smem_u32(&bars->a_full), (a_arms - 1) & 1) &&
                 gtime() - t0 < (unsigned long long)kWaitNs) {
          }
        }
      }
    }
  } else if (warp == kG1Warp) {
    // ------------------------------------------------------------ GEMM1 issuer (whole
    // warp; waits are polled by every lane, MMAs issued by one elected lane)
    const uint32_t id1 = idesc_bf16(BM, BN);
    const int nk1 = kx / 16;
    // descriptors of stage 0; a K-step of 16 elements (256 bytes) adds 16 to the
    // encoded start address, a stage adds its byte size >> 4
    const uint64_t dA = sdesc(smem_u32(sA), 128, (uint32_t)kx * 16);
    const uint64_t dB0 = sdesc(smem_u32(sB), 128, (uint32_t)kx * 16);
    const uint64_t b_step = b_bytes >> 4;
    uint32_t a_par = 0;
    Ring sr{0, 0}, br{0, 0};   // smem stage ring, TMEM S-buffer ring
    for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x) {
      const int ch = u % g.nchunks;
      const int j0 = ch * g.tiles_per_chunk;
      const int nt = min(g.ntiles, j0 + g.tiles_per_chunk) - j0;
      if (!mbar_wait(smem_u32(&bars->a_full), a_par, abort, g.err, 21)) break;
      a_par ^= 1;
      bool ok = true;
      for (int jj = 0; jj < nt; ++jj) {
        const uint32_t st = sr.idx, buf = br.idx;
        if (!mbar_wait(smem_u32(&bars->fullB[st]), sr.phase, abort, g.err, 22) ||
            !mbar_wait(smem_u32(&bars->s_free[buf]), br.phase ^ 1, abort, g.err, 23)) {
          ok = false;
          break;
        }
        __syncwarp();
        tc_fence_after();
        const uint64_t db = dB0 + st * b_step;
        const uint32_t ts = tmem + buf * 128;
        for (int q = 0; q < nk1; ++q)   // kx / 16 K steps (4 .. 13)
          mma_ss(ts, dA + (uint64_t)q * 16, db + (uint64_t)q * 16, id1, q > 0 ? 1u : 0u);
        mma_commit(smem_u32(&bars->s_full[buf]));
        mma_commit(smem_u32(&bars->emptyB[st]));
        if (jj == nt - 1) mma_commit(smem_u32(&bars->a_free));
        sr.next(nsb);
        br.next(kSBuf);
      }
      if (!ok) break;
    }
    // drain: a final commit completes once every MMA this warp issued is done
    __syncwarp();
    mma_commit(smem_u32(&bars->drain1));
    const unsigned long long t0 = gtime();
    while (!mbar_try_wait(smem_u32(&bars->drain1), 0) &&
           gtime() - t0 < (unsigned long long)kWaitNs) {
    }
  } else if (warp == 2) {
    // ------------------------------------------------------------ GEMM2 issuer
    const uint32_t id2 = idesc_f16(BM, 2 * tp);   // B = [V_hi; V_lo], N = 2 tp
    uint32_t t2 = 0;                              // tiles issued (p_free is per tile parity)
    const uint64_t dV0 = sdesc(smem_u32(sV), 128, BN * 16);
    const uint64_t v_step = v_bytes >> 4;
    uint32_t o_par = 0;
    Ring sr{0, 0}, br{0, 0};
    bool first_unit = true;
    for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x) {
      const int ch = u % g.nchunks;
      const int j0 = ch * g.tiles_per_chunk;
      const int nt = min(g.ntiles, j0 + g.tiles_per_chunk) - j0;
      bool ok = true;
      for (int jj = 0; jj < nt; ++jj) {
        const uint32_t st = sr.idx, buf = br.idx;   // br: ring of P buffers here
        if (!mbar_wait(smem_u32(&bars->fullV[st]), sr.phase, abort, g.err, 26) ||
            !mbar_wait(smem_u32(&bars->p_ready[buf]), br.phase, abort, g.err, 24)) {
          ok = false;
          break;
        }
        // O is overwritten by this unit's first product: wait until the epilogue
        // has read the previous unit's O
        if (jj == 0 && !first_unit) {
          if (!mbar_wait(smem_u32(&bars->o_free), o_par, abort, g.err, 25)) {
            ok = false;
            break;
          }
          o_par ^= 1;
        }
        __syncwarp();
        tc_fence_after();
        // K elements 16 kk .. 16 kk + 15: FP16 P in TMEM columns 8 kk .. 8 kk + 7 of the
        // P buffer.  P [V_hi | V_lo] goes into O columns [0, tp) and [tp, 2 tp): the hi
        // and lo parts of the V tile are adjacent 8-row groups, so one descriptor with
        // N = 2 tp covers both.
        const uint64_t dv = dV0 + st * v_step;
        const uint32_t tpb = tmem + 256 + buf * 64;
        const uint32_t acc0 = jj > 0 ? 1u : 0u;
#pragma unroll
        for (int kk = 0; kk < BN / 16; ++kk)
          mma_ts(t_o, tpb + kk * 8, dv + (uint64_t)kk * 16, id2, (kk > 0) ? 1u : acc0);
        if (split) {   // P_lo [V_hi | V_lo] into the same O columns
#pragma unroll
          for (int kk = 0; kk < BN / 16; ++kk)
            mma_ts(t_o, tpb + 64 + kk * 8, dv + (uint64_t)kk * 16, id2, 1u);
        }
        mma_commit(smem_u32(&bars->emptyV[st]));
        mma_commit(smem_u32(&bars->p_free[t2 & 1u]));
        ++t2;
        if (jj == nt - 1) mma_commit(smem_u32(&bars->o_full));
        sr.next(nsv);
        br.next(npb);
      }
      first_unit = false;
      if (!ok) break;
    }
    __syncwarp();
    mma_commit(smem_u32(&bars->drain2));
    const unsigned long long t0 = gtime();
    while (!mbar_try_wait(smem_u32(&bars->drain2), 0) &&
           gtime() - t0 < (unsigned long long)kWaitNs) {
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    // (warps kEpiWarp0 .. kEpiWarp0 + 15) in two teams of eight that take alternate
    // tiles: team 0 the even tiles of the CTA's tile sequence (S buffer 0), team 1 the
    // odd ones (S buffer 1).  Each warp owns one TMEM lane quarter (its scheduler's)
    // and 64 columns of its team's tiles, processed as two chunks of 32.  With two
    // tiles in flight, one team's TMEM loads / stores and barrier waits overlap the
    // other team's exponentials, which keep the MUFU pipe busy.
    const int e = warp - kEpiWarp0;
    const int team = e >> 3;
    const int half = (e >> 2) & 1;                // columns 64 half .. 64 half + 63
    const int quarter = warp & 3;                 // TMEM lane quarter of this warp
    const int row = quarter * 32 + lane;          // row within the tile
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t sbuf = (uint32_t)team;         // tile t uses S buffer t % 2
    uint32_t of_par = 0, gt = 0, mine = 0;        // CTA tile count, this team's count
    for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x) {
      const int rt = u / g.nchunks, ch = u % g.nchunks;
      const int j0 = ch * g.tiles_per_chunk;
      const int j1 = min(g.ntiles, j0 + g.tiles_per_chunk);
      bool ok = true;
      for (int j = j0; j < j1; ++j, ++gt) {
        if ((gt & 1u) != (uint32_t)team) continue;
        if (!mbar_wait(smem_u32(&bars->s_full[sbuf]), mine & 1u, abort, g.err, 31)) {
          ok = false;
          break;
        }
        const uint32_t k = mine++;                // this team's tile index
        tc_fence_after();
        // P buffer of this tile and the GEMM2 that must have completed before it is
        // rewritten.  p_free[b] completes once per GEMM2 of a tile of parity b, i.e. of
        // team b's tiles, so every wait below stays within one phase of its barrier
        // (a parity wait cannot tell phases two apart).
        //   fast mode (two P buffers): buffer `team`, free after GEMM2 of the team's
        //     previous tile: phase k - 1 of p_free[team];
        //   split mode (one P buffer): free after GEMM2 of the previous tile, i.e. of
        //     the other team's latest tile: phase k - 1 (team 0) or k (team 1) of
        //     p_free[1 - team].
        const uint32_t pb = split ? 0u : sbuf;
        const uint32_t fb = split ? 1u - sbuf : sbuf;
        const bool wait_p = (split && team == 1) || k >= 1;
        const uint32_t p_par = (split && team == 1) ? (k & 1u) : ((k - 1u) & 1u);
        if (!split) {
          // fast mode: both 32-column chunks are loaded first, so the S buffer goes back
          // to GEMM1 before any exponential, and one store wait covers both chunks
          uint32_t v0[32], v1[32];
          GP_TMEM_LD32(tmem + sbuf * 128 + lane_off + half * 64, v0);
          GP_TMEM_LD32(tmem + sbuf * 128 + lane_off + half * 64 + 32, v1);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars->s_free[sbuf]));
          if (g.dbg && u == (int)blockIdx.x && blockIdx.x == 0 && j == j0) {
            for (int q = 0; q < 32; ++q) {
              g.dbg[row * BN + half * 64 + q] = __uint_as_float(v0[q]);
              g.dbg[row * BN + half * 64 + 32 + q] = __uint_as_float(v1[q]);
            }
          }
          uint32_t pk0[16], pk1[16];
          if (g.kind == GP_RBF) p_from_s<GP_RBF>(v0, pk0, pk0, false);
          else if (g.kind == GP_MATERN32) p_from_s<GP_MATERN32>(v0, pk0, pk0, false);
          else if (g.kind == GP_RATQUAD) p_from_s<GP_RATQUAD>(v0, pk0, pk0, false);
          else p_from_s<GP_MATERN52>(v0, pk0, pk0, false);
          if (wait_p && !mbar_wait(smem_u32(&bars->p_free[fb]), p_par, abort, g.err, 33)) {
            ok = false;
            break;
          }
          tc_fence_after();
          GP_TMEM_ST16(tmem + 256 + pb * 64 + lane_off + half * 32, pk0);
          if (g.kind == GP_RBF) p_from_s<GP_RBF>(v1, pk1, pk1, false);
          else if (g.kind == GP_MATERN32) p_from_s<GP_MATERN32>(v1, pk1, pk1, false);
          else if (g.kind == GP_RATQUAD) p_from_s<GP_RATQUAD>(v1, pk1, pk1, false);
          else p_from_s<GP_MATERN52>(v1, pk1, pk1, false);
          GP_TMEM_ST16(tmem + 256 + pb * 64 + lane_off + half * 32 + 16, pk1);
          // tcgen05.st reads its source registers asynchronously
          tmem_wait_st();
        }
        if (split) {
          // split mode, in the same order: both chunks loaded, the S buffer returned to
          // GEMM1 before any exponential; each chunk's P_hi and P_lo stored as soon as
          // they are formed (the second chunk reuses the first one's registers only
          // after its stores have completed)
          uint32_t v0[32], v1[32];
          GP_TMEM_LD32(tmem + sbuf * 128 + lane_off + half * 64, v0);
          GP_TMEM_LD32(tmem + sbuf * 128 + lane_off + half * 64 + 32, v1);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars->s_free[sbuf]));
          if (g.dbg && u == (int)blockIdx.x && blockIdx.x == 0 && j == j0) {
            for (int q = 0; q < 32; ++q) {
              g.dbg[row * BN + half * 64 + q] = __uint_as_float(v0[q]);
              g.dbg[row * BN + half * 64 + 32 + q] = __uint_as_float(v1[q]);
            }
          }
          uint32_t pk[16], pl[16];
          if (g.kind == GP_RBF) p_from_s<GP_RBF>(v0, pk, pl, true);
          else if (g.kind == GP_MATERN32) p_from_s<GP_MATERN32>(v0, pk, pl, true);
          else if (g.kind == GP_RATQUAD) p_from_s<GP_RATQUAD>(v0, pk, pl, true);
          else p_from_s<GP_MATERN52>(v0, pk, pl, true);
          if (wait_p && !mbar_wait(smem_u32(&bars->p_free[fb]), p_par, abort, g.err, 33)) {
            ok = false;
            break;
          }
          tc_fence_after();
          GP_TMEM_ST16(tmem + 256 + pb * 64 + lane_off + half * 32, pk);
          GP_TMEM_ST16(tmem + 256 + 64 + lane_off + half * 32, pl);
          tmem_wait_st();          // pk / pl are reused below
          if (g.kind == GP_RBF) p_from_s<GP_RBF>(v1, pk, pl, true);
          else if (g.kind == GP_MATERN32) p_from_s<GP_MATERN32>(v1, pk, pl, true);
          else if (g.kind == GP_RATQUAD) p_from_s<GP_RATQUAD>(v1, pk, pl, true);
          else p_from_s<GP_MATERN52>(v1, pk, pl, true);
          GP_TMEM_ST16(tmem + 256 + pb * 64 + lane_off + half * 32 + 16, pk);
          GP_TMEM_ST16(tmem + 256 + 64 + lane_off + half * 32 + 16, pl);
          tmem_wait_st();
        }
        if (!ok) break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->p_ready[pb]));
      }
      if (!ok) break;
      if (e >= 4) continue;
      // the unit's product is complete: O -> partial output (warps kEpiWarp0 .. + 3,
      // one per lane quarter)
      if (!mbar_wait(smem_u32(&bars->o_full), of_par, abort, g.err, 32)) break;
      of_par ^= 1;
      tc_fence_after();
      const int grow = rt * BM + row;
      float* dst = g.part + (size_t)ch * tp * g.npad;
#pragma unroll 1
      for (int c0 = 0; c0 < tp; c0 += 16) {
        // O = columns [0, tp) (V_hi) + [tp, 2 tp) (V_lo); when tp is an odd multiple
        // of 8 the last 16-column load runs past tp (at most to column 2 tp + 7 <= 119
        // of O, inside the allocation) and the columns >= t are not stored
        uint32_t v[16], w[16];
        GP_TMEM_LD16(t_o + lane_off + c0, v);
        GP_TMEM_LD16(t_o + lane_off + tp + c0, w);
        tmem_wait_ld();
        if (grow < g.n) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float o = __uint_as_float(v[q]) + __uint_as_float(w[q]);
            if (c0 + q < g.t) dst[(size_t)(c0 + q) * g.npad + grow] = o;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&bars->o_free));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kG1Warp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- packing kernels ------------------------------------------------------------------
// Augmented exponent operands in the canonical tile layout:
// A_i = [c x, 1, -c |x|^2/2] ; B_j = [x, -c |x|^2/2, 1], each entry split into BF16
// parts v = p0 + p1 (+ p2), p_m = bf16(v - p_0 - .. - p_{m-1}).  Segments of d + 2
// columns pair the parts whose products are kept:
//   two parts:   (p0, p0), (p0, p1), (p1, p0)                              (~16 bits)
//   three parts: (p0, p0), (p0, p1), (p1, p0), (p0, p2), (p1, p1), (p2, p0)  (~24 bits)
// so that A' . B' = sum of the kept products; zero padded to kx.
__device__ __forceinline__ void bf16_parts(double v, float (&pt)[3]) {
  const float p0 = __bfloat162float(__float2bfloat16_rn((float)v));
  const float p1 = __bfloat162float(__float2bfloat16_rn((float)(v - (double)p0)));
  const float p2 =
      __bfloat162float(__float2bfloat16_rn((float)(v - (double)p0 - (double)p1)));
  pt[0] = p0;
  pt[1] = p1;
  pt[2] = p2;
}

__global__ void pack_x_kernel(int n, int ntiles, int d, int kx, int parts,
                              const float* __restrict__ Xs, int kind,
                              __nv_bfloat16* __restrict__ xa, __nv_bfloat16* __restrict__ xb,
                              float* __restrict__ norms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntiles * BM) return;
  const double c = (kind == GP_RBF) ? 1.4426950408889634 : 1.0;
  const int L = d + 2;
  // part of A (first) and of B (second) in each segment
  constexpr int kSegA[6] = {0, 0, 1, 0, 1, 2};
  constexpr int kSegB[6] = {0, 1, 0, 2, 1, 0};
  const int nseg = parts == 3 ? 6 : 3;
  double av[kMaxD + 2], bv[kMaxD + 2];
  double nrm = 0.0;
  const bool valid = i < n;
  for (int q = 0; q < d; ++q) {
    double x = valid ? (double)Xs[(size_t)i * d + q] : 0.0;
    nrm += x * x;
    av[q] = c * x;
    bv[q] = x;
  }
  av[d] = valid ? 1.0 : 0.0;
  av[d + 1] = valid ? -0.5 * c * nrm : 0.0;
  bv[d] = valid ? -0.5 * c * nrm : 0.0;
  bv[d + 1] = valid ? 1.0 : 0.0;
  if (valid && norms) norms[i] = (float)nrm;
  const int tile = i / BM, r = i % BM;
  unsigned char* ta = reinterpret_cast<unsigned char*>(xa) + (size_t)tile * BM * kx * 2;
  unsigned char* tb = reinterpret_cast<unsigned char*>(xb) + (size_t)tile * BN * kx * 2;
  for (int k = 0; k < kx; ++k) {
    float va = 0.f, vb = 0.f;
    const int seg = k / L, q = k % L;
    if (seg < nseg) {
      float pa[3], pb[3];
      bf16_parts(av[q], pa);
      bf16_parts(bv[q], pb);
      va = pa[kSegA[seg]];
      vb = pb[kSegB[seg]];
    }
    *reinterpret_cast<__nv_bfloat16*>(ta + tile_off(r, k, kx)) = __float2bfloat16_rn(va);
    *reinterpret_cast<__nv_bfloat16*>(tb + tile_off(r, k, kx)) = __float2bfloat16_rn(vb);
  }
}

// Power-of-two column scales of V: scale_c = 2^e_c with max_j |V_jc| scale_c in
// [2^13, 2^14) (1 for an all-zero or non-finite column).  vscale[c] = scale_c,
// vscale[kMaxT64 + c] = 1 / scale_c.  Grid (kScaleParts, t): block (b, c) takes the
// maximum over one row range of column c into vscale[2 kMaxT64 + c kScaleParts + b];
// the last block of column c to finish (counter cnt[c], reset by that block) forms
// the scale.
constexpr int kMaxT64 = 64;
constexpr int kScaleParts = 16;
__global__ void colscale_kernel(int n, const float* __restrict__ V, int64_t ldv,
                                float* __restrict__ vscale, unsigned* __restrict__ cnt,
                                const int* gate) {
  if (gate && *gate == 0) return;
  const int c = blockIdx.y, b = blockIdx.x;
  const int per = (n + kScaleParts - 1) / kScaleParts;
  const int r0 = b * per, r1 = min(n, r0 + per);
  float m = 0.f;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) m = fmaxf(m, fabsf(V[i + (int64_t)c * ldv]));
  __shared__ float red[32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    vscale[2 * kMaxT64 + c * kScaleParts + b] = m;
    __threadfence();
    last = atomicAdd(&cnt[c], 1u) == kScaleParts - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const volatile float* parts = vscale + 2 * kMaxT64 + c * kScaleParts;
  float mx = 0.f;
  for (int q = 0; q < kScaleParts; ++q) mx = fmaxf(mx, parts[q]);
  int e = 0;
  if (mx > 0.f && mx <= 3.0e38f) {
    int ex;
    frexpf(mx, &ex);                      // mx = f 2^ex, f in [0.5, 1)
    e = max(-120, min(120, 14 - ex));     // mx 2^e in [2^13, 2^14)
  }
  vscale[c] = ldexpf(1.0f, e);
  vscale[kMaxT64 + c] = ldexpf(1.0f, -e);
  cnt[c] = 0;
}

// V (n x t FP32, column-major) -> tiles of 2 tp x BN FP16: rows [0, tp) the hi parts
// and rows [tp, 2 tp) the lo parts of the scaled columns (rows = columns of V).
__global__ void pack_v_kernel(int n, int ntiles, int t, int tp, const float* __restrict__ V,
                              int64_t ldv, const float* __restrict__ vscale,
                              __half* __restrict__ vp, const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)ntiles * BN * tp;
  if (e >= total) return;
  const int j = (int)(e % ((int64_t)ntiles * BN));
  const int c = (int)(e / ((int64_t)ntiles * BN));
  const float v = (j < n && c < t) ? V[j + (int64_t)c * ldv] * vscale[c] : 0.f;
  const int tile = j / BN, k = j % BN;
  const size_t part = (size_t)tp * BN * 2;
  unsigned char* tv = reinterpret_cast<unsigned char*>(vp) + (size_t)tile * part * 2;
  const __half hi = __float2half_rn(v);
  *reinterpret_cast<__half*>(tv + tile_off(c, k, BN)) = hi;
  *reinterpret_cast<__half*>(tv + part + tile_off(c, k, BN)) = __float2half_rn(v - __half2float(hi));
}

// W = s / scale_c * (sum over chunks) + sigma^2 V (NaN on a device-side abort).  The
// chunk partials are added with Neumaier's compensated summation in FP32 (FP64
// arithmetic runs at 1/64 of the FP32 rate on this part, which made this pass a few
// percent of every product).
__global__ void tc_reduce_kernel(int n, int npad, int t, int tp, int nchunks,
                                 const float* __restrict__ part,
                                 const float* __restrict__ V, int64_t ldv,
                                 const double* __restrict__ theta, int D,
                                 const float* __restrict__ vscale, float* __restrict__ W,
                                 int64_t ldw, const int* gate, const int* err) {
  if (gate && *gate == 0) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * t) return;
  const int c = (int)(e / n), i = (int)(e % n);
  float sum = 0.f, comp = 0.f;
  for (int ch = 0; ch < nchunks; ++ch) {
    const float x = part[((size_t)ch * tp + c) * npad + i];
    const float tsum = __fadd_rn(sum, x);
    comp = __fadd_rn(comp, fabsf(sum) >= fabsf(x) ? __fadd_rn(__fadd_rn(sum, -tsum), x)
                                                   : __fadd_rn(__fadd_rn(x, -tsum), sum));
    sum = tsum;
  }
  const float acc = __fadd_rn(sum, comp) * ((float)theta[D] * vscale[kMaxT64 + c]);
  float w = fmaf((float)theta[D + 1], V[i + (int64_t)c * ldv], acc);
  if (*err) w = __int_as_float(0x7fc00000);
  W[i + (int64_t)c * ldw] = w;
}

int sm_count() {
  static int cnt = 0;
  if (cnt == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || cnt <= 0)
      cnt = 148;
  }
  return cnt;
}

int kx_for(int d) { return 3 * (d + 2) <= 64 ? 64 : 128; }
int kx3_for(int d) { return (6 * (d + 2) + 15) / 16 * 16; }   // three-part form
int tp_for(int t) { return (t + 7) / 8 * 8; }
int ntiles_for(int64_t n) { return (int)cdiv(n, BM); }
// Large problems split every row's sum into chunks of at most kChunkTiles column tiles:
// each output then accumulates in FP32 (TMEM) over at most 8 kChunkTiles MMA steps and
// the chunk partials are added with compensation.  One FP32 accumulator over all 3,907 column
// tiles of n = 5e5 (31k MMA steps) leaves rounding of ~1e-5 (|K||v|)_i, which in the
// small-eigenvalue directions of an ill-conditioned K (lambda_max / sigma^2 ~ 1e5) is of
// the order of sigma^2 itself, and CG on probe vectors diverged there.  (The partials
// are summed with compensation in tc_reduce_kernel.)
constexpr int kChunkTiles = 64;
constexpr int kLongRow = 1024;   // rows of more column tiles than this are chunked
int min_chunks_for(int ntiles) {
  return ntiles > kLongRow ? (int)cdiv(ntiles, kChunkTiles) : 1;
}
int nchunks_for(int ntiles) {
  int want = (int)cdiv(8LL * 152, ntiles);
  int maxc = std::max(1, ntiles / 16);
  return std::max(min_chunks_for(ntiles), std::max(1, std::min(want, maxc)));
}
// Largest column-chunk count the autotuner may pick (the partial-sum buffer is sized
// for it): chunks of at least 4 tiles, and no more than ~16 work units per SM.
int max_chunks_for(int ntiles) {
  const int a = std::max(1, std::min(ntiles / 4, (int)cdiv(16LL * 152, ntiles)));
  return std::max(a, nchunks_for(ntiles));
}

// ---- autotuned launch configurations ----------------------------------------------------
// Key: exponent operand width kx, padded t, kernel kind, split mode and the tile-count
// bucket ceil(log2(ntiles)); value: column chunks and the B / V ring depths.
struct TcConfig {
  int nchunks = 0, nsb = 0, nsv = 0;
};
std::mutex g_tune_mu;
std::map<uint64_t, TcConfig> g_tune;
uint64_t tune_key(int kx, int tp, int kind, int split, int ntiles) {
  int b = 0;
  while ((1 << b) < ntiles) ++b;
  return ((uint64_t)kx << 40) | ((uint64_t)tp << 32) | ((uint64_t)kind << 24) |
         ((uint64_t)(split ? 1 : 0) << 16) | (uint64_t)b;
}
bool tune_lookup(uint64_t key, TcConfig* c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *c = it->second;
  return true;
}
constexpr size_t kSmemCap = 220 * 1024;
size_t smem_bytes(int kx, int tp, int nsb, int nsv) {
  size_t b = (size_t)BM * kx * 2 + (size_t)nsb * BN * kx * 2 + (size_t)nsv * tp * BN * 2 * 2 +
             sizeof(Bars) + 1024;
  // keep one CTA per SM: it owns all 512 TMEM columns
  return std::max<size_t>(b, 120 * 1024);
}
// Deepest B and V rings (2 .. 4 stages each, V first) that fit the shared-memory cap.
void stages_for(int kx, int tp, int* nsb, int* nsv) {
  for (int total = 2 * kMaxStages; total >= 4; --total)
    for (int v = std::min(kMaxStages, total - 2); v >= 2 && total - v <= kMaxStages; --v)
      if (smem_bytes(kx, tp, total - v, v) <= kSmemCap) {
        *nsb = total - v;
        *nsv = v;
        return;
      }
  *nsb = 2;
  *nsv = 2;
}

}  // namespace

size_t tc_xpack_bytes(int64_t n, int d, int prec) {
  (void)prec;
  // A and B forms of the two-part split, then of the three-part split
  return (size_t)ntiles_for(n) * BM * (kx_for(d) + kx3_for(d)) * 2 * 2;
}
size_t tc_vpack_bytes(int64_t n, int t, int prec) {
  (void)prec;
  return (size_t)ntiles_for(n) * BN * tp_for(t) * 2 * 2;   // hi and lo parts
}
size_t tc_part_elems(int64_t n, int t) {
  const int nt = ntiles_for(n);
  return (size_t)max_chunks_for(nt) * tp_for(t) * nt * BM;
}
bool tc_supported(const Prob& pb, int t) {
  return pb.prec == GP_BF16 && t >= 1 && t <= 64 && pb.d <= kMaxD;
}

gp_status tc_prepare_inputs(const Prob& pb, const void* Xs, const TcBufs& tb, cudaStream_t st) {
  const int nt = ntiles_for(pb.n), kx = kx_for(pb.d), kx3 = kx3_for(pb.d);
  __nv_bfloat16* xa = static_cast<__nv_bfloat16*>(tb.xpack);
  __nv_bfloat16* xb = xa + (size_t)nt * BM * kx;
  __nv_bfloat16* xa3 = xb + (size_t)nt * BN * kx;
  __nv_bfloat16* xb3 = xa3 + (size_t)nt * BM * kx3;
  const unsigned blocks = (unsigned)cdiv((int64_t)nt * BM, 128);
  pack_x_kernel<<<blocks, 128, 0, st>>>((int)pb.n, nt, pb.d, kx, 2,
                                        static_cast<const float*>(Xs), pb.kind, xa, xb,
                                        tb.norms);
  GP_LAUNCH_CHECK();
  pack_x_kernel<<<blocks, 128, 0, st>>>((int)pb.n, nt, pb.d, kx3, 3,
                                        static_cast<const float*>(Xs), pb.kind, xa3, xb3,
                                        nullptr);
  GP_LAUNCH_CHECK();
  return GP_OK;
}

gp_status kmvm_tc(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t, float* W,
                  int64_t ldw, const int* gate, int mode, cudaStream_t st) {
  return kmvm_tc_debug(pb, tb, V, ldv, t, W, ldw, gate, nullptr, mode, st);
}

namespace {
// mode: 0 = fast (the split flag is known to be off), 1 = split (known on), 2 = read
// on the device (shared memory sized for the wider split-mode operands).
gp_status kmvm_tc_cfg(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                      float* W, int64_t ldw, const int* gate, float* dbg, const TcConfig* cfg,
                      int mode, cudaStream_t st) {
  const int n = (int)pb.n;
  const int nt = ntiles_for(pb.n), kx = kx_for(pb.d), kx3 = kx3_for(pb.d), tp = tp_for(t);
  // Operand width the shared memory is sized for.  Invariant: the kernel never uses
  // a wider form than this (it takes the three-part form only when kx3 <= kxs, and
  // kxs >= kx always), whatever the split flag holds at launch.  kx3 can be narrower
  // than kx (small d: kx is padded to 64), so the width is the larger of the two
  // whenever the flag may be on; when the three-part tiles do not fit at all, split
  // mode keeps the two-part exponent.
  const int kwide = std::max(kx, kx3);
  const bool fit3 = smem_bytes(kwide, tp, 2, 2) <= kSmemCap;
  const int kxs = (mode != 0 && fit3) ? kwide : kx;
  const int nch = cfg ? std::max(min_chunks_for(nt), std::min(cfg->nchunks, max_chunks_for(nt)))
                      : nchunks_for(nt);
  const int npad = nt * BM;
  __nv_bfloat16* xa = static_cast<__nv_bfloat16*>(tb.xpack);
  __nv_bfloat16* xb = xa + (size_t)nt * BM * kx;
  __half* vp = static_cast<__half*>(tb.vpack);
  int* err = tb.err;
  const int64_t vtotal = (int64_t)nt * BN * tp;
  colscale_kernel<<<dim3(kScaleParts, t), 256, 0, st>>>(
      n, V, ldv, tb.vscale, reinterpret_cast<unsigned*>(tb.err + kTcErrCounters), gate);
  GP_LAUNCH_CHECK();
  pack_v_kernel<<<(unsigned)cdiv(vtotal, 256), 256, 0, st>>>(n, nt, t, tp, V, ldv, tb.vscale, vp,
                                                              gate);
  GP_LAUNCH_CHECK();
  TcArgs a;
  a.xa = xa;
  a.xb = xb;
  a.xa3 = xb + (size_t)nt * BN * kx;
  a.xb3 = a.xa3 + (size_t)nt * BM * kx3;
  a.vp = vp;
  a.part = tb.part;
  a.n = n;
  a.npad = npad;
  a.ntiles = nt;
  a.nchunks = nch;
  a.tiles_per_chunk = (int)cdiv(nt, nch);
  a.kx = kx;
  a.kx3 = kx3;
  a.kx3_ok = kx3 <= kxs ? 1 : 0;
  a.tp = tp;
  a.t = t;
  a.kind = pb.kind;
  a.D = pb.D;
  stages_for(kxs, tp, &a.nsb, &a.nsv);
  if (cfg && cfg->nsb >= 2 && cfg->nsv >= 2 && smem_bytes(kxs, tp, cfg->nsb, cfg->nsv) <= kSmemCap) {
    a.nsb = cfg->nsb;
    a.nsv = cfg->nsv;
  }
  a.gate = gate;
  a.err = err;
  a.dbg = dbg;
  // the chunk count must not leave an empty chunk
  a.nchunks = (int)cdiv(nt, a.tiles_per_chunk);
  const size_t sm = smem_bytes(kxs, tp, a.nsb, a.nsv);
  static bool attr_set = false;
  if (!attr_set) {
    GP_CUDA_TRY(cudaFuncSetAttribute(kmvm_tc_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    GP_CUDA_TRY(cudaFuncSetAttribute(kmvm_tc_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    attr_set = true;
  }
  const int units = nt * a.nchunks;
  const int grid = std::min(units, sm_count());
  if (mode == 0) kmvm_tc_kernel<false><<<grid, kThreads, sm, st>>>(a);
  else kmvm_tc_kernel<true><<<grid, kThreads, sm, st>>>(a);
  GP_LAUNCH_CHECK();
  tc_reduce_kernel<<<(unsigned)cdiv((int64_t)n * t, 256), 256, 0, st>>>(
      n, npad, t, tp, a.nchunks, tb.part, V, ldv, pb.theta, pb.D, tb.vscale, W, ldw, gate, err);
  GP_LAUNCH_CHECK();
  return GP_OK;
}
}  // namespace

gp_status kmvm_tc_debug(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                        float* W, int64_t ldw, const int* gate, float* dbg, int mode,
                        cudaStream_t st) {
  // the split flag is on the device; the tuned table is keyed on fast mode, which is
  // what the tuner times (split mode has the same tiling and ring structure)
  TcConfig c;
  const bool tuned = tune_lookup(tune_key(kx_for(pb.d), tp_for(t), pb.kind, 0, ntiles_for(pb.n)), &c);
  return kmvm_tc_cfg(pb, tb, V, ldv, t, W, ldw, gate, dbg, tuned ? &c : nullptr, mode, st);
}

// Times the candidate configurations for this problem shape (one warm-up and three
// timed products each, CUDA events on `st`), records the fastest in the table and
// leaves its product in W.  Synchronises with `st`.
gp_status tc_autotune(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t,
                      float* W, int64_t ldw, cudaStream_t st, int* best_out) {
  const int nt = ntiles_for(pb.n), kx = kx_for(pb.d), tp = tp_for(t);
  std::vector<TcConfig> cands;
  const int rings[3][2] = {{kMaxStages, kMaxStages}, {3, 3}, {2, 2}};
  const int chunk_opts[] = {1, 2, 3, 4, 6, 8, 12, 16, 24};
  for (int c : chunk_opts) {
    if (c > max_chunks_for(nt)) break;
    for (auto& r : rings)
      if (smem_bytes(kx, tp, r[0], r[1]) <= kSmemCap) cands.push_back(TcConfig{c, r[0], r[1]});
  }
  cudaEvent_t e0, e1;
  GP_CUDA_TRY(cudaEventCreate(&e0));
  GP_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  TcConfig bc;
  gp_status rs = GP_OK;
  for (const TcConfig& c : cands) {
    rs = kmvm_tc_cfg(pb, tb, V, ldv, t, W, ldw, nullptr, nullptr, &c, 0, st);
    if (rs != GP_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && rs == GP_OK; ++r)
      rs = kmvm_tc_cfg(pb, tb, V, ldv, t, W, ldw, nullptr, nullptr, &c, 0, st);
    cudaEventRecord(e1, st);
    if (rs != GP_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rs = GP_ERR_CUDA;
      break;
    }
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != GP_OK) return rs;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(kx, tp, pb.kind, 0, nt)] = bc;
  }
  if (best_out) {
    best_out[0] = bc.nchunks;
    best_out[1] = bc.nsb;
    best_out[2] = bc.nsv;
    best_out[3] = (int)cands.size();
  }
  // W from the chosen configuration
  return kmvm_tc_cfg(pb, tb, V, ldv, t, W, ldw, nullptr, nullptr, &bc, 0, st);
}

// The configuration the product uses for this shape: {nchunks, nsb, nsv, tuned}.
void tc_config(const Prob& pb, int t, int* out4) {
  const int nt = ntiles_for(pb.n), kx = kx_for(pb.d), tp = tp_for(t);
  TcConfig c;
  const bool tuned = tune_lookup(tune_key(kx, tp, pb.kind, 0, nt), &c);
  int nsb, nsv;
  stages_for(kx, tp, &nsb, &nsv);
  out4[0] = tuned ? std::min(c.nchunks, max_chunks_for(nt)) : nchunks_for(nt);
  out4[1] = tuned ? c.nsb : nsb;
  out4[2] = tuned ? c.nsv : nsv;
  out4[3] = tuned ? 1 : 0;
}

}  // namespace gp
