// Tensor-core (tcgen05) kernel-matrix products for the TF32 / BF16 precisions.
#include "ops.h"

namespace gp {

size_t tc_xpack_bytes(int64_t n, int d, int prec) { (void)n; (void)d; (void)prec; return 0; }
size_t tc_vpack_bytes(int64_t n, int t, int prec) { (void)n; (void)t; (void)prec; return 0; }
size_t tc_part_elems(int64_t n, int t) { (void)n; (void)t; return 0; }
bool tc_supported(const Prob& pb, int t) { (void)pb; (void)t; return false; }
gp_status tc_prepare_inputs(const Prob& pb, const void* Xs, const TcBufs& tb, cudaStream_t st) {
  (void)pb; (void)Xs; (void)tb; (void)st;
  set_error("tensor-core path not available");
  return GP_ERR_INVALID_ARG;
}
gp_status kmvm_tc(const Prob& pb, const TcBufs& tb, const float* V, int64_t ldv, int t, float* W,
                  int64_t ldw, const int* gate, cudaStream_t st) {
  (void)pb; (void)tb; (void)V; (void)ldv; (void)t; (void)W; (void)ldw; (void)gate; (void)st;
  set_error("tensor-core path not available");
  return GP_ERR_INVALID_ARG;
}

}  // namespace gp
