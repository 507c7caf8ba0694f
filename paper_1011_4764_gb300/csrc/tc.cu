// Tensor-core (tcgen05) pair contraction: TF32, BF16 and BF16 hi+lo split.
#include "ofm_internal.h"

struct TcPlan {};

ofm_status ofm_plan_extra(ofm_ctx* c) { (void)c; return OFM_OK; }
void ofm_tc_free(ofm_ctx* c) { delete c->tc; c->tc = nullptr; }
ofm_status ofm_contract_tc(ofm_ctx* c, ofm_precision prec) {
  (void)prec;
  return ofm_fail(c, OFM_ERR_INVALID, "tensor-core contraction is not built yet");
}
ofm_status ofm_window_vectors(ofm_ctx* c, int m, double* C_out) {
  (void)m; (void)C_out;
  return ofm_fail(c, OFM_ERR_INVALID, "window eigenvectors are not built yet");
}
