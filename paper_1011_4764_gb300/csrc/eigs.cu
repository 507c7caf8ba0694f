// Batched fragment eigensolver (placeholder until the kernels land).
#include "ofm_internal.h"

extern "C" ofm_status ofm_fragment_eigs(ofm_ctx* c, const ofm_eig_opts* opts, double* eps_out,
                                        double* resid_out) {
  (void)opts; (void)eps_out; (void)resid_out;
  if (!c) return OFM_ERR_INVALID;
  return ofm_fail(c, OFM_ERR_INVALID, "fragment eigensolver is not built yet");
}
