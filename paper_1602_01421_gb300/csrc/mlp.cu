// Learned start block (an MLP over SpMM-derived vertex features).  Built in a later step.
#include "fe_internal.cuh"

namespace fe {
int mlp_start_block(fe_csr, const float*, int, int, uint64_t, double*, cudaStream_t) {
  return set_error(FE_ERR_INVALID, "learned start block is not available yet");
}
}  // namespace fe
