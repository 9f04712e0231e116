// Semi-external SpMM (Section 3.3): the sparse matrix stays in pinned host memory and row
// panels stream to the device.  (Built in a later step; until then creating a capped handle
// fails with FE_ERR_INVALID.)
#include "fe_internal.cuh"

namespace fe {
int semiext_create(fe_csr h, const int64_t*, const int32_t*, const fe_csr_opts&) {
  (void)h;
  return set_error(FE_ERR_INVALID, "semi-external mode (device_mem_cap_bytes > 0) is not available yet");
}
int semiext_spmm(fe_csr, const void*, void*, int, fe_dtype, cudaStream_t) {
  return set_error(FE_ERR_INVALID, "semi-external mode is not available yet");
}
void semiext_destroy(fe_csr) {}
int64_t semiext_panels(fe_csr) { return 0; }
}  // namespace fe
