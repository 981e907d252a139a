// Tensor-core (tcgen05) forms of the two contractions.
#include "yy_internal.h"

namespace yy {

yy_status tc_prepare(yy_grid *, yy_precision) { return YY_ERR_NOT_SUPPORTED; }
void tc_free(yy_grid *) {}
cudaError_t tc_analysis(yy_grid *, yy_precision, const double *, const double *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t tc_pack_coefficients(yy_grid *, yy_precision, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_synthesis(yy_grid *, yy_precision, int, double *, double *, double *, double *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace yy
