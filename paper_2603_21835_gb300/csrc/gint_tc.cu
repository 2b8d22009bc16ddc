// gint_tc.cu -- tensor-core (tcgen05) brick kernels.  Placeholder until the kernels land.
#include "gint_handle.cuh"

int gint_tc_rho(gint_handle *, int, const double *, double *, const double *, double *, cudaStream_t) {
  return GINT_EUNSUPPORTED;
}
int gint_tc_vlocal(gint_handle *, int, const double *, double *, cudaStream_t) { return GINT_EUNSUPPORTED; }
