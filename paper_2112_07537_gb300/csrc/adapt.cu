// adapt.cu -- block criterion and grid adaptation (Alg. SM3) on the device.
#include "mr_internal.cuh"

namespace mr {

int launch_criterion(mr_grid *g, const double *P64, int Gi, double *maxdet) {
  (void)g, (void)P64, (void)Gi, (void)maxdet;
  set_error("criterion not built yet");
  return MR_ERR_UNSUPPORTED;
}

int adapt_iteration(mr_grid *g, int crit_fid, double er, double ec, int flags, int *nch) {
  (void)g, (void)crit_fid, (void)er, (void)ec, (void)flags, (void)nch;
  set_error("adaptation not built yet");
  return MR_ERR_UNSUPPORTED;
}

}  // namespace mr
