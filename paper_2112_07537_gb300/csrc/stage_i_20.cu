// Instantiation of the FP32 fused stage kernels for the 2.0 wavelet.
#include "stage_kernels.cuh"

namespace mr {
template int fused_launch<2, 0>(mr_grid *, const float *, const float *, const float *, int, const float *,
                                   float *, int, double, const double *, int, bool, const float *);
}  // namespace mr
