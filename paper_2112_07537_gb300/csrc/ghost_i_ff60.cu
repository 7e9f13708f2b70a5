// ghost_i_ff60.cu -- the ghost kernels instantiated for float fields, float
// padded blocks and the 6.0 wavelet, compiled on their own so that the
// instantiations build in parallel.
#include "ghost_kernels.cuh"

namespace mr {
template int ghost_impl<float, float, 6, 0>(mr_grid *, const float *, float *, int, float *, float *, int, int, const int *);
}  // namespace mr
