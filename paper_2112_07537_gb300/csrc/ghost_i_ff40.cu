// ghost_i_ff40.cu -- the ghost kernels instantiated for float fields, float
// padded blocks and the 4.0 wavelet, compiled on their own so that the
// instantiations build in parallel.
#include "ghost_kernels.cuh"

namespace mr {
template int ghost_impl<float, float, 4, 0>(mr_grid *, const float *, float *, int, float *, float *, int, int, const int *);
}  // namespace mr
