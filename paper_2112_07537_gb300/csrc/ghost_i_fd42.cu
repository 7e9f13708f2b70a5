// ghost_i_fd42.cu -- the ghost kernels instantiated for float fields, double
// padded blocks and the 4.2 wavelet, compiled on their own so that the
// instantiations build in parallel.
#include "ghost_kernels.cuh"

namespace mr {
template int ghost_impl<float, double, 4, 2>(mr_grid *, const float *, float *, int, double *, double *, int, int, const int *);
}  // namespace mr
