// ghost_i_dd22.cu -- the ghost kernels instantiated for double fields, double
// padded blocks and the 2.2 wavelet, compiled on their own so that the
// instantiations build in parallel.
#include "ghost_kernels.cuh"

namespace mr {
template int ghost_impl<double, double, 2, 2>(mr_grid *, const double *, double *, int, double *, double *, int, int, const int *);
}  // namespace mr
