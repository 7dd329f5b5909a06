// kern_fwd_half.cu -- integration kernels with two cells per warp (half a warp each).
#include "kern_forward.cuh"

namespace chemgb {

template const void* plain_kernel<GrpH>();
template cudaError_t launch_plain_g<GrpH>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&, int, double*,
                                  const double*, double*, const double*, double*, int*, int*, int*, const IntOpts&,
                                  const unsigned long long*, unsigned long long);
template const void* persistent_kernel<GrpH>();
template cudaError_t launch_persistent_g<GrpH>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&, int,
                                       double*, const double*, double*, const double*, double*, int*, int*, int*,
                                       const int*, unsigned long long*, int, const IntOpts&,
                                       const unsigned long long*, unsigned long long);

}  // namespace chemgb
