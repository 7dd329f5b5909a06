// kern_fwd_warp_plain.cu -- the plain integration kernel with one warp per cell.
#include "kern_forward.cuh"

namespace chemgb {

template const void* plain_kernel<Grp1>();
template cudaError_t launch_plain_g<Grp1>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&, int, double*,
                                  const double*, double*, const double*, double*, int*, int*, int*, const IntOpts&,
                                  const unsigned long long*, unsigned long long);

}  // namespace chemgb
