// kern_fwd_warp.cu -- the persistent integration kernel with one warp per cell, and the dispatch over lane
// groups.
#include "kern_forward.cuh"

namespace chemgb {

template const void* persistent_kernel<Grp1>();
template cudaError_t launch_persistent_g<Grp1>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&, int,
                                       double*, const double*, double*, const double*, double*, int*, int*, int*,
                                       const int*, unsigned long long*, int, const IntOpts&,
                                       const unsigned long long*, unsigned long long);

// instantiated in the other lane groups' translation units (kern_fwd_warp_plain.cu, kern_fwd_pair.cu,
// kern_fwd_half.cu): declared here so that the dispatch below does not instantiate them again
extern template const void* plain_kernel<Grp1>();
extern template cudaError_t launch_plain_g<Grp1>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&,
                                               int, double*, const double*, double*, const double*, double*, int*,
                                               int*, int*, const IntOpts&, const unsigned long long*,
                                               unsigned long long);
extern template const void* plain_kernel<Grp2>();
extern template cudaError_t launch_plain_g<Grp2>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&,
                                               int, double*, const double*, double*, const double*, double*, int*,
                                               int*, int*, const IntOpts&, const unsigned long long*,
                                               unsigned long long);
extern template const void* persistent_kernel<Grp2>();
extern template cudaError_t launch_persistent_g<Grp2>(dim3, dim3, size_t, cudaStream_t, const MechView&,
                                                    const CellLayout&, int, double*, const double*, double*,
                                                    const double*, double*, int*, int*, int*, const int*,
                                                    unsigned long long*, int, const IntOpts&,
                                                    const unsigned long long*, unsigned long long);
extern template const void* plain_kernel<GrpH>();
extern template cudaError_t launch_plain_g<GrpH>(dim3, dim3, size_t, cudaStream_t, const MechView&, const CellLayout&,
                                               int, double*, const double*, double*, const double*, double*, int*,
                                               int*, int*, const IntOpts&, const unsigned long long*,
                                               unsigned long long);
extern template const void* persistent_kernel<GrpH>();
extern template cudaError_t launch_persistent_g<GrpH>(dim3, dim3, size_t, cudaStream_t, const MechView&,
                                                    const CellLayout&, int, double*, const double*, double*,
                                                    const double*, double*, int*, int*, int*, const int*,
                                                    unsigned long long*, int, const IntOpts&,
                                                    const unsigned long long*, unsigned long long);

const void* forward_kernel(ForwardKernel kind, int g) {
  if (kind == KF_PLAIN) return g == 0 ? plain_kernel<Grp1>() : g == 1 ? plain_kernel<Grp2>() : plain_kernel<GrpH>();
  return g == 0 ? persistent_kernel<Grp1>() : g == 1 ? persistent_kernel<Grp2>() : persistent_kernel<GrpH>();
}

cudaError_t launch_integrate_plain(int g, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                            const CellLayout& L, int N, double* T, const double* p, double* Y, const double* dt,
                            double* h_io, int* nsub, int* status, int* nacc_out, const IntOpts& o,
                            const unsigned long long* stamp, unsigned long long budget_ns) {
  auto f = g == 0 ? launch_plain_g<Grp1> : g == 1 ? launch_plain_g<Grp2> : launch_plain_g<GrpH>;
  return f(grid, block, smem, stream, M, L, N, T, p, Y, dt, h_io, nsub, status, nacc_out, o, stamp, budget_ns);
}

cudaError_t launch_integrate_persistent(int g, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                                 const CellLayout& L, int N, double* T, const double* p, double* Y,
                                 const double* dt, double* h_io, int* nsub, int* status, int* nacc_out,
                                 const int* perm, unsigned long long* head, int chunk, const IntOpts& o,
                                 const unsigned long long* stamp, unsigned long long budget_ns) {
  auto f = g == 0 ? launch_persistent_g<Grp1> : g == 1 ? launch_persistent_g<Grp2> : launch_persistent_g<GrpH>;
  return f(grid, block, smem, stream, M, L, N, T, p, Y, dt, h_io, nsub, status, nacc_out, perm, head, chunk, o, stamp,
           budget_ns);
}

}  // namespace chemgb
