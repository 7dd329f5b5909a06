// kern_forward.cuh -- host-side handles and launchers of the integration kernels (integrate.cuh), included
// by one translation unit per lane group and form (kern_fwd_warp*.cu, kern_fwd_pair.cu, kern_fwd_half.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "integrate.cuh"
#include "kernels.cuh"

namespace chemgb {

// Host-side handles and launches of the instantiations for lane group Gp (explicitly instantiated in one
// translation unit per group and form).
template <class Gp>
const void* plain_kernel() {
  return (const void*)k_integrate_plain<Gp>;
}

template <class Gp>
const void* persistent_kernel() {
  return (const void*)k_integrate_persistent<Gp>;
}

template <class Gp>
cudaError_t launch_plain_g(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                           const CellLayout& L, int N, double* T, const double* p, double* Y, const double* dt,
                           double* h_io, int* nsub, int* status, int* nacc_out, const IntOpts& o,
                           const unsigned long long* stamp, unsigned long long budget_ns) {
  if (block.x % Gp::size != 0 || block.x % kWarp != 0 || block.y != 1 || block.z != 1) return cudaErrorInvalidValue;
  k_integrate_plain<Gp><<<grid, block, smem, stream>>>(M, L, N, T, p, Y, dt, h_io, nsub, status, nacc_out, o, stamp,
                                                       budget_ns);
  return cudaSuccess;
}

template <class Gp>
cudaError_t launch_persistent_g(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                                const CellLayout& L, int N, double* T, const double* p, double* Y, const double* dt,
                                double* h_io, int* nsub, int* status, int* nacc_out, const int* perm,
                                unsigned long long* head, int chunk, const IntOpts& o,
                                const unsigned long long* stamp, unsigned long long budget_ns) {
  if (block.x % Gp::size != 0 || block.x % kWarp != 0 || block.y != 1 || block.z != 1) return cudaErrorInvalidValue;
  k_integrate_persistent<Gp><<<grid, block, smem, stream>>>(M, L, N, T, p, Y, dt, h_io, nsub, status, nacc_out, perm,
                                                            head, chunk, o, stamp, budget_ns);
  return cudaSuccess;
}

}  // namespace chemgb
