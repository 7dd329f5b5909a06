// kernels.cuh -- the integration, rate, Jacobian and adjoint kernels, declared for the C ABI.
//
// The kernels are compiled in several translation units (one per lane group of the integration kernels,
// kern_fwd_*.cu, and kern_adjoint.cu) so that the library builds in parallel; capi.cu launches them
// through these declarations.
#pragma once
#include "adjoint.cuh"
#include "device.cuh"

namespace chemgb {

__global__ void k_rates(MechView M, CellLayout L, int N, const double* __restrict__ T, const double* __restrict__ p,
                        const double* __restrict__ Y, double* __restrict__ dTdt, double* __restrict__ dYdt,
                        double* __restrict__ wdot);

__global__ void k_jacobian(MechView M, CellLayout L, int N, const double* __restrict__ T, const double* __restrict__ p,
                           const double* __restrict__ Y, double* __restrict__ Sv, double* __restrict__ u,
                           double* __restrict__ v);

// The integration kernels are templates on the lane group (one warp, two warps or half a warp per cell);
// their instantiations keep internal linkage inside their translation unit, so the ABI reaches them
// through these host functions (group g: 0 one warp, 1 two warps, 2 half a warp per cell).
//   plain form: one lane group per cell, cells in index order;
//   persistent form: resident lane groups pull `chunk` cells at a time from the sorted queue `perm`.
enum ForwardKernel { KF_PLAIN = 0, KF_PERSISTENT = 1 };
// Host-side handle of the kernel (for cudaFuncSetAttribute, cudaFuncGetAttributes and occupancy queries).
const void* forward_kernel(ForwardKernel kind, int g);
cudaError_t launch_integrate_plain(int g, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                            const CellLayout& L, int N, double* T, const double* p, double* Y, const double* dt,
                            double* h_io, int* nsub, int* status, int* nacc_out, const IntOpts& o,
                            const unsigned long long* stamp, unsigned long long budget_ns);
cudaError_t launch_integrate_persistent(int g, dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                                 const CellLayout& L, int N, double* T, const double* p, double* Y,
                                 const double* dt, double* h_io, int* nsub, int* status, int* nacc_out,
                                 const int* perm, unsigned long long* head, int chunk, const IntOpts& o,
                                 const unsigned long long* stamp, unsigned long long budget_ns);

// Per-group pieces, one translation unit each.
template <class Gp>
const void* plain_kernel();
template <class Gp>
const void* persistent_kernel();
template <class Gp>
cudaError_t launch_plain_g(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M, const CellLayout& L,
                    int N, double* T, const double* p, double* Y, const double* dt, double* h_io, int* nsub,
                    int* status, int* nacc_out, const IntOpts& o, const unsigned long long* stamp,
                    unsigned long long budget_ns);
template <class Gp>
cudaError_t launch_persistent_g(dim3 grid, dim3 block, size_t smem, cudaStream_t stream, const MechView& M,
                         const CellLayout& L, int N, double* T, const double* p, double* Y, const double* dt,
                         double* h_io, int* nsub, int* status, int* nacc_out, const int* perm,
                         unsigned long long* head, int chunk, const IntOpts& o, const unsigned long long* stamp,
                         unsigned long long budget_ns);

// Discrete adjoint: resident warps (one per block) pull cells, longest tapes first; shared memory holds the
// forward cell layout, each warp's workspace (A.total doubles) and dual-number workspace are in global
// memory.
__global__ void k_adjoint(MechView M, AdjLayout A, int N, const double* __restrict__ p, const double* __restrict__ rec_h,
                          const double* __restrict__ rec_ck, const int* __restrict__ rec_n, int K,
                          const double* __restrict__ gT, const double* __restrict__ gY, double* __restrict__ grad_cell,
                          double* __restrict__ gT0, double* __restrict__ gY0, int* __restrict__ status,
                          int* __restrict__ head, const int* __restrict__ perm, Dual4* dual_ws, double* warp_ws,
                          IntOpts o);

__global__ void k_grad_reduce(int N, int P, const double* __restrict__ grad_cell, double* __restrict__ out1,
                              double* __restrict__ out2, int half);

__global__ void k_set_params(MechView M, const double* __restrict__ rxd0, double* __restrict__ rxd,
                             const double* __restrict__ dlnA, const double* __restrict__ dEa);

}  // namespace chemgb
