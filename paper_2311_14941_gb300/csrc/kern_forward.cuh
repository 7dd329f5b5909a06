// kern_forward.cuh -- the integration kernels (one lane group per cell) and the rate and Jacobian kernels,
// included by one translation unit per lane group (kern_fwd_warp.cu, kern_fwd_pair.cu, kern_fwd_half.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "kernels.cuh"

namespace chemgb {

__device__ __forceinline__ IntOpts with_deadline(IntOpts o, const unsigned long long* stamp,
                                                 unsigned long long budget_ns);

// Load one cell's state into y (lanes over state components).
template <class Gp>
__device__ __forceinline__ void load_state(double* y, int m, int N, int c, const double* T, const double* Y,
                                           const Gp& g) {
  for (int i = g.lane; i < m; i += g.size) y[i] = (i == 0) ? T[c] : Y[(size_t)(i - 1) * N + c];
  g.sync();
}

// The lane group of this thread (Gp: one warp, two warps or half a warp per cell); s = the cell's memory.
__device__ __forceinline__ void cell_slot(int gs, const CellLayout& L, double* smem, int& cell_in_block, double*& s) {
  cell_in_block = threadIdx.x / gs;
  s = smem + (size_t)cell_in_block * L.total;
}
template <class Gp>
__device__ __forceinline__ Gp cell_group(const CellLayout& L, double* smem, int& cell_in_block, double*& s);
template <>
__device__ __forceinline__ Grp1 cell_group<Grp1>(const CellLayout& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(Grp1::size, L, smem, cell_in_block, s);
  return Grp1{(int)threadIdx.x - cell_in_block * Grp1::size};
}
template <>
__device__ __forceinline__ Grp2 cell_group<Grp2>(const CellLayout& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(Grp2::size, L, smem, cell_in_block, s);
  return Grp2{(int)threadIdx.x - cell_in_block * Grp2::size, 1 + cell_in_block, s + L.misc};
}
template <>
__device__ __forceinline__ GrpH cell_group<GrpH>(const CellLayout& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(GrpH::size, L, smem, cell_in_block, s);
  const int half = (threadIdx.x / GrpH::size) & 1;
  return GrpH{(int)threadIdx.x - cell_in_block * GrpH::size, half ? 0xffff0000u : 0x0000ffffu};
}

// Cells taken per queue pull: a half-warp group pulls together with the other half of its warp (one
// atomic per warp, the two halves take consecutive slots of the sorted queue, so the two cells that
// share a warp have similar previous costs and run side by side); other groups pull alone.
template <class Gp>
struct PullOf {
  static constexpr int groups = 1;   // lane groups per pulling unit
};
template <>
struct PullOf<GrpH> {
  static constexpr int groups = 2;
};

// Block-cooperative coalesced load of the block's consecutive cells: adjacent threads read adjacent
// cells of the same state row (structure of arrays), then each lane group owns its cell's copy.
__device__ __forceinline__ void load_tile(double* smem, const CellLayout& L, int m, int N, int c0, int wpb,
                                          const double* T, const double* Y) {
  const int total = wpb * m;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = idx / wpb, w = idx - row * wpb;
    const int c = c0 + w;
    if (c < N) smem[(size_t)w * L.total + L.y + row] = (row == 0) ? T[c] : Y[(size_t)(row - 1) * N + c];
  }
  __syncthreads();
}

// Plain form: one lane group per cell, cells in index order, one launch.
template <class Gp>
__global__ void k_integrate_plain(MechView M, CellLayout L, int N, double* __restrict__ T, const double* __restrict__ p,
                                  double* __restrict__ Y, const double* __restrict__ dt, double* __restrict__ h_io,
                                  int* __restrict__ nsub, int* __restrict__ status, int* __restrict__ nacc_out,
                                  IntOpts o, const unsigned long long* stamp, unsigned long long budget_ns) {
  extern __shared__ double smem[];
  if (blockDim.x % Gp::size != 0 || blockDim.x % kWarp != 0) return;   // the launch wrapper rejects such shapes
  const int cpb = blockDim.x / Gp::size;
  int w = 0;
  double* s = nullptr;
  const Gp g = cell_group<Gp>(L, smem, w, s);
  const int c0 = blockIdx.x * cpb;
  load_tile(smem, L, M.m, N, c0, cpb, T, Y);
  const int c = c0 + w;
  if (c >= N) return;
  double h = h_io[c];
  int ns = 0, na = 0, st = 0;
  integrate_cell(M, s, L, p[c], dt[c], h, ns, na, st, with_deadline(o, stamp, budget_ns), g, c);
  const double* y = s + L.y;
  for (int i = g.lane; i < M.m; i += g.size) {
    if (i == 0) T[c] = y[0];
    else Y[(size_t)(i - 1) * N + c] = y[i];
  }
  if (g.lane == 0) {
    h_io[c] = h;
    nsub[c] = ns;
    status[c] = st;
    if (nacc_out) nacc_out[c] = na;
  }
}

__device__ __forceinline__ IntOpts with_deadline(IntOpts o, const unsigned long long* stamp,
                                                 unsigned long long budget_ns) {
  if (budget_ns && stamp) o.deadline_ns = *stamp + budget_ns;
  return o;
}

// Persistent form: grid sized to the resident capacity; every lane group (every warp of two half-warp
// groups) pulls `chunk` cells per group at a time from the sorted queue with one atomicAdd and
// integrates them one after the other.  No block-wide barrier: warps of a block finish independently.
template <class Gp>
__device__ __forceinline__ long long queue_pull(const Gp& g, unsigned long long* head, int chunk) {
  return gbcast(g, g.lane == 0 ? (long long)atomicAdd(head, (unsigned long long)chunk) : 0ll);
}
__device__ __forceinline__ long long queue_pull(const GrpH& g, unsigned long long* head, int chunk) {
  // one pull for the warp; the upper half takes the second `chunk` cells
  const unsigned lane = threadIdx.x & (kWarp - 1);
  long long b = 0;
  if (lane == 0) b = (long long)atomicAdd(head, 2ull * (unsigned long long)chunk);
  b = __shfl_sync(0xffffffffu, b, 0);
  return b + (lane >= (unsigned)GrpH::size ? chunk : 0);
}

template <class Gp>
__global__ void k_integrate_persistent(MechView M, CellLayout L, int N, double* __restrict__ T,
                                       const double* __restrict__ p, double* __restrict__ Y,
                                       const double* __restrict__ dt, double* __restrict__ h_io,
                                       int* __restrict__ nsub, int* __restrict__ status, int* __restrict__ nacc_out,
                                       const int* __restrict__ perm, unsigned long long* __restrict__ head, int chunk,
                                       IntOpts o, const unsigned long long* stamp, unsigned long long budget_ns) {
  extern __shared__ double smem[];
  if (blockDim.x % Gp::size != 0 || blockDim.x % kWarp != 0) return;   // the launch wrapper rejects such shapes
  int w = 0;
  double* s = nullptr;
  const Gp g = cell_group<Gp>(L, smem, w, s);
  const IntOpts oo = with_deadline(o, stamp, budget_ns);
  while (true) {
    // 64-bit queue head: every pull adds `chunk` per group, including the last pulls past the end, so a
    // 32-bit head could wrap for large N * lane groups * chunk.  The half-warp pull is warp-wide: both
    // halves leave the loop together (the first half's base decides), and a half whose share starts
    // past the end integrates nothing in that round.
    const long long base = queue_pull(g, head, chunk);
    const long long base0 = PullOf<Gp>::groups == 2 ? base - ((threadIdx.x & (kWarp - 1)) >= GrpH::size ? chunk : 0)
                                                    : base;
    if (base0 >= N) break;
    const int end = (int)min(base + (long long)chunk, (long long)N);
    for (int j = (int)min(base, (long long)N); j < end; ++j) {
      const int c = perm[j];
      load_state(s + L.y, M.m, N, c, T, Y, g);
      double h = h_io[c];
      int ns = 0, na = 0, st = 0;
      integrate_cell(M, s, L, p[c], dt[c], h, ns, na, st, oo, g, c);
      const double* y = s + L.y;
      for (int i = g.lane; i < M.m; i += g.size) {
        if (i == 0) T[c] = y[0];
        else Y[(size_t)(i - 1) * N + c] = y[i];
      }
      if (g.lane == 0) {
        h_io[c] = h;
        nsub[c] = ns;
        status[c] = st;
        if (nacc_out) nacc_out[c] = na;
      }
      g.sync();
    }
  }
}


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
