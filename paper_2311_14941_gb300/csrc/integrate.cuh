// integrate.cuh -- the integration kernels (one lane group per cell), device code only.
//
// Templates on the lane group Gp (one warp, two warps or half a warp per cell), the mechanism view MV and
// the cell layout LT.  The library instantiates them with the run-time MechView / CellLayout; the
// mechanism-specialised build compiles the same source at run time with views whose sizes are
// compile-time constants (derived types with the same data members).  Nothing here may need a C library
// header, so the run-time compiler can take it as it is.
#pragma once
#include "device.cuh"

namespace chemgb {

__device__ __forceinline__ IntOpts with_deadline(IntOpts o, const unsigned long long* stamp,
                                                 unsigned long long budget_ns) {
  if (budget_ns && stamp) o.deadline_ns = *stamp + budget_ns;
  return o;
}

// Load one cell's state into y (lanes over state components).
template <class Gp>
__device__ __forceinline__ void load_state(double* y, int m, int N, int c, const double* T, const double* Y,
                                           const Gp& g) {
  for (int i = g.lane; i < m; i += g.size) y[i] = (i == 0) ? T[c] : Y[(size_t)(i - 1) * N + c];
  g.sync();
}

// The lane group of this thread (Gp: one warp, two warps or half a warp per cell); s = the cell's memory.
template <class LT>
__device__ __forceinline__ void cell_slot(int gs, const LT& L, double* smem, int& cell_in_block, double*& s) {
  cell_in_block = threadIdx.x / gs;
  s = smem + (size_t)cell_in_block * L.total;
}
template <class LT>
__device__ __forceinline__ Grp1 make_group(const Grp1*, const LT& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(Grp1::size, L, smem, cell_in_block, s);
  return Grp1{(int)threadIdx.x - cell_in_block * Grp1::size};
}
template <class LT>
__device__ __forceinline__ Grp2 make_group(const Grp2*, const LT& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(Grp2::size, L, smem, cell_in_block, s);
  return Grp2{(int)threadIdx.x - cell_in_block * Grp2::size, 1 + cell_in_block, s + L.misc};
}
template <class LT>
__device__ __forceinline__ GrpH make_group(const GrpH*, const LT& L, double* smem, int& cell_in_block, double*& s) {
  cell_slot(GrpH::size, L, smem, cell_in_block, s);
  const int half = (threadIdx.x / GrpH::size) & 1;
  return GrpH{(int)threadIdx.x - cell_in_block * GrpH::size, half ? 0xffff0000u : 0x0000ffffu};
}
template <class Gp, class LT>
__device__ __forceinline__ Gp cell_group(const LT& L, double* smem, int& cell_in_block, double*& s) {
  return make_group(static_cast<const Gp*>(nullptr), L, smem, cell_in_block, s);
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
template <class LT>
__device__ __forceinline__ void load_tile(double* smem, const LT& L, int m, int N, int c0, int wpb, const double* T,
                                          const double* Y) {
  const int total = wpb * m;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = idx / wpb, w = idx - row * wpb;
    const int c = c0 + w;
    if (c < N) smem[(size_t)w * L.total + L.y + row] = (row == 0) ? T[c] : Y[(size_t)(row - 1) * N + c];
  }
  __syncthreads();
}

// Plain form: one lane group per cell, cells in index order, one launch.
template <class Gp, class MV = MechView, class LT = CellLayout>
__global__ void k_integrate_plain(MV M, LT L, int N, double* __restrict__ T, const double* __restrict__ p,
                                  double* __restrict__ Y, const double* __restrict__ dt, double* __restrict__ h_io,
                                  int* __restrict__ nsub, int* __restrict__ status, int* __restrict__ nacc_out,
                                  IntOpts o, const unsigned long long* stamp, unsigned long long budget_ns) {
  extern __shared__ double smem[];
  if (blockDim.x % Gp::size != 0 || blockDim.x % kWarp != 0) return;   // the launchers reject such shapes
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

template <class Gp, class MV = MechView, class LT = CellLayout>
__global__ void k_integrate_persistent(MV M, LT L, int N, double* __restrict__ T, const double* __restrict__ p,
                                       double* __restrict__ Y, const double* __restrict__ dt,
                                       double* __restrict__ h_io, int* __restrict__ nsub, int* __restrict__ status,
                                       int* __restrict__ nacc_out, const int* __restrict__ perm,
                                       unsigned long long* __restrict__ head, int chunk, IntOpts o,
                                       const unsigned long long* stamp, unsigned long long budget_ns) {
  extern __shared__ double smem[];
  if (blockDim.x % Gp::size != 0 || blockDim.x % kWarp != 0) return;   // the launchers reject such shapes
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

}  // namespace chemgb
