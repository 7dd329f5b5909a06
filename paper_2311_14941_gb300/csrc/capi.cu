// capi.cu -- C ABI: handle life cycle, table upload, kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/chem.h"
#include "compile.h"
#include "kernels.cuh"
#include "specialize.h"

using namespace chemgb;

static_assert(kCellOk == CHEM_CELL_OK && kCellMaxSteps == CHEM_CELL_MAXSTEPS && kCellHmin == CHEM_CELL_HMIN &&
                  kCellNonfinite == CHEM_CELL_NONFINITE && kCellBadInput == CHEM_CELL_BADINPUT &&
                  kCellTimeout == CHEM_CELL_TIMEOUT,
              "device status codes differ from chem.h");

namespace {

thread_local std::string g_err;

chem_status fail(chem_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

chem_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CHEM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

constexpr int kMaxBlockCells = 32;   // cells per block at most (half-warp cells: 16 warps)

struct chem_handle_s {
  int device = 0;
  HostMech hm;
  MechView view[kNumGroups]{};   // view[g]: the tables with the programs of lane group g (kGroupWidth)
  void* blob = nullptr;
  CellLayout L{};
  int cell_bytes = 0;
  int smem_optin = 0;
  int num_sms = 0;
  bool attr_set = false;
  bool adj_attr_set = false;
  const double* rxd0 = nullptr;   // the compiled (unshifted) reaction table
  // scratch of the sorted work queue and the time-budget stamp (grows on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* adj_scratch = nullptr;     // adjoint tape, gradients, dual workspaces (grows on demand)
  size_t adj_scratch_bytes = 0;
  void* map_scratch = nullptr;     // zonal mapping: zone table and the compacted cells (grows on demand)
  size_t map_scratch_bytes = 0;
  // per warps-per-cell choice (set with the attributes): the largest block that launches (in cells), the
  // block size that fits the most cells per SM, and that number of cells
  int max_cells[kNumGroups] = {1, 1, 2};
  int default_cells[kNumGroups] = {1, 1, 2};
  int resident_cells[kNumGroups] = {0, 0, 0};
  int bps_cache[kNumGroups][kMaxBlockCells + 1] = {};   // resident blocks per SM of the persistent kernel
  int auto_wpc = 1;                // warps per cell when the caller leaves the choice to the library
  int auto_cpw = 1;                // cells per warp when the caller leaves the choice to the library
  // tabulated temperature functions (built at the first call that asks for a tolerance)
  HostTables tabs;
  void* tab_dev = nullptr;
  bool params_shifted = false;     // chem_set_params moved the Arrhenius parameters off the description's
  // mechanism-specialised one-warp kernels (chem_specialize), their largest block and occupancy
  SpecKernels spec;
  int spec_max_cells = 1;
  int spec_bps_cache[kMaxBlockCells + 1] = {};
  // CUDA graph of the persistent sequence, re-captured when its arguments change
  struct GraphKey {
    int N, mode, cpb, chunk, grp;
    const void* ptr[10];
    double d[6];
    int i[5];
    bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
  } gkey{};
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;
};

namespace {

// Shared-memory layout of one cell (offsets in doubles).
CellLayout make_layout(const HostMech& hm, bool separate_lu = false) {
  CellLayout L{};
  int o = 0;
  const int m = hm.m, n = hm.n, R = hm.R;
  auto take = [&](int cnt) { int at = o; o += cnt; return at; };
  L.y = take(m); L.ytmp = take(m); L.f0 = take(m); L.U1 = take(m); L.U2 = take(m); L.U3 = take(m);
  L.U4 = take(m); L.x = take(m); L.z = take(m); L.u = take(m); L.v = take(m);
  L.C = take(n); L.hRT = take(n); L.eg = take(n); L.emg = take(n); L.cpR = take(n);
  L.q = take(std::max(R, 1));
  L.S = take(hm.nnz_S);
  // the Jacobian passes' dq/dT values and derivative slots are dead once S is assembled; the factor and
  // 1/diag reuse their space (the adjoint keeps the factor apart: separate_lu)
  const int lu_part = hm.nnz_LU + m;
  if (separate_lu) {
    L.D = take(std::max(hm.jreg, 1));
    L.LU = take(hm.nnz_LU);
    L.dinv = take(m);
  } else {
    const int reuse = std::max(lu_part, hm.jreg);
    L.D = o;
    L.LU = o;
    L.dinv = o + hm.nnz_LU;
    o += reuse;
  }
  int np = 1;
  for (const HostProg& P : hm.prog) {
    for (const HostGather* g : {&P.g_omega, &P.g_row, &P.g_col}) np = std::max(np, g->n_partial);
    for (const HostGather& g : P.g_jac) np = std::max(np, g.n_partial);
  }
  L.part = take(np);
  L.misc = take(16);
  L.total = o;
  return L;
}

// Reverse-pass layout: shared memory = the forward cell layout; the per-warp global workspace below.
AdjLayout make_adj_layout(const HostMech& hm, int K) {
  AdjLayout A{};
  A.L = make_layout(hm);
  int o = 0;
  const int m = hm.m;
  // 256-byte aligned pieces (32 doubles): coalesced lane-strided access
  auto take = [&](int cnt) { int at = o; o += (cnt + 31) / 32 * 32; return at; };
  A.Y3 = take(m); A.Y4 = take(m); A.W1 = take(m); A.W2 = take(m); A.W3 = take(m); A.W4 = take(m);
  A.MU1 = take(m); A.MU2 = take(m); A.MU3 = take(m); A.MU4 = take(m); A.LAM = take(m); A.G = take(m);
  A.ZT = take(m); A.WS = take(m);
  {   // one step record: offsets within it
    int r = 0;
    auto rtake = [&](int cnt) { int at = r; r += (cnt + 31) / 32 * 32; return at; };
    A.SY = rtake(hm.nnz_S); A.UY = rtake(m); A.VY = rtake(m); A.HY = rtake(hm.n); A.QY = rtake(std::max(hm.R, 1));
    A.SC = rtake(8); A.LUG = rtake(hm.nnz_LU + m);
    A.jstride = r;
  }
  A.JREC = take(K * A.jstride);
  A.UST = take(K * 4 * m);
  A.SEG = take(K * m);
  A.GA = take(std::max(hm.R, 1));
  A.GE = take(std::max(hm.R, 1));
  A.total = o;
  return A;
}

template <class T>
size_t put(std::vector<char>& buf, const std::vector<T>& v) {
  size_t off = align_up(buf.size(), 256);
  buf.resize(off + v.size() * sizeof(T) + 8);
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

}  // namespace

// =============================================================================================== kernels
namespace chemgb {

// ---- sorted work queue (the on-chip form of the paper's dynamic load balancing)
constexpr int kBuckets = 32;

// Scratch layout (bytes): [0, 128) bucket counts, [128, 256) bucket cursors, [256, 264) queue head
// (64-bit), [264, 272) start stamp (ns), [512, 512 + 4N) permutation.
constexpr size_t kScrCounts = 0, kScrCursor = 128, kScrHead = 256, kScrStamp = 264, kScrPerm = 512;

// Scratch for chem_integrate_noalloc: a fixed array in the module's static device memory, so that
// entry point never allocates.  Same layout as the handle scratch; room for kNoAllocMaxCells cells.
constexpr int kNoAllocMaxCells = 1 << 20;
constexpr size_t kNoAllocBytes = kScrPerm + (size_t)kNoAllocMaxCells * sizeof(int);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__device__ __forceinline__ int cost_bucket(int ns) { return ns <= 1 ? 0 : min(kBuckets - 1, 31 - __clz(ns)); }

__global__ void k_stamp(unsigned long long* stamp) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *stamp = global_ns();
}

__global__ void k_sort_count(int N, const int* __restrict__ nsub_prev, int* __restrict__ counts) {
  __shared__ int sh[kBuckets];
  for (int t = threadIdx.x; t < kBuckets; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
    atomicAdd(&sh[cost_bucket(nsub_prev[c])], 1);
  __syncthreads();
  for (int t = threadIdx.x; t < kBuckets; t += blockDim.x)
    if (sh[t]) atomicAdd(&counts[t], sh[t]);
}

// Costliest bucket first (largest previous substep count): long cells start early, cheap cells fill
// the tail.
__global__ void k_sort_scatter(int N, const int* __restrict__ nsub_prev, const int* __restrict__ counts,
                               int* __restrict__ cursor, int* __restrict__ perm) {
  __shared__ int off[kBuckets];
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = kBuckets - 1; b >= 0; --b) { off[b] = acc; acc += counts[b]; }
  }
  __syncthreads();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int b = cost_bucket(nsub_prev[c]);
    perm[off[b] + atomicAdd(&cursor[b], 1)] = c;
  }
}

}  // namespace chemgb

// =============================================================================================== ABI
namespace {

// The handle's device is made current for the duration of an entry point; the caller's current device
// is put back when the scope ends, so a call never leaves another device selected.
struct DeviceScope {
  int prev = -1;
  int cur = -1;
  cudaError_t enter(int device) {
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) { prev = -1; return e; }
    cur = prev;
    if (device == prev) return cudaSuccess;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) cur = device;
    return e;
  }
  ~DeviceScope() {
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

chem_status check_handle(chem_handle h, DeviceScope& ds) {
  if (!h) return fail(CHEM_EINVAL, "null handle");
  if (h->device < 0) return fail(CHEM_EINVAL, "handle was compiled on the host only (device -1)");
  cudaError_t e = ds.enter(h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return CHEM_OK;
}

int max_cells_per_block(const chem_handle h, int grp) { return h->max_cells[grp]; }

chem_status set_attrs(chem_handle h) {
  if (h->attr_set) return CHEM_OK;
  const int bytes = h->smem_optin;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_rates, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_jacobian, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return cuda_fail(e, "cudaFuncSetAttribute");
  for (int grp = 0; grp < kNumGroups; ++grp)
    for (ForwardKernel kind : {KF_PLAIN, KF_PERSISTENT})
      if ((e = cudaFuncSetAttribute(forward_kernel(kind, grp), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) !=
          cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
  // largest block per lane group: shared memory, the threads the kernels' registers allow (both forms),
  // at most 16 cells (32 half-warp cells), for two-warp cells the 15 named barriers besides barrier 0, and
  // for half-warp cells an even count (whole warps)
  for (int grp = 0; grp < kNumGroups; ++grp) {
    cudaFuncAttributes fa1, fa2;
    if ((e = cudaFuncGetAttributes(&fa1, forward_kernel(KF_PLAIN, grp))) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa2, forward_kernel(KF_PERSISTENT, grp))) != cudaSuccess)
      return cuda_fail(e, "cudaFuncGetAttributes");
    const int width = kGroupWidth[grp];
    int c = std::max(1, h->smem_optin / std::max(h->cell_bytes, 1));
    c = std::min(c, std::min(fa1.maxThreadsPerBlock, fa2.maxThreadsPerBlock) / width);
    if (grp == 1) c = std::min(c, 15);
    c = std::min(c, grp == 2 ? kMaxBlockCells : 16);
    if (grp == 2) c &= ~1;
    h->max_cells[grp] = std::max(grp == 2 ? 2 : 1, c);
  }
  // default block shape per lane group: the most resident cells per SM (each block also reserves some
  // shared memory, so a few cells per block can fit one more cell per SM than single-cell blocks);
  // ties -> fewer cells per block
  for (int grp = 0; grp < kNumGroups; ++grp) {
    const int step = grp == 2 ? 2 : 1;
    int best_c = step, best_cells = 0;
    for (int c = step; c <= max_cells_per_block(h, grp); c += step) {
      int blocks = 0;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_kernel(KF_PERSISTENT, grp),
                                                             c * kGroupWidth[grp], (size_t)c * h->cell_bytes)) !=
          cudaSuccess)
        return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (blocks * c > best_cells) { best_cells = blocks * c; best_c = c; }
    }
    h->default_cells[grp] = best_c;
    h->resident_cells[grp] = best_cells;
  }
  // automatic choice: two warps per cell when one-warp cells leave fewer than 6 warps per SM (a cell
  // larger than ~35 KB of shared memory) and two-warp cells fit as many cells
  h->auto_wpc = (h->resident_cells[0] < 6 && h->resident_cells[1] >= h->resident_cells[0]) ? 2 : 1;
  // two cells per warp for mechanisms whose species loops fit half a warp, unless shared memory would
  // then hold fewer cells per SM
  h->auto_cpw = (h->hm.n <= 16 && h->resident_cells[2] >= h->resident_cells[0]) ? 2 : 1;
  h->attr_set = true;
  return CHEM_OK;
}

// Cells per block: the request (0: the default of the warps-per-cell choice) bounded by the largest block
// that launches.
int cells_per_block(const chem_handle h, int requested, int grp) {
  int c = requested > 0 ? requested : h->default_cells[grp];
  c = std::max(1, std::min(c, max_cells_per_block(h, grp)));
  if (grp == 2) c = std::max(2, c & ~1);   // half-warp cells fill whole warps
  return c;
}

chem_status ensure_scratch(chem_handle h, int N) {
  const size_t need = kScrPerm + (size_t)std::max(N, 1) * sizeof(int);
  if (h->scratch_bytes >= need) return CHEM_OK;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  if (h->scratch) cudaFree(h->scratch);
  h->scratch = nullptr;
  h->scratch_bytes = 0;
  const size_t bytes = std::max(need, need + need / 4);
  if (cudaMalloc(&h->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(CHEM_ENOMEM, "cudaMalloc of integrator scratch failed");
  }
  h->scratch_bytes = bytes;
  return CHEM_OK;
}

chem_status launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return CHEM_OK;
}

// Resident blocks per SM of the persistent kernel for a launch shape (cached per shape; spec: the
// mechanism-specialised kernel, one warp per cell).
chem_status persistent_blocks_per_sm(chem_handle h, int grp, int cpb, int& bps, bool spec = false) {
  int& cached = spec ? h->spec_bps_cache[cpb] : h->bps_cache[grp][cpb];
  if (cached == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached,
                                                                  spec ? h->spec.persistent
                                                                       : forward_kernel(KF_PERSISTENT, grp),
                                                                  cpb * kGroupWidth[grp],
                                                                  (size_t)cpb * h->cell_bytes);
    if (e != cudaSuccess) { cached = 0; return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"); }
    cached = std::max(cached, 1);
  }
  bps = cached;
  return CHEM_OK;
}

// Defaults and checks of the step-control fields of chem_integrate_opts (tolerances, step limits,
// method, trace), common to every integrating entry point.
chem_status tolerance_opts(const chem_integrate_opts& o, int N, IntOpts& io) {
  io = IntOpts{};
  io.rtol = o.rtol > 0.0 ? o.rtol : 1e-6;
  io.atol = o.atol > 0.0 ? o.atol : 1e-12;
  io.h_init = o.h_init > 0.0 ? o.h_init : 1e-7;
  io.h_min = o.h_min > 0.0 ? o.h_min : 1e-20;
  io.max_substeps = o.max_substeps > 0 ? o.max_substeps : 100000;
  io.max_nonfinite = o.max_nonfinite > 0 ? o.max_nonfinite : 10;
  io.deadline_ns = 0;
  io.trace = o.trace;
  io.trace_cap = o.trace ? o.trace_cap : 0;
  io.N = N;
  io.rec_h = nullptr; io.rec_ck = nullptr; io.rec_n = nullptr; io.rec_cap = 0; io.rec_K = 1;
  if (o.method < 0 || o.method > 2) return fail(CHEM_EINVAL, "method must be 0 (RODAS3), 1 (ROS2) or 2 (RODAS4)");
  io.method = o.method;
  if (o.trace && o.trace_cap < 1) return fail(CHEM_EINVAL, "trace_cap must be >= 1 when trace is given");
  if (!(std::isfinite(io.rtol) && std::isfinite(io.atol) && std::isfinite(io.h_init) && std::isfinite(io.h_min)))
    return fail(CHEM_EINVAL, "non-finite option");
  return CHEM_OK;
}

// One integration call's options after defaults and checks, and its launch shape.  Shared by
// chem_integrate and chem_integrate_noalloc so that the two entry points cannot drift apart.
struct IntCall {
  chem_integrate_opts o{};
  IntOpts io{};
  unsigned long long budget_ns = 0;
  int grp = 0;     // lane group: 0 one warp, 1 two warps, 2 half a warp per cell
  int cpb = 1;     // cells per block
  int grid = 1;    // persistent form: resident blocks on the device
  int chunk = 1;   // persistent form: cells per queue pull
  int tab = 0;     // tabulated temperature functions
  double tab_tol = 0.0;
  int spec = 0;    // the mechanism-specialised kernels (one warp per cell)
};

chem_status parse_integrate(chem_handle h, int N, const chem_integrate_opts* opts, IntCall& c) {
  chem_integrate_opts& o = c.o;
  if (opts) o = *opts;
  chem_status st = tolerance_opts(o, N, c.io);
  if (st != CHEM_OK) return st;
  if (o.mode != 0 && o.mode != 1) return fail(CHEM_EINVAL, "mode must be 0 (plain) or 1 (persistent)");
  if (o.warps_per_cell < 0 || o.warps_per_cell > kMaxWarpsPerCell)
    return fail(CHEM_EINVAL, "warps_per_cell must be 0 (automatic), 1 or 2");
  if (o.cells_per_warp < 0 || o.cells_per_warp > 2)
    return fail(CHEM_EINVAL, "cells_per_warp must be 0 (automatic), 1 or 2");
  if (o.cells_per_warp == 2 && o.warps_per_cell == 2)
    return fail(CHEM_EINVAL, "cells_per_warp = 2 needs warps_per_cell 0 or 1");
  if (!(o.time_budget_s >= 0.0) || !std::isfinite(o.time_budget_s)) return fail(CHEM_EINVAL, "bad time_budget_s");
  if (o.tabulate != 0 && o.tabulate != 1) return fail(CHEM_EINVAL, "tabulate must be 0 or 1");
  if (!(o.tab_tol >= 0.0 && o.tab_tol < 1.0)) return fail(CHEM_EINVAL, "tab_tol must lie in [0, 1)");
  c.tab = o.tabulate;
  c.tab_tol = o.tab_tol > 0.0 ? o.tab_tol : 1e-10;
  if (c.tab && h->params_shifted)
    return fail(CHEM_EINVAL, "tabulate: the tables hold the description's parameters, which chem_set_params shifted");
  if (o.specialized != 0 && o.specialized != 1) return fail(CHEM_EINVAL, "specialized must be 0 or 1");
  c.spec = o.specialized;
  if (c.spec && !h->spec.plain)
    return fail(CHEM_EINVAL, "specialized: chem_specialize has not compiled this handle's kernels");
  if (c.spec && (o.warps_per_cell > 1 || o.cells_per_warp > 1))
    return fail(CHEM_EINVAL, "specialized kernels integrate one cell per warp (warps_per_cell, cells_per_warp <= 1)");
  if ((st = set_attrs(h)) != CHEM_OK) return st;
  c.budget_ns = (unsigned long long)(o.time_budget_s * 1e9);
  if (c.spec) c.grp = 0;
  else if (o.cells_per_warp == 2) c.grp = 2;
  else if (o.cells_per_warp == 0 && o.warps_per_cell == 0 && h->auto_cpw == 2) c.grp = 2;
  else c.grp = (o.warps_per_cell > 0 ? o.warps_per_cell : h->auto_wpc) - 1;
  c.cpb = cells_per_block(h, o.block_cells, c.grp);
  if (c.spec) c.cpb = std::min(c.cpb, h->spec_max_cells);
  int bps = 1;
  if ((st = persistent_blocks_per_sm(h, c.grp, c.cpb, bps, c.spec != 0)) != CHEM_OK) return st;
  c.grid = h->num_sms * bps;
  // a pull larger than an even share of the cells over the resident lane groups only leaves groups idle
  const long long groups = (long long)c.grid * c.cpb;
  const long long share = std::max(1LL, ((long long)N + groups - 1) / groups);
  c.chunk = (int)std::min<long long>(o.chunk > 0 ? o.chunk : 1, share);
  return CHEM_OK;
}

// Launches of the integration kernel chosen by an integration call: the library's instantiation of lane
// group c.grp, or the mechanism-specialised kernel (same parameters, launched through its handle).
cudaError_t launch_plain(const chem_handle h, const IntCall& c, dim3 grid, dim3 block, size_t smem,
                         cudaStream_t strm, const MechView& V, int N, double* T, const double* p, double* Y,
                         const double* dt, double* h_io, int* nsub, int* status, const unsigned long long* stamp) {
  if (!c.spec)
    return launch_integrate_plain(c.grp, grid, block, smem, strm, V, h->L, N, T, p, Y, dt, h_io, nsub, status,
                                  c.o.naccept, c.io, stamp, c.budget_ns);
  if (block.x % kWarp != 0 || block.y != 1 || block.z != 1) return cudaErrorInvalidValue;
  MechView v = V;
  CellLayout L = h->L;
  int* nacc = c.o.naccept;
  IntOpts io = c.io;
  unsigned long long budget = c.budget_ns;
  void* args[] = {&v, &L, &N, &T, (void*)&p, &Y, (void*)&dt, &h_io, &nsub, &status, &nacc, &io, (void*)&stamp, &budget};
  return cudaLaunchKernel(h->spec.plain, grid, block, args, smem, strm);
}

cudaError_t launch_persistent(const chem_handle h, const IntCall& c, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t strm, const MechView& V, int N, double* T, const double* p, double* Y,
                              const double* dt, double* h_io, int* nsub, int* status, const int* perm,
                              unsigned long long* head, const unsigned long long* stamp) {
  if (!c.spec)
    return launch_integrate_persistent(c.grp, grid, block, smem, strm, V, h->L, N, T, p, Y, dt, h_io, nsub, status,
                                       c.o.naccept, perm, head, c.chunk, c.io, stamp, c.budget_ns);
  if (block.x % kWarp != 0 || block.y != 1 || block.z != 1) return cudaErrorInvalidValue;
  MechView v = V;
  CellLayout L = h->L;
  int* nacc = c.o.naccept;
  int chunk = c.chunk;
  IntOpts io = c.io;
  unsigned long long budget = c.budget_ns;
  void* args[] = {&v,    &L,     &N,    &T,         (void*)&p, &Y,  (void*)&dt,     &h_io,  &nsub,
                  &status, &nacc, (void*)&perm, &head, &chunk,   &io, (void*)&stamp, &budget};
  return cudaLaunchKernel(h->spec.persistent, grid, block, args, smem, strm);
}

// The tables of tolerance tol in device memory: built on the host and uploaded when the handle holds
// none for tol (allocating; may_allocate false: only tables already built are accepted).
chem_status ensure_tables(chem_handle h, double tol, bool may_allocate) {
  if (h->tab_dev && h->tabs.tol == tol) return CHEM_OK;
  if (!may_allocate)
    return fail(CHEM_EINVAL, "tabulate: no tables of this tab_tol in the handle yet (chem_integrate builds them)");
  std::string err;
  HostTables t;
  chem_status st = build_tables(h->hm, tol, t, err);
  if (st != CHEM_OK) return fail(st, err);
  size_t bytes = 0;
  for (int c = 0; c < kTabClasses; ++c) bytes += align_up(t.coef[c].size() * sizeof(double), 256);
  void* dev = nullptr;
  if (bytes > 0 && cudaMalloc(&dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(CHEM_ENOMEM, "cudaMalloc of the tables failed");
  }
  size_t off = 0;
  for (int c = 0; c < kTabClasses; ++c) {
    if (!t.coef[c].empty()) {
      cudaError_t e = cudaMemcpy((char*)dev + off, t.coef[c].data(), t.coef[c].size() * sizeof(double),
                                 cudaMemcpyHostToDevice);
      if (e != cudaSuccess) { cudaFree(dev); return cuda_fail(e, "cudaMemcpy of the tables"); }
    }
    off += align_up(t.coef[c].size() * sizeof(double), 256);
  }
  if (h->tab_dev) cudaFree(h->tab_dev);
  h->tab_dev = dev;
  h->tabs = std::move(t);
  return CHEM_OK;
}

// The view of lane group grp, with the handle's tables switched on when tab is set.
MechView view_for(const chem_handle h, int grp, int tab) {
  MechView V = h->view[grp];
  V.tab_on = 0;
  if (!tab || !h->tab_dev) return V;
  V.tab_on = 1;
  size_t off = 0;
  for (int c = 0; c < kTabClasses; ++c) {
    V.tab_deg[c] = h->tabs.deg[c];
    V.tab[c] = h->tabs.deg[c] > 0 ? (const double*)((const char*)h->tab_dev + off) : nullptr;
    off += align_up(h->tabs.coef[c].size() * sizeof(double), 256);
  }
  V.tab_ulo = h->tabs.u_lo;
  V.tab_du = h->tabs.du;
  V.tab_tlo = kTabTlo;
  V.tab_thi = kTabThi;
  V.tab_ni = kTabIntervals;
  return V;
}

}  // namespace

extern "C" {

const char* chem_last_error(void) { return g_err.c_str(); }

chem_status chem_create(const chem_mech_desc* desc, int device, chem_handle* out) {
  g_err.clear();
  if (!desc || !out) return fail(CHEM_EINVAL, "desc and out must not be NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = device == -1 ? cudaSuccess : cudaGetDeviceCount(&ndev);
  const bool host_only = device == -1;
  if (host_only) {
    chem_handle h = new (std::nothrow) chem_handle_s();
    if (!h) return fail(CHEM_ENOMEM, "host allocation failed");
    h->device = -1;
    std::string err;
    chem_status st = compile_mechanism(*desc, h->hm, err);
    if (st != CHEM_OK) { delete h; return fail(st, err); }
    h->L = make_layout(h->hm);
    h->cell_bytes = h->L.total * (int)sizeof(double);
    *out = h;
    return CHEM_OK;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(CHEM_EINVAL, "device index out of range");
  DeviceScope ds;
  if ((e = ds.enter(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  chem_handle h = new (std::nothrow) chem_handle_s();
  if (!h) return fail(CHEM_ENOMEM, "host allocation failed");
  h->device = device;
  std::string err;
  chem_status st = compile_mechanism(*desc, h->hm, err);
  if (st != CHEM_OK) { delete h; return fail(st, err); }
  const HostMech& hm = h->hm;
  h->L = make_layout(hm);
  h->cell_bytes = h->L.total * (int)sizeof(double);
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDeviceProperties"); }
  h->smem_optin = (int)prop.sharedMemPerBlockOptin;
  h->num_sms = prop.multiProcessorCount;
  if (h->cell_bytes > h->smem_optin) {
    delete h;
    return fail(CHEM_EUNSUPPORTED, "mechanism needs " + std::to_string(h->L.total * 8) +
                                       " bytes of shared memory per cell, more than the device allows");
  }
  // pack every table into one device allocation
  std::vector<char> buf;
  size_t o_sp = put(buf, hm.sp), o_rxd = put(buf, hm.rxd), o_rxi = put(buf, hm.rxi), o_esp = put(buf, hm.eff_sp),
         o_eam = put(buf, hm.eff_am1), o_dsp = put(buf, hm.dslot_sp), o_dmask = put(buf, hm.dslot_mask),
         o_dam = put(buf, hm.dslot_am1), o_er = put(buf, hm.entry_row), o_ec = put(buf, hm.entry_col),
         o_ew = put(buf, hm.entry_wratio), o_lsrc = put(buf, hm.lu_src), o_ldiag = put(buf, hm.lu_diag),
         o_sout = put(buf, hm.s_out), o_rxo = put(buf, hm.rx_order), o_rxd0 = put(buf, hm.rxd);
  const int n_jp = (int)hm.jpass.size() / 4;
  if (n_jp > kMaxJPass) { delete h; return fail(CHEM_EUNSUPPORTED, "too many Jacobian passes"); }
  constexpr int kMaxG = 3 + kMaxJPass;
  size_t o_g[kNumGroups][kMaxG][2], o_lops[kNumGroups], o_sops[kNumGroups], o_tops[kNumGroups];
  const HostGather* gs[kNumGroups][kMaxG];
  for (int w = 0; w < kNumGroups; ++w) {
    const HostProg& P = hm.prog[w];
    gs[w][0] = &P.g_omega; gs[w][1] = &P.g_row; gs[w][2] = &P.g_col;
    for (int i = 0; i < n_jp; ++i) gs[w][3 + i] = &P.g_jac[i];
    for (int i = 0; i < 3 + n_jp; ++i) { o_g[w][i][0] = put(buf, gs[w][i]->ops); o_g[w][i][1] = put(buf, gs[w][i]->comb); }
    o_lops[w] = put(buf, P.lu_ops); o_sops[w] = put(buf, P.sv_ops); o_tops[w] = put(buf, P.svT_ops);
  }
  if ((e = cudaMalloc(&h->blob, buf.size())) != cudaSuccess) { delete h; return fail(CHEM_ENOMEM, "cudaMalloc of mechanism tables failed"); }
  if ((e = cudaMemcpy(h->blob, buf.data(), buf.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(h->blob);
    delete h;
    return cuda_fail(e, "cudaMemcpy of mechanism tables");
  }
  char* b = (char*)h->blob;
  h->rxd0 = (const double*)(b + o_rxd0);
  for (int w = 0; w < kNumGroups; ++w) {
    const HostProg& P = hm.prog[w];
    MechView& V = h->view[w];
    V.width = P.width;
    V.n = hm.n; V.R = hm.R; V.m = hm.m; V.n_troe = hm.n_troe; V.n_tb = hm.n_tb; V.nY = hm.nY; V.nnz_S = hm.nnz_S;
    V.nnz_LU = hm.nnz_LU; V.n_dslot = hm.n_dslot;
    V.sp = (const double*)(b + o_sp); V.rxd = (const double*)(b + o_rxd); V.rxi = (const int*)(b + o_rxi);
    V.eff_sp = (const int*)(b + o_esp); V.eff_am1 = (const double*)(b + o_eam);
    V.dslot_sp = (const int*)(b + o_dsp); V.dslot_mask = (const int*)(b + o_dmask);
    V.dslot_am1 = (const double*)(b + o_dam);
    V.entry_row = (const int*)(b + o_er); V.entry_col = (const int*)(b + o_ec);
    V.entry_wratio = (const double*)(b + o_ew);
    V.lu_src = (const int*)(b + o_lsrc); V.lu_diag = (const int*)(b + o_ldiag);
    V.lu_ops = (const ElimOp*)(b + o_lops[w]); V.lu_steps = (int)P.lu_kind.size();
    V.sv_ops = (const ElimOp*)(b + o_sops[w]); V.sv_steps = (int)P.sv_kind.size();
    V.svT_ops = (const ElimOp*)(b + o_tops[w]); V.svT_steps = (int)P.svT_kind.size();
    V.s_out = (const int*)(b + o_sout);
    V.rx_order = (const int*)(b + o_rxo);
    V.n_jpass = n_jp;
    for (int i = 0; i < n_jp; ++i)
      for (int j = 0; j < 4; ++j) V.jpass[i][j] = hm.jpass[(size_t)i * 4 + j];
    Gather* vg[kMaxG] = {&V.g_omega, &V.g_row, &V.g_col};
    for (int i = 0; i < n_jp; ++i) vg[3 + i] = &V.g_jac[i];
    for (int i = 0; i < 3 + n_jp; ++i) {
      vg[i]->ops = (const GatherOp*)(b + o_g[w][i][0]);
      vg[i]->steps = gs[w][i]->steps;
      vg[i]->n_partial = gs[w][i]->n_partial;
      vg[i]->comb = (const int*)(b + o_g[w][i][1]);
      vg[i]->n_comb = (int)gs[w][i]->comb.size() / 3;
    }
  }
  *out = h;
  return CHEM_OK;
}

chem_status chem_balance_plan(int world, const int64_t* counts, const double* costs, int32_t* dest) {
  g_err.clear();
  std::string err;
  const chem_status st = balance_plan(world, counts, costs, dest, err);
  return st == CHEM_OK ? CHEM_OK : fail(st, err);
}

chem_status chem_create_from_json(const char* json_text, int device, chem_handle* out) {
  g_err.clear();
  if (!out) return fail(CHEM_EINVAL, "out must not be NULL");
  *out = nullptr;
  JsonMech jm;
  std::string err;
  const chem_status st = parse_mech_json(json_text, jm, err);
  if (st != CHEM_OK) return fail(st, err);
  return chem_create(&jm.desc, device, out);   // compiles into the handle's own tables
}

chem_status chem_destroy(chem_handle h) {
  if (!h) return CHEM_OK;
  if (h->device < 0) { delete h; return CHEM_OK; }
  DeviceScope ds;
  ds.enter(h->device);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->blob) cudaFree(h->blob);
  if (h->scratch) cudaFree(h->scratch);
  if (h->adj_scratch) cudaFree(h->adj_scratch);
  if (h->map_scratch) cudaFree(h->map_scratch);
  if (h->tab_dev) cudaFree(h->tab_dev);
  release_specialized(h->spec);
  delete h;
  return CHEM_OK;
}

chem_status chem_specialize(chem_handle h, double* compile_s) {
  if (h && h->device < 0) {   // host-only handle: compile into the cache, load nothing
    std::string err;
    SpecKernels k;
    chem_status st = compile_specialized(h->hm, h->L, false, k, err);
    if (st != CHEM_OK) return fail(st, err);
    if (compile_s) *compile_s = k.compile_s;
    return CHEM_OK;
  }
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (h->spec.plain) {   // already compiled for this handle (graphs may hold the loaded kernels)
    if (compile_s) *compile_s = 0.0;
    return CHEM_OK;
  }
  if ((st = set_attrs(h)) != CHEM_OK) return st;
  std::string err;
  SpecKernels k;
  if ((st = compile_specialized(h->hm, h->L, true, k, err)) != CHEM_OK) return fail(st, err);
  cudaError_t e = cudaSuccess;
  cudaFuncAttributes fa1, fa2;
  for (const void* f : {k.plain, k.persistent})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa1, k.plain);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa2, k.persistent);
  if (e != cudaSuccess) {
    release_specialized(k);
    return cuda_fail(e, "attributes of the specialised kernels");
  }
  // largest block: the generic one-warp bound and the threads the specialised kernels' registers allow
  h->spec_max_cells =
      std::max(1, std::min(h->max_cells[0], std::min(fa1.maxThreadsPerBlock, fa2.maxThreadsPerBlock) / kWarp));
  h->spec = k;
  if (compile_s) *compile_s = k.compile_s;
  return CHEM_OK;
}

chem_status chem_specialized_source(chem_handle h, char* buf, int* len) {
  if (!h || !len) return fail(CHEM_EINVAL, "null argument");
  const std::string src = specialized_source(h->hm, h->L);
  const int need = (int)src.size() + 1;
  if (buf && *len >= need) std::memcpy(buf, src.c_str(), (size_t)need);
  const bool small = buf && *len < need;
  *len = need;
  return small ? fail(CHEM_EINVAL, "buffer too small (len now holds the size needed)") : CHEM_OK;
}

chem_status chem_info(chem_handle h, chem_info_t* info) {
  if (!h || !info) return fail(CHEM_EINVAL, "null argument");
  info->n_species = h->hm.n;
  info->n_reactions = h->hm.R;
  info->n_state = h->hm.m;
  info->nnz_S = h->hm.nnz_S;
  info->nnz_LU = h->hm.nnz_LU;
  info->lu_steps = (int)h->hm.prog[0].lu_kind.size();
  info->solve_steps = (int)h->hm.prog[0].sv_kind.size();
  info->smem_per_cell = h->cell_bytes;
  info->n_dslots = h->hm.n_dslot;
  info->jac_passes = (int)h->hm.jpass.size() / 4;
  info->smem_adjoint_per_cell = make_adj_layout(h->hm, 16).L.total * (int)sizeof(double);
  for (int w = 0; w < kNumGroups; ++w) { info->max_block_cells[w] = 0; info->resident_cells[w] = 0; }
  info->auto_warps_per_cell = 0;
  info->auto_cells_per_warp = 0;
  if (h->device >= 0) {
    DeviceScope ds;
    chem_status st = check_handle(h, ds);
    if (st == CHEM_OK) st = set_attrs(h);
    if (st != CHEM_OK) return st;
    for (int w = 0; w < kNumGroups; ++w) {
      info->max_block_cells[w] = h->max_cells[w];
      info->resident_cells[w] = h->resident_cells[w];
    }
    info->auto_warps_per_cell = h->auto_wpc;
    info->auto_cells_per_warp = h->auto_cpw;
  }
  return CHEM_OK;
}

chem_status chem_jacobian_pattern(chem_handle h, int* row_ptr, int* col_idx) {
  if (!h || !row_ptr || !col_idx) return fail(CHEM_EINVAL, "null argument");
  std::copy(h->hm.csr_ptr.begin(), h->hm.csr_ptr.end(), row_ptr);
  std::copy(h->hm.csr_col.begin(), h->hm.csr_col.end(), col_idx);
  return CHEM_OK;
}

chem_status chem_export_plan(chem_handle h, int which, int* out, int* count) {
  if (!h || !count) return fail(CHEM_EINVAL, "null argument");
  const HostMech& hm = h->hm;
  std::vector<int> v;
  auto prog = [&](const std::vector<ElimOp>& ops, const std::vector<uint8_t>& kinds, int width) {
    for (size_t st = 0; st < kinds.size(); ++st)
      for (int l = 0; l < width; ++l) {
        const ElimOp& o = ops[st * width + l];
        v.push_back(kinds[st]); v.push_back(o.t); v.push_back(o.a); v.push_back(o.b);
      }
  };
  const HostProg& P1 = hm.prog[0];
  const HostProg& P2 = hm.prog[1];
  switch (which) {
    case 0: prog(P1.lu_ops, P1.lu_kind, P1.width); break;
    case 1: prog(P1.sv_ops, P1.sv_kind, P1.width); break;
    case 2: v = hm.perm; break;
    case 3: v = hm.lu_rowptr; v.insert(v.end(), hm.lu_col.begin(), hm.lu_col.end()); break;
    case 4: v = hm.lu_src; break;
    case 5: v = hm.s_out; break;
    case 6: prog(P1.svT_ops, P1.svT_kind, P1.width); break;
    case 7: v = hm.rx_order; break;
    case 8: prog(P2.lu_ops, P2.lu_kind, P2.width); break;
    case 9: prog(P2.sv_ops, P2.sv_kind, P2.width); break;
    case 10: prog(P2.svT_ops, P2.svT_kind, P2.width); break;
    case 11: prog(hm.prog[2].lu_ops, hm.prog[2].lu_kind, hm.prog[2].width); break;
    case 12: prog(hm.prog[2].sv_ops, hm.prog[2].sv_kind, hm.prog[2].width); break;
    case 13: prog(hm.prog[2].svT_ops, hm.prog[2].svT_kind, hm.prog[2].width); break;
    default: return fail(CHEM_EINVAL, "unknown plan part");
  }
  if (out) std::copy(v.begin(), v.end(), out);
  *count = (int)v.size();
  return CHEM_OK;
}

chem_status chem_rates(chem_handle h, int N, const double* T, const double* p, const double* Y, double* dTdt,
                       double* dYdt, double* wdot, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !dTdt || !dYdt) return fail(CHEM_EINVAL, "null array argument");
  if ((st = set_attrs(h)) != CHEM_OK) return st;
  const int wpb = cells_per_block(h, 4, 0);
  k_rates<<<(N + wpb - 1) / wpb, wpb * kWarp, wpb * h->cell_bytes, (cudaStream_t)stream>>>(h->view[0], h->L, N, T, p, Y,
                                                                                           dTdt, dYdt, wdot);
  return launch_check("chem_rates launch");
}

chem_status chem_jacobian(chem_handle h, int N, const double* T, const double* p, const double* Y, double* S_vals,
                          double* u, double* v, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !S_vals || !u || !v) return fail(CHEM_EINVAL, "null array argument");
  if ((st = set_attrs(h)) != CHEM_OK) return st;
  const int wpb = cells_per_block(h, 4, 0);
  k_jacobian<<<(N + wpb - 1) / wpb, wpb * kWarp, wpb * h->cell_bytes, (cudaStream_t)stream>>>(h->view[0], h->L, N, T, p,
                                                                                              Y, S_vals, u, v);
  return launch_check("chem_jacobian launch");
}

chem_status chem_integrate(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                           double* h_io, int* nsub, int* status, const chem_integrate_opts* opts, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !dt || !h_io || !nsub || !status) return fail(CHEM_EINVAL, "null array argument");
  IntCall c;
  if ((st = parse_integrate(h, N, opts, c)) != CHEM_OK) return st;
  const chem_integrate_opts& o = c.o;
  const IntOpts& io = c.io;
  const unsigned long long budget_ns = c.budget_ns;
  cudaStream_t strm = (cudaStream_t)stream;
  cudaError_t e;
  const int grp = c.grp;
  const int width = kGroupWidth[grp];
  if (c.tab && (st = ensure_tables(h, c.tab_tol, true)) != CHEM_OK) return st;
  const MechView V = view_for(h, grp, c.tab);
  const int cpb = c.cpb;
  if (o.mode == 0) {
    unsigned long long* stamp = nullptr;
    if (budget_ns) {
      if ((st = ensure_scratch(h, 1)) != CHEM_OK) return st;
      stamp = (unsigned long long*)((char*)h->scratch + kScrStamp);
      k_stamp<<<1, 32, 0, strm>>>(stamp);
    }
    if ((e = launch_plain(h, c, (N + cpb - 1) / cpb, cpb * width, cpb * h->cell_bytes, strm, V, N, T, p, Y, dt, h_io,
                          nsub, status, stamp)) != cudaSuccess)
      return cuda_fail(e, "chem_integrate launch shape");
    return launch_check("chem_integrate launch");
  }
  // persistent mode: sort by previous cost, then one resident grid pulling from the queue; the whole
  // sequence is one CUDA graph, captured once per argument set and replayed on `stream`
  if ((st = ensure_scratch(h, N)) != CHEM_OK) return st;
  const int chunk = c.chunk;
  chem_handle_s::GraphKey key{};
  key.N = N; key.mode = 1; key.cpb = cpb; key.chunk = chunk; key.grp = grp;
  const void* ptrs[10] = {T, p, Y, dt, h_io, nsub, status, o.naccept, o.trace, h->scratch};
  for (int i = 0; i < 10; ++i) key.ptr[i] = ptrs[i];
  key.d[0] = io.rtol; key.d[1] = io.atol; key.d[2] = io.h_init; key.d[3] = io.h_min; key.d[4] = o.time_budget_s;
  key.i[0] = io.max_substeps; key.i[1] = io.max_nonfinite; key.i[2] = io.trace_cap; key.i[3] = io.method;
  key.i[4] = c.tab + 2 * c.spec;
  key.d[5] = c.tab ? c.tab_tol : 0.0;
  if (!h->gexec || !(h->gkey == key)) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (!h->cap_stream && (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    const int grid = std::min(c.grid, (N + cpb - 1) / cpb);
    char* scr = (char*)h->scratch;
    int* counts = (int*)(scr + kScrCounts);
    int* cursor = (int*)(scr + kScrCursor);
    unsigned long long* head = (unsigned long long*)(scr + kScrHead);
    unsigned long long* stamp = (unsigned long long*)(scr + kScrStamp);
    int* perm = (int*)(scr + kScrPerm);
    const int sblocks = std::min(4 * h->num_sms, (N + 255) / 256);
    cudaStream_t cs = h->cap_stream;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamBeginCapture");
    cudaMemsetAsync(scr, 0, kScrHead + 8, cs);
    k_stamp<<<1, 32, 0, cs>>>(stamp);
    k_sort_count<<<sblocks, 256, 0, cs>>>(N, nsub, counts);
    k_sort_scatter<<<sblocks, 256, 0, cs>>>(N, nsub, counts, cursor, perm);
    const cudaError_t se = launch_persistent(h, c, grid, cpb * width, cpb * h->cell_bytes, cs, V, N, T, p, Y, dt,
                                             h_io, nsub, status, perm, head, stamp);
    cudaGraph_t graph = nullptr;
    cudaError_t le = se != cudaSuccess ? se : cudaGetLastError();
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(le, "persistent launch capture"); }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { h->gexec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    h->gkey = key;
  }
  if ((e = cudaGraphLaunch(h->gexec, strm)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return launch_check("chem_integrate launch");
}

}  // extern "C"

extern "C" chem_status chem_set_params(chem_handle h, const double* dlnA, const double* dEa, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  h->params_shifted = dlnA != nullptr || dEa != nullptr;
  if (h->hm.R == 0) return CHEM_OK;
  k_set_params<<<(h->hm.R + 127) / 128, 128, 0, (cudaStream_t)stream>>>(h->view[0], h->rxd0, (double*)h->view[0].rxd,
                                                                         dlnA, dEa);
  return launch_check("chem_set_params launch");
}

extern "C" chem_status chem_adjoint(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                                    const double* gT, const double* gY, double* grad_lnA, double* grad_Ea,
                                    double* grad_cell, double* gT0, double* gY0, int* status,
                                    const chem_integrate_opts* opts, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !dt || !gT || !gY || !grad_lnA || !grad_Ea || !status)
    return fail(CHEM_EINVAL, "null array argument");
  chem_integrate_opts o{};
  if (opts) o = *opts;
  if (o.method != 0) return fail(CHEM_EINVAL, "chem_adjoint differentiates RODAS3 steps only (method 0)");
  if (o.tabulate) return fail(CHEM_EINVAL, "chem_adjoint differentiates the exact functions only (tabulate 0)");
  o.trace = nullptr;   // the adjoint records its own tape instead
  IntOpts io;
  if ((st = tolerance_opts(o, N, io)) != CHEM_OK) return st;
  const int K = o.ckpt_every > 0 ? o.ckpt_every : 16;
  const int cap = o.tape_steps > 0 ? o.tape_steps : 4096;
  if (K > 64) return fail(CHEM_EINVAL, "ckpt_every must be <= 64");
  if ((st = set_attrs(h)) != CHEM_OK) return st;
  const HostMech& hm = h->hm;
  const int m = hm.m;
  const AdjLayout A = make_adj_layout(hm, K);
  const int adj_bytes = A.L.total * (int)sizeof(double);
  if (adj_bytes > h->smem_optin)
    return fail(CHEM_EUNSUPPORTED, "adjoint needs " + std::to_string(adj_bytes) + " bytes of shared memory per cell");
  cudaError_t e;
  if (!h->adj_attr_set) {
    if ((e = cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem_optin)) != cudaSuccess)
      return cuda_fail(e, "cudaFuncSetAttribute");
    h->adj_attr_set = true;
  }
  int bps = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_adjoint, kWarp, (size_t)adj_bytes)) != cudaSuccess)
    return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  bps = std::max(bps, 1);
  const int grid = std::min(h->num_sms * bps, N);
  // scratch: head, tape (h, checkpoints, counts), h_io/nsub of the forward pass, per-cell gradients,
  // dual workspaces
  const size_t nck = (size_t)(cap / K + 1);
  const size_t b_head = 256;
  const size_t b_rh = align_up((size_t)cap * N * 8, 256);
  const size_t b_ck = align_up(nck * m * N * 8, 256);
  const size_t b_rn = align_up((size_t)N * 4, 256);
  const size_t b_hio = align_up((size_t)N * 8, 256);
  const size_t b_ns = align_up((size_t)N * 4, 256);
  const size_t b_gc = grad_cell ? 0 : align_up((size_t)2 * hm.R * N * 8, 256);
  const size_t b_dw = align_up((size_t)grid * h->L.total * sizeof(Dual4), 256);
  const size_t b_ww = align_up((size_t)grid * (size_t)A.total * 8, 256);
  const size_t need = b_head + b_rh + b_ck + b_rn + b_hio + b_ns + b_gc + b_dw + b_ww;
  if (need > h->adj_scratch_bytes) {
    if (h->adj_scratch) cudaFree(h->adj_scratch);
    h->adj_scratch = nullptr;
    h->adj_scratch_bytes = 0;
    if (cudaMalloc(&h->adj_scratch, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(CHEM_ENOMEM, "cudaMalloc of adjoint scratch (" + std::to_string(need) + " bytes) failed");
    }
    h->adj_scratch_bytes = need;
  }
  char* q = (char*)h->adj_scratch;
  int* head = (int*)q; q += b_head;
  double* rec_h = (double*)q; q += b_rh;
  double* rec_ck = (double*)q; q += b_ck;
  int* rec_n = (int*)q; q += b_rn;
  double* hio = (double*)q; q += b_hio;
  int* nsub = (int*)q; q += b_ns;
  double* gcell = grad_cell;
  if (!gcell) { gcell = (double*)q; q += b_gc; }
  Dual4* dws = (Dual4*)q; q += b_dw;
  double* wws = (double*)q;
  cudaStream_t strm = (cudaStream_t)stream;
  // forward pass with the tape
  io.rec_h = rec_h; io.rec_ck = rec_ck; io.rec_n = rec_n; io.rec_cap = cap; io.rec_K = K;
  if ((e = cudaMemsetAsync(hio, 0, (size_t)N * 8, strm)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if ((e = launch_integrate_plain(0, N, kWarp, h->cell_bytes, strm, h->view[0], h->L, N, T, p, Y, dt, hio, nsub, status,
                                  nullptr, io, nullptr, 0ull)) != cudaSuccess)
    return cuda_fail(e, "chem_adjoint forward launch shape");
  if ((st = launch_check("chem_adjoint forward launch")) != CHEM_OK) return st;
  // reverse pass, cells ordered by tape length (longest first) as in the sorted work queue
  io.rec_h = nullptr; io.rec_ck = nullptr; io.rec_n = nullptr;
  if ((st = ensure_scratch(h, N)) != CHEM_OK) return st;
  char* scr = (char*)h->scratch;
  int* perm = (int*)(scr + kScrPerm);
  if ((e = cudaMemsetAsync(scr, 0, kScrHead + 8, strm)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const int sblocks = std::min(4 * h->num_sms, (N + 255) / 256);
  k_sort_count<<<sblocks, 256, 0, strm>>>(N, rec_n, (int*)(scr + kScrCounts));
  k_sort_scatter<<<sblocks, 256, 0, strm>>>(N, rec_n, (int*)(scr + kScrCounts), (int*)(scr + kScrCursor), perm);
  if ((e = cudaMemsetAsync(head, 0, 4, strm)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  k_adjoint<<<grid, kWarp, adj_bytes, strm>>>(h->view[0], A, N, p, rec_h, rec_ck, rec_n, K, gT, gY, gcell, gT0, gY0,
                                               status, head, perm, dws, wws, io);
  if ((st = launch_check("chem_adjoint reverse launch")) != CHEM_OK) return st;
  const int P = 2 * hm.R;
  if (P > 0) {
    k_grad_reduce<<<(P * kWarp + 255) / 256, 256, 0, strm>>>(N, P, gcell, grad_lnA, grad_Ea, hm.R);
    if ((st = launch_check("chem_adjoint reduction launch")) != CHEM_OK) return st;
  }
  return CHEM_OK;
}

// Device address of the static scratch array on the current device.  In host code the array's name
// only stands for it; the real address is looked up once per device and kept.
namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

chem_status noalloc_scratch_address(int device, char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= kNoAllocMaxDevices) return fail(CHEM_EUNSUPPORTED, "device index too large");
  if (!g_noalloc_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_noalloc_addr[device] = ptr;
  }
  *out = (char*)g_noalloc_addr[device];
  return CHEM_OK;
}
}  // namespace

extern "C" chem_status chem_integrate_noalloc(chem_handle h, int N, double* T, const double* p, double* Y,
                                              const double* dt, double* h_io, int* nsub, int* status,
                                              const chem_integrate_opts* opts, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N > kNoAllocMaxCells)
    return fail(CHEM_EINVAL, "chem_integrate_noalloc handles at most " + std::to_string(kNoAllocMaxCells) +
                                 " cells per call (fixed static scratch); got " + std::to_string(N));
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !dt || !h_io || !nsub || !status) return fail(CHEM_EINVAL, "null array argument");
  chem_integrate_opts o1{};
  if (opts) o1 = *opts;
  o1.mode = 1;   // always the sorted work queue
  IntCall c;
  if ((st = parse_integrate(h, N, &o1, c)) != CHEM_OK) return st;
  if (c.tab && (st = ensure_tables(h, c.tab_tol, false)) != CHEM_OK) return st;
  char* scr = nullptr;
  if ((st = noalloc_scratch_address(h->device, &scr)) != CHEM_OK) return st;
  const int grp = c.grp, wpb = c.cpb;
  const int grid = std::min(c.grid, (N + wpb - 1) / wpb);
  const int sblocks = std::min(4 * h->num_sms, (N + 255) / 256);
  int* counts = (int*)(scr + kScrCounts);
  int* cursor = (int*)(scr + kScrCursor);
  unsigned long long* head = (unsigned long long*)(scr + kScrHead);
  unsigned long long* stamp = (unsigned long long*)(scr + kScrStamp);
  int* perm = (int*)(scr + kScrPerm);
  cudaStream_t strm = (cudaStream_t)stream;
  cudaError_t e;
  // the array keeps the previous call's contents: clear the counters and the queue head first
  if ((e = cudaMemsetAsync(scr, 0, kScrHead + 8, strm)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  k_stamp<<<1, 32, 0, strm>>>(stamp);
  k_sort_count<<<sblocks, 256, 0, strm>>>(N, nsub, counts);
  k_sort_scatter<<<sblocks, 256, 0, strm>>>(N, nsub, counts, cursor, perm);
  if ((e = launch_persistent(h, c, grid, wpb * kGroupWidth[grp], wpb * h->cell_bytes, strm, view_for(h, grp, c.tab),
                             N, T, p, Y, dt, h_io, nsub, status, perm, head, stamp)) != cudaSuccess)
    return cuda_fail(e, "chem_integrate_noalloc launch shape");
  return launch_check("chem_integrate_noalloc launch");
}

namespace {
__global__ void k_elementary(int fn, int N, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double v = x[i];
  y[i] = fn == 0 ? fast_exp(v) : fn == 1 ? exp(v) : fn == 2 ? fast_log(v) : log(v);
}
}  // namespace

extern "C" chem_status chem_eval_elementary(int fn, int N, const double* x, double* y, chem_stream stream) {
  if (fn < 0 || fn > 3)
    return fail(CHEM_EINVAL, "fn must be 0 (library exp), 1 (CUDA exp), 2 (library log) or 3 (CUDA log)");
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N == 0) return CHEM_OK;
  if (!x || !y) return fail(CHEM_EINVAL, "null array argument");
  k_elementary<<<(N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(fn, N, x, y);
  return launch_check("chem_eval_elementary launch");
}

// ===================================================================== zonal reference-cell mapping
// Sec. 2.5: where the reactivity is low, a cell's chemistry solution is mapped from a reference cell.
// Zones are found with one open-addressing hash table over the zone keys: every candidate inserts its
// key and lowers the slot's cell index to its own (atomicMin), so each zone's reference is its lowest
// index whatever the thread order; a candidate then compares its quantised key with that reference's
// (a 64-bit hash collision between two zones therefore only costs mapping, never correctness).  The
// cells to integrate are compacted, integrated by chem_integrate, and the members of each zone take
// their reference's change before the integrated results are scattered back.
namespace {

struct MapKey {
  double T_max, dT;
  int ns;
  int sp[8];
  double dY[8];
};

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// The zone of cell c: q[0] = floor(T/dT), q[1 + i] = floor(Y_s_i / dY_i); false if c is not a candidate
// (T >= T_max, a non-finite key value, p or dt, or a quotient of magnitude 2^62 or more).
__device__ bool zone_of(const MapKey& mk, int N, int c, const double* T, const double* p, const double* Y,
                        const double* dt, long long* q) {
  const double t = T[c];
  if (!(isfinite(t) && t < mk.T_max) || !isfinite(p[c]) || !isfinite(dt[c])) return false;
  for (int i = 0; i <= mk.ns; ++i) {
    const double x = i == 0 ? t : Y[(size_t)mk.sp[i - 1] * N + c];
    const double d = i == 0 ? mk.dT : mk.dY[i - 1];
    if (!isfinite(x)) return false;
    const double r = x / d;
    if (!(fabs(r) < 4611686018427387904.0)) return false;   // 2^62
    q[i] = (long long)floor(r);
  }
  return true;
}

__device__ unsigned long long zone_hash(const long long* q, int nq, double p, double dt) {
  unsigned long long h = mix64((unsigned long long)__double_as_longlong(p + 0.0));   // -0 and +0 alike
  h = mix64(h ^ (unsigned long long)__double_as_longlong(dt + 0.0));
  for (int i = 0; i < nq; ++i) h = mix64(h ^ (unsigned long long)q[i]);
  return h ? h : 1ull;   // 0 marks an empty slot and a non-candidate
}

__global__ void k_fill_int(int n, int* __restrict__ a, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_map_insert(MapKey mk, int N, const double* __restrict__ T, const double* __restrict__ p,
                             const double* __restrict__ Y, const double* __restrict__ dt,
                             unsigned long long* __restrict__ key, unsigned long long* tkey, int* tref,
                             unsigned tmask) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  long long q[9];
  if (!zone_of(mk, N, c, T, p, Y, dt, q)) { key[c] = 0ull; return; }
  const unsigned long long hs = zone_hash(q, mk.ns + 1, p[c], dt[c]);
  key[c] = hs;
  unsigned s = (unsigned)hs & tmask;
  for (unsigned it = 0; it <= tmask; ++it, s = (s + 1u) & tmask) {   // the table is at least half empty
    const unsigned long long prev = atomicCAS(&tkey[s], 0ull, hs);
    if (prev == 0ull || prev == hs) { atomicMin(&tref[s], c); return; }
  }
}

__global__ void k_map_resolve(MapKey mk, int N, const double* __restrict__ T, const double* __restrict__ p,
                              const double* __restrict__ Y, const double* __restrict__ dt,
                              const unsigned long long* __restrict__ key, const unsigned long long* __restrict__ tkey,
                              const int* __restrict__ tref, unsigned tmask, int* __restrict__ ref,
                              int* __restrict__ pos, int* __restrict__ list, int* count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  int r = c;
  const unsigned long long hs = key[c];
  if (hs) {
    unsigned s = (unsigned)hs & tmask;
    for (unsigned it = 0; it <= tmask; ++it, s = (s + 1u) & tmask) {
      const unsigned long long k = tkey[s];
      if (k == hs) { r = tref[s]; break; }
      if (k == 0ull) break;
    }
    if (r < 0 || r >= N) r = c;
    if (r != c) {
      long long qa[9], qb[9];
      bool same = zone_of(mk, N, c, T, p, Y, dt, qa) && zone_of(mk, N, r, T, p, Y, dt, qb) && p[c] == p[r] &&
                  dt[c] == dt[r];
      for (int i = 0; same && i <= mk.ns; ++i) same = qa[i] == qb[i];
      if (!same) r = c;
    }
  }
  ref[c] = r;
  if (r == c) {
    const int j = atomicAdd(count, 1);
    list[j] = c;
    pos[c] = j;
  }
}

__global__ void k_map_gather(int M, const int* __restrict__ list, int N, int n, const double* __restrict__ T,
                             const double* __restrict__ p, const double* __restrict__ Y,
                             const double* __restrict__ dt, const double* __restrict__ h_io,
                             const int* __restrict__ nsub, double* __restrict__ cT, double* __restrict__ cp,
                             double* __restrict__ cY, double* __restrict__ cdt, double* __restrict__ ch,
                             int* __restrict__ cns) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int c = list[j];
  cT[j] = T[c]; cp[j] = p[c]; cdt[j] = dt[c]; ch[j] = h_io[c]; cns[j] = nsub[c];
  for (int k = 0; k < n; ++k) cY[(size_t)k * M + j] = Y[(size_t)k * N + c];
}

// members take their reference's change; runs before the scatter, so T[r], Y[.., r] still hold the
// references' initial states
__global__ void k_map_apply(int N, int n, const int* __restrict__ ref, const int* __restrict__ pos,
                            double* __restrict__ T, double* __restrict__ Y, int* __restrict__ nsub,
                            int* __restrict__ status, const double* __restrict__ cT, const double* __restrict__ cY,
                            const int* __restrict__ cst, int M) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int r = ref[c];
  if (r == c) return;
  const int j = pos[r];
  T[c] = T[c] + (cT[j] - T[r]);
  for (int k = 0; k < n; ++k) {
    const size_t o = (size_t)k * N;
    Y[o + c] = Y[o + c] + (cY[(size_t)k * M + j] - Y[o + r]);
  }
  status[c] = cst[j];
  nsub[c] = 0;
}

__global__ void k_map_scatter(int M, const int* __restrict__ list, int N, int n, const double* __restrict__ cT,
                              const double* __restrict__ cY, const double* __restrict__ ch,
                              const int* __restrict__ cns, const int* __restrict__ cst, double* __restrict__ T,
                              double* __restrict__ Y, double* __restrict__ h_io, int* __restrict__ nsub,
                              int* __restrict__ status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int c = list[j];
  T[c] = cT[j]; h_io[c] = ch[j]; nsub[c] = cns[j]; status[c] = cst[j];
  for (int k = 0; k < n; ++k) Y[(size_t)k * N + c] = cY[(size_t)k * M + j];
}

// scratch of one call, 256-byte aligned pieces
struct MapScratch {
  unsigned long long *key, *tkey;
  int *tref, *pos, *list, *count, *cns, *cst;
  double *cT, *cp, *cdt, *ch, *cY;
  unsigned tmask;
  size_t bytes;
};

MapScratch map_layout(char* base, int N, int n) {
  unsigned S = 1024;
  while (S < 2u * (unsigned)N) S <<= 1;
  MapScratch m{};
  size_t o = 0;
  // base == nullptr: only the size is wanted
  auto take = [&](size_t b) { size_t at = o; o = align_up(o + b, 256); return base ? base + at : nullptr; };
  m.key = (unsigned long long*)take((size_t)N * 8);
  m.tkey = (unsigned long long*)take((size_t)S * 8);
  m.tref = (int*)take((size_t)S * 4);
  m.pos = (int*)take((size_t)N * 4);
  m.list = (int*)take((size_t)N * 4);
  m.count = (int*)take(4);
  m.cns = (int*)take((size_t)N * 4);
  m.cst = (int*)take((size_t)N * 4);
  m.cT = (double*)take((size_t)N * 8);
  m.cp = (double*)take((size_t)N * 8);
  m.cdt = (double*)take((size_t)N * 8);
  m.ch = (double*)take((size_t)N * 8);
  m.cY = (double*)take((size_t)N * n * 8);
  m.tmask = S - 1;
  m.bytes = o;
  return m;
}

}  // namespace

extern "C" chem_status chem_integrate_mapped(chem_handle h, int N, double* T, const double* p, double* Y,
                                             const double* dt, double* h_io, int* nsub, int* status,
                                             const chem_integrate_opts* opts, const chem_map_opts* map, int* ref,
                                             int* n_integrated, chem_stream stream) {
  DeviceScope ds;
  chem_status st = check_handle(h, ds);
  if (st != CHEM_OK) return st;
  if (n_integrated) *n_integrated = 0;
  if (N < 0) return fail(CHEM_EINVAL, "N must be >= 0");
  if (N > (1 << 29)) return fail(CHEM_EINVAL, "N must be <= 2^29 for chem_integrate_mapped");
  if (N == 0) return CHEM_OK;
  if (!T || !p || !Y || !dt || !h_io || !nsub || !status || !ref) return fail(CHEM_EINVAL, "null array argument");
  chem_integrate_opts o{};
  if (opts) o = *opts;
  if (o.trace || o.naccept) return fail(CHEM_EINVAL, "chem_integrate_mapped takes no trace and no naccept");
  const int n = h->hm.n;
  MapKey mk{};
  mk.T_max = -INFINITY;   // no candidates
  mk.dT = 1.0;
  if (map) {
    if (std::isnan(map->T_max)) return fail(CHEM_EINVAL, "map->T_max is NaN");
    if (!(map->dT > 0.0) || !std::isfinite(map->dT)) return fail(CHEM_EINVAL, "map->dT must be finite and > 0");
    if (map->n_species < 0 || map->n_species > 8) return fail(CHEM_EINVAL, "map->n_species must be 0..8");
    mk.T_max = map->T_max;
    mk.dT = map->dT;
    mk.ns = map->n_species;
    for (int i = 0; i < mk.ns; ++i) {
      const int s = map->species[i];
      if (s < 0 || s >= n) return fail(CHEM_EINVAL, "map->species out of range");
      for (int j = 0; j < i; ++j)
        if (map->species[j] == s) return fail(CHEM_EINVAL, "map->species repeats a species");
      if (!(map->dY[i] > 0.0) || !std::isfinite(map->dY[i])) return fail(CHEM_EINVAL, "map->dY must be finite and > 0");
      mk.sp[i] = s;
      mk.dY[i] = map->dY[i];
    }
  }
  cudaError_t e;
  const size_t need = map_layout(nullptr, N, n).bytes;
  if (h->map_scratch_bytes < need) {
    if (h->map_scratch) cudaFree(h->map_scratch);
    h->map_scratch = nullptr;
    h->map_scratch_bytes = 0;
    const size_t bytes = need + need / 4;
    if (cudaMalloc(&h->map_scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(CHEM_ENOMEM, "cudaMalloc of mapping scratch failed");
    }
    h->map_scratch_bytes = bytes;
  }
  const MapScratch m = map_layout((char*)h->map_scratch, N, n);
  cudaStream_t strm = (cudaStream_t)stream;
  const int S = (int)(m.tmask + 1u);
  cudaMemsetAsync(m.tkey, 0, (size_t)S * 8, strm);
  cudaMemsetAsync(m.count, 0, 4, strm);
  k_fill_int<<<(S + 255) / 256, 256, 0, strm>>>(S, m.tref, INT_MAX);
  const int gb = (N + 255) / 256;
  k_map_insert<<<gb, 256, 0, strm>>>(mk, N, T, p, Y, dt, m.key, m.tkey, m.tref, m.tmask);
  k_map_resolve<<<gb, 256, 0, strm>>>(mk, N, T, p, Y, dt, m.key, m.tkey, m.tref, m.tmask, ref, m.pos, m.list,
                                       m.count);
  if ((st = launch_check("chem_integrate_mapped zone launch")) != CHEM_OK) return st;
  int M = 0;
  if ((e = cudaMemcpyAsync(&M, m.count, 4, cudaMemcpyDeviceToHost, strm)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync");
  if ((e = cudaStreamSynchronize(strm)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (M < 1 || M > N) return fail(CHEM_ECUDA, "internal error: bad count of cells to integrate");
  const int gm = (M + 255) / 256;
  k_map_gather<<<gm, 256, 0, strm>>>(M, m.list, N, n, T, p, Y, dt, h_io, nsub, m.cT, m.cp, m.cY, m.cdt, m.ch, m.cns);
  if ((st = launch_check("chem_integrate_mapped gather launch")) != CHEM_OK) return st;
  if ((st = chem_integrate(h, M, m.cT, m.cp, m.cY, m.cdt, m.ch, m.cns, m.cst, &o, stream)) != CHEM_OK) return st;
  k_map_apply<<<gb, 256, 0, strm>>>(N, n, ref, m.pos, T, Y, nsub, status, m.cT, m.cY, m.cst, M);
  k_map_scatter<<<gm, 256, 0, strm>>>(M, m.list, N, n, m.cT, m.cY, m.ch, m.cns, m.cst, T, Y, h_io, nsub, status);
  if ((st = launch_check("chem_integrate_mapped launch")) != CHEM_OK) return st;
  if (n_integrated) *n_integrated = M;
  return CHEM_OK;
}
