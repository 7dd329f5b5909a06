// kern_rates.cu -- the rate (chem_rates) and Jacobian (chem_jacobian) kernels, one warp per cell.
#include "kern_forward.cuh"

namespace chemgb {

__global__ void k_rates(MechView M, CellLayout L, int N, const double* __restrict__ T, const double* __restrict__ p,
                        const double* __restrict__ Y, double* __restrict__ dTdt, double* __restrict__ dYdt,
                        double* __restrict__ wdot) {
  extern __shared__ double smem[];
  const int wpb = blockDim.x / kWarp, w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int c0 = blockIdx.x * wpb;
  double* s = smem + (size_t)w * L.total;
  load_tile(smem, L, M.m, N, c0, wpb, T, Y);
  const int c = c0 + w;
  if (c >= N) return;
  const Grp1 g{lane};
  double* f = s + L.f0;
  Scal sc = eval_f<double>(M, s, L, s + L.y, p[c], f, g);
  for (int i = lane; i < M.m; i += kWarp) {
    if (i == 0) dTdt[c] = f[0];
    else dYdt[(size_t)(i - 1) * N + c] = f[i];
  }
  if (wdot) {
    for (int k = lane; k < M.n; k += kWarp) wdot[(size_t)k * N + c] = f[1 + k] * sc.rho * __ldg(M.sp + (size_t)k * SP_STRIDE);
  }
}

__global__ void k_jacobian(MechView M, CellLayout L, int N, const double* __restrict__ T, const double* __restrict__ p,
                           const double* __restrict__ Y, double* __restrict__ Sv, double* __restrict__ u,
                           double* __restrict__ v) {
  extern __shared__ double smem[];
  const int wpb = blockDim.x / kWarp, w = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const int c0 = blockIdx.x * wpb;
  double* s = smem + (size_t)w * L.total;
  load_tile(smem, L, M.m, N, c0, wpb, T, Y);
  const int c = c0 + w;
  if (c >= N) return;
  eval_jac<double>(M, s, L, s + L.y, p[c], Grp1{lane});
  for (int e = lane; e < M.nnz_S; e += kWarp) Sv[(size_t)__ldg(M.s_out + e) * N + c] = s[L.S + e];
  for (int i = lane; i < M.m; i += kWarp) {
    u[(size_t)i * N + c] = s[L.u + i];
    v[(size_t)i * N + c] = s[L.v + i];
  }
}

}  // namespace chemgb
