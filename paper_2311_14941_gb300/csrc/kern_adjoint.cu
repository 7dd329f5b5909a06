// kern_adjoint.cu -- the discrete-adjoint reverse pass, the per-parameter gradient reduction and the
// parameter shifts.
#include <cuda_runtime.h>

#include "../../include/chem.h"
#include "kernels.cuh"

namespace chemgb {

// ---- discrete adjoint: resident warps pull cells (longest tapes first).  Shared memory: the forward cell
// layout; each warp's workspace (AdjLayout offsets) and dual-number workspace are in global memory.
__global__ void __launch_bounds__(32, 8)
k_adjoint(MechView M, AdjLayout A, int N, const double* __restrict__ p, const double* __restrict__ rec_h,
          const double* __restrict__ rec_ck, const int* __restrict__ rec_n, int K, const double* __restrict__ gT,
          const double* __restrict__ gY, double* __restrict__ grad_cell, double* __restrict__ gT0,
          double* __restrict__ gY0, int* __restrict__ status, int* __restrict__ head, const int* __restrict__ perm,
          Dual4* dual_ws, double* warp_ws, IntOpts o) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x % kWarp;
  const int gw = blockIdx.x;   // one warp per block
  double* s = smem;
  Dual4* dw = dual_ws + (size_t)gw * A.L.total;
  double* ws = warp_ws + (size_t)gw * A.total;
  const int m = M.m;
  double* LAM = ws + A.LAM;
  double* GA = ws + A.GA;
  double* GE = ws + A.GE;
  while (true) {
    int c = 0;
    if (lane == 0) c = atomicAdd(head, 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= N) break;
    c = perm[c];   // costliest cells (longest tapes) first
    const int na = rec_n[c];
    for (int i = lane; i < m; i += kWarp) LAM[i] = (i == 0) ? gT[c] : gY[(size_t)(i - 1) * N + c];
    for (int r = lane; r < M.R; r += kWarp) { GA[r] = 0.0; GE[r] = 0.0; }
    __syncwarp();
    bool ok = na >= 0;
    if (ok) ok = adjoint_cell(M, s, ws, A, dw, p[c], na, rec_h, rec_ck, K, N, c, Grp1{lane}, o);
    if (!ok) {
      for (int i = lane; i < m; i += kWarp) LAM[i] = 0.0;
      for (int r = lane; r < M.R; r += kWarp) { GA[r] = 0.0; GE[r] = 0.0; }
      __syncwarp();
    }
    for (int r = lane; r < M.R; r += kWarp) {
      const int d = __ldg(M.rx_order + r);
      grad_cell[(size_t)d * N + c] = GA[r];
      grad_cell[(size_t)(M.R + d) * N + c] = GE[r];
    }
    if (gT0 && lane == 0) gT0[c] = LAM[0];
    if (gY0)
      for (int i = 1 + lane; i < m; i += kWarp) gY0[(size_t)(i - 1) * N + c] = LAM[i];
    if (status && lane == 0 && !ok && status[c] == CHEM_CELL_OK) status[c] = CHEM_CELL_NOTAPE;
    __syncwarp();
  }
}

// sums over cells in a fixed order (one warp per parameter): deterministic gradients
__global__ void k_grad_reduce(int N, int P, const double* __restrict__ grad_cell, double* __restrict__ out1,
                              double* __restrict__ out2, int half) {
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) / kWarp, lane = threadIdx.x % kWarp;
  if (wg >= P) return;
  double acc = 0.0;
  for (int c = lane; c < N; c += kWarp) acc += grad_cell[(size_t)wg * N + c];
  acc = warp_sum(acc);
  if (lane == 0) {
    if (wg < half) out1[wg] = acc;
    else out2[wg - half] = acc;
  }
}

// parameter shifts: ln A_r = ln A_r,0 + dlnA[d], Ea_r = Ea_r,0 + dEa[d] (d: description index of
// compiled reaction r); Troe low-pressure limits shift jointly
__global__ void k_set_params(MechView M, const double* __restrict__ rxd0, double* __restrict__ rxd,
                             const double* __restrict__ dlnA, const double* __restrict__ dEa) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M.R) return;
  const int d = __ldg(M.rx_order + r);
  const double a = dlnA ? dlnA[d] : 0.0, e = dEa ? dEa[d] / kRu : 0.0;
  const double* src = rxd0 + (size_t)r * RX_D;
  double* dst = rxd + (size_t)r * RX_D;
  dst[0] = src[0] + a;
  dst[2] = src[2] + e;
  if (__ldg((const int*)(M.rxi + (size_t)r * RX_I)) == 2) {
    dst[3] = src[3] + a;
    dst[5] = src[5] + e;
  }
}

}  // namespace chemgb
