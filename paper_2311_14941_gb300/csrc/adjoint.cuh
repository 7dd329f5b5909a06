// adjoint.cuh -- discrete adjoint of the RODAS3 integration (one warp per cell).
//
// The forward pass records the accepted step sizes and a checkpoint every K accepted steps.  The reverse
// pass walks the segments backwards, recomputes a segment's states from its checkpoint with the same
// arithmetic as the forward pass, and applies the adjoint of each step in reverse order.  Gradients are
// those of the discrete map with the accepted step sizes frozen.
//
// Adjoint of one step (transformed form, M = I/(h gamma) - J(y), A U_i = r_i):
//   mu_i = m_i lambda';  for i = 4..1:  w_i = M^-T mu_i;  mu_j += (c_ij/h) w_i (j < i);
//     stage states Y_i = y + sum_j a_ij U_j:  g_i = J(Y_i)^T w_i,  lambda += g_i,  mu_j += a_ij g_i;
//     Hessian term (J depends on y):           lambda += d/de [J(y + e U_i)^T w_i]
//     parameters theta_j = (ln A_j, Ea_j):     dL/dtheta += w_i^T f_theta(Y_i) + w_i^T J_theta(y) U_i
//   lambda (= dL/dy_n) = lambda' + sum of the above.
// With J = S + u v^T: J^T w = S^T w + v (u.w), and M^-T x by Sherman-Morrison on the transposed factor.
// A shift of ln A_j scales reaction j's forward and reverse rates (both fall-off limits for Troe), so
// d f / d lnA_j = e_j q_j with e_j = d f / d q_j, and d f / d Ea_j = -e_j q_j / (Ru T); w^T e_j is a
// sum over the reaction's participants of a_k = W_k w_k / rho - w_T H_k / (rho c_p).
// The Hessian and the mixed parameter terms use forward-mode dual numbers through the same rate and
// Jacobian code (exact, no finite differences).
#pragma once
#include "device.cuh"

namespace chemgb {

struct AdjLayout {
  CellLayout L;        // base workspace (factor kept apart from the derivative slots)
  int Y3, Y4, AU1, AU2, AU3, AU4, W1, W2, W3, W4, MU1, MU2, MU3, MU4, LAM, G, ZT, WS;   // m-vectors
  int SY, UY, VY;      // S, u, v at y (the step's own Jacobian)
  int A;               // n: participant coefficients of the parameter terms
  int total;
};
// Per-warp global memory of the reverse pass (touched once per step, so kept out of shared memory):
// the recomputed states of one segment (K*m) and the cell's gradient accumulators (2R, compiled
// reaction order).

// out = J^T w = S^T w + v (u . w) with S in the internal entry order
template <class Sc>
__device__ __forceinline__ void vjp(const MechView& M, const Sc* S, const Sc* u, const Sc* v, const double* w, Sc* out,
                                    Sc* part, const Grp1& g) {
  run_gather(M.g_col, out + 1, part, [&](int a, int b) { return S[a] * w[1 + b]; }, g);
  Sc t0 = Sc(0.0), uw = Sc(0.0);
  for (int k = g.lane; k < M.n; k += g.size) t0 = sfma(S[M.nY + k], Sc(w[1 + k]), t0);
  for (int i = g.lane; i < M.m; i += g.size) uw = sfma(u[i], Sc(w[i]), uw);
  t0 = gsum(g, t0);
  uw = gsum(g, uw);
  for (int c = g.lane; c < M.m; c += g.size) {
    const Sc base = (c == 0) ? t0 : out[c];
    out[c] = sfma(v[c], uw, sfma(S[M.nY + M.n + c], Sc(w[0]), base));
  }
  g.sync();
}

__device__ __forceinline__ void acc_theta(double& g, double c) { g += c; }
__device__ __forceinline__ void acc_theta(double& g, const Dual& c) { g += c.d; }

// dL/dtheta += w^T f_theta at the evaluated state (value part for double, tangent part for Dual):
// for reaction r, q_r * E_r with E_r = sum_products a_k - sum_reactants a_k.
template <class Sc>
__device__ __forceinline__ void theta_terms(const MechView& M, const Sc* s, const CellLayout& L, const ScalT<Sc>& sc,
                                            const double* w, Sc* a, double* GA, double* GE, const Grp1& g) {
  const Sc c1 = (w[0] * kRu) * sc.T / (sc.rho * sc.cp);
  for (int k = g.lane; k < M.n; k += g.size)
    a[k] = sfma(Sc(__ldg(M.sp + (size_t)k * SP_STRIDE + 1) * w[1 + k]), sc.irho, -(c1 * s[L.hRT + k]));
  g.sync();
  const Sc iRT = 1.0 / (kRu * sc.T);
  for (int r = g.lane; r < M.R; r += g.size) {
    const int* I = M.rxi + (size_t)r * RX_I;
    const int nro = __ldg(I + 2), npo = __ldg(I + 3);
    Sc E = Sc(0.0);
    for (int i = 0; i < npo; ++i) E += a[__ldg(I + 7 + i)];
    for (int i = 0; i < nro; ++i) E -= a[__ldg(I + 4 + i)];
    const Sc qE = s[L.q + r] * E;
    acc_theta(GA[r], qE);
    acc_theta(GE[r], -(qE * iRT));
  }
  g.sync();
}

// x <- A^-T x (transposed substitution with the same factor)
__device__ __forceinline__ void lu_solveT(const MechView& M, const double* s, const CellLayout& L, double* x, const Grp1& g) {
  const double* LU = s + L.LU;
  const double* dinv = s + L.dinv;
  const ElimOp* op = M.svT_ops + g.lane;
  for (int st = 0; st < M.svT_steps; ++st, op += g.size) {
    const ElimOp o = ld_eop(op);
    if (o.t != OP_IDLE) {
      if (o.kind == K_UPDATE) x[o.t] = fma(-LU[o.a], x[o.b], x[o.t]);
      else x[o.t] *= dinv[o.a];
    }
    g.sync();
  }
}

// x <- M^-T x with M^T = A^T - v u^T:  x = A^-T x + zt (u . A^-T x) / (1 - u . zt),  zt = A^-T v
__device__ __forceinline__ void smT_solve(const MechView& M, const double* s, const AdjLayout& A, double* x,
                                          double idenT, const Grp1& g) {
  lu_solveT(M, s, A.L, x, g);
  const double* u = s + A.UY;
  const double* zt = s + A.ZT;
  double d = 0.0;
  for (int i = g.lane; i < M.m; i += g.size) d = fma(u[i], x[i], d);
  d = gsum(g, d) * idenT;
  for (int i = g.lane; i < M.m; i += g.size) x[i] = fma(zt[i], d, x[i]);
  g.sync();
}

__device__ __forceinline__ void vset(double* dst, const double* src, int m, const Grp1& g) {
  for (int i = g.lane; i < m; i += g.size) dst[i] = src[i];
  g.sync();
}

// sum_st (d_st J)^T W_st into out (m), J = S + u v^T at the dual point (d_st: tangent st):
//   d(J^T w) = dS^T w + dv (u . w) + v (du . w).
__device__ __forceinline__ void vjp_tangents(const MechView& M, const Dual4* S, const Dual4* u, const Dual4* v,
                                             const double* const* Ws, double* out, double* part, const Grp1& g) {
  run_gather(M.g_col, out + 1, part, [&](int a, int b) {
    double acc = 0.0;
#pragma unroll
    for (int st = 0; st < 4; ++st) acc = fma(S[a].d[st], Ws[st][1 + b], acc);
    return acc;
  }, g);
  double t0 = 0.0, uw[4] = {0.0, 0.0, 0.0, 0.0}, duw[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = g.lane; k < M.n; k += g.size)
#pragma unroll
    for (int st = 0; st < 4; ++st) t0 = fma(S[M.nY + k].d[st], Ws[st][1 + k], t0);
  for (int i = g.lane; i < M.m; i += g.size)
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      uw[st] = fma(u[i].v, Ws[st][i], uw[st]);
      duw[st] = fma(u[i].d[st], Ws[st][i], duw[st]);
    }
  t0 = gsum(g, t0);
#pragma unroll
  for (int st = 0; st < 4; ++st) { uw[st] = gsum(g, uw[st]); duw[st] = gsum(g, duw[st]); }
  for (int c = g.lane; c < M.m; c += g.size) {
    double acc = (c == 0) ? t0 : out[c];
    const Dual4& vc = v[c];
    const Dual4& sT = S[M.nY + M.n + c];
#pragma unroll
    for (int st = 0; st < 4; ++st)
      acc += fma(vc.d[st], uw[st], fma(vc.v, duw[st], sT.d[st] * Ws[st][0]));
    out[c] = acc;
  }
  g.sync();
}

__device__ __forceinline__ Dual tangent_of(const Dual4& x, int st) { return Dual(x.v, x.d[st]); }

// The mixed parameter terms of the four stages: GA_r, GE_r += sum_st d_st [q_r E_r(W_st)] with the
// parameter contraction of theta_terms evaluated in the dual number of tangent st.
__device__ __forceinline__ void theta_tangents(const MechView& M, const Dual4* s, const CellLayout& L,
                                               const ScalT<Dual4>& sc, const double* const* Ws, Dual* a,
                                               double* GA, double* GE, const Grp1& g) {
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const double* w = Ws[st];
    const Dual T = tangent_of(sc.T, st), rho = tangent_of(sc.rho, st), cp = tangent_of(sc.cp, st);
    const Dual irho = tangent_of(sc.irho, st);
    const Dual c1 = (w[0] * kRu) * T / (rho * cp);
    for (int k = g.lane; k < M.n; k += g.size)
      a[k] = sfma(Dual(__ldg(M.sp + (size_t)k * SP_STRIDE + 1) * w[1 + k]), irho, -(c1 * tangent_of(s[L.hRT + k], st)));
    g.sync();
    const Dual iRT = 1.0 / (kRu * T);
    for (int r = g.lane; r < M.R; r += g.size) {
      const int* I = M.rxi + (size_t)r * RX_I;
      const int nro = __ldg(I + 2), npo = __ldg(I + 3);
      Dual E = Dual(0.0);
      for (int i = 0; i < npo; ++i) E += a[__ldg(I + 7 + i)];
      for (int i = 0; i < nro; ++i) E -= a[__ldg(I + 4 + i)];
      const Dual qE = tangent_of(s[L.q + r], st) * E;
      GA[r] += qE.d;
      GE[r] += (-(qE * iRT)).d;
    }
    g.sync();
  }
}

// All second-order terms of one step: the Jacobian at y differentiated along U1..U4 at once, then the
// state part into LAM and the parameter part into GA, GE.  tmp: m doubles of scratch.
__device__ __forceinline__ void second_order_terms(const MechView& M, Dual4* dw, const CellLayout& Ld,
                                                   const double* y, double p, const double* const* Us,
                                                   const double* const* Ws, double* LAM, double* tmp, double* GA,
                                                   double* GE, const Grp1& g) {
  Dual4* yd = dw + Ld.y;
  for (int i = g.lane; i < M.m; i += g.size) {
    Dual4 x(y[i]);
#pragma unroll
    for (int st = 0; st < 4; ++st) x.d[st] = Us[st][i];
    yd[i] = x;
  }
  g.sync();
  const ScalT<Dual4> scd = eval_jac<Dual4>(M, dw, Ld, yd, p, g);
  vjp_tangents(M, dw + Ld.S, dw + Ld.u, dw + Ld.v, Ws, tmp, reinterpret_cast<double*>(dw + Ld.part), g);
  for (int i = g.lane; i < M.m; i += g.size) LAM[i] += tmp[i];
  g.sync();
  theta_tangents(M, dw, Ld, scd, Ws, reinterpret_cast<Dual*>(dw + Ld.z), GA, GE, g);
}

// One adjoint step at state y (a row of the segment) with step h.  lambda (A.LAM) is updated in place,
// the parameter gradients accumulate into GA, GE.  Returns false if the factor is singular (cannot
// happen for a step the forward pass accepted).
__device__ __forceinline__ bool adjoint_step(const MechView& M, double* s, const AdjLayout& A, Dual4* dw,
                                             const CellLayout& Ld, const double* y, double p, double h,
                                             double* GA, double* GE, const Grp1& g) {
  const CellLayout& L = A.L;
  const int m = M.m;
  const double ih = 1.0 / h;
  double* U1 = s + A.AU1; double* U2 = s + A.AU2; double* U3 = s + A.AU3; double* U4 = s + A.AU4;
  double* W1 = s + A.W1; double* W2 = s + A.W2; double* W3 = s + A.W3; double* W4 = s + A.W4;
  double* MU1 = s + A.MU1; double* MU2 = s + A.MU2; double* MU3 = s + A.MU3; double* MU4 = s + A.MU4;
  double* LAM = s + A.LAM; double* G = s + A.G; double* Y3 = s + A.Y3; double* Y4 = s + A.Y4;
  // ---- forward quantities of the step (same arithmetic as the forward attempt)
  vset(s + L.y, y, m, g);
  eval_jac<double>(M, s, L, s + L.y, p, g);
  vset(s + A.SY, s + L.S, M.nnz_S, g);
  vset(s + A.UY, s + L.u, m, g);
  vset(s + A.VY, s + L.v, m, g);
  if (!lu_build_factor(M, s, L, ih * (1.0 / RG), g)) return false;
  double* z = s + L.z;
  const double* u = s + A.UY;
  const double* v = s + A.VY;
  const double* f0 = s + L.f0;
  for (int i = g.lane; i < m; i += g.size) { z[i] = u[i]; U1[i] = f0[i]; }
  g.sync();
  lu_solve_impl<true>(M, s, L, z, U1, g);
  double vz = 0.0, vx = 0.0;
  for (int i = g.lane; i < m; i += g.size) { vz = fma(v[i], z[i], vz); vx = fma(v[i], U1[i], vx); }
  vz = gsum(g, vz);
  vx = gsum(g, vx);
  const double iden = 1.0 / (1.0 - vz);
  vx *= iden;
  for (int i = g.lane; i < m; i += g.size) U1[i] = fma(z[i], vx, U1[i]);
  g.sync();
  for (int i = g.lane; i < m; i += g.size) U2[i] = fma(C21 * ih, U1[i], f0[i]);
  g.sync();
  sm_solve(M, s, L, U2, iden, g);
  for (int i = g.lane; i < m; i += g.size) Y3[i] = fma(A31, U1[i], y[i]);
  g.sync();
  eval_f<double>(M, s, L, Y3, p, U3, g);
  for (int i = g.lane; i < m; i += g.size) U3[i] = fma(ih, fma(C31, U1[i], C32 * U2[i]), U3[i]);
  g.sync();
  sm_solve(M, s, L, U3, iden, g);
  for (int i = g.lane; i < m; i += g.size) Y4[i] = fma(A43, U3[i], fma(A41, U1[i], y[i]));
  g.sync();
  eval_f<double>(M, s, L, Y4, p, U4, g);
  for (int i = g.lane; i < m; i += g.size) U4[i] = fma(ih, fma(C41, U1[i], fma(C42, U2[i], C43 * U3[i])), U4[i]);
  g.sync();
  sm_solve(M, s, L, U4, iden, g);
  // transposed Sherman-Morrison vector
  double* zt = s + A.ZT;
  vset(zt, v, m, g);
  lu_solveT(M, s, L, zt, g);
  double uz = 0.0;
  for (int i = g.lane; i < m; i += g.size) uz = fma(u[i], zt[i], uz);
  uz = gsum(g, uz);
  const double idenT = 1.0 / (1.0 - uz);
  // ---- reverse sweep over the stages
  for (int i = g.lane; i < m; i += g.size) {
    MU1[i] = M1 * LAM[i]; MU2[i] = 0.0; MU3[i] = M3 * LAM[i]; MU4[i] = M4 * LAM[i];
  }
  g.sync();
  // stage 4: r4 = f(Y4) + (c41 U1 + c42 U2 + c43 U3)/h, Y4 = y + a41 U1 + a43 U3
  vset(W4, MU4, m, g);
  smT_solve(M, s, A, W4, idenT, g);
  {
    ScalT<double> sc = eval_jac<double>(M, s, L, Y4, p, g);
    theta_terms<double>(M, s, L, sc, W4, s + A.A, GA, GE, g);
    vjp<double>(M, s + L.S, s + L.u, s + L.v, W4, G, s + L.part, g);
  }
  for (int i = g.lane; i < m; i += g.size) {
    MU1[i] = fma(C41 * ih, W4[i], fma(A41, G[i], MU1[i]));
    MU2[i] = fma(C42 * ih, W4[i], MU2[i]);
    MU3[i] = fma(C43 * ih, W4[i], fma(A43, G[i], MU3[i]));
    LAM[i] += G[i];
  }
  g.sync();
  // stage 3: r3 = f(Y3) + (c31 U1 + c32 U2)/h, Y3 = y + a31 U1
  vset(W3, MU3, m, g);
  smT_solve(M, s, A, W3, idenT, g);
  {
    ScalT<double> sc = eval_jac<double>(M, s, L, Y3, p, g);
    theta_terms<double>(M, s, L, sc, W3, s + A.A, GA, GE, g);
    vjp<double>(M, s + L.S, s + L.u, s + L.v, W3, G, s + L.part, g);
  }
  for (int i = g.lane; i < m; i += g.size) {
    MU1[i] = fma(C31 * ih, W3[i], fma(A31, G[i], MU1[i]));
    MU2[i] = fma(C32 * ih, W3[i], MU2[i]);
    LAM[i] += G[i];
  }
  g.sync();
  // stage 2: r2 = f(y) + (c21/h) U1;  stage 1: r1 = f(y)
  vset(W2, MU2, m, g);
  smT_solve(M, s, A, W2, idenT, g);
  for (int i = g.lane; i < m; i += g.size) MU1[i] = fma(C21 * ih, W2[i], MU1[i]);
  g.sync();
  vset(W1, MU1, m, g);
  smT_solve(M, s, A, W1, idenT, g);
  double* WS = s + A.WS;
  for (int i = g.lane; i < m; i += g.size) WS[i] = W1[i] + W2[i];
  g.sync();
  vjp<double>(M, s + A.SY, s + A.UY, s + A.VY, WS, G, s + L.part, g);
  for (int i = g.lane; i < m; i += g.size) LAM[i] += G[i];
  g.sync();
  {
    vset(s + L.y, y, m, g);
    ScalT<double> sc = eval_f<double>(M, s, L, s + L.y, p, s + L.f0, g);
    theta_terms<double>(M, s, L, sc, WS, s + A.A, GA, GE, g);
  }
  // ---- Hessian and mixed parameter terms: derivative of J(y) along U_i, contracted with w_i, for the
  //      four stages in one evaluation of the Jacobian with four tangents
  const double* Us[4] = {U1, U2, U3, U4};
  const double* Ws[4] = {W1, W2, W3, W4};
  second_order_terms(M, dw, Ld, y, p, Us, Ws, LAM, G, GA, GE, g);
  return true;
}

// Reverse pass of one cell from its tape.  Returns false on a singular factor.
__device__ __forceinline__ bool adjoint_cell(const MechView& M, double* s, const AdjLayout& A, Dual4* dw,
                                             const CellLayout& Ld, double p, int n_acc, const double* rec_h,
                                             const double* rec_ck, int K, int N, int cell, const Grp1& g,
                                             const IntOpts& o, double* seg, double* GA, double* GE) {
  const int m = M.m;
  const CellLayout& L = A.L;
  const int nseg = (n_acc + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int n0 = sg * K, n1 = min(n_acc, n0 + K);
    for (int i = g.lane; i < m; i += g.size) seg[i] = rec_ck[((size_t)sg * m + i) * N + cell];
    g.sync();
    // recompute the segment's states with the forward arithmetic
    for (int nn = n0; nn < n1 - 1; ++nn) {
      vset(s + L.y, seg + (size_t)(nn - n0) * m, m, g);
      eval_jac<double>(M, s, L, s + L.y, p, g);
      const StepOut so = ros_attempt(M, s, L, p, rec_h[(size_t)nn * N + cell], o.rtol, o.atol, g);
      if (!so.good) return false;
      vset(seg + (size_t)(nn - n0 + 1) * m, s + L.ytmp, m, g);
    }
    for (int nn = n1 - 1; nn >= n0; --nn)
      if (!adjoint_step(M, s, A, dw, Ld, seg + (size_t)(nn - n0) * m, p, rec_h[(size_t)nn * N + cell], GA, GE,
                        g))
        return false;
  }
  return true;
}

}  // namespace chemgb
