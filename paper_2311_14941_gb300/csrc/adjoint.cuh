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

// Memory of the reverse pass.  Shared memory holds the forward cell layout L only (the factor shares
// its region with the Jacobian's pass scratch, as in the integrator), so as many warps per SM fit as
// for the forward pass.  Everything else of a warp lives in its own slice of global memory (offsets in
// doubles below), read and written lane-strided, except the step records (the step's Jacobian and
// factor), which the transposed solves and the products with J(y)^T read by index.
struct AdjLayout {
  CellLayout L;        // shared memory: the forward layout
  int Y3, Y4, W1, W2, W3, W4, MU1, MU2, MU3, MU4, LAM, G, ZT, WS;   // m-vectors
  // step record, kept by the segment recompute for every step of the segment (offsets within a record):
  int SY;              // nnz_S: S at y (the step's own Jacobian)
  int UY, VY;          // m each: the rank-one part u v^T at y
  int HY;              // n: h/RT at y
  int QY;              // R: rates of progress at y
  int SC;              // 8: T, rho, c_p, 1/rho at y
  int LUG;             // nnz_LU + m: the step's factor and its reciprocal pivots
  int JREC, jstride;   // K records of jstride doubles
  int UST;             // K * 4m: U1..U4 of every step of the current segment
  int SEG;             // K * m: the segment's states
  int GA, GE;          // R each: the cell's gradient accumulators (compiled reaction order)
  int total;           // doubles per warp
};

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

// dL/dtheta += w^T f_theta at an evaluated state: for reaction r, q_r * E_r with E_r = sum_products a_k -
// sum_reactants a_k, a_k = W_k w_k / rho - w_T H_k / (rho c_p).  hRT, q: the evaluation's h/RT and rates
// of progress; a: n doubles of scratch (shared memory, read by index).
__device__ __forceinline__ void theta_terms(const MechView& M, const double* hRT, const double* q, double T,
                                            double rho, double cp, double irho, const double* w, double* a,
                                            double* GA, double* GE, const Grp1& g) {
  const double c1 = (w[0] * kRu) * T / (rho * cp);
  for (int k = g.lane; k < M.n; k += g.size)
    a[k] = fma(__ldg(M.sp + (size_t)k * SP_STRIDE + 1) * w[1 + k], irho, -(c1 * hRT[k]));
  g.sync();
  const double iRT = 1.0 / (kRu * T);
  for (int r = g.lane; r < M.R; r += g.size) {
    const int* I = M.rxi + (size_t)r * RX_I;
    const int nro = __ldg(I + 2), npo = __ldg(I + 3);
    double E = 0.0;
    for (int i = 0; i < npo; ++i) E += a[__ldg(I + 7 + i)];
    for (int i = 0; i < nro; ++i) E -= a[__ldg(I + 4 + i)];
    const double qE = q[r] * E;
    GA[r] += qE;
    GE[r] += -(qE * iRT);
  }
  g.sync();
}

// x <- A^-T x (transposed substitution with the factor LU, dinv; x in shared memory)
__device__ __forceinline__ void lu_solveT(const MechView& M, const double* LU, const double* dinv, double* x,
                                          const Grp1& g) {
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
__device__ __forceinline__ void smT_solve(const MechView& M, const double* LU, const double* dinv, const double* u,
                                          const double* zt, double* x, double idenT, const Grp1& g) {
  lu_solveT(M, LU, dinv, x, g);
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

// Tangents carried per dual-number evaluation of the Jacobian in the second-order terms: the four stages
// take 4 / kTangentsPerPass passes (fewer live registers per dual number against a little more
// arithmetic per pass).
constexpr int kTangentsPerPass = 2;

// sum_st (d_st J)^T W_st into out (m), J = S + u v^T at the dual point (d_st: tangent st):
//   d(J^T w) = dS^T w + dv (u . w) + v (du . w).
template <int NT>
__device__ __forceinline__ void vjp_tangents(const MechView& M, const DualN<NT>* S, const DualN<NT>* u,
                                             const DualN<NT>* v, const double* const* Ws, double* out, double* part,
                                             const Grp1& g) {
  run_gather(M.g_col, out + 1, part, [&](int a, int b) {
    double acc = 0.0;
#pragma unroll
    for (int st = 0; st < NT; ++st) acc = fma(S[a].d[st], Ws[st][1 + b], acc);
    return acc;
  }, g);
  double t0 = 0.0, uw[NT], duw[NT];
#pragma unroll
  for (int st = 0; st < NT; ++st) { uw[st] = 0.0; duw[st] = 0.0; }
  for (int k = g.lane; k < M.n; k += g.size)
#pragma unroll
    for (int st = 0; st < NT; ++st) t0 = fma(S[M.nY + k].d[st], Ws[st][1 + k], t0);
  for (int i = g.lane; i < M.m; i += g.size)
#pragma unroll
    for (int st = 0; st < NT; ++st) {
      uw[st] = fma(u[i].v, Ws[st][i], uw[st]);
      duw[st] = fma(u[i].d[st], Ws[st][i], duw[st]);
    }
  t0 = gsum(g, t0);
#pragma unroll
  for (int st = 0; st < NT; ++st) { uw[st] = gsum(g, uw[st]); duw[st] = gsum(g, duw[st]); }
  for (int c = g.lane; c < M.m; c += g.size) {
    double acc = (c == 0) ? t0 : out[c];
    const DualN<NT>& vc = v[c];
    const DualN<NT>& sT = S[M.nY + M.n + c];
#pragma unroll
    for (int st = 0; st < NT; ++st)
      acc += fma(vc.d[st], uw[st], fma(vc.v, duw[st], sT.d[st] * Ws[st][0]));
    out[c] = acc;
  }
  g.sync();
}

template <int NT>
__device__ __forceinline__ Dual tangent_of(const DualN<NT>& x, int st) { return Dual(x.v, x.d[st]); }

// The mixed parameter terms of the stages of this pass: GA_r, GE_r += sum_st d_st [q_r E_r(W_st)] with
// the parameter contraction of theta_terms evaluated in the dual number of tangent st.
template <int NT>
__device__ __forceinline__ void theta_tangents(const MechView& M, const DualN<NT>* s, const CellLayout& L,
                                               const ScalT<DualN<NT>>& sc, const double* const* Ws, Dual* a,
                                               double* GA, double* GE, const Grp1& g) {
#pragma unroll
  for (int st = 0; st < NT; ++st) {
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

// Second-order terms of NT stages of one step: the Jacobian at y differentiated along their U_i at once,
// then the state part into LAM and the parameter part into GA, GE.  dwv: the dual workspace (the cell
// layout in DualN<NT>); tmp: m doubles of scratch.
template <int NT>
__device__ __forceinline__ void second_order_terms(const MechView& M, void* dwv, const CellLayout& Ld,
                                                   const double* y, double p, const double* const* Us,
                                                   const double* const* Ws, double* LAM, double* tmp, double* GA,
                                                   double* GE, const Grp1& g) {
  using DT = DualN<NT>;
  DT* dw = static_cast<DT*>(dwv);
  DT* yd = dw + Ld.y;
  for (int i = g.lane; i < M.m; i += g.size) {
    DT x(y[i]);
#pragma unroll
    for (int st = 0; st < NT; ++st) x.d[st] = Us[st][i];
    yd[i] = x;
  }
  g.sync();
  const ScalT<DT> scd = eval_jac<DT>(M, dw, Ld, yd, p, g);
  vjp_tangents<NT>(M, dw + Ld.S, dw + Ld.u, dw + Ld.v, Ws, tmp, reinterpret_cast<double*>(dw + Ld.part), g);
  for (int i = g.lane; i < M.m; i += g.size) LAM[i] += tmp[i];
  g.sync();
  theta_tangents<NT>(M, dw, Ld, scd, Ws, reinterpret_cast<Dual*>(dw + Ld.z), GA, GE, g);
}

// One adjoint step at state y with step h, whose stage vectors U1..U4 and step record jr (the Jacobian
// at y and the factor of the step) the segment recompute kept.  lambda (A.LAM) is updated in place, the
// parameter gradients accumulate into GA, GE.
__device__ __forceinline__ void adjoint_step(const MechView& M, double* s, double* ws, const AdjLayout& A, Dual4* dw,
                                             const double* jr, const double* y, const double* U1, const double* U2,
                                             const double* U3, const double* U4, double p, double h, double* GA,
                                             double* GE, const Grp1& g) {
  const CellLayout& L = A.L;
  const int m = M.m;
  const double ih = 1.0 / h;
  double* W1 = ws + A.W1; double* W2 = ws + A.W2; double* W3 = ws + A.W3; double* W4 = ws + A.W4;
  double* MU1 = ws + A.MU1; double* MU2 = ws + A.MU2; double* MU3 = ws + A.MU3; double* MU4 = ws + A.MU4;
  double* LAM = ws + A.LAM; double* G = ws + A.G; double* Y3 = ws + A.Y3; double* Y4 = ws + A.Y4;
  const double* UY = jr + A.UY; const double* VY = jr + A.VY; double* ZT = ws + A.ZT;
  const double* LUg = jr + A.LUG;
  double* X = s + L.U3;      // shared scratch of the transposed solves
  double* a = s + L.ytmp;    // shared scratch of the parameter terms (n <= m)
  // ---- the step's factor (kept by the recompute) into shared memory for the first solves
  vset(s + L.LU, LUg, M.nnz_LU + m, g);
  const double* LUs = s + L.LU;
  const double* dinvs = s + L.dinv;
  // transposed Sherman-Morrison vector zt = A^-T v
  vset(X, VY, m, g);
  lu_solveT(M, LUs, dinvs, X, g);
  double uz = 0.0;
  for (int i = g.lane; i < m; i += g.size) uz = fma(UY[i], X[i], uz);
  uz = gsum(g, uz);
  const double idenT = 1.0 / (1.0 - uz);
  vset(ZT, X, m, g);
  // ---- reverse sweep over the stages, one pass of the loop per stage, so that the kernel holds one copy
  //      of the transposed solve and of the stage Jacobian code (written out, the stages overflowed the
  //      instruction cache)
  for (int i = g.lane; i < m; i += g.size) {
    MU1[i] = M1 * LAM[i]; MU2[i] = 0.0; MU3[i] = M3 * LAM[i]; MU4[i] = M4 * LAM[i];
    Y4[i] = fma(A43, U3[i], fma(A41, U1[i], y[i]));
    Y3[i] = fma(A31, U1[i], y[i]);
  }
  g.sync();
  double* const Wv[4] = {W1, W2, W3, W4};
  double* const MUv[4] = {MU1, MU2, MU3, MU4};
#pragma unroll 1
  for (int st = 3; st >= 0; --st) {   // stage st + 1
    // the factor back into shared memory where a stage Jacobian took its region
    if (st == 2 || st == 1) vset(s + L.LU, LUg, M.nnz_LU + m, g);
    vset(X, MUv[st], m, g);
    smT_solve(M, LUs, dinvs, UY, ZT, X, idenT, g);
    double* W = Wv[st];
    vset(W, X, m, g);
    if (st >= 2) {
      // stage 4: r4 = f(Y4) + (c41 U1 + c42 U2 + c43 U3)/h, Y4 = y + a41 U1 + a43 U3;
      // stage 3: r3 = f(Y3) + (c31 U1 + c32 U2)/h,          Y3 = y + a31 U1
      const ScalT<double> sc = eval_jac<double>(M, s, L, st == 3 ? Y4 : Y3, p, g);
      theta_terms(M, s + L.hRT, s + L.q, sc.T, sc.rho, sc.cp, sc.irho, W, a, GA, GE, g);
      vjp<double>(M, s + L.S, s + L.u, s + L.v, W, G, s + L.part, g);
      if (st == 3) {
        for (int i = g.lane; i < m; i += g.size) {
          MU1[i] = fma(C41 * ih, W4[i], fma(A41, G[i], MU1[i]));
          MU2[i] = fma(C42 * ih, W4[i], MU2[i]);
          MU3[i] = fma(C43 * ih, W4[i], fma(A43, G[i], MU3[i]));
          LAM[i] += G[i];
        }
      } else {
        for (int i = g.lane; i < m; i += g.size) {
          MU1[i] = fma(C31 * ih, W3[i], fma(A31, G[i], MU1[i]));
          MU2[i] = fma(C32 * ih, W3[i], MU2[i]);
          LAM[i] += G[i];
        }
      }
    } else if (st == 1) {   // stage 2: r2 = f(y) + (c21/h) U1 (stage 1: r1 = f(y), nothing to propagate)
      for (int i = g.lane; i < m; i += g.size) MU1[i] = fma(C21 * ih, W2[i], MU1[i]);
    }
    g.sync();
  }
  double* WS = ws + A.WS;
  for (int i = g.lane; i < m; i += g.size) WS[i] = W1[i] + W2[i];
  g.sync();
  vjp<double>(M, jr + A.SY, UY, VY, WS, G, s + L.part, g);
  for (int i = g.lane; i < m; i += g.size) LAM[i] += G[i];
  g.sync();
  theta_terms(M, jr + A.HY, jr + A.QY, jr[A.SC], jr[A.SC + 1], jr[A.SC + 2], jr[A.SC + 3], WS, a, GA, GE, g);
  // ---- Hessian and mixed parameter terms: derivative of J(y) along U_i, contracted with w_i, for the
  //      four stages in one evaluation of the Jacobian with four tangents
  const double* Us[4] = {U1, U2, U3, U4};
  const double* Ws[4] = {W1, W2, W3, W4};
#pragma unroll 1
  for (int s0 = 0; s0 < 4; s0 += kTangentsPerPass)
    second_order_terms<kTangentsPerPass>(M, dw, L, y, p, Us + s0, Ws + s0, LAM, G, GA, GE, g);
}

// Reverse pass of one cell from its tape.  ws: the warp's global workspace.  Returns false on a singular
// factor.
__device__ __forceinline__ bool adjoint_cell(const MechView& M, double* s, double* ws, const AdjLayout& A, Dual4* dw,
                                             double p, int n_acc, const double* rec_h, const double* rec_ck, int K,
                                             int N, int cell, const Grp1& g, const IntOpts& o) {
  const int m = M.m;
  const CellLayout& L = A.L;
  double* seg = ws + A.SEG;
  double* ust = ws + A.UST;
  double* GA = ws + A.GA;
  double* GE = ws + A.GE;
  const int nseg = (n_acc + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int n0 = sg * K, n1 = min(n_acc, n0 + K);
    for (int i = g.lane; i < m; i += g.size) seg[i] = rec_ck[((size_t)sg * m + i) * N + cell];
    g.sync();
    // recompute the segment's states and stage vectors with the forward arithmetic, and keep each step's
    // Jacobian at y and its factor for the reverse sweep
    for (int nn = n0; nn < n1; ++nn) {
      double* jr = ws + A.JREC + (size_t)(nn - n0) * A.jstride;
      vset(s + L.y, seg + (size_t)(nn - n0) * m, m, g);
      const ScalT<double> sy = eval_jac<double>(M, s, L, s + L.y, p, g);
      vset(jr + A.SY, s + L.S, M.nnz_S, g);
      vset(jr + A.UY, s + L.u, m, g);
      vset(jr + A.VY, s + L.v, m, g);
      vset(jr + A.QY, s + L.q, M.R, g);
      vset(jr + A.HY, s + L.hRT, M.n, g);
      if (g.lane == 0) {
        jr[A.SC] = sy.T; jr[A.SC + 1] = sy.rho; jr[A.SC + 2] = sy.cp; jr[A.SC + 3] = sy.irho;
      }
      const StepOut so = ros_attempt(M, s, L, p, rec_h[(size_t)nn * N + cell], o.rtol, o.atol, g);
      if (!so.good) return false;   // also a singular factor (cannot happen for a step the forward pass accepted)
      vset(jr + A.LUG, s + L.LU, M.nnz_LU + m, g);
      double* u4 = ust + (size_t)(nn - n0) * 4 * m;
      for (int i = g.lane; i < m; i += g.size) {
        u4[i] = s[L.U1 + i]; u4[m + i] = s[L.U2 + i]; u4[2 * m + i] = s[L.U3 + i]; u4[3 * m + i] = s[L.U4 + i];
        if (nn + 1 < n1) seg[(size_t)(nn - n0 + 1) * m + i] = s[L.ytmp + i];
      }
      g.sync();
    }
    for (int nn = n1 - 1; nn >= n0; --nn) {
      const double* u4 = ust + (size_t)(nn - n0) * 4 * m;
      adjoint_step(M, s, ws, A, dw, ws + A.JREC + (size_t)(nn - n0) * A.jstride, seg + (size_t)(nn - n0) * m, u4,
                   u4 + m, u4 + 2 * m, u4 + 3 * m, p, rec_h[(size_t)nn * N + cell], GA, GE, g);
    }
  }
  return true;
}

}  // namespace chemgb
