// device.cuh -- warp-level device routines: one warp owns one reactor cell, its state and its sparse
// factor in shared memory.
//
// Mathematical content (the paper names the techniques, Sec. 2.5; the formulas are the standard ones):
//   f(y):  y = (T, Y_1..Y_n) at fixed p.  C_k = rho Y_k / W_k, rho = p Wbar / (Ru T).
//          k_f = exp(ln A + b ln T - Ea/(Ru T)); third-body [M]; Troe fall-off; k_r = k_f / Kc with
//          1/Kc = prod_k exp(g_k)^nu_k (Ru T / p0)^(sum nu), g_k = h_k/(Ru T) - s_k/Ru (NASA-7), so a
//          reaction's reverse rate costs multiplications only (one exp per species, not per reaction).
//          dY_k/dt = W_k w_k / rho,  dT/dt = -sum_k H_k w_k / (rho c_p).
//   J(y):  exact Jacobian written as S + u v^T.  With [M] = p/(Ru T) + sum_listed (alpha_j - 1) C_j (the
//          default efficiencies add up to the total concentration, a function of T alone at fixed p),
//          d w / d C is sparse: Dtil = sum_r nu_r (d q_r / d C).  Then, with g_k = sum_j Dtil_kj C_j,
//            S_kj = (W_k/W_j) Dtil_kj,  u_k = (W_k/rho)(w_k - g_k),  v_j = Wbar / W_j,
//            S_kT = (W_k/rho)(w_T,k - g_k/T) + f_k/T      (w_T = d w / d T at fixed C)
//            S_Tj = -(Ru T sum_k hRT_k Dtil_kj + f_T cpR_j Ru) / (W_j c_p)
//            S_TT = -sum_k [Cp_k w_k + H_k (w_T,k - g_k/T)] / (rho c_p) + f_T (1/T - Ru sum Y dcpR/dT / W / c_p)
//            u_T  = sum_k H_k g_k / (rho c_p) + f_T.
//   Step:  RODAS3 (Sandu et al. 1997) in the transformed form of Hairer & Wanner (Vol. II, IV.7):
//            (I/(h gamma) - J) U_i = f(y + sum_j a_ij U_j) + sum_j (c_ij / h) U_j,
//            y_new = y + sum m_i U_i,  err = sum e_i U_i,
//          where J = S + u v^T is inverted by Sherman-Morrison around the sparse LU of I/(h gamma) - S.
#pragma once
#include <cstdint>

#include "mech.h"

namespace chemgb {

// RODAS3 in transformed form.  a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1,
// e = (b - bhat) Gamma^-1, obtained from the published alpha_ij, gamma_ij, b, bhat (gamma = 1/2).
// Zero coefficients are exploited below: a21 = a32 = a42 = 0 (stage 2 reuses f(y)), m2 = 0,
// e = (0, 0, 0, 1).
constexpr double RG = 0.5;
constexpr double A31 = 2.0, A41 = 2.0, A43 = 1.0;
constexpr double C21 = 4.0, C31 = 1.0, C32 = -1.0, C41 = 1.0, C42 = -1.0, C43 = -8.0 / 3.0;
constexpr double M1 = 2.0, M3 = 1.0, M4 = 1.0;

constexpr double kInvLn10 = 0.43429448190325182765;
constexpr double kLn10 = 2.30258509299404568402;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;   // identical on every lane (each butterfly stage adds the same pair of operands)
}

__device__ __forceinline__ GatherOp ld_gop(const GatherOp* p) {
  uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  GatherOp o;
  o.a = (uint16_t)(v.x & 0xFFFF); o.b = (uint16_t)(v.x >> 16);
  o.dst = (uint16_t)(v.y & 0xFFFF); o.flags = (uint16_t)(v.y >> 16);
  return o;
}

__device__ __forceinline__ ElimOp ld_eop(const ElimOp* p) {
  uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  ElimOp o;
  o.t = (uint16_t)(v.x & 0xFFFF); o.a = (uint16_t)(v.x >> 16);
  o.b = (uint16_t)(v.y & 0xFFFF); o.pad = 0;
  return o;
}

// Per-cell scalars shared by all lanes (every lane holds the same values).
struct Scal {
  double T, lnT, invT, Wbar, rho, irho, cp, ctot, rtp, irtp, dcps;
};

// -------------------------------------------------------------------------------------- gathers
// out[g] = sum over the group's terms of val(a, b); partial sums of split groups are combined after.
template <class F>
__device__ __forceinline__ void run_gather(const Gather& G, double* out, double* part, F val, int lane) {
  double acc = 0.0;
  const GatherOp* op = G.ops + lane;
  for (int s = 0; s < G.steps; ++s, op += kWarp) {
    GatherOp o = ld_gop(op);
    if (!(o.flags & 1)) acc += val(o.a, o.b);
    if (o.dst != DST_NONE) {
      if (o.dst & PARTIAL_BIT) part[o.dst & 0x7FFF] = acc; else out[o.dst] = acc;
      acc = 0.0;
    }
  }
  __syncwarp();
  for (int c = lane; c < G.n_comb; c += kWarp) {
    const int dst = __ldg(G.comb + 3 * c), f = __ldg(G.comb + 3 * c + 1), cnt = __ldg(G.comb + 3 * c + 2);
    double s = 0.0;
    for (int i = 0; i < cnt; ++i) s += part[f + i];
    out[dst] = s;
  }
  __syncwarp();
}

// Same program, two accumulators: out1[g] = sum nu q[r], out2[g] = sum nu dq[r].
__device__ __forceinline__ void run_gather2(const Gather& G, double* out1, double* out2, double* part,
                                            const double* q, const double* dq, int lane) {
  double acc1 = 0.0, acc2 = 0.0;
  const GatherOp* op = G.ops + lane;
  for (int s = 0; s < G.steps; ++s, op += kWarp) {
    GatherOp o = ld_gop(op);
    if (!(o.flags & 1)) {
      const double nu = (double)(int16_t)o.b;
      acc1 = fma(nu, q[o.a], acc1);
      acc2 = fma(nu, dq[o.a], acc2);
    }
    if (o.dst != DST_NONE) {
      if (o.dst & PARTIAL_BIT) {
        part[2 * (o.dst & 0x7FFF)] = acc1;
        part[2 * (o.dst & 0x7FFF) + 1] = acc2;
      } else {
        out1[o.dst] = acc1;
        out2[o.dst] = acc2;
      }
      acc1 = acc2 = 0.0;
    }
  }
  __syncwarp();
  for (int c = lane; c < G.n_comb; c += kWarp) {
    const int dst = __ldg(G.comb + 3 * c), f = __ldg(G.comb + 3 * c + 1), cnt = __ldg(G.comb + 3 * c + 2);
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < cnt; ++i) { s1 += part[2 * (f + i)]; s2 += part[2 * (f + i) + 1]; }
    out1[dst] = s1;
    out2[dst] = s2;
  }
  __syncwarp();
}

// -------------------------------------------------------------------------------------- thermo
// NASA-7 at T for every species (lanes over species); fills C, hRT, eg = exp(g), emg = 1/eg, cpR.
template <bool DERIV>
__device__ __forceinline__ Scal eval_species(const MechView& M, double* s, const CellLayout& L, const double* y,
                                             double p, int lane) {
  Scal sc;
  sc.T = y[0];
  sc.lnT = log(sc.T);
  sc.invT = 1.0 / sc.T;
  const double T = sc.T;
  double sig = 0.0, cps = 0.0, dcps = 0.0;
  for (int k = lane; k < M.n; k += kWarp) {
    const double* t = M.sp + (size_t)k * SP_STRIDE;
    const double iw = __ldg(t);
    const double* c = t + 4 + (T < __ldg(t + 2) ? 0 : SP_RANGE);
    const double a0 = __ldg(c + 0), a1 = __ldg(c + 1), a2 = __ldg(c + 2), a3 = __ldg(c + 3), a4 = __ldg(c + 4);
    const double cpR = fma(T, fma(T, fma(T, fma(T, a4, a3), a2), a1), a0);
    const double h = fma(T, fma(T, fma(T, fma(T, __ldg(c + 8), __ldg(c + 7)), __ldg(c + 6)), __ldg(c + 5)), a0);
    const double a5 = __ldg(c + 13), a6 = __ldg(c + 14);
    const double hRT = fma(a5, sc.invT, h);
    const double gp = fma(T, fma(T, fma(T, fma(T, __ldg(c + 12), __ldg(c + 11)), __ldg(c + 10)), __ldg(c + 9)),
                          fma(a5, sc.invT, -a6));
    const double g = fma(a0, 1.0 - sc.lnT, gp);
    const double eg = exp(g);
    const double yw = y[1 + k] * iw;
    sig += yw;
    cps = fma(yw, cpR, cps);
    if (DERIV) {
      const double dcp = fma(T, fma(T, __ldg(c + 17) * T + __ldg(c + 16), __ldg(c + 15)), a1);
      dcps = fma(yw, dcp, dcps);
    }
    s[L.hRT + k] = hRT;
    s[L.eg + k] = eg;
    s[L.emg + k] = 1.0 / eg;
    s[L.cpR + k] = cpR;
    s[L.C + k] = yw;
  }
  sig = warp_sum(sig);
  cps = warp_sum(cps);
  if (DERIV) dcps = warp_sum(dcps);
  sc.Wbar = 1.0 / sig;
  sc.ctot = p * sc.invT * (1.0 / kRu);
  sc.rho = sc.ctot * sc.Wbar;
  sc.irho = 1.0 / sc.rho;
  sc.cp = kRu * cps;
  sc.dcps = dcps;
  sc.rtp = kRu * T * (1.0 / kP0);
  sc.irtp = 1.0 / sc.rtp;
  for (int k = lane; k < M.n; k += kWarp) s[L.C + k] *= sc.rho;
  __syncwarp();
  return sc;
}

// -------------------------------------------------------------------------------------- reactions
// Rates of progress q (and, with DERIV, dq/dT at fixed C and the derivative slots dq/dC_j).
template <bool DERIV>
__device__ __forceinline__ void eval_reactions(const MechView& M, double* s, const CellLayout& L, const Scal& sc,
                                               int lane) {
  const double* C = s + L.C;
  const double* eg = s + L.eg;
  const double* emg = s + L.emg;
  const double* hRT = s + L.hRT;
  for (int r = lane; r < M.R; r += kWarp) {
    const int* I = M.rxi + (size_t)r * RX_I;
    const double* D = M.rxd + (size_t)r * RX_D;
    const int type = __ldg(I), rev = __ldg(I + 1), nro = __ldg(I + 2), npo = __ldg(I + 3);
    const int r0 = __ldg(I + 4), r1 = __ldg(I + 5), r2 = __ldg(I + 6);
    const int p0 = __ldg(I + 7), p1 = __ldg(I + 8), p2 = __ldg(I + 9);
    const double lnA = __ldg(D), bb = __ldg(D + 1), Ta = __ldg(D + 2);
    const double lnkinf = fma(-Ta, sc.invT, fma(bb, sc.lnT, lnA));
    double kf = exp(lnkinf);
    // concentration products and the partial products without one occurrence
    const double cr0 = C[r0], cr1 = nro > 1 ? C[r1] : 1.0, cr2 = nro > 2 ? C[r2] : 1.0;
    const double cp0 = C[p0], cp1 = npo > 1 ? C[p1] : 1.0, cp2 = npo > 2 ? C[p2] : 1.0;
    const double Pf = cr0 * cr1 * cr2, Pb = cp0 * cp1 * cp2;
    // third-body concentration: total concentration plus listed corrections
    double Mv = sc.ctot;
    if (type != 0) {
      const int eo = __ldg(I + 11), ec = __ldg(I + 12);
      for (int i = 0; i < ec; ++i) Mv = fma(__ldg(M.eff_am1 + eo + i), C[__ldg(M.eff_sp + eo + i)], Mv);
    }
    double dlnkf_dT = 0.0, dlnk_dlnM = 0.0, iM = 0.0;
    if (DERIV) dlnkf_dT = fma(Ta, sc.invT, bb) * sc.invT;
    if (type == 2) {
      // Troe fall-off: Pr = k0 [M] / k_inf, F from the broadening function of F_cent
      const double lnk0 = fma(-__ldg(D + 5), sc.invT, fma(__ldg(D + 4), sc.lnT, __ldg(D + 3)));
      const double lnM = log(Mv);
      const double lnPr = lnk0 - lnkinf + lnM;
      const double Pr = exp(lnPr);
      const double e3 = exp(-sc.T * __ldg(D + 8)), e1 = exp(-sc.T * __ldg(D + 9));
      const double T2 = __ldg(D + 10);
      const double e2 = T2 > 0.0 ? exp(-T2 * sc.invT) : 0.0;
      const double Fc = fma(__ldg(D + 6), e3, fma(__ldg(D + 7), e1, e2));
      const double Lc = log(Fc) * kInvLn10;
      const double cc = fma(-0.67, Lc, -0.4);
      const double nn = fma(-1.27, Lc, 0.75);
      const double x = fma(lnPr, kInvLn10, cc);
      const double den = fma(-0.14, x, nn);
      const double iden = 1.0 / den;
      const double f1 = x * iden;
      const double ib = 1.0 / fma(f1, f1, 1.0);
      const double log10F = Lc * ib;
      const double F = exp(log10F * kLn10);
      const double ipr1 = 1.0 / (1.0 + Pr);
      kf = kf * (Pr * ipr1) * F;
      if (DERIV) {
        const double dlnk0_dT = fma(__ldg(D + 5), sc.invT, __ldg(D + 4)) * sc.invT;
        const double dlnPr_dT = dlnk0_dT - dlnkf_dT;
        const double dFc_dT = -__ldg(D + 6) * __ldg(D + 8) * e3 - __ldg(D + 7) * __ldg(D + 9) * e1 +
                              T2 * sc.invT * sc.invT * e2;
        const double dLc_dT = dFc_dT / Fc * kInvLn10;
        const double dx_dT = fma(dlnPr_dT, kInvLn10, -0.67 * dLc_dT);
        const double dnn_dT = -1.27 * dLc_dT;
        const double df1_dT = (dx_dT * nn - x * dnn_dT) * iden * iden;
        const double dlog10F_dT = fma(dLc_dT, ib, -2.0 * Lc * f1 * df1_dT * ib * ib);
        dlnkf_dT = dlnkf_dT + dlnPr_dT * ipr1 + kLn10 * dlog10F_dT;
        const double df1_dlnM = nn * kInvLn10 * iden * iden;
        dlnk_dlnM = ipr1 - kLn10 * 2.0 * Lc * f1 * df1_dlnM * ib * ib;
        iM = exp(-lnM);
      }
    }
    // reverse rate: k_r = k_f * prod exp(g)^nu_products * prod exp(-g)^nu_reactants * (Ru T/p0)^sum(nu)
    double kr = 0.0, dlnKc_dT = 0.0;
    if (rev) {
      double ik = eg[p0] * emg[r0];
      if (npo > 1) ik *= eg[p1];
      if (npo > 2) ik *= eg[p2];
      if (nro > 1) ik *= emg[r1];
      if (nro > 2) ik *= emg[r2];
      const int dn = npo - nro;
      if (dn > 0) { ik *= sc.rtp; if (dn > 1) ik *= sc.rtp; if (dn > 2) ik *= sc.rtp; }
      if (dn < 0) { ik *= sc.irtp; if (dn < -1) ik *= sc.irtp; if (dn < -2) ik *= sc.irtp; }
      kr = kf * ik;
      if (DERIV) {
        double sh = hRT[p0] - hRT[r0];
        if (npo > 1) sh += hRT[p1];
        if (npo > 2) sh += hRT[p2];
        if (nro > 1) sh -= hRT[r1];
        if (nro > 2) sh -= hRT[r2];
        dlnKc_dT = (sh - (double)dn) * sc.invT;
      }
    }
    const double Mfac = (type == 1) ? Mv : 1.0;
    const double qn = fma(kf, Pf, -kr * Pb);
    const double q = Mfac * qn;
    s[L.q + r] = q;
    if (DERIV) {
      const double kfM = kf * Mfac, krM = kr * Mfac;
      const double qf = kfM * Pf, qr = krM * Pb;
      double dqdM = 0.0;
      if (type == 1) dqdM = qn;
      else if (type == 2) dqdM = dlnk_dlnM * q * iM;
      // dq/dT at fixed C; [M] depends on T through the total concentration p/(Ru T)
      const double dqdT = fma(dlnkf_dT, qf, -(dlnkf_dT - dlnKc_dT) * qr) - dqdM * sc.ctot * sc.invT;
      s[L.dqdT + r] = dqdT;
      // partial products: d(prod)/d(occurrence i) = product of the other occurrences
      const double dr0 = cr1 * cr2, dr1 = cr0 * cr2, dr2 = cr0 * cr1;
      const double dp0 = cp1 * cp2, dp1 = cp0 * cp2, dp2 = cp0 * cp1;
      const int so = __ldg(I + 13), scn = __ldg(I + 14);
      for (int i = 0; i < scn; ++i) {
        const int mask = __ldg(M.dslot_mask + so + i);
        double v = __ldg(M.dslot_am1 + so + i) * dqdM;
        double fr = 0.0, fp = 0.0;
        if (mask & 1) fr += dr0;
        if (mask & 2) fr += dr1;
        if (mask & 4) fr += dr2;
        if (mask & 8) fp += dp0;
        if (mask & 16) fp += dp1;
        if (mask & 32) fp += dp2;
        v = fma(kfM, fr, v);
        v = fma(-krM, fp, v);
        s[L.D + so + i] = v;
      }
    }
  }
  __syncwarp();
}

// -------------------------------------------------------------------------------------- f and J
// f(y) into out[m].  Uses C/hRT/eg/emg/cpR/q scratch.  Returns the scalars of the evaluation.
__device__ __forceinline__ Scal eval_f(const MechView& M, double* s, const CellLayout& L, const double* y, double p,
                                       double* out, int lane) {
  Scal sc = eval_species<false>(M, s, L, y, p, lane);
  eval_reactions<false>(M, s, L, sc, lane);
  const double* q = s + L.q;
  double* part = s + L.part;
  double* w = out + 1;   // production rates written in place, then scaled
  run_gather(M.g_omega, w, part, [&](int a, int b) { return (double)(int16_t)b * q[a]; }, lane);
  double Qs = 0.0;
  for (int k = lane; k < M.n; k += kWarp) {
    const double om = w[k];
    Qs = fma(s[L.hRT + k], om, Qs);
    w[k] = om * __ldg(M.sp + (size_t)k * SP_STRIDE + 1) * sc.irho;
  }
  Qs = warp_sum(Qs);
  if (lane == 0) out[0] = -kRu * sc.T * Qs / (sc.rho * sc.cp);
  __syncwarp();
  return sc;
}

// f(y) into f0[m], S[nnz_S] (internal order), u[m], v[m].  Scratch: C.., q, dqdT, D, x (w), z (w_T),
// U1 (g), U2 (t).
__device__ __forceinline__ void eval_jac(const MechView& M, double* s, const CellLayout& L, const double* y, double p,
                                         int lane) {
  Scal sc = eval_species<true>(M, s, L, y, p, lane);
  eval_reactions<true>(M, s, L, sc, lane);
  double* part = s + L.part;
  double* w = s + L.x;      // w_k
  double* wT = s + L.z;     // w_T,k
  double* gk = s + L.U1;
  double* tk = s + L.U2;
  double* S = s + L.S;
  const double* C = s + L.C;
  const double* hRT = s + L.hRT;
  const double* Dsl = s + L.D;
  run_gather2(M.g_omega, w, wT, part, s + L.q, s + L.dqdT, lane);
  run_gather(M.g_dtil, S, part, [&](int a, int b) { return (double)(int16_t)b * Dsl[a]; }, lane);
  run_gather(M.g_row, gk, part, [&](int a, int b) { return S[a] * C[b]; }, lane);
  run_gather(M.g_col, tk, part, [&](int a, int b) { return S[a] * hRT[b]; }, lane);
  double* f = s + L.f0;
  double* u = s + L.u;
  double* v = s + L.v;
  const double T = sc.T;
  // f, u and the T column; partial sums for the T row scalars
  double Qs = 0.0, A1 = 0.0, A2 = 0.0;
  for (int k = lane; k < M.n; k += kWarp) {
    const double Wk = __ldg(M.sp + (size_t)k * SP_STRIDE + 1);
    const double om = w[k], g = gk[k];
    const double fk = Wk * om * sc.irho;
    f[1 + k] = fk;
    u[1 + k] = Wk * sc.irho * (om - g);
    S[M.nY + k] = fma(Wk * sc.irho, fma(-g, sc.invT, wT[k]), fk * sc.invT);
    v[1 + k] = sc.Wbar * __ldg(M.sp + (size_t)k * SP_STRIDE);
    const double h = hRT[k];
    Qs = fma(h, om, Qs);
    A1 = fma(s[L.cpR + k], om, fma(T * h, fma(-g, sc.invT, wT[k]), A1));
    A2 = fma(h, g, A2);
  }
  Qs = warp_sum(Qs);
  A1 = warp_sum(A1);
  A2 = warp_sum(A2);
  const double rcp = sc.rho * sc.cp;
  const double fT = -kRu * T * Qs / rcp;
  // T row: S_Tj for species j, then S_TT; u_T; v_T
  for (int j = lane; j < M.n; j += kWarp) {
    const double iw = __ldg(M.sp + (size_t)j * SP_STRIDE);
    S[M.nY + M.n + 1 + j] = -kRu * fma(T, tk[j], fT * s[L.cpR + j]) * iw / sc.cp;
  }
  if (lane == 0) {
    f[0] = fT;
    S[M.nY + M.n] = -kRu * A1 / rcp + fT * (sc.invT - kRu * sc.dcps / sc.cp);
    u[0] = kRu * T * A2 / rcp + fT;
    v[0] = 0.0;
  }
  __syncwarp();
  // species block: S_kj = (W_k / W_j) Dtil_kj (after the row and column sums used Dtil)
  for (int e = lane; e < M.nY; e += kWarp) S[e] *= __ldg(M.entry_wratio + e);
  __syncwarp();
}

// -------------------------------------------------------------------------------------- linear algebra
// LU of A = I/(h gamma) - S, in place, by the precomputed elimination program.  false if a pivot is 0
// or not finite.
__device__ __forceinline__ bool lu_build_factor(const MechView& M, double* s, const CellLayout& L, double gh,
                                                int lane) {
  double* LU = s + L.LU;
  double* dinv = s + L.dinv;
  const double* S = s + L.S;
  for (int l = lane; l < M.nnz_LU; l += kWarp) {
    const int src = __ldg(M.lu_src + l);
    LU[l] = src >= 0 ? -S[src] : 0.0;
  }
  __syncwarp();
  for (int i = lane; i < M.m; i += kWarp) LU[__ldg(M.lu_diag + i)] += gh;
  __syncwarp();
  bool ok = true;
  const ElimOp* op = M.lu_ops + lane;
  ElimOp nx = M.lu_steps > 0 ? ld_eop(op) : ElimOp{OP_IDLE, 0, 0, 0};
  for (int st = 0; st < M.lu_steps; ++st) {
    const ElimOp o = nx;
    op += kWarp;
    if (st + 1 < M.lu_steps) nx = ld_eop(op);
    const int kind = __ldg(M.lu_kind + st);
    if (o.t != OP_IDLE) {
      if (kind == K_UPDATE) {
        LU[o.t] = fma(-LU[o.a], LU[o.b], LU[o.t]);
      } else if (kind == K_SCALE) {
        LU[o.t] *= dinv[o.a];
      } else {
        const double d = LU[o.a];
        const double r = 1.0 / d;
        ok = ok && (d != 0.0) && isfinite(r);
        dinv[o.t] = r;
      }
    }
    __syncwarp();
  }
  return __all_sync(0xffffffffu, ok);
}

// x <- A^{-1} x (forward and backward substitution by the precomputed program; state-order vector)
__device__ __forceinline__ void lu_solve(const MechView& M, const double* s, const CellLayout& L, double* x,
                                         int lane) {
  const double* LU = s + L.LU;
  const double* dinv = s + L.dinv;
  const ElimOp* op = M.sv_ops + lane;
  ElimOp nx = M.sv_steps > 0 ? ld_eop(op) : ElimOp{OP_IDLE, 0, 0, 0};
  for (int st = 0; st < M.sv_steps; ++st) {
    const ElimOp o = nx;
    op += kWarp;
    if (st + 1 < M.sv_steps) nx = ld_eop(op);
    const int kind = __ldg(M.sv_kind + st);
    if (o.t != OP_IDLE) {
      if (kind == K_UPDATE) x[o.t] = fma(-LU[o.a], x[o.b], x[o.t]);
      else x[o.t] *= dinv[o.a];
    }
    __syncwarp();
  }
}

// x <- M^{-1} x with M = A - u v^T:  x = A^-1 x + z (v . A^-1 x) / (1 - v . z),  z = A^-1 u
__device__ __forceinline__ void sm_solve(const MechView& M, const double* s, const CellLayout& L, double* x,
                                         double iden, int lane) {
  lu_solve(M, s, L, x, lane);
  const double* v = s + L.v;
  const double* z = s + L.z;
  double d = 0.0;
  for (int i = lane; i < M.m; i += kWarp) d = fma(v[i], x[i], d);
  d = warp_sum(d) * iden;
  for (int i = lane; i < M.m; i += kWarp) x[i] = fma(z[i], d, x[i]);
  __syncwarp();
}

// -------------------------------------------------------------------------------------- step
struct StepOut {
  bool good;
  double err;
};

// One RODAS3 attempt of size h from y (f0, S, u, v already evaluated at y).  ynew into ytmp, err into
// the return value.  U1..U4, x, z, LU are scratch.
__device__ __forceinline__ StepOut ros_attempt(const MechView& M, double* s, const CellLayout& L, double p, double h,
                                               double rtol, double atol, int lane) {
  StepOut so{false, 0.0};
  const int m = M.m;
  const double ih = 1.0 / h;
  if (!lu_build_factor(M, s, L, ih * (1.0 / RG), lane)) return so;
  double* y = s + L.y;
  double* yt = s + L.ytmp;
  double* f0 = s + L.f0;
  double* U1 = s + L.U1;
  double* U2 = s + L.U2;
  double* U3 = s + L.U3;
  double* U4 = s + L.U4;
  double* z = s + L.z;
  const double* u = s + L.u;
  const double* v = s + L.v;
  // z = A^-1 u and the Sherman-Morrison denominator
  for (int i = lane; i < m; i += kWarp) z[i] = u[i];
  __syncwarp();
  lu_solve(M, s, L, z, lane);
  double vz = 0.0;
  for (int i = lane; i < m; i += kWarp) vz = fma(v[i], z[i], vz);
  vz = warp_sum(vz);
  const double den = 1.0 - vz;
  if (!(den != 0.0) || !isfinite(den)) return so;
  const double iden = 1.0 / den;
  // stage 1
  for (int i = lane; i < m; i += kWarp) U1[i] = f0[i];
  __syncwarp();
  sm_solve(M, s, L, U1, iden, lane);
  // stage 2 (a21 = 0: f(y) again)
  for (int i = lane; i < m; i += kWarp) U2[i] = fma(C21 * ih, U1[i], f0[i]);
  __syncwarp();
  sm_solve(M, s, L, U2, iden, lane);
  // stage 3
  for (int i = lane; i < m; i += kWarp) yt[i] = fma(A31, U1[i], y[i]);
  __syncwarp();
  eval_f(M, s, L, yt, p, U3, lane);
  for (int i = lane; i < m; i += kWarp) U3[i] = fma(ih, fma(C31, U1[i], C32 * U2[i]), U3[i]);
  __syncwarp();
  sm_solve(M, s, L, U3, iden, lane);
  // stage 4
  for (int i = lane; i < m; i += kWarp) yt[i] = fma(A43, U3[i], fma(A41, U1[i], y[i]));
  __syncwarp();
  eval_f(M, s, L, yt, p, U4, lane);
  for (int i = lane; i < m; i += kWarp) U4[i] = fma(ih, fma(C41, U1[i], fma(C42, U2[i], C43 * U3[i])), U4[i]);
  __syncwarp();
  sm_solve(M, s, L, U4, iden, lane);
  // solution, embedded error, scaled RMS norm
  double e2 = 0.0;
  bool fin = true;
  for (int i = lane; i < m; i += kWarp) {
    const double yn = fma(M4, U4[i], fma(M3, U3[i], fma(M1, U1[i], y[i])));
    yt[i] = yn;
    const double sc = fma(rtol, fmax(fabs(y[i]), fabs(yn)), atol);
    const double e = U4[i] / sc;
    e2 = fma(e, e, e2);
    fin = fin && isfinite(yn);
  }
  e2 = warp_sum(e2);
  fin = __all_sync(0xffffffffu, fin);
  __syncwarp();
  so.err = sqrt(e2 / (double)m);
  so.good = fin;
  return so;
}

struct IntOpts {
  double rtol, atol, h_init, h_min;
  int max_substeps, max_nonfinite;
  unsigned long long deadline_ns;   // 0: none
  double* trace;                    // optional step trace (see chem_integrate_opts)
  int trace_cap;
  int N;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Adaptive integration of the cell whose state sits in y (shared memory) over [0, dt].
__device__ __forceinline__ void integrate_cell(const MechView& M, double* s, const CellLayout& L, double p, double dt,
                                               double& h_io, int& nsub, int& nacc, int& status, const IntOpts& o,
                                               int lane, int cell) {
  double* y = s + L.y;
  const int m = M.m;
  // input check
  bool ok = isfinite(p) && p > 0.0 && isfinite(dt) && dt >= 0.0 && isfinite(y[0]) && y[0] > 0.0;
  double sig = 0.0;
  for (int k = lane; k < M.n; k += kWarp) {
    const double yk = y[1 + k];
    ok = ok && isfinite(yk);
    sig = fma(yk, __ldg(M.sp + (size_t)k * SP_STRIDE), sig);
  }
  sig = warp_sum(sig);
  ok = __all_sync(0xffffffffu, ok) && sig > 0.0;
  nsub = 0;
  nacc = 0;
  if (!ok) { status = CHEM_CELL_BADINPUT; return; }
  double h = (h_io > 0.0 && isfinite(h_io)) ? h_io : o.h_init;
  if (dt > 0.0) h = fmin(h, dt);
  double t = 0.0;
  bool rejected_last = false, needJ = true;
  int nonfinite = 0, ns = 0, na = 0, st = CHEM_CELL_OK;
  while (t < dt) {
    if (ns >= o.max_substeps) { st = CHEM_CELL_MAXSTEPS; break; }
    if (o.deadline_ns) {
      unsigned long long now = lane == 0 ? global_ns() : 0ull;
      now = __shfl_sync(0xffffffffu, now, 0);
      if (now > o.deadline_ns) { st = CHEM_CELL_TIMEOUT; break; }
    }
    const bool last = (t + h >= dt * (1.0 - 1e-14));
    const double hu = last ? dt - t : h;
    if (hu < o.h_min) { st = CHEM_CELL_HMIN; break; }
    ++ns;
    if (needJ) {
      eval_jac(M, s, L, y, p, lane);
      needJ = false;
    }
    const StepOut so = ros_attempt(M, s, L, p, hu, o.rtol, o.atol, lane);
    if (o.trace && lane == 0 && ns <= o.trace_cap)
      o.trace[(size_t)(ns - 1) * o.N + cell] = (so.good && isfinite(so.err) && so.err <= 1.0) ? hu : -hu;
    if (!so.good || !isfinite(so.err)) {
      if (++nonfinite >= o.max_nonfinite) { st = CHEM_CELL_NONFINITE; break; }
      h = hu * 0.1;
      rejected_last = true;
      continue;
    }
    nonfinite = 0;
    const double fac = fmax(0.2, 0.9 * pow(so.err, -1.0 / 3.0));
    if (so.err <= 1.0) {
      t = last ? dt : t + hu;
      ++na;
      const double* yt = s + L.ytmp;
      for (int i = lane; i < m; i += kWarp) y[i] = yt[i];
      __syncwarp();
      h = hu * fmin(rejected_last ? 1.0 : 6.0, fac);
      rejected_last = false;
      needJ = true;
    } else {
      h = hu * fmin(1.0, fac);
      rejected_last = true;
    }
  }
  if (o.trace && lane == 0 && ns < o.trace_cap) o.trace[(size_t)ns * o.N + cell] = 0.0;
  h_io = h;
  nsub = ns;
  nacc = na;
  status = st;
}

}  // namespace chemgb
