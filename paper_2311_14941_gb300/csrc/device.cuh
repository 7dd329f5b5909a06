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
#include "mech.h"
#include "scalar.cuh"

namespace chemgb {

// -------------------------------------------------------------------------------------- lane groups
// The lanes that integrate one cell: one warp (GrpW<1>), or two consecutive warps of a block (GrpW<2>).
// Work inside a cell is strided over the group's lanes; shared-memory ordering inside the group is a
// warp barrier for one warp and a named barrier (bar.sync id, 64) for two.  Reductions add each warp's
// butterfly sum in warp order, so every lane of the group holds the same, reproducible value.  The
// group size is a compile-time constant: the one-warp code is the plain warp code.
template <int W>
struct GrpW;

template <>
struct GrpW<1> {
  static constexpr int size = kWarp;
  int lane;
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

template <>
struct GrpW<2> {
  static constexpr int size = 2 * kWarp;
  int lane;     // 0 .. 63
  int bar;      // named barrier of the group: 1 + the cell's index in its block
  double* xch;  // one exchange slot per warp in the cell's shared memory
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
  }
};

using Grp1 = GrpW<1>;
using Grp2 = GrpW<2>;

// Half a warp: two cells share a warp, 16 lanes each (mechanisms with few species, whose loops and
// sparse programs leave most of a warp's lanes idle).  Shared-memory ordering is a warp barrier over the
// group's own lanes, and reductions are butterflies within them, so the two cells of a warp may also
// run apart (different step sequences) without waiting for each other.
struct GrpH {
  static constexpr int size = kWarp / 2;
  int lane;        // 0 .. 15
  unsigned mask;   // the lanes of this half of the warp
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

__device__ __forceinline__ double gsum(const Grp1&, double v) { return warp_sum(v); }
__device__ __forceinline__ double gsum(const GrpH& g, double v) {
#pragma unroll
  for (int o = GrpH::size / 2; o > 0; o >>= 1) v += __shfl_xor_sync(g.mask, v, o);
  return v;
}
__device__ __forceinline__ double gsum(const Grp2& g, double v) {
  v = warp_sum(v);
  g.sync();   // earlier readers of the slots are done
  if ((g.lane & (kWarp - 1)) == 0) g.xch[g.lane / kWarp] = v;
  g.sync();
  return g.xch[0] + g.xch[1];
}
template <class G>
__device__ __forceinline__ Dual gsum(const G& g, Dual v) { return Dual(gsum(g, v.v), gsum(g, v.d)); }
template <class G, int K>
__device__ __forceinline__ DualN<K> gsum(const G& g, DualN<K> v) {
  v.v = gsum(g, v.v);
#pragma unroll
  for (int i = 0; i < K; ++i) v.d[i] = gsum(g, v.d[i]);
  return v;
}

__device__ __forceinline__ bool gall(const Grp1&, bool ok) { return __all_sync(0xffffffffu, ok); }
__device__ __forceinline__ bool gall(const GrpH& g, bool ok) { return __all_sync(g.mask, ok); }
__device__ __forceinline__ bool gall(const Grp2& g, bool ok) {
  ok = __all_sync(0xffffffffu, ok);
  g.sync();
  if ((g.lane & (kWarp - 1)) == 0) g.xch[g.lane / kWarp] = ok ? 1.0 : 0.0;
  g.sync();
  return g.xch[0] != 0.0 && g.xch[1] != 0.0;
}

// The value of lane 0, on every lane of the group.
__device__ __forceinline__ long long gbcast(const Grp1&, long long v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ long long gbcast(const GrpH& g, long long v) { return __shfl_sync(g.mask, v, 0, GrpH::size); }
__device__ __forceinline__ long long gbcast(const Grp2& g, long long v) {
  g.sync();
  if (g.lane == 0) g.xch[0] = __longlong_as_double(v);
  g.sync();
  const long long r = __double_as_longlong(g.xch[0]);
  g.sync();   // everyone has read the slot before it is reused
  return r;
}

// RODAS3 in transformed form.  a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1, m = b Gamma^-1,
// e = (b - bhat) Gamma^-1, obtained from the published alpha_ij, gamma_ij, b, bhat (gamma = 1/2).
// Zero coefficients are exploited below: a21 = a32 = a42 = 0 (stage 2 reuses f(y)), m2 = 0,
// e = (0, 0, 0, 1).
constexpr double RG = 0.5;
constexpr double A31 = 2.0, A41 = 2.0, A43 = 1.0;
constexpr double C21 = 4.0, C31 = 1.0, C32 = -1.0, C41 = 1.0, C42 = -1.0, C43 = -8.0 / 3.0;
constexpr double M1 = 2.0, M3 = 1.0, M4 = 1.0;

// ROS2 (Verwer, Spee, Blom and Hundsdorfer 1999), order 2 with a first-order embedded solution,
// L-stable with gamma = 1 + 1/sqrt(2).  Its published stages (I - gamma h J) k1 = f(y),
// (I - gamma h J) k2 = f(y + h k1) - 2 k1 give, with U_i = gamma h k_i, the transformed form
//   (I/(h gamma) - J) U1 = f(y),  (I/(h gamma) - J) U2 = f(y + U1/gamma) - (2/(gamma h)) U1,
//   y_new = y + (3/(2 gamma)) U1 + (1/(2 gamma)) U2,  err = (U1 + U2)/(2 gamma).
constexpr double RG2 = 0x1.b504f333f9de6p+0;   // 1 + 1/sqrt(2) rounded to double
constexpr double R2_A21 = 1.0 / RG2, R2_C21 = -2.0 / RG2, R2_M1 = 1.5 / RG2, R2_M2 = 0.5 / RG2, R2_E = 0.5 / RG2;

// RODAS4 (Hairer and Wanner, Solving ODEs II, Sec. VI.4), order 4 with an order-3 embedded solution,
// stiffly accurate and L-stable, gamma = 1/4, in its published transformed form:
//   (I/(h gamma) - J) U_i = f(y + sum_j a_ij U_j) + sum_j (c_ij / h) U_j.
// a_6j = a_5j (j < 5) and a_65 = 1, m = (a_51, a_52, a_53, a_54, 1, 1), e = (0, 0, 0, 0, 0, 1): stage 6
// starts from stage 5's point plus U5, y_new is stage 6's point plus U6, and U6 is the error estimate.
constexpr double RG4 = 0.25;
constexpr double R4_A21 = 1.544;
constexpr double R4_A31 = 0.9466785280815826, R4_A32 = 0.2557011698983284;
constexpr double R4_A41 = 3.314825187068521, R4_A42 = 2.896124015972201, R4_A43 = 0.9986419139977817;
constexpr double R4_A51 = 1.221224509226641, R4_A52 = 6.019134481288629, R4_A53 = 12.53708332932087,
                 R4_A54 = -0.6878860361058950;
constexpr double R4_C21 = -5.6688;
constexpr double R4_C31 = -2.430093356833875, R4_C32 = -0.2063599157091915;
constexpr double R4_C41 = -0.1073529058151375, R4_C42 = -9.594562251023355, R4_C43 = -20.47028614809616;
constexpr double R4_C51 = 7.496443313967647, R4_C52 = -10.24680431464352, R4_C53 = -33.99990352819905,
                 R4_C54 = 11.70890893206160;
constexpr double R4_C61 = 8.083246795921522, R4_C62 = -7.981132988064893, R4_C63 = -31.52159432874371,
                 R4_C64 = 16.31930543123136, R4_C65 = -6.058818238834054;
// The same coefficients as tables for the stage loop (row k - 2 of stage k; constant memory, read
// with warp-uniform indices).
static __constant__ double kR4A[4][4] = {{R4_A21, 0.0, 0.0, 0.0},
                                         {R4_A31, R4_A32, 0.0, 0.0},
                                         {R4_A41, R4_A42, R4_A43, 0.0},
                                         {R4_A51, R4_A52, R4_A53, R4_A54}};
static __constant__ double kR4C[5][5] = {{R4_C21, 0.0, 0.0, 0.0, 0.0},
                                         {R4_C31, R4_C32, 0.0, 0.0, 0.0},
                                         {R4_C41, R4_C42, R4_C43, 0.0, 0.0},
                                         {R4_C51, R4_C52, R4_C53, R4_C54, 0.0},
                                         {R4_C61, R4_C62, R4_C63, R4_C64, R4_C65}};

constexpr double kInvLn10 = 0.43429448190325182765;
constexpr double kLn10 = 2.30258509299404568402;


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
  o.b = (uint16_t)(v.y & 0xFFFF); o.kind = (uint16_t)(v.y >> 16);
  return o;
}

// Per-cell scalars shared by all lanes (every lane holds the same values).  tj, ttau: interval and local
// coordinate of T in the tables of tabulated temperature functions (tj < 0: exact evaluation).
template <class Sc>
struct ScalT {
  Sc T, lnT, invT, Wbar, rho, irho, cp, ctot, rtp, irtp, dcps;
  int tj;
  double ttau;
};

template <class A, class B>
struct same_type {
  static constexpr bool value = false;
};
template <class A>
struct same_type<A, A> {
  static constexpr bool value = true;
};
template <class Sc>
__host__ __device__ constexpr bool is_real() { return same_type<Sc, double>::value; }

// Polynomial in tau with coefficients c[0..d] (table memory, read-only path).
__device__ __forceinline__ double tab_poly(const double* c, int d, double tau) {
  double v = __ldg(c + d);
  for (int i = d - 1; i >= 0; --i) v = fma(v, tau, __ldg(c + i));
  return v;
}

// The table coordinates of T: interval j of u = 1/T and tau = 2 (u - u_j)/du - 1 (-1 outside the range or
// without tables; computed with the division, so that every implementation of the tables locates T alike).
template <class MV>
__device__ __forceinline__ void tab_locate(const MV& M, double T, double invT, int& tj, double& ttau) {
  tj = -1;
  ttau = 0.0;
  if (M.tab_on && T >= M.tab_tlo && T < M.tab_thi) {
    const double x = (invT - M.tab_ulo) / M.tab_du;
    const int j = min(M.tab_ni - 1, max(0, (int)floor(x)));
    tj = j;
    ttau = 2.0 * (x - j) - 1.0;
  }
}
using Scal = ScalT<double>;

// Coefficient nu of the omega and Dtil gather programs: the op carries the top 16 bits of the IEEE
// double nu (exact for +-1, +-2, +-3), rebuilt with integer instructions (no conversion on the FP64 pipe).
__device__ __forceinline__ double nu_of(int b) { return __hiloint2double(b << 16, 0); }

// -------------------------------------------------------------------------------------- gathers
// out[g] = sum over the group's terms of val(a, b); partial sums of split groups are combined after.
// ACC: out[g] += sum instead (outputs without terms in the program are left as they are).
template <bool ACC = false, class Sc, class F, class Gp, class GT>
__device__ __forceinline__ void run_gather(const GT& G, Sc* out, Sc* part, F valf, const Gp& g) {
  Sc acc = Sc(0.0);
  const GatherOp* op = G.ops + g.lane;
  const int NS = G.steps;
  const GatherOp idle{0, 0, DST_NONE, 1};
  GatherOp n1 = NS > 0 ? ld_gop(op) : idle;
  GatherOp n2 = NS > 1 ? ld_gop(op + g.size) : idle;
  for (int s = 0; s < NS; ++s) {
    const GatherOp o = n1;
    n1 = n2;
    if (s + 2 < NS) n2 = ld_gop(op + (size_t)(s + 2) * g.size);
    if (!(o.flags & 1)) acc += valf(o.a, o.b);
    if (o.dst != DST_NONE) {
      if (o.dst & PARTIAL_BIT) part[o.dst & 0x7FFF] = acc;
      else if (ACC) out[o.dst] += acc;
      else out[o.dst] = acc;
      acc = Sc(0.0);
    }
  }
  g.sync();
  for (int c = g.lane; c < G.n_comb; c += g.size) {
    const int dst = __ldg(G.comb + 3 * c), f = __ldg(G.comb + 3 * c + 1), cnt = __ldg(G.comb + 3 * c + 2);
    Sc s = Sc(0.0);
    for (int i = 0; i < cnt; ++i) s += part[f + i];
    if (ACC) out[dst] += s; else out[dst] = s;
  }
  g.sync();
}

// -------------------------------------------------------------------------------------- thermo
// One species at T: cp/R, h/RT, g = h/RT - s/R and its exponential (NASA-7, range by T vs T_mid).
template <class Sc>
struct SpOut {
  Sc cpR, hRT, eg, emg, yw, dcp;
};

template <class Sc, bool DERIV, class MV>
__device__ __forceinline__ SpOut<Sc> species_item(const MV& M, int k, const Sc* y, Sc T, Sc lnT, Sc invT,
                                                  int tj, double ttau) {
  const double* t = M.sp + (size_t)k * SP_STRIDE;
  const double iw = __ldg(t);
  const double* c = t + 4 + (val(T) < __ldg(t + 2) ? 0 : SP_RANGE);
  const Sc a0 = __ldg(c + 0), a1 = __ldg(c + 1), a2 = __ldg(c + 2), a3 = __ldg(c + 3), a4 = __ldg(c + 4);
  SpOut<Sc> o;
  o.cpR = sfma(T, sfma(T, sfma(T, sfma(T, a4, a3), a2), a1), a0);
  const Sc h = sfma(T, sfma(T, sfma(T, sfma(T, Sc(__ldg(c + 8)), Sc(__ldg(c + 7))), Sc(__ldg(c + 6))), Sc(__ldg(c + 5))),
                    a0);
  const Sc a5 = __ldg(c + 13), a6 = __ldg(c + 14);
  o.hRT = sfma(a5, invT, h);
  const Sc gp = sfma(T, sfma(T, sfma(T, sfma(T, Sc(__ldg(c + 12)), Sc(__ldg(c + 11))), Sc(__ldg(c + 10))),
                             Sc(__ldg(c + 9))),
                     sfma(a5, invT, -a6));
  bool tabd = false;
  if constexpr (is_real<Sc>()) {
    if (tj >= 0 && M.tab_deg[0] > 0 && M.tab_deg[1] > 0) {
      o.eg = tab_poly(M.tab[0] + ((size_t)tj * M.n + k) * (M.tab_deg[0] + 1), M.tab_deg[0], ttau);
      o.emg = tab_poly(M.tab[1] + ((size_t)tj * M.n + k) * (M.tab_deg[1] + 1), M.tab_deg[1], ttau);
      tabd = true;
    }
  }
  if (!tabd) {
    o.eg = sexp(sfma(a0, 1.0 - lnT, gp));
    o.emg = 1.0 / o.eg;
  }
  o.yw = y[1 + k] * iw;
  o.dcp = DERIV ? sfma(T, sfma(T, Sc(__ldg(c + 17)) * T + Sc(__ldg(c + 16)), Sc(__ldg(c + 15))), a1) : Sc(0.0);
  return o;
}

// NASA-7 at T for every species, two species per lane at a time (independent exp chains in flight);
// fills C, hRT, eg = exp(g), emg = 1/eg, cpR.
template <class Sc, bool DERIV, class Gp, class MV, class LT>
__device__ __forceinline__ ScalT<Sc> eval_species(const MV& M, Sc* s, const LT& L, const Sc* y,
                                                  double p, const Gp& g) {
  ScalT<Sc> sc;
  sc.T = y[0];
  sc.lnT = slog(sc.T);
  sc.invT = 1.0 / sc.T;
  sc.tj = -1;
  sc.ttau = 0.0;
  if constexpr (is_real<Sc>()) tab_locate(M, sc.T, sc.invT, sc.tj, sc.ttau);
  const Sc T = sc.T;
  Sc sig = Sc(0.0), cps = Sc(0.0), dcps = Sc(0.0);
  Sc* __restrict__ hRT = s + L.hRT;
  Sc* __restrict__ egv = s + L.eg;
  Sc* __restrict__ emg = s + L.emg;
  Sc* __restrict__ cpv = s + L.cpR;
  Sc* __restrict__ C = s + L.C;
  for (int k = g.lane; k < M.n; k += 2 * g.size) {
    const bool v2 = k + g.size < M.n;
    const int k2 = v2 ? k + g.size : k;
    const SpOut<Sc> a = species_item<Sc, DERIV>(M, k, y, T, sc.lnT, sc.invT, sc.tj, sc.ttau);
    const SpOut<Sc> b = species_item<Sc, DERIV>(M, k2, y, T, sc.lnT, sc.invT, sc.tj, sc.ttau);
    const Sc ia = a.emg, ib = b.emg;
    sig += a.yw + (v2 ? b.yw : Sc(0.0));
    cps = sfma(a.yw, a.cpR, cps);
    if (v2) cps = sfma(b.yw, b.cpR, cps);
    if (DERIV) {
      dcps = sfma(a.yw, a.dcp, dcps);
      if (v2) dcps = sfma(b.yw, b.dcp, dcps);
    }
    hRT[k] = a.hRT; egv[k] = a.eg; emg[k] = ia; cpv[k] = a.cpR; C[k] = a.yw;
    if (v2) { hRT[k2] = b.hRT; egv[k2] = b.eg; emg[k2] = ib; cpv[k2] = b.cpR; C[k2] = b.yw; }
  }
  sig = gsum(g, sig);
  cps = gsum(g, cps);
  if (DERIV) dcps = gsum(g, dcps);
  sc.Wbar = 1.0 / sig;
  sc.ctot = p * sc.invT * (1.0 / kRu);
  sc.rho = sc.ctot * sc.Wbar;
  sc.irho = 1.0 / sc.rho;
  sc.cp = kRu * cps;
  sc.dcps = dcps;
  sc.rtp = kRu * T * (1.0 / kP0);
  sc.irtp = 1.0 / sc.rtp;
  g.sync();
  for (int k = g.lane; k < M.n; k += g.size) C[k] *= sc.rho;
  g.sync();
  return sc;
}

// -------------------------------------------------------------------------------------- reactions
// Per-reaction quantities of the rate evaluation that the derivative part needs afterwards.
template <class Sc>
struct RxCore {
  Sc q, qn, kf, kr, Mfac, dlnkf_dT, dlnKc_dT, dlnk_dlnM, iM;
  Sc cr0, cr1, cr2, cp0, cp1, cp2;
  int so, scn;
  bool rep;   // a species occurs more than once on one side (coefficient 2 or 3)
};

// Rate of progress of reaction r, specialised on the reaction type (0 elementary, 1 third-body,
// 2 Troe).  Branch-free in the participant counts: absent occurrences read index 0 and count as 1.
template <class Sc, int TYPE, bool DERIV, class MV>
__device__ __forceinline__ RxCore<Sc> rx_core(const MV& M, int r, const Sc* __restrict__ C,
                                              const Sc* __restrict__ eg, const Sc* __restrict__ emg,
                                              const Sc* __restrict__ hRT, const ScalT<Sc>& sc) {
  const int* I = M.rxi + (size_t)r * RX_I;
  const double* D = M.rxd + (size_t)r * RX_D;
  const int rev = __ldg(I + 1), nro = __ldg(I + 2), npo = __ldg(I + 3);
  const int r0 = __ldg(I + 4), r1 = max(__ldg(I + 5), 0), r2 = max(__ldg(I + 6), 0);
  const int p0 = __ldg(I + 7), p1 = max(__ldg(I + 8), 0), p2 = max(__ldg(I + 9), 0);
  const Sc lnA = __ldg(D), bb = __ldg(D + 1), Ta = __ldg(D + 2);
  RxCore<Sc> x;
  x.rep = (nro > 1 && r1 == r0) || (nro > 2 && (r2 == r0 || r2 == r1)) || (npo > 1 && p1 == p0) ||
          (npo > 2 && (p2 == p0 || p2 == p1));
  const Sc lnkinf = sfma(-Ta, sc.invT, sfma(bb, sc.lnT, lnA));
  Sc kf;
  bool tkf = false;
  if constexpr (is_real<Sc>()) {
    if (sc.tj >= 0 && M.tab_deg[2] > 0) {
      kf = tab_poly(M.tab[2] + ((size_t)sc.tj * M.R + r) * (M.tab_deg[2] + 1), M.tab_deg[2], sc.ttau);
      tkf = true;
    }
  }
  if (!tkf) kf = sexp(lnkinf);
  x.cr0 = C[r0]; x.cr1 = nro > 1 ? C[r1] : Sc(1.0); x.cr2 = nro > 2 ? C[r2] : Sc(1.0);
  x.cp0 = C[p0]; x.cp1 = npo > 1 ? C[p1] : Sc(1.0); x.cp2 = npo > 2 ? C[p2] : Sc(1.0);
  const Sc Pf = x.cr0 * x.cr1 * x.cr2, Pb = x.cp0 * x.cp1 * x.cp2;
  Sc Mv = sc.ctot;
  if (TYPE != 0) {
    const int eo = __ldg(I + 11), ec = __ldg(I + 12);
    for (int i = 0; i < ec; ++i) Mv = sfma(Sc(__ldg(M.eff_am1 + eo + i)), C[__ldg(M.eff_sp + eo + i)], Mv);
  }
  x.dlnkf_dT = DERIV ? sfma(Ta, sc.invT, bb) * sc.invT : Sc(0.0);
  x.dlnk_dlnM = Sc(0.0);
  x.iM = Sc(0.0);
  if (TYPE == 2) {
    const Sc lnk0 = sfma(-Sc(__ldg(D + 5)), sc.invT, sfma(Sc(__ldg(D + 4)), sc.lnT, Sc(__ldg(D + 3))));
    const Sc lnM = slog(Mv);
    const Sc lnPr = lnk0 - lnkinf + lnM;
    const Sc Pr = sexp(lnPr);
    const double T2 = __ldg(D + 10);
    // the Troe centre: tabulated (Troe reactions are the first compiled ones), or from its three
    // exponentials, which the Jacobian's temperature derivative needs in any case
    bool tfc = false;
    if constexpr (is_real<Sc>()) tfc = sc.tj >= 0 && M.tab_deg[3] > 0;
    Sc e3 = Sc(0.0), e1 = Sc(0.0), e2 = Sc(0.0), Fc;
    if (!tfc || DERIV) {
      e3 = sexp(-sc.T * __ldg(D + 8));
      e1 = sexp(-sc.T * __ldg(D + 9));
      e2 = T2 > 0.0 ? sexp(-T2 * sc.invT) : Sc(0.0);
    }
    if constexpr (is_real<Sc>()) {
      if (tfc) Fc = tab_poly(M.tab[3] + ((size_t)sc.tj * M.n_troe + r) * (M.tab_deg[3] + 1), M.tab_deg[3], sc.ttau);
    }
    if (!tfc) Fc = sfma(Sc(__ldg(D + 6)), e3, sfma(Sc(__ldg(D + 7)), e1, e2));
    const Sc Lc = slog(Fc) * kInvLn10;
    const Sc cc = sfma(Sc(-0.67), Lc, Sc(-0.4));
    const Sc nn = sfma(Sc(-1.27), Lc, Sc(0.75));
    const Sc xx = sfma(lnPr, Sc(kInvLn10), cc);
    const Sc den = sfma(Sc(-0.14), xx, nn);
    // three reciprocals from one division: 1/den, 1/(1 + f1^2) = den^2/S2 with S2 = den^2 + xx^2, and
    // 1/(1 + Pr), all from R = 1/(den S2 (1 + Pr))
    const Sc pr1 = 1.0 + Pr;
    const Sc S2 = sfma(xx, xx, den * den);
    const Sc dp = den * pr1;
    const Sc R = 1.0 / (dp * S2);
    const Sc iden = S2 * pr1 * R;
    const Sc f1 = xx * iden;
    const Sc ib = den * dp * R * den;
    const Sc F = sexp(Lc * ib * kLn10);
    const Sc ipr1 = den * S2 * R;
    kf = kf * (Pr * ipr1) * F;
    if (DERIV) {
      const Sc dlnk0_dT = sfma(Sc(__ldg(D + 5)), sc.invT, Sc(__ldg(D + 4))) * sc.invT;
      const Sc dlnPr_dT = dlnk0_dT - x.dlnkf_dT;
      const Sc dFc_dT = -(__ldg(D + 6) * __ldg(D + 8)) * e3 - (__ldg(D + 7) * __ldg(D + 9)) * e1 +
                        T2 * sc.invT * sc.invT * e2;
      const Sc dLc_dT = dFc_dT / Fc * kInvLn10;
      const Sc dx_dT = sfma(dlnPr_dT, Sc(kInvLn10), -0.67 * dLc_dT);
      const Sc dnn_dT = -1.27 * dLc_dT;
      const Sc df1_dT = (dx_dT * nn - xx * dnn_dT) * iden * iden;
      const Sc dlog10F_dT = sfma(dLc_dT, ib, -2.0 * Lc * f1 * df1_dT * ib * ib);
      x.dlnkf_dT = x.dlnkf_dT + dlnPr_dT * ipr1 + kLn10 * dlog10F_dT;
      const Sc df1_dlnM = nn * kInvLn10 * iden * iden;
      x.dlnk_dlnM = ipr1 - kLn10 * 2.0 * Lc * f1 * df1_dlnM * ib * ib;
      x.iM = sexp(-lnM);
    }
  }
  // reverse rate: k_r = k_f * prod exp(g)^nu'' * prod exp(-g)^nu' * (Ru T/p0)^(sum nu)
  const int dn = npo - nro;
  Sc ik = eg[p0] * emg[r0];
  ik *= (npo > 1 ? eg[p1] : Sc(1.0)) * (npo > 2 ? eg[p2] : Sc(1.0));
  ik *= (nro > 1 ? emg[r1] : Sc(1.0)) * (nro > 2 ? emg[r2] : Sc(1.0));
  const Sc fp = dn > 0 ? sc.rtp : sc.irtp;
  const int adn = dn < 0 ? -dn : dn;
  ik *= (adn >= 1 ? fp : Sc(1.0)) * (adn >= 2 ? fp : Sc(1.0)) * (adn >= 3 ? fp : Sc(1.0));
  x.kr = rev ? kf * ik : Sc(0.0);
  x.kf = kf;
  if (DERIV) {
    Sc sh = hRT[p0] - hRT[r0];
    sh += (npo > 1 ? hRT[p1] : Sc(0.0)) + (npo > 2 ? hRT[p2] : Sc(0.0));
    sh -= (nro > 1 ? hRT[r1] : Sc(0.0)) + (nro > 2 ? hRT[r2] : Sc(0.0));
    const double dnd = dn == 0 ? 0.0 : dn == 1 ? 1.0 : dn == -1 ? -1.0 : dn == 2 ? 2.0 : dn == -2 ? -2.0 :
                       dn == 3 ? 3.0 : -3.0;
    x.dlnKc_dT = rev ? (sh - dnd) * sc.invT : Sc(0.0);
  } else {
    x.dlnKc_dT = Sc(0.0);
  }
  x.Mfac = (TYPE == 1) ? Mv : Sc(1.0);
  x.qn = sfma(kf, Pf, -(x.kr * Pb));
  x.q = x.Mfac * x.qn;
  x.so = DERIV ? __ldg(I + 13) : 0;
  x.scn = DERIV ? __ldg(I + 14) : 0;
  return x;
}

// Store q (and with DERIV: dq/dT at fixed C into s[dq_off + r], and the derivative slots dq/dC_j into
// s[d_off + slot]) of reaction r.
template <class Sc, int TYPE, bool DERIV, class MV, class LT>
__device__ __forceinline__ void rx_store(const MV& M, int r, const RxCore<Sc>& x, Sc* s, const LT& L,
                                         const ScalT<Sc>& sc, bool valid, int dq_off, int d_off) {
  if (!valid) return;
  s[L.q + r] = x.q;
  if (!DERIV) return;
  const Sc kfM = x.kf * x.Mfac, krM = x.kr * x.Mfac;
  const Sc qf = kfM * x.cr0 * x.cr1 * x.cr2, qr = krM * x.cp0 * x.cp1 * x.cp2;
  Sc dqdM = Sc(0.0);
  if (TYPE == 1) dqdM = x.qn;
  if (TYPE == 2) dqdM = x.dlnk_dlnM * x.q * x.iM;
  // [M] depends on T through the total concentration p/(Ru T)
  s[dq_off + r] = sfma(x.dlnkf_dT, qf, -((x.dlnkf_dT - x.dlnKc_dT) * qr)) - dqdM * sc.ctot * sc.invT;
  // partial products: d(prod)/d(occurrence i) = product of the other occurrences
  const Sc dr0 = x.cr1 * x.cr2, dr1 = x.cr0 * x.cr2, dr2 = x.cr0 * x.cr1;
  const Sc dp0 = x.cp1 * x.cp2, dp1 = x.cp0 * x.cp2, dp2 = x.cp0 * x.cp1;
  // a slot's factor is the sum over the slot species' occurrences; with no species repeated on a side in
  // any active lane of the warp, it is one occurrence factor (or none): select it instead of adding
  const bool any_rep = __any_sync(__activemask(), x.rep);
  for (int i = 0; i < x.scn; ++i) {
    const int mask = __ldg(M.dslot_mask + x.so + i);
    // elementary reactions list no colliders: their (efficiency - 1) is 0 and so is the [M] term
    Sc v = TYPE == 0 ? Sc(0.0) : __ldg(M.dslot_am1 + x.so + i) * dqdM;
    Sc fr, fq;
    if (any_rep) {           // a slot species may occur more than once on a side: sum its factors
      fr = Sc(0.0); fq = Sc(0.0);
      if (mask & 1) fr += dr0;
      if (mask & 2) fr += dr1;
      if (mask & 4) fr += dr2;
      if (mask & 8) fq += dp0;
      if (mask & 16) fq += dp1;
      if (mask & 32) fq += dp2;
    } else {                 // at most one occurrence per side: select it
      fr = (mask & 1) ? dr0 : (mask & 2) ? dr1 : (mask & 4) ? dr2 : Sc(0.0);
      fq = (mask & 8) ? dp0 : (mask & 16) ? dp1 : (mask & 32) ? dp2 : Sc(0.0);
    }
    v = sfma(kfM, fr, v);
    v = sfma(-krM, fq, v);
    s[d_off + x.so + i] = v;
  }
}

// Rates of progress of reactions [rb, re).  Reactions are ordered Troe, third-body, elementary, so every
// segment has warp-uniform control flow; elementary reactions go two per lane (two exp chains).
template <class Sc, bool DERIV, class Gp, class MV, class LT>
__device__ __forceinline__ void eval_reactions(const MV& M, Sc* s, const LT& L, const ScalT<Sc>& sc,
                                               const Gp& g, int rb, int re, int dq_off = 0, int d_off = 0) {
  const Sc* C = s + L.C;
  const Sc* eg = s + L.eg;
  const Sc* emg = s + L.emg;
  const Sc* hRT = s + L.hRT;
  const int t1 = min(re, M.n_troe), e0 = M.n_troe + M.n_tb, b1 = min(re, e0);
  for (int r = rb + g.lane; r < t1; r += g.size)
    rx_store<Sc, 2, DERIV>(M, r, rx_core<Sc, 2, DERIV>(M, r, C, eg, emg, hRT, sc), s, L, sc, true, dq_off, d_off);
  for (int r = max(rb, M.n_troe) + g.lane; r < b1; r += g.size)
    rx_store<Sc, 1, DERIV>(M, r, rx_core<Sc, 1, DERIV>(M, r, C, eg, emg, hRT, sc), s, L, sc, true, dq_off, d_off);
  for (int r = max(rb, e0) + g.lane; r < re; r += 2 * g.size) {
    const bool v2 = r + g.size < re;
    const int r2 = v2 ? r + g.size : r;
    const RxCore<Sc> a = rx_core<Sc, 0, DERIV>(M, r, C, eg, emg, hRT, sc);
    const RxCore<Sc> b = rx_core<Sc, 0, DERIV>(M, r2, C, eg, emg, hRT, sc);
    rx_store<Sc, 0, DERIV>(M, r, a, s, L, sc, true, dq_off, d_off);
    rx_store<Sc, 0, DERIV>(M, r2, b, s, L, sc, v2, dq_off, d_off);
  }
  g.sync();
}

// -------------------------------------------------------------------------------------- f and J
// f(y) into out[m].  Uses C/hRT/eg/emg/cpR/q scratch.  Returns the scalars of the evaluation.
template <class Sc, class Gp, class MV, class LT>
__device__ __forceinline__ ScalT<Sc> eval_f(const MV& M, Sc* s, const LT& L, const Sc* y, double p,
                                            Sc* out, const Gp& g) {
  ScalT<Sc> sc = eval_species<Sc, false>(M, s, L, y, p, g);
  eval_reactions<Sc, false>(M, s, L, sc, g, 0, M.R);
  const Sc* q = s + L.q;
  Sc* part = s + L.part;
  Sc* w = out + 1;   // production rates written in place, then scaled
  run_gather(M.g_omega, w, part, [&](int a, int b) { return nu_of(b) * q[a]; }, g);
  Sc Qs = Sc(0.0);
  for (int k = g.lane; k < M.n; k += g.size) {
    const Sc om = w[k];
    Qs = sfma(s[L.hRT + k], om, Qs);
    w[k] = om * __ldg(M.sp + (size_t)k * SP_STRIDE + 1) * sc.irho;
  }
  Qs = gsum(g, Qs);
  if (g.lane == 0) out[0] = -kRu * sc.T * Qs / (sc.rho * sc.cp);
  g.sync();
  return sc;
}

// f(y) into f0[m], S[nnz_S] (internal order), u[m], v[m].  Scratch: C.., q, the pass region D, x (w),
// U1 (g), U2 (t).  The reactions run in passes (see MechView::jpass): each pass leaves dq/dT and the
// derivative slots of its reactions in the region, and its gather adds them into the Y block of S
// (Dtil) and into the T-column slots of S, which hold w_T until the T column is formed below.
template <class Sc, class Gp, class MV, class LT>
__device__ __forceinline__ ScalT<Sc> eval_jac(const MV& M, Sc* s, const LT& L, const Sc* y, double p,
                                              const Gp& g) {
  ScalT<Sc> sc = eval_species<Sc, true>(M, s, L, y, p, g);
  Sc* part = s + L.part;
  Sc* w = s + L.x;      // w_k
  Sc* gk = s + L.U1;
  Sc* tk = s + L.U2;
  Sc* S = s + L.S;
  Sc* wT = S + M.nY;    // w_T,k, until overwritten by the T column
  const Sc* C = s + L.C;
  const Sc* hRT = s + L.hRT;
  const Sc* reg = s + L.D;
  for (int e = g.lane; e < M.nY + M.n; e += g.size) S[e] = Sc(0.0);
  for (int ps = 0; ps < M.n_jpass; ++ps) {
    const int rb = M.jpass[ps][JP_RB], cnt = M.jpass[ps][JP_CNT];
    eval_reactions<Sc, true>(M, s, L, sc, g, rb, M.jpass[ps][JP_RE], L.D - rb, L.D + cnt - M.jpass[ps][JP_SB]);
    run_gather<true>(M.g_jac[ps], S, part, [&](int a, int b) { return nu_of(b) * reg[a]; }, g);
  }
  const Sc* q = s + L.q;
  run_gather(M.g_omega, w, part, [&](int a, int b) { return nu_of(b) * q[a]; }, g);
  run_gather(M.g_row, gk, part, [&](int a, int b) { return S[a] * C[b]; }, g);
  run_gather(M.g_col, tk, part, [&](int a, int b) { return S[a] * hRT[b]; }, g);
  Sc* f = s + L.f0;
  Sc* u = s + L.u;
  Sc* v = s + L.v;
  const Sc T = sc.T;
  // f, u and the T column; partial sums for the T row scalars
  Sc Qs = Sc(0.0), A1 = Sc(0.0), A2 = Sc(0.0);
  for (int k = g.lane; k < M.n; k += g.size) {
    const double Wk = __ldg(M.sp + (size_t)k * SP_STRIDE + 1);
    const Sc om = w[k], g = gk[k];
    const Sc dwT = sfma(-g, sc.invT, wT[k]);   // read before the T column overwrites w_T
    const Sc fk = Wk * om * sc.irho;
    f[1 + k] = fk;
    u[1 + k] = Wk * sc.irho * (om - g);
    S[M.nY + k] = sfma(Wk * sc.irho, dwT, fk * sc.invT);
    v[1 + k] = sc.Wbar * __ldg(M.sp + (size_t)k * SP_STRIDE);
    const Sc h = hRT[k];
    Qs = sfma(h, om, Qs);
    A1 = sfma(s[L.cpR + k], om, sfma(T * h, dwT, A1));
    A2 = sfma(h, g, A2);
  }
  Qs = gsum(g, Qs);
  A1 = gsum(g, A1);
  A2 = gsum(g, A2);
  const Sc rcp = sc.rho * sc.cp;
  const Sc fT = -kRu * T * Qs / rcp;
  // T row: S_Tj for species j, then S_TT; u_T; v_T
  for (int j = g.lane; j < M.n; j += g.size) {
    const double iw = __ldg(M.sp + (size_t)j * SP_STRIDE);
    S[M.nY + M.n + 1 + j] = -kRu * sfma(T, tk[j], fT * s[L.cpR + j]) * iw / sc.cp;
  }
  if (g.lane == 0) {
    f[0] = fT;
    S[M.nY + M.n] = -kRu * A1 / rcp + fT * (sc.invT - kRu * sc.dcps / sc.cp);
    u[0] = kRu * T * A2 / rcp + fT;
    v[0] = Sc(0.0);
  }
  g.sync();
  // species block: S_kj = (W_k / W_j) Dtil_kj (after the row and column sums used Dtil)
  for (int e = g.lane; e < M.nY; e += g.size) S[e] *= __ldg(M.entry_wratio + e);
  g.sync();
  return sc;
}

// -------------------------------------------------------------------------------------- linear algebra
// LU of A = I/(h gamma) - S, in place, by the precomputed elimination program.  false if a pivot is 0
// or not finite.
template <class Gp, class MV, class LT>
__device__ __forceinline__ bool lu_build_factor(const MV& M, double* s, const LT& L, double gh,
                                                const Gp& g) {
  double* LU = s + L.LU;
  double* dinv = s + L.dinv;
  const double* S = s + L.S;
  for (int l = g.lane; l < M.nnz_LU; l += g.size) {
    const int src = __ldg(M.lu_src + l);
    LU[l] = src >= 0 ? -S[src] : 0.0;
  }
  g.sync();
  for (int i = g.lane; i < M.m; i += g.size) LU[__ldg(M.lu_diag + i)] += gh;
  g.sync();
  bool ok = true;
  const ElimOp* op = M.lu_ops + g.lane;
  const int NS = M.lu_steps;
  ElimOp n1 = NS > 0 ? ld_eop(op) : ElimOp{OP_IDLE, 0, 0, 0};
  ElimOp n2 = NS > 1 ? ld_eop(op + g.size) : ElimOp{OP_IDLE, 0, 0, 0};
  for (int st = 0; st < NS; ++st) {
    const ElimOp o = n1;
    n1 = n2;
    if (st + 2 < NS) n2 = ld_eop(op + (size_t)(st + 2) * g.size);
    const int kind = o.kind;
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
    g.sync();
  }
  return gall(g, ok);
}

// x <- A^{-1} x (forward and backward substitution by the precomputed program; state-order vector).
// With x2 != nullptr the same program solves a second right-hand side in the same steps.
template <bool TWO, class Gp, class MV, class LT>
__device__ __forceinline__ void lu_solve_impl(const MV& M, const double* s, const LT& L, double* x,
                                              double* x2, const Gp& g) {
  const double* LU = s + L.LU;
  const double* dinv = s + L.dinv;
  const ElimOp* op = M.sv_ops + g.lane;
  const int S = M.sv_steps;
  // the factor does not change during the solve: each step's coefficient (L/U entry or 1/pivot; idle
  // ops read entry 0) is loaded one step ahead, off the step-to-step dependence through x
  auto coef = [&](const ElimOp& o) { return (o.kind == K_UPDATE ? LU : dinv)[o.a]; };
  ElimOp n1 = S > 0 ? ld_eop(op) : ElimOp{OP_IDLE, 0, 0, K_SCALE};
  ElimOp n2 = S > 1 ? ld_eop(op + g.size) : ElimOp{OP_IDLE, 0, 0, K_SCALE};
  double c1 = coef(n1);
  for (int st = 0; st < S; ++st) {
    const ElimOp o = n1;
    const double c = c1;
    n1 = n2;
    c1 = coef(n1);
    if (st + 2 < S) n2 = ld_eop(op + (size_t)(st + 2) * g.size);
    if (o.t != OP_IDLE) {
      if (o.kind == K_UPDATE) {
        x[o.t] = fma(-c, x[o.b], x[o.t]);
        if (TWO) x2[o.t] = fma(-c, x2[o.b], x2[o.t]);
      } else {
        x[o.t] *= c;
        if (TWO) x2[o.t] *= c;
      }
    }
    g.sync();
  }
}

template <class Gp, class MV, class LT>
__device__ __forceinline__ void lu_solve(const MV& M, const double* s, const LT& L, double* x,
                                         const Gp& g) {
  lu_solve_impl<false>(M, s, L, x, nullptr, g);
}

// x <- M^{-1} x with M = A - u v^T:  x = A^-1 x + z (v . A^-1 x) / (1 - v . z),  z = A^-1 u
template <class Gp, class MV, class LT>
__device__ __forceinline__ void sm_solve(const MV& M, const double* s, const LT& L, double* x,
                                         double iden, const Gp& g) {
  lu_solve(M, s, L, x, g);
  const double* v = s + L.v;
  const double* z = s + L.z;
  double d = 0.0;
  for (int i = g.lane; i < M.m; i += g.size) d = fma(v[i], x[i], d);
  d = gsum(g, d) * iden;
  for (int i = g.lane; i < M.m; i += g.size) x[i] = fma(z[i], d, x[i]);
  g.sync();
}

// -------------------------------------------------------------------------------------- step
struct StepOut {
  bool good;
  double err;
};

// One RODAS3 attempt of size h from y (f0, S, u, v already evaluated at y).  ynew into ytmp, err into
// the return value.  U1..U4, x, z, LU are scratch.
template <class Gp, class MV, class LT>
__device__ __forceinline__ StepOut ros_attempt(const MV& M, double* s, const LT& L, double p, double h,
                                               double rtol, double atol, const Gp& g) {
  StepOut so{false, 0.0};
  const int m = M.m;
  const double ih = 1.0 / h;
  if (!lu_build_factor(M, s, L, ih * (1.0 / RG), g)) return so;
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
  // z = A^-1 u (the Sherman-Morrison vector) and stage 1's A^-1 f0, in one pass of the solve program
  for (int i = g.lane; i < m; i += g.size) { z[i] = u[i]; U1[i] = f0[i]; }
  g.sync();
  lu_solve_impl<true>(M, s, L, z, U1, g);
  double vz = 0.0, vx = 0.0;
  for (int i = g.lane; i < m; i += g.size) { vz = fma(v[i], z[i], vz); vx = fma(v[i], U1[i], vx); }
  vz = gsum(g, vz);
  vx = gsum(g, vx);
  const double den = 1.0 - vz;
  if (!(den != 0.0) || !isfinite(den)) return so;
  const double iden = 1.0 / den;
  // stage 1: Sherman-Morrison correction of A^-1 f0
  vx *= iden;
  for (int i = g.lane; i < m; i += g.size) U1[i] = fma(z[i], vx, U1[i]);
  g.sync();
  // stage 2 (a21 = 0: f(y) again)
  for (int i = g.lane; i < m; i += g.size) U2[i] = fma(C21 * ih, U1[i], f0[i]);
  g.sync();
  sm_solve(M, s, L, U2, iden, g);
  // stage 3
  for (int i = g.lane; i < m; i += g.size) yt[i] = fma(A31, U1[i], y[i]);
  g.sync();
  eval_f<double>(M, s, L, yt, p, U3, g);
  for (int i = g.lane; i < m; i += g.size) U3[i] = fma(ih, fma(C31, U1[i], C32 * U2[i]), U3[i]);
  g.sync();
  sm_solve(M, s, L, U3, iden, g);
  // stage 4
  for (int i = g.lane; i < m; i += g.size) yt[i] = fma(A43, U3[i], fma(A41, U1[i], y[i]));
  g.sync();
  eval_f<double>(M, s, L, yt, p, U4, g);
  for (int i = g.lane; i < m; i += g.size) U4[i] = fma(ih, fma(C41, U1[i], fma(C42, U2[i], C43 * U3[i])), U4[i]);
  g.sync();
  sm_solve(M, s, L, U4, iden, g);
  // solution, embedded error, scaled RMS norm
  double e2 = 0.0;
  bool fin = true;
  for (int i = g.lane; i < m; i += g.size) {
    const double yn = fma(M4, U4[i], fma(M3, U3[i], fma(M1, U1[i], y[i])));
    yt[i] = yn;
    const double sc = fma(rtol, fmax(fabs(y[i]), fabs(yn)), atol);
    const double e = U4[i] / sc;
    e2 = fma(e, e, e2);
    fin = fin && isfinite(yn);
  }
  e2 = gsum(g, e2);
  fin = gall(g, fin);
  g.sync();
  so.err = sqrt(e2 / (double)m);
  so.good = fin;
  return so;
}

// One ROS2 attempt of size h from y (f0, S, u, v already evaluated at y); ynew into ytmp.
template <class Gp, class MV, class LT>
__device__ __forceinline__ StepOut ros2_attempt(const MV& M, double* s, const LT& L, double p, double h,
                                                double rtol, double atol, const Gp& g) {
  StepOut so{false, 0.0};
  const int m = M.m;
  const double ih = 1.0 / h;
  if (!lu_build_factor(M, s, L, ih * (1.0 / RG2), g)) return so;
  double* y = s + L.y;
  double* yt = s + L.ytmp;
  double* f0 = s + L.f0;
  double* U1 = s + L.U1;
  double* U2 = s + L.U2;
  double* z = s + L.z;
  const double* u = s + L.u;
  const double* v = s + L.v;
  for (int i = g.lane; i < m; i += g.size) { z[i] = u[i]; U1[i] = f0[i]; }
  g.sync();
  lu_solve_impl<true>(M, s, L, z, U1, g);
  double vz = 0.0, vx = 0.0;
  for (int i = g.lane; i < m; i += g.size) { vz = fma(v[i], z[i], vz); vx = fma(v[i], U1[i], vx); }
  vz = gsum(g, vz);
  vx = gsum(g, vx);
  const double den = 1.0 - vz;
  if (!(den != 0.0) || !isfinite(den)) return so;
  const double iden = 1.0 / den;
  vx *= iden;
  for (int i = g.lane; i < m; i += g.size) U1[i] = fma(z[i], vx, U1[i]);
  g.sync();
  // stage 2
  for (int i = g.lane; i < m; i += g.size) yt[i] = fma(R2_A21, U1[i], y[i]);
  g.sync();
  eval_f<double>(M, s, L, yt, p, U2, g);
  for (int i = g.lane; i < m; i += g.size) U2[i] = fma(R2_C21 * ih, U1[i], U2[i]);
  g.sync();
  sm_solve(M, s, L, U2, iden, g);
  double e2 = 0.0;
  bool fin = true;
  for (int i = g.lane; i < m; i += g.size) {
    const double yn = fma(R2_M2, U2[i], fma(R2_M1, U1[i], y[i]));
    yt[i] = yn;
    const double sc = fma(rtol, fmax(fabs(y[i]), fabs(yn)), atol);
    const double e = R2_E * (U1[i] + U2[i]) / sc;
    e2 = fma(e, e, e2);
    fin = fin && isfinite(yn);
  }
  e2 = gsum(g, e2);
  fin = gall(g, fin);
  g.sync();
  so.err = sqrt(e2 / (double)m);
  so.good = fin;
  return so;
}

// One RODAS4 attempt of size h from y (f0, S, u, v already evaluated at y); ynew into ytmp.  U5 lives in
// the Jacobian's w_k vector (x), which is scratch until the next Jacobian evaluation; stage 6's
// coefficient sum is gathered into U1 and its solution U6 takes U2's place, so the attempt needs no
// shared memory beyond RODAS3's.
template <class Gp, class MV, class LT>
__device__ __forceinline__ StepOut ros4_attempt(const MV& M, double* s, const LT& L, double p, double h,
                                                double rtol, double atol, const Gp& g) {
  StepOut so{false, 0.0};
  const int m = M.m;
  const double ih = 1.0 / h;
  if (!lu_build_factor(M, s, L, ih * (1.0 / RG4), g)) return so;
  double* y = s + L.y;
  double* yt = s + L.ytmp;
  double* f0 = s + L.f0;
  double* U1 = s + L.U1;
  double* U2 = s + L.U2;
  double* U3 = s + L.U3;
  double* U4 = s + L.U4;
  double* U5 = s + L.x;
  double* z = s + L.z;
  const double* u = s + L.u;
  const double* v = s + L.v;
  // z = A^-1 u and stage 1's A^-1 f0 in one pass of the solve program, then the Sherman-Morrison
  // correction of stage 1
  for (int i = g.lane; i < m; i += g.size) { z[i] = u[i]; U1[i] = f0[i]; }
  g.sync();
  lu_solve_impl<true>(M, s, L, z, U1, g);
  double vz = 0.0, vx = 0.0;
  for (int i = g.lane; i < m; i += g.size) { vz = fma(v[i], z[i], vz); vx = fma(v[i], U1[i], vx); }
  vz = gsum(g, vz);
  vx = gsum(g, vx);
  const double den = 1.0 - vz;
  if (!(den != 0.0) || !isfinite(den)) return so;
  const double iden = 1.0 / den;
  vx *= iden;
  for (int i = g.lane; i < m; i += g.size) U1[i] = fma(z[i], vx, U1[i]);
  g.sync();
  // stages 2..6 in one loop (one copy of the right-hand side and solve code: the six stages written out
  // overflowed the instruction cache).  Stage k's point is y + sum_j a_kj U_j (stage 6: stage 5's point
  // plus U5), its vector solves A U_k = f(point) + (1/h) sum_j c_kj U_j; the coefficient sums are formed
  // in the order of the written-out stages, so the arithmetic is unchanged.
  double* Us[5] = {U1, U2, U3, U4, U5};
#pragma unroll 1
  for (int k = 1; k < 6; ++k) {   // stage k + 1
    double* out = k < 5 ? Us[k] : U2;   // stage 6's vector overwrites U2, dead by then
    if (k < 5) {
      for (int i = g.lane; i < m; i += g.size) {
        double acc = y[i];
        for (int j = 0; j < k; ++j) acc = fma(kR4A[k - 1][j], Us[j][i], acc);
        yt[i] = acc;
      }
    } else {   // stage 6: the coefficient sum of U1..U5 goes into U1 (not read afterwards)
      for (int i = g.lane; i < m; i += g.size) {
        yt[i] += U5[i];
        double acc = kR4C[4][4] * U5[i];
        for (int j = 3; j >= 0; --j) acc = fma(kR4C[4][j], Us[j][i], acc);
        U1[i] = ih * acc;
      }
    }
    g.sync();
    eval_f<double>(M, s, L, yt, p, out, g);
    if (k == 1) {
      for (int i = g.lane; i < m; i += g.size) out[i] = fma(R4_C21 * ih, U1[i], out[i]);
    } else if (k < 5) {
      for (int i = g.lane; i < m; i += g.size) {
        double acc = kR4C[k - 1][k - 1] * Us[k - 1][i];
        for (int j = k - 2; j >= 0; --j) acc = fma(kR4C[k - 1][j], Us[j][i], acc);
        out[i] = fma(ih, acc, out[i]);
      }
    } else {
      for (int i = g.lane; i < m; i += g.size) out[i] += U1[i];
    }
    g.sync();
    sm_solve(M, s, L, out, iden, g);
  }
  // solution = stage 6's point + U6, error estimate U6, scaled RMS norm
  double e2 = 0.0;
  bool fin = true;
  for (int i = g.lane; i < m; i += g.size) {
    const double yn = yt[i] + U2[i];
    yt[i] = yn;
    const double sc = fma(rtol, fmax(fabs(y[i]), fabs(yn)), atol);
    const double e = U2[i] / sc;
    e2 = fma(e, e, e2);
    fin = fin && isfinite(yn);
  }
  e2 = gsum(g, e2);
  fin = gall(g, fin);
  g.sync();
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
  // optional tape for the discrete adjoint: accepted step sizes rec_h[i*N + c] (i < rec_cap) and
  // checkpoints rec_ck[(j*m + l)*N + c] = state component l after j*rec_K accepted steps; rec_n[c] is the
  // number of accepted steps, or -1 when the tape overflowed
  double* rec_h;
  double* rec_ck;
  int* rec_n;
  int rec_cap, rec_K;
  int method;   // 0 RODAS3, 1 ROS2, 2 RODAS4
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Adaptive integration of the cell whose state sits in y (shared memory) over [0, dt].
template <class Gp, class MV, class LT>
__device__ __forceinline__ void integrate_cell(const MV& M, double* s, const LT& L, double p, double dt,
                                               double& h_io, int& nsub, int& nacc, int& status, const IntOpts& o,
                                               const Gp& g, int cell) {
  double* y = s + L.y;
  const int m = M.m;
  // input check
  bool ok = isfinite(p) && p > 0.0 && isfinite(dt) && dt >= 0.0 && isfinite(y[0]) && y[0] > 0.0;
  double sig = 0.0;
  for (int k = g.lane; k < M.n; k += g.size) {
    const double yk = y[1 + k];
    ok = ok && isfinite(yk);
    sig = fma(yk, __ldg(M.sp + (size_t)k * SP_STRIDE), sig);
  }
  sig = gsum(g, sig);
  ok = gall(g, ok) && sig > 0.0;
  nsub = 0;
  nacc = 0;
  if (!ok) {
    status = kCellBadInput;
    if (o.rec_h && g.lane == 0) o.rec_n[cell] = -1;
    return;
  }
  double h = (h_io > 0.0 && isfinite(h_io)) ? h_io : o.h_init;
  if (dt > 0.0) h = fmin(h, dt);
  double t = 0.0;
  bool rejected_last = false, needJ = true;
  int nonfinite = 0, ns = 0, na = 0, st = kCellOk;
  if (o.rec_h)
    for (int i = g.lane; i < m; i += g.size) o.rec_ck[(size_t)i * o.N + cell] = y[i];
  while (t < dt) {
    if (ns >= o.max_substeps) { st = kCellMaxSteps; break; }
    if (o.deadline_ns) {
      const unsigned long long now = (unsigned long long)gbcast(g, g.lane == 0 ? (long long)global_ns() : 0ll);
      if (now > o.deadline_ns) { st = kCellTimeout; break; }
    }
    const bool last = (t + h >= dt * (1.0 - 1e-14));
    const double hu = last ? dt - t : h;
    if (hu < o.h_min) { st = kCellHmin; break; }
    ++ns;
    if (needJ) {
      eval_jac<double>(M, s, L, y, p, g);
      needJ = false;
    }
    const StepOut so = o.method == 1   ? ros2_attempt(M, s, L, p, hu, o.rtol, o.atol, g)
                       : o.method == 2 ? ros4_attempt(M, s, L, p, hu, o.rtol, o.atol, g)
                                       : ros_attempt(M, s, L, p, hu, o.rtol, o.atol, g);
    if (o.trace && g.lane == 0 && ns <= o.trace_cap)
      o.trace[(size_t)(ns - 1) * o.N + cell] = (so.good && isfinite(so.err) && so.err <= 1.0) ? hu : -hu;
    if (!so.good || !isfinite(so.err)) {
      if (++nonfinite >= o.max_nonfinite) { st = kCellNonfinite; break; }
      h = hu * 0.1;
      rejected_last = true;
      continue;
    }
    nonfinite = 0;
    // step-size factor: err^(-1/(embedded order + 1)): 3 for RODAS3, 2 for ROS2, 4 for RODAS4
    const double fac =
        fmax(0.2, 0.9 * pow(so.err, o.method == 1 ? -0.5 : o.method == 2 ? -0.25 : -1.0 / 3.0));
    if (so.err <= 1.0) {
      t = last ? dt : t + hu;
      ++na;
      const double* yt = s + L.ytmp;
      for (int i = g.lane; i < m; i += g.size) y[i] = yt[i];
      g.sync();
      if (o.rec_h && na <= o.rec_cap) {
        if (g.lane == 0) o.rec_h[(size_t)(na - 1) * o.N + cell] = hu;
        if (na % o.rec_K == 0)
          for (int i = g.lane; i < m; i += g.size) o.rec_ck[((size_t)(na / o.rec_K) * m + i) * o.N + cell] = y[i];
      }
      h = hu * fmin(rejected_last ? 1.0 : 6.0, fac);
      rejected_last = false;
      needJ = true;
    } else {
      h = hu * fmin(1.0, fac);
      rejected_last = true;
    }
  }
  if (o.trace && g.lane == 0 && ns < o.trace_cap) o.trace[(size_t)ns * o.N + cell] = 0.0;
  if (o.rec_h && g.lane == 0) o.rec_n[cell] = (na <= o.rec_cap && st == kCellOk) ? na : -1;
  h_io = h;
  nsub = ns;
  nacc = na;
  status = st;
}

}  // namespace chemgb
