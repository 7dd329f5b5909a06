/*
 * chem_oracle.cpp -- plain CPU reference for constant-pressure homogeneous-reactor chemistry.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load this library.  It shares no code with the CUDA library: its own mechanism struct,
 * its own loops, dense linear algebra, FP64 throughout.  It is written for a reader checking it against
 * the definitions, not for speed.
 *
 * What it computes.  The paper treats every CFD cell as an independent homogeneous gas-phase reactor
 * whose species equations are integrated by a stiff ODE solver with a sparse analytical Jacobian
 * (Sec. 1 and Sec. 2.5).  The paper states none of the formulas, so each ingredient below is the
 * standard definition of the named technique:
 *   - state y = (T, Y_1..Y_n) at fixed pressure p; W = 1/sum(Y_k/W_k); rho = p W / (Ru T);
 *     C_k = rho Y_k / W_k;  dY_k/dt = W_k w_k / rho;  dT/dt = -sum_k H_k w_k / (rho c_p);
 *   - NASA-7 polynomials for cp/R, h/RT, s/R (low set below T_mid, high set at or above it);
 *   - modified Arrhenius k = A T^b exp(-Ea/(Ru T)); third-body concentration [M] = sum_k alpha_k C_k
 *     (alpha_k = 1 unless listed); Troe fall-off k = k_inf Pr/(1+Pr) F (Gilbert-Luther-Troe form);
 *   - reverse rates k_r = k_f / Kc with Kc = exp(-dG/(Ru T)) (p0/(Ru T))^(sum nu), p0 = 101325 Pa;
 *   - Jacobian d f / d y written out densely by the chain rule through C(T, Y), rho(T, Y), c_p(T, Y);
 *   - the 4-stage L-stable Rosenbrock method RODAS3 (Sandu et al. 1997; also ROS2 and RODAS4) in its
 *     k-form
 *       (I - h g J) k_i = h f(y + sum_j a_ij k_j) + h J sum_j g_ij k_j,
 *       y1 = y + sum b_i k_i,  err = sum (b_i - bhat_i) k_i,
 *     with dense partial-pivot LU, and the Hairer-Wanner step-size controller.
 * Every function is templated on the scalar type so that the same code runs on complex numbers for
 * complex-step derivatives (the Jacobian check and the discrete sensitivities).
 */
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cplx = std::complex<double>;

constexpr double kRu = 8.314462618;   // J/(mol K), CODATA 2018 exact
constexpr double kP0 = 101325.0;      // Pa, standard-state pressure of Kc
constexpr double kLn10 = 2.302585092994045684;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
template <class S> inline double mag(const S& x) { return std::fabs(re(x)); }
inline bool finite_(double x) { return std::isfinite(x); }
inline bool finite_(const cplx& x) { return std::isfinite(x.real()) && std::isfinite(x.imag()); }

}  // namespace

extern "C" {
/* Mechanism as flat arrays (all caller-owned; see the package's synthetic generator for the layout). */
typedef struct {
  int n, R;
  const double* W;        /* [n] kg/mol */
  const double* lo;       /* [n*7] NASA-7 low range */
  const double* hi;       /* [n*7] NASA-7 high range */
  const double* Tmid;     /* [n] */
  const int *rptr, *rsp, *rnu;   /* reactants: CSR by reaction */
  const int *pptr, *psp, *pnu;   /* products */
  const double *A, *b, *Ea;      /* forward Arrhenius (k_inf for Troe), Ea in J/mol */
  const int* type;               /* 0 elementary, 1 third-body, 2 Troe */
  const int* rev;                /* 1 reversible */
  const int *eptr, *esp;         /* listed efficiencies: CSR by reaction */
  const double* eval;
  const double* troe;            /* [R*4] alpha, T3, T1, T2 (T2 <= 0: absent) */
  const double* low;             /* [R*3] A0, b0, Ea0 */
} OMech;
}

namespace {

/* Optional parameter shifts: k_f,r of reaction j multiplied by exp(dlnA[j]) (both limits for Troe) and
   every activation energy of reaction j shifted by dEa[j]; used for complex-step sensitivities. */
struct OTab;

template <class S> struct Perturb {
  const S* dlnA = nullptr;
  const S* dEa = nullptr;
  const OTab* tab = nullptr;   // tabulated temperature functions (real arithmetic only), see below
};

/* ---------------------------------------------------------------- tabulated temperature functions
   An opt-in approximation (Sec. 2.5: SpeedCHEM evaluates costly thermodynamic functions by interpolation
   of optimal degree).  Reading taken here: the temperature functions that each cost one or more
   exponentials -- every species' exp(g_k) and exp(-g_k) with g_k = h_k/(Ru T) - s_k/Ru (the factors of
   the equilibrium constants), every reaction's forward rate coefficient (the high-pressure limit of a
   fall-off reaction) and each fall-off reaction's Troe centre F_cent -- are replaced, for
   kTabTlo <= T < kTabThi, by piecewise polynomials in u = 1/T:
     - kTabNI equal intervals of u over [1/kTabThi, 1/kTabTlo] (T = 1000 K, the usual NASA-7 switch, is a
       boundary);
     - on interval j, with tau = 2 (u - u_j)/du - 1 in [-1, 1], the polynomial of degree d through the
       d + 1 Chebyshev points tau_i = cos(pi (2i + 1) / (2d + 2)), kept as monomial coefficients in tau;
     - one degree per class of functions (the four classes above), the smallest d in 1..8 for which every
       function of the class is within the relative tolerance of its exact value at 17 equispaced points
       of every interval ("optimal degree"); a class that no degree up to 8 meets stays exact.
   Outside the range the exact functions are used.  The fall-off variable P_r = k_0 [M] / k_inf stays
   exact (a ratio of two Arrhenius forms), and so do the logarithmic temperature derivatives of the
   Jacobian. */
constexpr int kTabNI = 640;
constexpr double kTabTlo = 250.0, kTabThi = 4000.0;
constexpr int kTabMaxDeg = 8;
enum { TAB_E = 0, TAB_IE = 1, TAB_KF = 2, TAB_FC = 3, TAB_CLASSES = 4 };

struct OTab {
  double tol = 0.0;
  double u_lo = 0.0, du = 0.0;
  int deg[TAB_CLASSES] = {0, 0, 0, 0};          // 0: the class is evaluated exactly
  int nfun[TAB_CLASSES] = {0, 0, 0, 0};
  std::vector<double> coef[TAB_CLASSES];        // [function][interval][deg + 1]
  std::vector<int> troe_slot;                   // reaction -> index among the fall-off reactions, -1
};

/* Interval and local coordinate of T; false outside the tabulated range. */
inline bool tab_locate(const OTab& t, double T, int& j, double& tau) {
  if (!(T >= kTabTlo && T < kTabThi)) return false;
  const double x = (1.0 / T - t.u_lo) / t.du;
  j = std::min(kTabNI - 1, std::max(0, (int)std::floor(x)));
  tau = 2.0 * (x - j) - 1.0;
  return true;
}

inline double tab_poly(const double* c, int d, double tau) {
  double v = c[d];
  for (int i = d - 1; i >= 0; --i) v = v * tau + c[i];
  return v;
}

/* Tabulated value of function f of class cls at (j, tau). */
inline double tab_value(const OTab& t, int cls, int f, int j, double tau) {
  const int d = t.deg[cls];
  return tab_poly(&t.coef[cls][((size_t)f * kTabNI + j) * (d + 1)], d, tau);
}

/* ---------------------------------------------------------------- thermo (NASA-7) */
template <class S> struct Thermo {
  std::vector<S> cp_R, h_RT, s_R, dcp_R_dT;
  std::vector<double> E, iE;   // tabulated exp(g_k), exp(-g_k) (filled by rates() when a table is in use)
};

template <class S> void thermo(const OMech& m, const S& T, Thermo<S>& th) {
  th.cp_R.assign(m.n, S(0)); th.h_RT.assign(m.n, S(0)); th.s_R.assign(m.n, S(0)); th.dcp_R_dT.assign(m.n, S(0));
  for (int k = 0; k < m.n; ++k) {
    const double* a = (re(T) < m.Tmid[k]) ? &m.lo[7 * k] : &m.hi[7 * k];
    S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    th.cp_R[k] = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    th.h_RT[k] = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    th.s_R[k] = a[0] * std::log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
    th.dcp_R_dT[k] = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T2 + 4.0 * a[4] * T3;
  }
}

/* ---------------------------------------------------------------- mixture */
template <class S> struct Mix {
  S Wbar, rho, cp;          // cp: mass-specific, J/(kg K)
  std::vector<S> C;         // mol/m^3
};

template <class S> void mixture(const OMech& m, const S& T, double p, const S* Y, const Thermo<S>& th, Mix<S>& mx) {
  S sig = 0.0;
  for (int k = 0; k < m.n; ++k) sig += Y[k] / m.W[k];
  mx.Wbar = 1.0 / sig;
  mx.rho = p * mx.Wbar / (kRu * T);
  mx.C.assign(m.n, S(0));
  mx.cp = 0.0;
  for (int k = 0; k < m.n; ++k) {
    mx.C[k] = mx.rho * Y[k] / m.W[k];
    mx.cp += Y[k] * (kRu * th.cp_R[k]) / m.W[k];
  }
}

/* ---------------------------------------------------------------- reaction rates */
template <class S> struct Rates {
  std::vector<S> kf, kr, M, qf, qr;            // per reaction; M is [M] (third-body and Troe)
  std::vector<S> dlnkf_dT, dlnkf_dlnM, dlnKc_dT;
  std::vector<double> nu;                       // [R*n] net stoichiometric coefficients nu'' - nu'
};

template <class S> S product_pow(const S& x, int nu) {
  S r = 1.0;
  for (int i = 0; i < nu; ++i) r *= x;
  return r;
}

template <class S>
void rates(const OMech& m, const S& T, double p, const Thermo<S>& th, const Mix<S>& mx, const Perturb<S>& pt,
           Rates<S>& rr) {
  const int R = m.R, n = m.n;
  rr.kf.assign(R, S(0)); rr.kr.assign(R, S(0)); rr.M.assign(R, S(0)); rr.qf.assign(R, S(0)); rr.qr.assign(R, S(0));
  rr.dlnkf_dT.assign(R, S(0)); rr.dlnkf_dlnM.assign(R, S(0)); rr.dlnKc_dT.assign(R, S(0));
  rr.nu.assign((size_t)R * n, 0.0);
  (void)p;
  // tabulated temperature functions: real arithmetic, no parameter shifts, T inside the table
  int tj = 0;
  double ttau = 0.0;
  const bool tab = std::is_same<S, double>::value && pt.tab && !pt.dlnA && !pt.dEa &&
                   tab_locate(*pt.tab, re(T), tj, ttau);
  std::vector<double> tE, tiE;
  if (tab && pt.tab->deg[TAB_E] > 0 && pt.tab->deg[TAB_IE] > 0) {
    tE.resize(n); tiE.resize(n);
    for (int k = 0; k < n; ++k) {
      tE[k] = tab_value(*pt.tab, TAB_E, k, tj, ttau);
      tiE[k] = tab_value(*pt.tab, TAB_IE, k, tj, ttau);
    }
  }
  for (int r = 0; r < R; ++r) {
    for (int i = m.rptr[r]; i < m.rptr[r + 1]; ++i) rr.nu[(size_t)r * n + m.rsp[i]] -= m.rnu[i];
    for (int i = m.pptr[r]; i < m.pptr[r + 1]; ++i) rr.nu[(size_t)r * n + m.psp[i]] += m.pnu[i];
    S dlnA = pt.dlnA ? pt.dlnA[r] : S(0.0);
    S dEa = pt.dEa ? pt.dEa[r] : S(0.0);
    S Ea = m.Ea[r] + dEa;
    // modified Arrhenius
    const S kinf_exact = m.A[r] * std::exp(dlnA) * std::pow(T, m.b[r]) * std::exp(-Ea / (kRu * T));
    const S kinf = (tab && pt.tab->deg[TAB_KF] > 0) ? S(tab_value(*pt.tab, TAB_KF, r, tj, ttau)) : kinf_exact;
    S dlnkinf_dT = m.b[r] / T + Ea / (kRu * T * T);
    // third-body concentration
    S M = 0.0;
    if (m.type[r] != 0) {
      std::vector<double> alpha(n, 1.0);
      for (int i = m.eptr[r]; i < m.eptr[r + 1]; ++i) alpha[m.esp[i]] = m.eval[i];
      for (int k = 0; k < n; ++k) M += alpha[k] * mx.C[k];
    }
    rr.M[r] = M;
    S kf = kinf, dlnkf_dT = dlnkinf_dT, dlnkf_dlnM = 0.0;
    if (m.type[r] == 2) {
      const double* tr = &m.troe[4 * r];
      const double* lw = &m.low[3 * r];
      S Ea0 = lw[2] + dEa;
      const int ts = pt.tab ? pt.tab->troe_slot[r] : -1;
      S k0 = lw[0] * std::exp(dlnA) * std::pow(T, lw[1]) * std::exp(-Ea0 / (kRu * T));
      S dlnk0_dT = lw[1] / T + Ea0 / (kRu * T * T);
      S Pr = k0 * M / kinf_exact;
      if (re(Pr) == 0.0) {
        kf = 0.0; dlnkf_dT = 0.0; dlnkf_dlnM = 0.0;
      } else {
        double alpha = tr[0], T3 = tr[1], T1 = tr[2], T2 = tr[3];
        S Fc = (1.0 - alpha) * std::exp(-T / T3) + alpha * std::exp(-T / T1);
        S dFc_dT = -(1.0 - alpha) / T3 * std::exp(-T / T3) - alpha / T1 * std::exp(-T / T1);
        if (T2 > 0.0) {
          Fc += std::exp(-T2 / T);
          dFc_dT += T2 / (T * T) * std::exp(-T2 / T);
        }
        if (tab && pt.tab->deg[TAB_FC] > 0) Fc = S(tab_value(*pt.tab, TAB_FC, ts, tj, ttau));
        S Lc = std::log10(Fc);
        S c = -0.4 - 0.67 * Lc;
        S nn = 0.75 - 1.27 * Lc;
        S Lp = std::log10(Pr);
        S x = Lp + c;
        S den = nn - 0.14 * x;
        S f1 = x / den;
        S log10F = Lc / (1.0 + f1 * f1);
        S F = std::pow(10.0, log10F);
        kf = kinf * (Pr / (1.0 + Pr)) * F;
        // derivatives of ln k with respect to T (at fixed [M]) and ln [M]
        S dlnPr_dT = dlnk0_dT - dlnkinf_dT;
        S dLc_dT = dFc_dT / (Fc * kLn10);
        S dx_dT = dlnPr_dT / kLn10 - 0.67 * dLc_dT;
        S dnn_dT = -1.27 * dLc_dT;
        S df1_dT = (dx_dT * nn - x * dnn_dT) / (den * den);
        S dlog10F_dT = dLc_dT / (1.0 + f1 * f1) - Lc * 2.0 * f1 * df1_dT / ((1.0 + f1 * f1) * (1.0 + f1 * f1));
        dlnkf_dT = dlnkinf_dT + dlnPr_dT / (1.0 + Pr) + kLn10 * dlog10F_dT;
        S df1_dlnM = (nn / kLn10) / (den * den);
        S dlog10F_dlnM = -Lc * 2.0 * f1 * df1_dlnM / ((1.0 + f1 * f1) * (1.0 + f1 * f1));
        dlnkf_dlnM = 1.0 / (1.0 + Pr) + kLn10 * dlog10F_dlnM;
      }
    }
    rr.kf[r] = kf;
    rr.dlnkf_dT[r] = dlnkf_dT;
    rr.dlnkf_dlnM[r] = dlnkf_dlnM;
    // equilibrium constant from NASA-7 Gibbs energies
    if (m.rev[r]) {
      S dG = 0.0, dH = 0.0;
      double dnu = 0.0;
      for (int k = 0; k < n; ++k) {
        double v = rr.nu[(size_t)r * n + k];
        if (v == 0.0) continue;
        dG += v * (th.h_RT[k] - th.s_R[k]);
        dH += v * th.h_RT[k];
        dnu += v;
      }
      S emdG = std::exp(-dG);
      if (!tE.empty()) {   // exp(-dG) = prod over products exp(-g)^nu * prod over reactants exp(g)^|nu|
        double e = 1.0;
        for (int k = 0; k < n; ++k) {
          const double v = rr.nu[(size_t)r * n + k];
          if (v > 0.0) e *= product_pow(tiE[k], (int)v);
          if (v < 0.0) e *= product_pow(tE[k], (int)(-v));
        }
        emdG = S(e);
      }
      S Kc = emdG * std::pow(kP0 / (kRu * T), dnu);
      rr.kr[r] = kf / Kc;
      rr.dlnKc_dT[r] = (dH - dnu) / T;
    }
    // rates of progress
    S Pf = 1.0, Pb = 1.0;
    for (int i = m.rptr[r]; i < m.rptr[r + 1]; ++i) Pf *= product_pow(mx.C[m.rsp[i]], m.rnu[i]);
    for (int i = m.pptr[r]; i < m.pptr[r + 1]; ++i) Pb *= product_pow(mx.C[m.psp[i]], m.pnu[i]);
    S Mfac = (m.type[r] == 1) ? M : S(1.0);
    rr.qf[r] = rr.kf[r] * Mfac * Pf;
    rr.qr[r] = m.rev[r] ? rr.kr[r] * Mfac * Pb : S(0.0);
  }
}

/* The exact value of function f of class cls at T (the functions the table stands for). */
double tab_exact(const OMech& m, const OTab& t, int cls, int f, double T) {
  if (cls == TAB_E || cls == TAB_IE) {
    const double* a = (T < m.Tmid[f]) ? &m.lo[7 * f] : &m.hi[7 * f];
    const double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    const double hRT = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    const double sR = a[0] * std::log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
    return cls == TAB_E ? std::exp(hRT - sR) : std::exp(sR - hRT);
  }
  if (cls == TAB_KF) return m.A[f] * std::pow(T, m.b[f]) * std::exp(-m.Ea[f] / (kRu * T));
  int r = 0;   // the f-th fall-off reaction
  for (int q = 0; q < m.R; ++q) if (t.troe_slot[q] == f) { r = q; break; }
  const double* tr = &m.troe[4 * r];
  double Fc = (1.0 - tr[0]) * std::exp(-T / tr[1]) + tr[0] * std::exp(-T / tr[2]);
  if (tr[3] > 0.0) Fc += std::exp(-tr[3] / T);
  return Fc;
}

/* Monomial coefficients (in tau) of the degree-d polynomial through the Chebyshev points of the interval
   [u0, u0 + du] of function f. */
void tab_fit(const OMech& m, const OTab& t, int cls, int f, double u0, int d, double* c) {
  const double pi = 3.14159265358979323846;
  std::vector<double> fv(d + 1), tv(d + 1), a(d + 1, 0.0);
  for (int i = 0; i <= d; ++i) {
    tv[i] = std::cos(pi * (2.0 * i + 1.0) / (2.0 * d + 2.0));
    fv[i] = tab_exact(m, t, cls, f, 1.0 / (u0 + 0.5 * (tv[i] + 1.0) * t.du));
  }
  // Chebyshev coefficients a_k = (2/(d+1)) sum_i f_i T_k(tau_i), a_0 halved
  for (int k = 0; k <= d; ++k) {
    double acc = 0.0;
    for (int i = 0; i <= d; ++i) acc += fv[i] * std::cos(k * std::acos(tv[i]));
    a[k] = 2.0 * acc / (d + 1);
  }
  a[0] *= 0.5;
  // sum_k a_k T_k(tau) in monomials: T_0 = 1, T_1 = tau, T_{k+1} = 2 tau T_k - T_{k-1}
  std::vector<double> Tm1(d + 1, 0.0), T0(d + 1, 0.0), Tn(d + 1, 0.0);
  for (int i = 0; i <= d; ++i) c[i] = 0.0;
  T0[0] = 1.0;
  for (int k = 0; k <= d; ++k) {
    for (int i = 0; i <= d; ++i) c[i] += a[k] * T0[i];
    std::fill(Tn.begin(), Tn.end(), 0.0);
    for (int i = 0; i < d; ++i) Tn[i + 1] += (k == 0 ? 1.0 : 2.0) * T0[i];
    if (k > 0)
      for (int i = 0; i <= d; ++i) Tn[i] -= Tm1[i];
    Tm1 = T0;
    T0 = Tn;
  }
}

/* Builds the tables of every class: the smallest degree that meets tol for every function of the class on
   every interval, checked at 17 equispaced points per interval against the exact functions. */
OTab* tab_build(const OMech& m, double tol) {
  OTab* t = new OTab();
  t->tol = tol;
  t->u_lo = 1.0 / kTabThi;
  t->du = (1.0 / kTabTlo - 1.0 / kTabThi) / kTabNI;
  t->troe_slot.assign(m.R, -1);
  int nt = 0;
  for (int r = 0; r < m.R; ++r) if (m.type[r] == 2) t->troe_slot[r] = nt++;
  const int nf[TAB_CLASSES] = {m.n, m.n, m.R, nt};
  for (int cls = 0; cls < TAB_CLASSES; ++cls) {
    t->nfun[cls] = nf[cls];
    t->deg[cls] = 0;
    if (nf[cls] == 0) continue;
    for (int d = 1; d <= kTabMaxDeg; ++d) {
      std::vector<double> cf((size_t)nf[cls] * kTabNI * (d + 1));
      bool ok = true;
      for (int f = 0; f < nf[cls] && ok; ++f)
        for (int j = 0; j < kTabNI && ok; ++j) {
          const double u0 = t->u_lo + j * t->du;
          double* c = &cf[((size_t)f * kTabNI + j) * (d + 1)];
          tab_fit(m, *t, cls, f, u0, d, c);
          for (int k = 0; k <= 16 && ok; ++k) {
            const double tau = -1.0 + k / 8.0;
            const double ex = tab_exact(m, *t, cls, f, 1.0 / (u0 + 0.5 * (tau + 1.0) * t->du));
            const double ap = tab_poly(c, d, tau);
            ok = std::fabs(ap - ex) <= tol * std::fabs(ex);
          }
        }
      if (ok) { t->deg[cls] = d; t->coef[cls].swap(cf); break; }
    }
  }
  return t;
}

/* ---------------------------------------------------------------- right-hand side */
template <class S> struct Eval {
  Thermo<S> th;
  Mix<S> mx;
  Rates<S> rr;
  std::vector<S> wdot;
};

template <class S>
void rhs(const OMech& m, double p, const Perturb<S>& pt, const S* y, S* f, Eval<S>& ev, double* gross_f = nullptr) {
  const int n = m.n;
  const S T = y[0];
  const S* Y = y + 1;
  thermo(m, T, ev.th);
  mixture(m, T, p, Y, ev.th, ev.mx);
  rates(m, T, p, ev.th, ev.mx, pt, ev.rr);
  ev.wdot.assign(n, S(0));
  std::vector<double> gw(n, 0.0);
  for (int r = 0; r < m.R; ++r)
    for (int k = 0; k < n; ++k) {
      double v = ev.rr.nu[(size_t)r * n + k];
      if (v == 0.0) continue;
      ev.wdot[k] += v * (ev.rr.qf[r] - ev.rr.qr[r]);
      gw[k] += std::fabs(v) * (mag(ev.rr.qf[r]) + mag(ev.rr.qr[r]));
    }
  S hw = 0.0;
  double ghw = 0.0;
  for (int k = 0; k < n; ++k) {
    S H = kRu * T * ev.th.h_RT[k];
    hw += H * ev.wdot[k];
    ghw += mag(H) * gw[k];
    f[1 + k] = m.W[k] * ev.wdot[k] / ev.mx.rho;
    if (gross_f) gross_f[1 + k] = m.W[k] * gw[k] / mag(ev.mx.rho);
  }
  f[0] = -hw / (ev.mx.rho * ev.mx.cp);
  if (gross_f) gross_f[0] = ghw / mag(ev.mx.rho * ev.mx.cp);
}

/* ---------------------------------------------------------------- Jacobian
   f = sum_r q_r e_r(y) with q_r = qf_r - qr_r and e_r = (-dH_r/(rho c_p), W_k nu_kr / rho), so
   J = sum_r [ e_r (grad qf_r - grad qr_r)^T + q_r (grad e_r)^T ].  Gradients are dense m-vectors in
   y = (T, Y_1..Y_n).  Alongside each gradient we accumulate the sum of magnitudes of its terms (the
   "gross" size) so a comparison can be scaled by the terms that cancel. */
template <class S> struct Grad {
  std::vector<S> v;
  std::vector<double> g;
  explicit Grad(int m = 0) : v(m, S(0)), g(m, 0.0) {}
  void zero() { std::fill(v.begin(), v.end(), S(0)); std::fill(g.begin(), g.end(), 0.0); }
  void axpy(const S& a, const Grad& x) {
    for (size_t i = 0; i < v.size(); ++i) { v[i] += a * x.v[i]; g[i] += mag(a) * x.g[i]; }
  }
  void add_T(const S& a) { v[0] += a; g[0] += mag(a); }
};

template <class S>
void jacobian(const OMech& m, double p, const Perturb<S>& pt, const S* y, S* J, double* G, Eval<S>& ev) {
  const int n = m.n, mm = n + 1;
  std::vector<S> f(mm);
  rhs(m, p, pt, y, f.data(), ev);
  const S T = y[0];
  const S* Y = y + 1;
  const auto& th = ev.th;
  const auto& mx = ev.mx;
  const auto& rr = ev.rr;
  for (int i = 0; i < mm * mm; ++i) J[i] = 0.0;
  if (G) for (int i = 0; i < mm * mm; ++i) G[i] = 0.0;
  // gradients of C_j, rho and c_p
  std::vector<Grad<S>> gC(n, Grad<S>(mm));
  for (int j = 0; j < n; ++j) {
    gC[j].add_T(-mx.C[j] / T);
    for (int i = 0; i < n; ++i) {
      if (i == j) { gC[j].v[1 + i] += mx.rho / m.W[j]; gC[j].g[1 + i] += mag(mx.rho / m.W[j]); }
      S t = -mx.C[j] * mx.Wbar / m.W[i];
      gC[j].v[1 + i] += t; gC[j].g[1 + i] += mag(t);
    }
  }
  Grad<S> grho(mm), gcp(mm);
  grho.add_T(-mx.rho / T);
  for (int i = 0; i < n; ++i) { grho.v[1 + i] = -mx.rho * mx.Wbar / m.W[i]; grho.g[1 + i] = mag(grho.v[1 + i]); }
  for (int k = 0; k < n; ++k) gcp.add_T(Y[k] * kRu * th.dcp_R_dT[k] / m.W[k]);
  for (int i = 0; i < n; ++i) { gcp.v[1 + i] = kRu * th.cp_R[i] / m.W[i]; gcp.g[1 + i] = mag(gcp.v[1 + i]); }
  const S rcp = mx.rho * mx.cp;

  Grad<S> gM(mm), glnkf(mm), gqf(mm), gqr(mm), gPf(mm), gPb(mm), geT(mm);
  std::vector<double> alpha(n);
  for (int r = 0; r < m.R; ++r) {
    gM.zero(); glnkf.zero(); gqf.zero(); gqr.zero(); gPf.zero(); gPb.zero(); geT.zero();
    const bool tb = m.type[r] != 0;
    if (tb) {
      std::fill(alpha.begin(), alpha.end(), 1.0);
      for (int i = m.eptr[r]; i < m.eptr[r + 1]; ++i) alpha[m.esp[i]] = m.eval[i];
      for (int j = 0; j < n; ++j) gM.axpy(S(alpha[j]), gC[j]);
    }
    // grad ln kf = dlnkf/dT e_T + dlnkf/dlnM grad M / M
    glnkf.add_T(rr.dlnkf_dT[r]);
    if (m.type[r] == 2 && re(rr.M[r]) != 0.0) glnkf.axpy(rr.dlnkf_dlnM[r] / rr.M[r], gM);
    // concentration products and their gradients
    S Pf = 1.0, Pb = 1.0;
    for (int i = m.rptr[r]; i < m.rptr[r + 1]; ++i) Pf *= product_pow(mx.C[m.rsp[i]], m.rnu[i]);
    for (int i = m.pptr[r]; i < m.pptr[r + 1]; ++i) Pb *= product_pow(mx.C[m.psp[i]], m.pnu[i]);
    for (int i = m.rptr[r]; i < m.rptr[r + 1]; ++i) {
      S d = S(double(m.rnu[i])) * product_pow(mx.C[m.rsp[i]], m.rnu[i] - 1);
      for (int l = m.rptr[r]; l < m.rptr[r + 1]; ++l) if (l != i) d *= product_pow(mx.C[m.rsp[l]], m.rnu[l]);
      gPf.axpy(d, gC[m.rsp[i]]);
    }
    for (int i = m.pptr[r]; i < m.pptr[r + 1]; ++i) {
      S d = S(double(m.pnu[i])) * product_pow(mx.C[m.psp[i]], m.pnu[i] - 1);
      for (int l = m.pptr[r]; l < m.pptr[r + 1]; ++l) if (l != i) d *= product_pow(mx.C[m.psp[l]], m.pnu[l]);
      gPb.axpy(d, gC[m.psp[i]]);
    }
    S Mfac = (m.type[r] == 1) ? rr.M[r] : S(1.0);
    // grad qf = qf grad ln kf + kf Pf grad Mfac + kf Mfac grad Pf
    gqf.axpy(rr.qf[r], glnkf);
    if (m.type[r] == 1) gqf.axpy(rr.kf[r] * Pf, gM);
    gqf.axpy(rr.kf[r] * Mfac, gPf);
    if (m.rev[r]) {
      // ln kr = ln kf - ln Kc
      gqr.axpy(rr.qr[r], glnkf);
      gqr.add_T(-rr.qr[r] * rr.dlnKc_dT[r]);
      if (m.type[r] == 1) gqr.axpy(rr.kr[r] * Pb, gM);
      gqr.axpy(rr.kr[r] * Mfac, gPb);
    }
    // e_r and its gradient
    S dH = 0.0, dCp = 0.0;
    for (int k = 0; k < n; ++k) {
      double v = rr.nu[(size_t)r * n + k];
      if (v == 0.0) continue;
      dH += v * kRu * T * th.h_RT[k];
      dCp += v * kRu * th.cp_R[k];
    }
    S eT = -dH / rcp;
    geT.add_T(-dCp / rcp);
    geT.axpy(dH * mx.cp / (rcp * rcp), grho);
    geT.axpy(dH * mx.rho / (rcp * rcp), gcp);
    const S q = rr.qf[r] - rr.qr[r];
    const double gq = mag(rr.qf[r]) + mag(rr.qr[r]);
    // T row
    for (int j = 0; j < mm; ++j) {
      J[j] += eT * (gqf.v[j] - gqr.v[j]) + q * geT.v[j];
      if (G) G[j] += mag(eT) * (gqf.g[j] + gqr.g[j]) + gq * geT.g[j];
    }
    // species rows
    for (int k = 0; k < n; ++k) {
      double v = rr.nu[(size_t)r * n + k];
      if (v == 0.0) continue;
      S eY = m.W[k] * v / mx.rho;
      S c2 = -m.W[k] * v / (mx.rho * mx.rho);   // grad eY = c2 grad rho
      S* Jrow = J + (size_t)(1 + k) * mm;
      double* Grow = G ? G + (size_t)(1 + k) * mm : nullptr;
      for (int j = 0; j < mm; ++j) {
        Jrow[j] += eY * (gqf.v[j] - gqr.v[j]) + q * c2 * grho.v[j];
        if (Grow) Grow[j] += mag(eY) * (gqf.g[j] + gqr.g[j]) + gq * mag(c2) * grho.g[j];
      }
    }
  }
}

/* ---------------------------------------------------------------- dense LU, partial pivoting */
template <class S> bool lu_factor(int m, S* A, int* piv) {
  for (int k = 0; k < m; ++k) {
    int pr = k;
    double best = mag(A[k * m + k]);
    for (int i = k + 1; i < m; ++i)
      if (mag(A[i * m + k]) > best) { best = mag(A[i * m + k]); pr = i; }
    piv[k] = pr;
    if (!(best > 0.0)) return false;
    if (pr != k)
      for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[pr * m + j]);
    for (int i = k + 1; i < m; ++i) {
      A[i * m + k] /= A[k * m + k];
      for (int j = k + 1; j < m; ++j) A[i * m + j] -= A[i * m + k] * A[k * m + j];
    }
  }
  return true;
}

template <class S> void lu_solve(int m, const S* LU, const int* piv, S* b) {
  for (int k = 0; k < m; ++k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) b[i] -= LU[i * m + j] * b[j];
  for (int i = m - 1; i >= 0; --i) {
    for (int j = i + 1; j < m; ++j) b[i] -= LU[i * m + j] * b[j];
    b[i] /= LU[i * m + i];
  }
}

/* ---------------------------------------------------------------- Rosenbrock methods (k-form)
   (I - h gamma J) k_i = h f(y + sum_j alpha_ij k_j) + h J sum_j gamma_ij k_j,
   y_new = y + sum_i b_i k_i, error = sum_i (b_i - bhat_i) k_i; the controller's exponent is
   -1/err_order (the order of the embedded pair plus one). */
constexpr int kMaxStages = 6;

struct Tableau {
  int s;
  double gamma;
  double a[kMaxStages][kMaxStages];   // alpha_ij, j < i
  double g[kMaxStages][kMaxStages];   // gamma_ij, j < i
  double b[kMaxStages], bhat[kMaxStages];
  int err_order;                      // the error estimate is O(h^err_order): controller exponent -1/err_order
};

/* RODAS3 (Sandu et al., Atmos. Environ. 31, 1997): 4 stages, order 3, embedded order 2, L-stable. */

const Tableau kRodas3 = {
    4, 0.5,
    {{0, 0, 0, 0}, {0, 0, 0, 0}, {1.0, 0, 0, 0}, {3.0 / 4.0, -1.0 / 4.0, 1.0 / 2.0, 0}},
    {{0, 0, 0, 0}, {1.0, 0, 0, 0}, {-1.0 / 4.0, -1.0 / 4.0, 0, 0}, {1.0 / 12.0, 1.0 / 12.0, -2.0 / 3.0, 0}},
    {5.0 / 6.0, -1.0 / 6.0, -1.0 / 6.0, 1.0 / 2.0},
    {3.0 / 4.0, -1.0 / 4.0, 1.0 / 2.0, 0.0},
    3};

/* ROS2 (Verwer, Spee, Blom and Hundsdorfer, SIAM J. Sci. Comput. 20, 1999): 2 stages, order 2,
   L-stable with gamma = 1 + 1/sqrt(2); its published form (I - gamma h J) k1 = f(y),
   (I - gamma h J) k2 = f(y + h k1) - 2 k1, y_new = y + h (3 k1 + k2)/2, with the embedded first-order
   solution y + h k1, is in this k-form (k = h k_published): alpha_21 = 1, gamma_21 = -2 gamma,
   b = (1/2, 1/2), bhat = (1, 0). */
const double kRos2Gamma = 0x1.b504f333f9de6p+0;   // 1 + 1/sqrt(2) rounded to double
const Tableau kRos2 = {
    2, kRos2Gamma,
    {{0, 0, 0, 0}, {1.0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {{0, 0, 0, 0}, {-2.0 * kRos2Gamma, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
    {0.5, 0.5, 0.0, 0.0},
    {1.0, 0.0, 0.0, 0.0},
    2};

/* RODAS4 (Hairer and Wanner, Solving Ordinary Differential Equations II, Sec. VI.4): 6 stages, order 4,
   embedded order 3, stiffly accurate, L-stable, gamma = 1/4.  The method is published in the transformed
   variables u_i = sum_j Gamma_ij k_j (Gamma lower triangular with diagonal gamma):
     (I/(h gamma) - J) u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij / h) u_j,
     y_new = y + sum_i m_i u_i,   error estimate sum_i e_i u_i.
   Those published numbers are kept here as printed, and the k-form of this oracle's step follows from
   them: Gamma^-1 = I/gamma - C (C = the strictly lower c_ij), alpha = A Gamma, b = m Gamma, and the
   embedded weights bhat = (m - e) Gamma. */
Tableau rodas4_tableau() {
  const int s = 6;
  const double gamma = 0.25;
  double A[6][6] = {}, Cm[6][6] = {};
  A[1][0] = 1.544;
  A[2][0] = 0.9466785280815826; A[2][1] = 0.2557011698983284;
  A[3][0] = 3.314825187068521; A[3][1] = 2.896124015972201; A[3][2] = 0.9986419139977817;
  A[4][0] = 1.221224509226641; A[4][1] = 6.019134481288629; A[4][2] = 12.53708332932087;
  A[4][3] = -0.6878860361058950;
  for (int j = 0; j < 4; ++j) A[5][j] = A[4][j];   // stage 6 starts from stage 5's point plus u_5
  A[5][4] = 1.0;
  Cm[1][0] = -5.6688;
  Cm[2][0] = -2.430093356833875; Cm[2][1] = -0.2063599157091915;
  Cm[3][0] = -0.1073529058151375; Cm[3][1] = -9.594562251023355; Cm[3][2] = -20.47028614809616;
  Cm[4][0] = 7.496443313967647; Cm[4][1] = -10.24680431464352; Cm[4][2] = -33.99990352819905;
  Cm[4][3] = 11.70890893206160;
  Cm[5][0] = 8.083246795921522; Cm[5][1] = -7.981132988064893; Cm[5][2] = -31.52159432874371;
  Cm[5][3] = 16.31930543123136; Cm[5][4] = -6.058818238834054;
  const double mw[6] = {A[4][0], A[4][1], A[4][2], A[4][3], 1.0, 1.0};
  const double ew[6] = {0, 0, 0, 0, 0, 1.0};
  // Gamma from its inverse G = I/gamma - C (lower triangular): column by column, forward substitution
  double Gi[6][6] = {}, Gm[6][6] = {};
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) Gi[i][j] = (i == j ? 1.0 / gamma : 0.0) - Cm[i][j];
  for (int c = 0; c < s; ++c)
    for (int i = 0; i < s; ++i) {
      double r = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) r -= Gi[i][k] * Gm[k][c];
      Gm[i][c] = r / Gi[i][i];
    }
  Tableau t{};
  t.s = s;
  t.gamma = gamma;
  t.err_order = 4;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < i; ++j) {
      double al = 0.0;
      for (int k = j; k < i; ++k) al += A[i][k] * Gm[k][j];
      t.a[i][j] = al;
      t.g[i][j] = Gm[i][j];
    }
  for (int j = 0; j < s; ++j) {
    double bb = 0.0, bh = 0.0;
    for (int i = j; i < s; ++i) { bb += mw[i] * Gm[i][j]; bh += (mw[i] - ew[i]) * Gm[i][j]; }
    t.b[j] = bb;
    t.bhat[j] = bh;
  }
  return t;
}
const Tableau kRodas4 = rodas4_tableau();

const Tableau& method_tableau(int method) { return method == 1 ? kRos2 : method == 2 ? kRodas4 : kRodas3; }

/* One Rosenbrock step of size h from y.  Returns false if the iteration matrix is singular. */
template <class S>
bool ros_step(const OMech& m, double p, const Perturb<S>& pt, const S* y, double h, S* ynew, S* yerr, Eval<S>& ev,
              const Tableau& tb = kRodas3) {
  const int mm = m.n + 1;
  std::vector<S> J((size_t)mm * mm), A((size_t)mm * mm);
  std::vector<int> piv(mm);
  jacobian(m, p, pt, y, J.data(), nullptr, ev);
  for (int i = 0; i < mm; ++i)
    for (int j = 0; j < mm; ++j) A[i * mm + j] = (i == j ? S(1.0) : S(0.0)) - h * tb.gamma * J[i * mm + j];
  if (!lu_factor(mm, A.data(), piv.data())) return false;
  std::vector<std::vector<S>> k(tb.s, std::vector<S>(mm));
  std::vector<S> yi(mm), fi(mm), gs(mm), rhsv(mm);
  for (int i = 0; i < tb.s; ++i) {
    for (int l = 0; l < mm; ++l) {
      yi[l] = y[l];
      gs[l] = 0.0;
      for (int j = 0; j < i; ++j) { yi[l] += tb.a[i][j] * k[j][l]; gs[l] += tb.g[i][j] * k[j][l]; }
    }
    rhs(m, p, pt, yi.data(), fi.data(), ev);
    for (int l = 0; l < mm; ++l) {
      S Jg = 0.0;
      for (int c = 0; c < mm; ++c) Jg += J[l * mm + c] * gs[c];
      rhsv[l] = h * fi[l] + h * Jg;
    }
    lu_solve(mm, A.data(), piv.data(), rhsv.data());
    k[i] = rhsv;
  }
  for (int l = 0; l < mm; ++l) {
    ynew[l] = y[l];
    yerr[l] = 0.0;
    for (int i = 0; i < tb.s; ++i) { ynew[l] += tb.b[i] * k[i][l]; yerr[l] += (tb.b[i] - tb.bhat[i]) * k[i][l]; }
  }
  return true;
}

enum { ST_OK = 0, ST_MAXSTEPS = 1, ST_HMIN = 2, ST_NONFINITE = 3, ST_BADINPUT = 4 };

struct Controls {
  double rtol, atol, h_default, h_min, fac_min, fac_max, safety;
  int max_steps;
  int max_nonfinite;   // consecutive non-finite attempts (each divides h by 10) before giving up
};

/* Adaptive integration of one cell over [0, dt].  y (m values) is overwritten with the result. */
int integrate_cell(const OMech& m, double p, double* y, double dt, const Controls& cc, double h_in, double* h_out,
                   int* nsub, int* nacc, std::vector<double>* tr_h, std::vector<int>* tr_acc,
                   const Tableau& tb = kRodas3, const OTab* tab = nullptr) {
  const int mm = m.n + 1;
  *nsub = 0; *nacc = 0;
  bool ok = finite_(y[0]) && y[0] > 0.0 && finite_(p) && p > 0.0 && finite_(dt) && dt >= 0.0;
  double sig = 0.0;
  for (int l = 1; l < mm; ++l) { ok = ok && finite_(y[l]); sig += y[l] / m.W[l - 1]; }
  if (!ok || !(sig > 0.0)) { *h_out = h_in; return ST_BADINPUT; }
  double h = (h_in > 0.0 && finite_(h_in)) ? h_in : cc.h_default;
  if (dt > 0.0) h = std::min(h, dt);
  double t = 0.0;
  bool rejected_last = false;
  int nonfinite = 0;
  Eval<double> ev;
  Perturb<double> pt;
  pt.tab = tab;
  std::vector<double> ynew(mm), yerr(mm);
  while (t < dt) {
    if (*nsub >= cc.max_steps) { *h_out = h; return ST_MAXSTEPS; }
    const bool last = (t + h >= dt * (1.0 - 1e-14));
    const double hu = last ? dt - t : h;
    if (hu < cc.h_min) { *h_out = h; return ST_HMIN; }
    ++*nsub;
    bool good = ros_step(m, p, pt, y, hu, ynew.data(), yerr.data(), ev, tb);
    double err = 0.0;
    if (good) {
      double s2 = 0.0;
      for (int l = 0; l < mm; ++l) {
        double sc = cc.atol + cc.rtol * std::max(std::fabs(y[l]), std::fabs(ynew[l]));
        double e = yerr[l] / sc;
        s2 += e * e;
      }
      err = std::sqrt(s2 / mm);
    }
    if (!good || !finite_(err)) {
      if (tr_h) { tr_h->push_back(hu); tr_acc->push_back(0); }
      if (++nonfinite >= cc.max_nonfinite) { *h_out = h; return ST_NONFINITE; }
      h = hu * 0.1;
      rejected_last = true;
      continue;
    }
    nonfinite = 0;
    const double fac = std::max(cc.fac_min, cc.safety * std::pow(err, -1.0 / tb.err_order));
    if (err <= 1.0) {
      if (tr_h) { tr_h->push_back(hu); tr_acc->push_back(1); }
      ++*nacc;
      t = last ? dt : t + hu;
      for (int l = 0; l < mm; ++l) y[l] = ynew[l];
      h = hu * std::min(rejected_last ? 1.0 : cc.fac_max, fac);
      rejected_last = false;
    } else {
      if (tr_h) { tr_h->push_back(hu); tr_acc->push_back(0); }
      h = hu * std::min(1.0, fac);
      rejected_last = true;
    }
  }
  *h_out = h;
  return ST_OK;
}

/* Replay: apply the given accepted step sizes, without error control. */
template <class S>
bool replay_cell(const OMech& m, double p, const Perturb<S>& pt, S* y, const double* hs, int nh,
                 const Tableau& tb = kRodas3) {
  const int mm = m.n + 1;
  Eval<S> ev;
  std::vector<S> ynew(mm), yerr(mm);
  for (int s = 0; s < nh; ++s) {
    if (!ros_step(m, p, pt, y, hs[s], ynew.data(), yerr.data(), ev, tb)) return false;
    for (int l = 0; l < mm; ++l) y[l] = ynew[l];
  }
  return true;
}

Controls make_controls(double rtol, double atol, int max_steps) {
  Controls c;
  c.rtol = rtol; c.atol = atol; c.h_default = 1e-7; c.h_min = 1e-20;
  c.fac_min = 0.2; c.fac_max = 6.0; c.safety = 0.9;
  c.max_steps = max_steps > 0 ? max_steps : 100000;
  c.max_nonfinite = 10;
  return c;
}

}  // namespace

/* ================================================================== C entry points (test use only) */
extern "C" {

/* f = dy/dt at y = (T, Y); optional wdot [n] (mol/m^3/s), gross_f [m], qf/qr [R], kf/kr [R]. */
int oracle_rhs(const OMech* m, double p, const double* y, double* f, double* wdot, double* gross_f, double* qf,
               double* qr, double* kf, double* kr) {
  Eval<double> ev;
  Perturb<double> pt;
  rhs(*m, p, pt, y, f, ev, gross_f);
  for (int k = 0; wdot && k < m->n; ++k) wdot[k] = ev.wdot[k];
  for (int r = 0; r < m->R; ++r) {
    if (qf) qf[r] = ev.rr.qf[r];
    if (qr) qr[r] = ev.rr.qr[r];
    if (kf) kf[r] = ev.rr.kf[r];
    if (kr) kr[r] = ev.rr.kr[r];
  }
  return 0;
}

/* NASA-7 values of every species at T: cp/R, h/RT, s/R. */
int oracle_thermo(const OMech* m, double T, double* cp_R, double* h_RT, double* s_R) {
  Thermo<double> th;
  thermo(*m, T, th);
  for (int k = 0; k < m->n; ++k) { cp_R[k] = th.cp_R[k]; h_RT[k] = th.h_RT[k]; s_R[k] = th.s_R[k]; }
  return 0;
}

/* Analytical dense Jacobian J[m*m] (row-major, J[i*m+j] = d f_i / d y_j) and optional gross sizes G. */
int oracle_jacobian(const OMech* m, double p, const double* y, double* J, double* G) {
  Eval<double> ev;
  Perturb<double> pt;
  jacobian(*m, p, pt, y, J, G, ev);
  return 0;
}

/* Complex-step Jacobian of oracle_rhs: column j = Im f(y + i eps e_j) / eps. */
int oracle_jacobian_cs(const OMech* m, double p, const double* y, double eps, double* J) {
  const int mm = m->n + 1;
  std::vector<cplx> yc(mm), fc(mm);
  Eval<cplx> ev;
  Perturb<cplx> pt;
  for (int j = 0; j < mm; ++j) {
    for (int l = 0; l < mm; ++l) yc[l] = cplx(y[l], l == j ? eps : 0.0);
    rhs(*m, p, pt, yc.data(), fc.data(), ev);
    for (int i = 0; i < mm; ++i) J[i * mm + j] = fc[i].imag() / eps;
  }
  return 0;
}

/* Complex-step derivative of f with respect to ln A_j (kind 0) or Ea_j (kind 1). */
int oracle_rhs_param_cs(const OMech* m, double p, const double* y, int kind, int j, double eps, double* df) {
  const int mm = m->n + 1;
  std::vector<cplx> yc(mm), fc(mm), d(m->R, cplx(0.0));
  for (int l = 0; l < mm; ++l) yc[l] = y[l];
  d[j] = cplx(0.0, eps);
  Perturb<cplx> pt;
  if (kind == 0) pt.dlnA = d.data(); else pt.dEa = d.data();
  Eval<cplx> ev;
  rhs(*m, p, pt, yc.data(), fc.data(), ev);
  for (int i = 0; i < mm; ++i) df[i] = fc[i].imag() / eps;
  return 0;
}

/* A method's coefficients (method 0 RODAS3, 1 ROS2, 2 RODAS4), padded to S = 6 stages: out[0] = s,
   out[1] = gamma, then alpha[S][S], gamma_ij[S][S], b[S], bhat[S], and err_order last (87 values). */
int oracle_tableau(int method, double* out) {
  const Tableau& t = method_tableau(method);
  constexpr int S = kMaxStages, SS = S * S;
  out[0] = t.s; out[1] = t.gamma; out[2 + 2 * SS + 2 * S] = t.err_order;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) { out[2 + S * i + j] = t.a[i][j]; out[2 + SS + S * i + j] = t.g[i][j]; }
  for (int i = 0; i < S; ++i) { out[2 + 2 * SS + i] = t.b[i]; out[2 + 2 * SS + S + i] = t.bhat[i]; }
  return 0;
}

/* One Rosenbrock step (k-form; method 0 RODAS3, 1 ROS2, 2 RODAS4): ynew, yerr. */
int oracle_step(const OMech* m, double p, const double* y, double h, double* ynew, double* yerr, int method) {
  Eval<double> ev;
  Perturb<double> pt;
  return ros_step(*m, p, pt, y, h, ynew, yerr, ev, method_tableau(method)) ? 0 : 1;
}

/* Adaptive integration of one cell.  y[m] in/out.  Optional trace of attempted steps (h, accepted). */
int oracle_integrate(const OMech* m, double p, double* y, double dt, double rtol, double atol, double h_in,
                     int max_steps, double* h_out, int* nsub, int* nacc, double* tr_h, int* tr_acc, int tr_cap,
                     int* tr_len, int method) {
  Controls cc = make_controls(rtol, atol, max_steps);
  std::vector<double> th;
  std::vector<int> ta;
  int st = integrate_cell(*m, p, y, dt, cc, h_in, h_out, nsub, nacc, tr_h ? &th : nullptr, tr_h ? &ta : nullptr,
                          method_tableau(method));
  if (tr_h) {
    int L = (int)th.size();
    *tr_len = L;
    for (int i = 0; i < std::min(L, tr_cap); ++i) { tr_h[i] = th[i]; tr_acc[i] = ta[i]; }
  }
  return st;
}

/* Replay a sequence of step sizes from y (in/out) without error control. */
int oracle_replay(const OMech* m, double p, double* y, const double* hs, int nh, int method) {
  Perturb<double> pt;
  return replay_cell(*m, p, pt, y, hs, nh, method_tableau(method)) ? 0 : 1;
}

/* The same with the tabulated temperature functions of tab (oracle_tab_build). */
int oracle_replay_tab(const OMech* m, double p, double* y, const double* hs, int nh, int method, const void* tab) {
  Perturb<double> pt;
  pt.tab = (const OTab*)tab;
  return replay_cell(*m, p, pt, y, hs, nh, method_tableau(method)) ? 0 : 1;
}

/* Tabulated temperature functions of the mechanism for relative tolerance tol (see tab_build); the caller
   frees them with oracle_tab_free. */
void* oracle_tab_build(const OMech* m, double tol) { return tab_build(*m, tol); }
void oracle_tab_free(void* tab) { delete (OTab*)tab; }

/* deg[4]: the degree of each class (0: exact), range[4]: T_lo, T_hi, u_lo, du; returns the interval count. */
int oracle_tab_info(const void* tab, int* deg, double* range) {
  const OTab* t = (const OTab*)tab;
  for (int c = 0; c < TAB_CLASSES; ++c) deg[c] = t->deg[c];
  range[0] = kTabTlo; range[1] = kTabThi; range[2] = t->u_lo; range[3] = t->du;
  return kTabNI;
}

/* Value of function f of class cls (0 exp(g_k), 1 exp(-g_k), 2 k_f of reaction f, 3 F_cent of the f-th
   fall-off reaction) at T: tabulated inside the range (for a tabulated class), else exact. */
double oracle_tab_eval(const OMech* m, const void* tab, int cls, int f, double T) {
  const OTab* t = (const OTab*)tab;
  int j = 0;
  double tau = 0.0;
  if (t->deg[cls] > 0 && tab_locate(*t, T, j, tau)) return tab_value(*t, cls, f, j, tau);
  return tab_exact(*m, *t, cls, f, T);
}

/* Complex-step derivative of the replayed final state with respect to one input:
   kind 0: ln A_j, kind 1: Ea_j, kind 2: initial state component y0_j.  dy[m] = d y_final / d theta. */
int oracle_replay_sens_cs(const OMech* m, double p, const double* y0, const double* hs, int nh, int kind, int j,
                          double eps, double* dy) {
  const int mm = m->n + 1;
  std::vector<cplx> y(mm), d(m->R, cplx(0.0));
  for (int l = 0; l < mm; ++l) y[l] = y0[l];
  Perturb<cplx> pt;
  if (kind == 0) { d[j] = cplx(0.0, eps); pt.dlnA = d.data(); }
  else if (kind == 1) { d[j] = cplx(0.0, eps); pt.dEa = d.data(); }
  else { y[j] += cplx(0.0, eps); }
  bool ok = replay_cell(*m, p, pt, y.data(), hs, nh);
  for (int l = 0; l < mm; ++l) dy[l] = y[l].imag() / eps;
  return ok ? 0 : 1;
}

/* Batch driver over N cells (structure of arrays: Y[k*N + c]); OpenMP dynamic schedule over cells, one
   cell at a time (a cell's integration takes milliseconds to seconds, so small samples keep every core
   busy).
   h_io: in initial step (<= 0: default), out last proposed step.  Optional trace [trace_cap*N]: attempt i
   of cell c at trace[i*N + c], +h accepted, -h rejected, 0 after the last.  Returns the thread count. */
int oracle_integrate_batch_tab(const OMech* m, int N, double* T, const double* p, double* Y, const double* dt,
                               double rtol, double atol, int max_steps, double* h_io, int* nsub, int* nacc,
                               int* status, int nthreads, double* trace, int trace_cap, int method, const void* tab);

int oracle_integrate_batch(const OMech* m, int N, double* T, const double* p, double* Y, const double* dt,
                           double rtol, double atol, int max_steps, double* h_io, int* nsub, int* nacc, int* status,
                           int nthreads, double* trace, int trace_cap, int method) {
  return oracle_integrate_batch_tab(m, N, T, p, Y, dt, rtol, atol, max_steps, h_io, nsub, nacc, status, nthreads,
                                    trace, trace_cap, method, nullptr);
}

/* The batch driver with the tabulated temperature functions of tab (NULL: exact). */
int oracle_integrate_batch_tab(const OMech* m, int N, double* T, const double* p, double* Y, const double* dt,
                               double rtol, double atol, int max_steps, double* h_io, int* nsub, int* nacc,
                               int* status, int nthreads, double* trace, int trace_cap, int method, const void* tab) {
  const Tableau& tb = method_tableau(method);
  Controls cc = make_controls(rtol, atol, max_steps);
  const int mm = m->n + 1;
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
  }
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int c = 0; c < N; ++c) {
    std::vector<double> y(mm);
    y[0] = T[c];
    for (int k = 0; k < m->n; ++k) y[1 + k] = Y[(size_t)k * N + c];
    double hout;
    int ns, na;
    std::vector<double> th;
    std::vector<int> ta;
    int st = integrate_cell(*m, p[c], y.data(), dt[c], cc, h_io ? h_io[c] : 0.0, &hout, &ns, &na,
                            trace ? &th : nullptr, trace ? &ta : nullptr, tb, (const OTab*)tab);
    if (trace) {
      for (int i = 0; i < trace_cap; ++i)
        trace[(size_t)i * N + c] = i < (int)th.size() ? (ta[i] ? th[i] : -th[i]) : 0.0;
    }
    T[c] = y[0];
    for (int k = 0; k < m->n; ++k) Y[(size_t)k * N + c] = y[1 + k];
    if (h_io) h_io[c] = hout;
    if (nsub) nsub[c] = ns;
    if (nacc) nacc[c] = na;
    if (status) status[c] = st;
  }
  return used;
}

}  // extern "C"
