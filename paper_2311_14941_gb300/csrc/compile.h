// compile.h -- host mechanism compiler: description -> tables and warp programs.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/chem.h"
#include "mech.h"

namespace chemgb {

struct HostGather {
  std::vector<GatherOp> ops;   // [steps * width]
  int steps = 0;
  int n_partial = 0;
  std::vector<int> comb;   // triples
};

// The warp programs for one group width (the lanes that integrate a cell: 32, 64 or 16).
struct HostProg {
  int width = kWarp;
  HostGather g_omega, g_row, g_col;
  std::vector<HostGather> g_jac;       // one gather program per Jacobian pass
  std::vector<ElimOp> lu_ops, sv_ops, svT_ops;   // [steps * width]
  std::vector<uint8_t> lu_kind, sv_kind, svT_kind;
};

struct HostMech {
  int n = 0, R = 0, m = 0, n_troe = 0, n_tb = 0, nY = 0, nnz_S = 0, nnz_LU = 0, n_dslot = 0;
  std::vector<int> rx_order;           // compiled reaction index -> description index
  std::vector<double> sp, rxd, eff_am1, dslot_am1, entry_wratio;
  std::vector<int> rxi, eff_sp, dslot_sp, dslot_mask, entry_row, entry_col;
  HostProg prog[kNumGroups];           // prog[g]: programs for lane group g (widths kGroupWidth)
  std::vector<int> jpass;              // [passes * 4]: first reaction, end reaction, first slot, reactions
  int jreg = 0;                        // doubles of the largest pass (dq/dT values + derivative slots)
  std::vector<int> perm, iperm;        // LU position -> state index, and back
  std::vector<int> lu_src, lu_diag, s_out;
  std::vector<int> lu_rowptr, lu_col;  // factor pattern, CSR in LU (permuted) order
  std::vector<int> csr_ptr, csr_col;   // S pattern in natural state order
  long long lu_flops = 0;              // multiply-adds of one factorisation (algorithmic)
};

// Validates and compiles; returns CHEM_OK or an error code with a message in err.
chem_status compile_mechanism(const chem_mech_desc& d, HostMech& hm, std::string& err);

// Tabulated temperature functions (the opt-in approximation of chem_integrate_opts.tabulate): per class
// TC_E exp(g_k), TC_IE exp(-g_k) (species), TC_KF the forward rate coefficient (compiled reaction order;
// the high-pressure limit of a fall-off reaction), TC_FC the Troe centre of the fall-off reactions (the
// first n_troe compiled reactions), a polynomial in tau on each of kTabIntervals equal intervals of
// u = 1/T over [1/kTabThi, 1/kTabTlo]; coefficients of class c at
// coef[c][((j * nfun_c + f) * (deg[c] + 1)) + i] (interval j, function f, power i of tau).
enum : int { TC_E = 0, TC_IE = 1, TC_KF = 2, TC_FC = 3, kTabClasses = 4 };
constexpr int kTabIntervals = 640;
constexpr double kTabTlo = 250.0, kTabThi = 4000.0;
struct HostTables {
  double tol = 0.0;
  double u_lo = 0.0, du = 0.0;
  int deg[kTabClasses] = {0, 0, 0, 0};   // 0: the class stays exact (no degree up to 8 meets tol)
  int nfun[kTabClasses] = {0, 0, 0, 0};
  std::vector<double> coef[kTabClasses];
};
// Builds the tables for relative tolerance tol (0 < tol < 1).
chem_status build_tables(const HostMech& hm, double tol, HostTables& t, std::string& err);

// A mechanism description read from JSON: the arrays, and a chem_mech_desc pointing into them.
struct JsonMech {
  std::vector<double> W, T_mid, nasa_lo, nasa_hi, A, b, Ea, eff_alpha, troe, low;
  std::vector<int> comp, reac_ptr, reac_sp, reac_nu, prod_ptr, prod_sp, prod_nu, rtype, reversible, eff_ptr, eff_sp;
  int n_elements = 0;
  chem_mech_desc desc{};
};
// Parses the JSON form of a description (keys named as the chem_mech_desc fields; two-dimensional
// arrays as nested rows or flat; other keys ignored).  CHEM_EINVAL with a message on malformed text,
// missing keys or inconsistent lengths; the description itself is validated by compile_mechanism.
chem_status parse_mech_json(const char* text, JsonMech& jm, std::string& err);

// Destination rank of every cell of every rank for an even chemistry load (chem_balance_plan).
chem_status balance_plan(int world, const int64_t* counts, const double* costs, int32_t* dest, std::string& err);

}  // namespace chemgb
