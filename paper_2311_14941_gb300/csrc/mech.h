// mech.h -- layout of a compiled mechanism, shared by the host compiler and the device kernels.
//
// All tables live in one device allocation; MechView carries typed pointers into it and is passed to
// kernels by value.  Index fields of the warp programs are 16 bits wide, which bounds reactions,
// derivative slots and factor entries to 65535 (chem_create reports CHEM_EUNSUPPORTED beyond).
#pragma once
#ifdef __CUDACC_RTC__
// run-time compilation (mechanism-specialised kernels) has no C library headers
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <cstdint>
#endif

namespace chemgb {

// Per-cell status codes of the device code (the same values as chem.h's CHEM_CELL_*, checked there).
enum : int { kCellOk = 0, kCellMaxSteps = 1, kCellHmin = 2, kCellNonfinite = 3, kCellBadInput = 4, kCellTimeout = 5 };

constexpr double kRu = 8.314462618;   // J/(mol K)
constexpr double kP0 = 101325.0;      // Pa, standard state of Kc
constexpr int kWarp = 32;
constexpr int kMaxWarpsPerCell = 2;   // a cell is integrated by one warp or by two
// Lane groups that integrate one cell, and the width their warp programs are built for:
//   group 0: one warp (32 lanes), group 1: two warps of a block (64 lanes), group 2: half a warp
//   (16 lanes; two cells share a warp, for mechanisms with few species).
constexpr int kNumGroups = 3;
constexpr int kGroupWidth[kNumGroups] = {32, 64, 16};

// ---- species table: SP_STRIDE doubles per species
//   [0] 1/W  [1] W  [2] T_mid  [3] unused
//   [4 .. 4+RANGE)   low range, [4+RANGE .. 4+2 RANGE) high range, each:
//   a0 a1 a2 a3 a4 | h1..h4 = a1/2 a2/3 a3/4 a4/5 | g1..g4 = -a1/2 -a2/6 -a3/12 -a4/20 | a5 a6 |
//   d2 d3 d4 = 2a2 3a3 4a4
// so cp/R = a0 + T(a1 + T(a2 + T(a3 + T a4))), h/RT = a0 + T(h1 + ...) + a5/T,
// g = h/RT - s/R = a0 (1 - ln T) + T(g1 + T(g2 + T(g3 + T g4))) + a5/T - a6,
// d(cp/R)/dT = a1 + T(d2 + T(d3 + T d4)).
constexpr int SP_RANGE = 18;
constexpr int SP_STRIDE = 4 + 2 * SP_RANGE;

// ---- reaction tables (reactions ordered: Troe, then third-body, then elementary)
// doubles, RX_D per reaction:
//   [0] ln A  [1] b  [2] Ea/Ru  [3] ln A0  [4] b0  [5] Ea0/Ru  [6] 1-alpha  [7] alpha  [8] 1/T3  [9] 1/T1
//   [10] T2 (0: absent)  [11] unused
constexpr int RX_D = 12;
// ints, RX_I per reaction:
//   [0] type (0 elementary, 1 third-body, 2 Troe)  [1] reversible  [2] reactant occurrences (1..3)
//   [3] product occurrences (1..3)  [4..6] reactant species per occurrence (coefficient nu expands into
//   nu occurrences)  [7..9] product occurrences  [10] sum of net coefficients  [11] efficiency offset
//   [12] efficiency count  [13] derivative-slot offset  [14] derivative-slot count  [15] unused
constexpr int RX_I = 16;

// ---- warp programs, compiled for a group of `width` lanes (one warp per cell: 32, two: 64, half: 16)
// Gather ("flattened segmented reduction"): step s, lane l executes op[s*width + l]:
//   acc = fma(value(a, b), acc); if dst != NONE: out[dst] = acc, acc = 0.
// dst >= PARTIAL_BIT selects the partial-sum buffer; a combine list then adds partials into outputs.
struct GatherOp {
  uint16_t a, b, dst, flags;   // flags bit 0: padding (no accumulation)
};
constexpr uint16_t DST_NONE = 0xFFFF;
constexpr uint16_t PARTIAL_BIT = 0x8000;

// Elimination / solve program: step s has one kind; lane l executes op[s*width + l] (t == OP_IDLE: idle).
//   LU:    K_RECIP  dinv[t] = 1 / LU[a]      K_SCALE  LU[t] *= dinv[a]     K_UPDATE LU[t] -= LU[a] * LU[b]
//   solve: K_SCALE  x[t] *= dinv[a]          K_UPDATE x[t] -= LU[a] * x[b]
// Every op of a step, idle ones included, carries the step's kind.
struct ElimOp {
  uint16_t t, a, b, kind;
};
constexpr uint16_t OP_IDLE = 0xFFFF;
enum : int { K_RECIP = 0, K_SCALE = 1, K_UPDATE = 2 };

struct Gather {
  const GatherOp* ops;   // [steps * 32]
  int steps;
  int n_partial;
  const int* comb;       // [n_comb * 3]: dst, first partial, count
  int n_comb;
};

// The Jacobian's reaction loop runs in passes over consecutive reaction ranges so that a pass's
// dq/dT values and derivative slots fit in the region the LU factor occupies during a step.
constexpr int kMaxJPass = 8;
enum : int { JP_RB = 0, JP_RE = 1, JP_SB = 2, JP_CNT = 3 };   // first/end reaction, first slot, reactions

struct MechView {
  int width;                 // lanes of the programs below: the lane group's width (32, 64 or 16)
  int n, R, m;
  int n_troe, n_tb;          // reactions [0, n_troe) Troe, [n_troe, n_troe + n_tb) third-body
  int nY;                    // Y-block entries of S (row-major by species, diagonal included)
  int nnz_S;                 // nY + n (T column) + m (T row)
  int nnz_LU;
  int n_dslot;
  const double* sp;          // [n * SP_STRIDE]
  const double* rxd;         // [R * RX_D]
  const int* rxi;            // [R * RX_I]
  const int* eff_sp;         // listed efficiencies
  const double* eff_am1;     // alpha - 1
  const int* dslot_sp;       // [n_dslot] column species of each derivative slot
  const int* dslot_mask;     // [n_dslot] bits 0..2 reactant occurrences, 3..5 product occurrences equal
  const double* dslot_am1;   // [n_dslot] (efficiency - 1) of the slot species, 0 if not listed
  const int* entry_row;      // [nY] species k of Y-block entry
  const int* entry_col;      // [nY] species j
  const double* entry_wratio;// [nY] W_k / W_j
  Gather g_omega;            // species <- reactions (a = reaction, b = top 16 bits of double(nu))
  int n_jpass;               // Jacobian passes
  int jpass[kMaxJPass][4];   // per pass: JP_RB, JP_RE, JP_SB, JP_CNT
  Gather g_jac[kMaxJPass];   // per pass: S[0 .. nY + n) += nu * region[a] (a < cnt: dq/dT of reaction
                             // rb + a into the T column; a >= cnt: derivative slot sb + a - cnt into the
                             // Y block), b = top 16 bits of double(nu)
  Gather g_row;              // species k <- sum_j Dtil_kj C_j (a = entry, b = species j)
  Gather g_col;              // species i <- sum_k h_k Dtil_ki (a = entry, b = species k)
  const int* lu_src;         // [nnz_LU] S index feeding the slot (-1: fill)
  const int* lu_diag;        // [m] LU slot of the diagonal of state index s (natural order)
  const ElimOp* lu_ops;      // [lu_steps * width]
  int lu_steps;
  const ElimOp* sv_ops;      // forward + backward substitution program, vector indices in state order
  int sv_steps;
  const ElimOp* svT_ops;     // transposed substitution program (A^T x = b)
  int svT_steps;
  const int* rx_order;       // [R] compiled reaction -> description index
  const int* s_out;          // [nnz_S] position of internal S entry in the CSR output order
  // tabulated temperature functions (an opt-in approximation; tab_on == 0: every function exact):
  // class c (0 exp(g_k), 1 exp(-g_k), 2 forward rate coefficient, 3 Troe centre) at interval j, function f
  // has its deg[c] + 1 polynomial coefficients (powers of tau) at tab[c] + (j * nfun_c + f) * (deg[c] + 1)
  int tab_on;
  int tab_deg[4];            // 0: the class stays exact
  const double* tab[4];
  double tab_ulo, tab_du;    // interval j covers u = 1/T in [tab_ulo + j du, tab_ulo + (j + 1) du)
  double tab_tlo, tab_thi;   // tabulated range of T
  int tab_ni;                // intervals
};

// Per-cell shared-memory layout (offsets in doubles).
struct CellLayout {
  int y, ytmp, f0, U1, U2, U3, U4, x, z, u, v;   // m-vectors
  int C, hRT, eg, emg, cpR;                       // n-vectors
  int q;                                          // R-vector
  int S;                                          // nnz_S
  int LU, dinv;                                   // nnz_LU, m
  int D;                                          // Jacobian pass region (aliases LU and dinv)
  int part;                                       // partial sums of the gathers
  int misc;                                       // 16 scalars
  int total;                                      // doubles per cell
};

}  // namespace chemgb
