// compile.cpp -- host mechanism compiler.
//
// The paper's chemistry library gets its speed from three mechanism-level preparations (Sec. 2.5):
// internal sparse management of mechanism quantities, a sparse analytical Jacobian, and (for the stiff
// solver) sparse linear algebra.  Here all of that is decided once, on the host, when a handle is
// created:
//   1. validation and reordering of reactions by type (Troe, third-body, elementary) so that warp lanes
//      working on consecutive reactions take the same branch;
//   2. the static pattern of the sparse Jacobian part S (T row and column, species couplings through
//      shared reactions and listed collision efficiencies);
//   3. a minimum-degree ordering of the species block with T last, the symbolic LU (fill) of
//      I/(h gamma) - S in that order, and DAG-scheduled warp programs for the numeric factorisation and
//      the two triangular solves;
//   4. load-balanced warp "gather" programs for every sparse reduction of the rate and Jacobian
//      evaluation (production rates, Jacobian entries, row and column sums).
#include "compile.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <set>

namespace chemgb {
namespace {

bool fin(double x) { return std::isfinite(x); }

// Gather coefficient nu as the top 16 bits of the IEEE double nu (+-1, +-2, +-3 have 16 trailing zero
// bits in their high word), so that the device rebuilds it with integer instructions only.
int enc_nu(int nu) {
  const double d = (double)nu;
  uint64_t bits;
  std::memcpy(&bits, &d, 8);
  return (int)(bits >> 48);
}

// ------------------------------------------------------------------------ gather programs
// groups[g] = list of (a, b) terms summed into output g.  Terms are dealt to the 32 lanes so that the
// longest lane is as short as possible: a group longer than the per-lane target is split into pieces
// whose partial sums are combined afterwards; pieces go to lanes largest first (LPT).  With skip_empty,
// outputs without terms are left untouched (programs that accumulate into their outputs); otherwise
// they are written with 0.
bool build_gather(const std::vector<std::vector<std::pair<int, int>>>& groups, HostGather& G, std::string& err,
                  int width, bool skip_empty = false) {
  G = HostGather();
  long total = 0;
  for (auto& g : groups) total += skip_empty ? (long)g.size() : (long)std::max<size_t>(g.size(), 1);
  if (groups.empty()) return true;
  const long cap = std::max<long>(1, (total + width - 1) / width);
  struct Piece { int g; int first; int count; int partial; };
  std::vector<Piece> pieces;
  int n_partial = 0;
  for (size_t g = 0; g < groups.size(); ++g) {
    const int L = (int)groups[g].size();
    if (L == 0 && skip_empty) continue;
    if (L <= cap) {
      pieces.push_back({(int)g, 0, L, -1});
    } else {
      const int np = (int)((L + cap - 1) / cap);
      const int per = (L + np - 1) / np;
      G.comb.push_back((int)g);
      G.comb.push_back(n_partial);
      G.comb.push_back(np);
      for (int p = 0; p < np; ++p) {
        int f = p * per, c = std::min(per, L - f);
        pieces.push_back({(int)g, f, c, n_partial++});
      }
    }
  }
  G.n_partial = n_partial;
  if (pieces.empty()) return true;
  std::vector<int> order(pieces.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return std::max(pieces[x].count, 1) > std::max(pieces[y].count, 1); });
  std::vector<std::vector<int>> lane(width);
  std::vector<long> load(width, 0);
  for (int pi : order) {
    int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lane[l].push_back(pi);
    load[l] += std::max(pieces[pi].count, 1);
  }
  G.steps = (int)*std::max_element(load.begin(), load.end());
  G.ops.assign((size_t)G.steps * width, GatherOp{0, 0, DST_NONE, 1});
  for (int l = 0; l < width; ++l) {
    int s = 0;
    for (int pi : lane[l]) {
      const Piece& P = pieces[pi];
      const auto& terms = groups[P.g];
      const int cnt = std::max(P.count, 1);
      for (int t = 0; t < cnt; ++t, ++s) {
        GatherOp op{0, 0, DST_NONE, 1};
        if (P.count > 0) {
          auto ab = terms[P.first + t];
          if (ab.first < 0 || ab.first > 0xFFFF || ab.second < -32768 || ab.second > 0xFFFF) {
            err = "mechanism too large for 16-bit program indices";
            return false;
          }
          op.a = (uint16_t)ab.first;
          op.b = (uint16_t)(ab.second & 0xFFFF);
          op.flags = 0;
        }
        if (t == cnt - 1) {
          int dst = P.partial >= 0 ? (PARTIAL_BIT | P.partial) : P.g;
          if (P.partial < 0 && P.g >= PARTIAL_BIT) { err = "too many gather outputs"; return false; }
          op.dst = (uint16_t)dst;
        }
        G.ops[(size_t)s * width + l] = op;
      }
    }
  }
  return true;
}

// ------------------------------------------------------------------------ DAG list scheduler
struct DagOp {
  int kind;
  int target;      // location written (distinct within a step)
  ElimOp enc;
  std::vector<int> succ;
  int npred = 0;
  int prio = 0;
};

// Steps of one kind, at most 32 ops, distinct targets; ops become ready when all predecessors are done.
// Priority = longest path to the end of the DAG (critical path first).
bool schedule(std::vector<DagOp>& ops, std::vector<ElimOp>& out, std::vector<uint8_t>& kinds, std::string& err,
              int width) {
  const int N = (int)ops.size();
  std::vector<int> indeg(N, 0), topo;
  topo.reserve(N);
  for (auto& o : ops) for (int s : o.succ) indeg[s]++;
  for (int i = 0; i < N; ++i) ops[i].npred = indeg[i];
  std::vector<int> q;
  for (int i = 0; i < N; ++i) if (indeg[i] == 0) q.push_back(i);
  for (size_t h = 0; h < q.size(); ++h) {
    int v = q[h];
    topo.push_back(v);
    for (int s : ops[v].succ) if (--indeg[s] == 0) q.push_back(s);
  }
  if ((int)topo.size() != N) { err = "internal error: cyclic elimination DAG"; return false; }
  for (int i = N - 1; i >= 0; --i) {
    int v = topo[i];
    int best = 0;
    for (int s : ops[v].succ) best = std::max(best, ops[s].prio);
    ops[v].prio = best + 1;
  }
  std::vector<char> done(N, 0);
  std::vector<int> ready;
  for (int i = 0; i < N; ++i) if (ops[i].npred == 0) ready.push_back(i);
  int remaining = N;
  out.clear();
  kinds.clear();
  std::vector<int> newly;
  while (remaining > 0) {
    if (ready.empty()) { err = "internal error: scheduler stalled"; return false; }
    std::stable_sort(ready.begin(), ready.end(), [&](int a, int b) {
      if (ops[a].prio != ops[b].prio) return ops[a].prio > ops[b].prio;
      return a < b;
    });
    const int K = ops[ready[0]].kind;
    std::vector<int> step;
    std::set<int> used;
    std::vector<int> keep;
    for (int v : ready) {
      if ((int)step.size() < width && ops[v].kind == K && !used.count(ops[v].target)) {
        step.push_back(v);
        used.insert(ops[v].target);
      } else {
        keep.push_back(v);
      }
    }
    for (int l = 0; l < width; ++l) {   // every lane's op carries the step's kind
      ElimOp e = l < (int)step.size() ? ops[step[l]].enc : ElimOp{OP_IDLE, 0, 0, 0};
      e.kind = (uint16_t)K;
      out.push_back(e);
    }
    kinds.push_back((uint8_t)K);
    newly.clear();
    for (int v : step) {
      done[v] = 1;
      --remaining;
      for (int s : ops[v].succ) if (--ops[s].npred == 0) newly.push_back(s);
    }
    ready = keep;
    ready.insert(ready.end(), newly.begin(), newly.end());
  }
  return true;
}

// exact minimum-degree ordering on the elimination graph; `last` is eliminated last
std::vector<int> min_degree_order(int m, const std::vector<std::vector<char>>& adj0, int last) {
  std::vector<std::vector<char>> adj = adj0;
  std::vector<char> alive(m, 1);
  std::vector<int> order;
  for (int step = 0; step < m - 1; ++step) {
    int best = -1, bdeg = 1 << 30;
    for (int v = 0; v < m; ++v) {
      if (!alive[v] || v == last) continue;
      int d = 0;
      for (int u = 0; u < m; ++u) d += (alive[u] && adj[v][u]) ? 1 : 0;
      if (d < bdeg) { bdeg = d; best = v; }
    }
    std::vector<int> nb;
    for (int u = 0; u < m; ++u) if (alive[u] && adj[best][u]) nb.push_back(u);
    for (int a : nb)
      for (int b : nb)
        if (a != b) adj[a][b] = 1;
    alive[best] = 0;
    order.push_back(best);
  }
  order.push_back(last);
  return order;
}

}  // namespace

chem_status compile_mechanism(const chem_mech_desc& d, HostMech& hm, std::string& err) {
  hm = HostMech();
  for (int g = 0; g < kNumGroups; ++g) hm.prog[g].width = kGroupWidth[g];
  const int n = d.n_species, R = d.n_reactions;
  if (n < 1 || R < 0) { err = "n_species must be >= 1 and n_reactions >= 0"; return CHEM_EINVAL; }
  if (!d.W || !d.nasa_lo || !d.nasa_hi || !d.T_mid) { err = "species arrays must not be NULL"; return CHEM_EINVAL; }
  if (R > 0 && (!d.reac_ptr || !d.reac_sp || !d.reac_nu || !d.prod_ptr || !d.prod_sp || !d.prod_nu || !d.A || !d.b ||
                !d.Ea || !d.rtype || !d.reversible || !d.eff_ptr || !d.troe || !d.low)) {
    err = "reaction arrays must not be NULL";
    return CHEM_EINVAL;
  }
  for (int k = 0; k < n; ++k) {
    if (!(d.W[k] > 0.0) || !fin(d.W[k])) { err = "molar mass of species " + std::to_string(k) + " must be positive"; return CHEM_EINVAL; }
    if (!(d.T_mid[k] > 0.0) || !fin(d.T_mid[k])) { err = "T_mid of species " + std::to_string(k) + " must be positive"; return CHEM_EINVAL; }
    for (int i = 0; i < 7; ++i)
      if (!fin(d.nasa_lo[7 * k + i]) || !fin(d.nasa_hi[7 * k + i])) { err = "non-finite NASA-7 coefficient"; return CHEM_EINVAL; }
  }
  // ---- reactions: validate and expand
  struct Rx {
    int type, rev;
    std::vector<int> ro, po;      // occurrences
    std::vector<std::pair<int, double>> eff;
    double A, b, Ea, A0, b0, Ea0, alpha, T3, T1, T2;
  };
  std::vector<Rx> rx(R);
  for (int r = 0; r < R; ++r) {
    Rx& x = rx[r];
    x.type = d.rtype[r];
    x.rev = d.reversible[r];
    if (x.type < 0 || x.type > 2) { err = "reaction " + std::to_string(r) + ": type must be 0, 1 or 2"; return CHEM_EINVAL; }
    if (x.rev != 0 && x.rev != 1) { err = "reaction " + std::to_string(r) + ": reversible must be 0 or 1"; return CHEM_EINVAL; }
    for (int side = 0; side < 2; ++side) {
      const int* ptr = side ? d.prod_ptr : d.reac_ptr;
      const int* sp = side ? d.prod_sp : d.reac_sp;
      const int* nu = side ? d.prod_nu : d.reac_nu;
      if (ptr[r + 1] < ptr[r]) { err = "reaction " + std::to_string(r) + ": bad participant pointers"; return CHEM_EINVAL; }
      std::vector<int>& occ = side ? x.po : x.ro;
      std::set<int> seen;
      for (int i = ptr[r]; i < ptr[r + 1]; ++i) {
        if (sp[i] < 0 || sp[i] >= n) { err = "reaction " + std::to_string(r) + ": species index out of range"; return CHEM_EINVAL; }
        if (nu[i] < 1 || nu[i] > 3) { err = "reaction " + std::to_string(r) + ": coefficients must be 1..3"; return CHEM_EINVAL; }
        if (seen.count(sp[i])) { err = "reaction " + std::to_string(r) + ": species listed twice on one side"; return CHEM_EINVAL; }
        seen.insert(sp[i]);
        for (int c = 0; c < nu[i]; ++c) occ.push_back(sp[i]);
      }
      if (occ.empty()) { err = "reaction " + std::to_string(r) + ": empty side"; return CHEM_EINVAL; }
      if (occ.size() > 3) { err = "reaction " + std::to_string(r) + ": order above 3 on one side"; return CHEM_EUNSUPPORTED; }
    }
    x.A = d.A[r]; x.b = d.b[r]; x.Ea = d.Ea[r];
    if (!(x.A > 0.0) || !fin(x.A) || !fin(x.b) || !fin(x.Ea)) { err = "reaction " + std::to_string(r) + ": Arrhenius parameters must be finite with A > 0"; return CHEM_EINVAL; }
    if (x.type != 0) {
      if (d.eff_ptr[r + 1] < d.eff_ptr[r]) { err = "reaction " + std::to_string(r) + ": bad efficiency pointers"; return CHEM_EINVAL; }
      std::set<int> seen;
      for (int i = d.eff_ptr[r]; i < d.eff_ptr[r + 1]; ++i) {
        int s = d.eff_sp[i];
        double a = d.eff_alpha[i];
        if (s < 0 || s >= n || seen.count(s)) { err = "reaction " + std::to_string(r) + ": bad efficiency species"; return CHEM_EINVAL; }
        if (!(a >= 0.0) || !fin(a)) { err = "reaction " + std::to_string(r) + ": efficiency must be finite and >= 0"; return CHEM_EINVAL; }
        seen.insert(s);
        if (a != 1.0) x.eff.push_back({s, a});
      }
    }
    x.A0 = x.b0 = x.Ea0 = x.alpha = x.T3 = x.T1 = x.T2 = 0.0;
    if (x.type == 2) {
      x.alpha = d.troe[4 * r]; x.T3 = d.troe[4 * r + 1]; x.T1 = d.troe[4 * r + 2]; x.T2 = d.troe[4 * r + 3];
      x.A0 = d.low[3 * r]; x.b0 = d.low[3 * r + 1]; x.Ea0 = d.low[3 * r + 2];
      if (!fin(x.alpha) || !(x.T3 > 0.0) || !(x.T1 > 0.0) || !fin(x.T2) || !(x.A0 > 0.0) || !fin(x.A0) || !fin(x.b0) || !fin(x.Ea0)) {
        err = "reaction " + std::to_string(r) + ": invalid Troe parameters";
        return CHEM_EINVAL;
      }
    }
    if (d.comp && d.n_elements > 0) {
      for (int e = 0; e < d.n_elements; ++e) {
        long bal = 0;
        for (int s : x.ro) bal -= d.comp[s * d.n_elements + e];
        for (int s : x.po) bal += d.comp[s * d.n_elements + e];
        if (bal != 0) { err = "reaction " + std::to_string(r) + " is not element balanced"; return CHEM_EINVAL; }
      }
    }
  }
  // ---- reorder: Troe, third-body, elementary (stable)
  hm.n = n; hm.R = R; hm.m = n + 1;
  const int m = n + 1;
  for (int t : {2, 1, 0})
    for (int r = 0; r < R; ++r) if (rx[r].type == t) hm.rx_order.push_back(r);
  for (int r = 0; r < R; ++r) { if (rx[r].type == 2) hm.n_troe++; if (rx[r].type == 1) hm.n_tb++; }

  // ---- species table
  hm.sp.assign((size_t)n * SP_STRIDE, 0.0);
  for (int k = 0; k < n; ++k) {
    double* s = &hm.sp[(size_t)k * SP_STRIDE];
    s[0] = 1.0 / d.W[k]; s[1] = d.W[k]; s[2] = d.T_mid[k];
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = rg ? &d.nasa_hi[7 * k] : &d.nasa_lo[7 * k];
      double* c = s + 4 + rg * SP_RANGE;
      for (int i = 0; i < 5; ++i) c[i] = a[i];
      c[5] = a[1] / 2.0; c[6] = a[2] / 3.0; c[7] = a[3] / 4.0; c[8] = a[4] / 5.0;
      c[9] = -a[1] / 2.0; c[10] = -a[2] / 6.0; c[11] = -a[3] / 12.0; c[12] = -a[4] / 20.0;
      c[13] = a[5]; c[14] = a[6];
      c[15] = 2.0 * a[2]; c[16] = 3.0 * a[3]; c[17] = 4.0 * a[4];
    }
  }
  // ---- reaction tables, derivative slots
  hm.rxd.assign((size_t)R * RX_D, 0.0);
  hm.rxi.assign((size_t)R * RX_I, -1);
  std::vector<std::vector<int>> net(R, std::vector<int>());   // per compiled reaction: (species, nu) pairs
  std::vector<std::map<int, int>> netmap(R);
  std::vector<std::vector<int>> slots_sp(R);
  for (int r = 0; r < R; ++r) {
    const Rx& x = rx[hm.rx_order[r]];
    double* D = &hm.rxd[(size_t)r * RX_D];
    D[0] = std::log(x.A); D[1] = x.b; D[2] = x.Ea / kRu;
    if (x.type == 2) {
      D[3] = std::log(x.A0); D[4] = x.b0; D[5] = x.Ea0 / kRu;
      D[6] = 1.0 - x.alpha; D[7] = x.alpha; D[8] = 1.0 / x.T3; D[9] = 1.0 / x.T1; D[10] = x.T2 > 0.0 ? x.T2 : 0.0;
    }
    int* I = &hm.rxi[(size_t)r * RX_I];
    I[0] = x.type; I[1] = x.rev; I[2] = (int)x.ro.size(); I[3] = (int)x.po.size();
    for (size_t i = 0; i < x.ro.size(); ++i) I[4 + i] = x.ro[i];
    for (size_t i = 0; i < x.po.size(); ++i) I[7 + i] = x.po[i];
    I[10] = (int)x.po.size() - (int)x.ro.size();
    I[11] = (int)hm.eff_sp.size();
    I[12] = (int)x.eff.size();
    for (auto& e : x.eff) { hm.eff_sp.push_back(e.first); hm.eff_am1.push_back(e.second - 1.0); }
    for (int s : x.ro) netmap[r][s] -= 1;
    for (int s : x.po) netmap[r][s] += 1;
    // distinct column species: reactants, products, listed colliders
    std::vector<int> cols;
    auto addc = [&](int s) { if (std::find(cols.begin(), cols.end(), s) == cols.end()) cols.push_back(s); };
    for (int s : x.ro) addc(s);
    for (int s : x.po) addc(s);
    if (x.type != 0) for (auto& e : x.eff) addc(e.first);
    I[13] = hm.n_dslot;
    I[14] = (int)cols.size();
    for (int s : cols) {
      int mask = 0;
      for (size_t i = 0; i < x.ro.size(); ++i) if (x.ro[i] == s) mask |= 1 << i;
      for (size_t i = 0; i < x.po.size(); ++i) if (x.po[i] == s) mask |= 1 << (3 + i);
      double am1 = 0.0;
      if (x.type != 0) for (auto& e : x.eff) if (e.first == s) am1 = e.second - 1.0;
      hm.dslot_sp.push_back(s);
      hm.dslot_mask.push_back(mask);
      hm.dslot_am1.push_back(am1);
      hm.n_dslot++;
    }
    slots_sp[r] = cols;
  }
  if (R > 0xFFFF || hm.n_dslot > 0xFFFF) { err = "mechanism too large for 16-bit program indices"; return CHEM_EUNSUPPORTED; }

  // ---- S pattern, Y block (species k row, species j column)
  std::vector<std::vector<char>> Yp(n, std::vector<char>(n, 0));
  for (int k = 0; k < n; ++k) Yp[k][k] = 1;
  for (int r = 0; r < R; ++r)
    for (auto& kv : netmap[r]) {
      if (kv.second == 0) continue;
      for (int j : slots_sp[r]) Yp[kv.first][j] = 1;
    }
  std::vector<std::vector<int>> eidx(n, std::vector<int>(n, -1));
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      if (Yp[k][j]) {
        eidx[k][j] = hm.nY++;
        hm.entry_row.push_back(k);
        hm.entry_col.push_back(j);
        hm.entry_wratio.push_back(d.W[k] / d.W[j]);
      }
  hm.nnz_S = hm.nY + n + m;
  if (hm.nnz_S > 0xFFFF) { err = "Jacobian pattern too large for 16-bit program indices"; return CHEM_EUNSUPPORTED; }
  // state-index pattern: s_index(row, col) -> internal S index
  auto s_index = [&](int row, int col) -> int {
    if (row == 0) return hm.nY + n + col;          // T row (col 0 = TT)
    if (col == 0) return hm.nY + (row - 1);        // T column
    return eidx[row - 1][col - 1];
  };
  // natural CSR order for output
  hm.csr_ptr.assign(m + 1, 0);
  hm.s_out.assign(hm.nnz_S, -1);
  {
    int pos = 0;
    for (int row = 0; row < m; ++row) {
      hm.csr_ptr[row] = pos;
      for (int col = 0; col < m; ++col) {
        int e = (row == 0 || col == 0) ? s_index(row, col) : eidx[row - 1][col - 1];
        if (e < 0) continue;
        hm.csr_col.push_back(col);
        hm.s_out[e] = pos++;
      }
    }
    hm.csr_ptr[m] = pos;
    if (pos != hm.nnz_S) { err = "internal error: pattern size mismatch"; return CHEM_EINVAL; }
  }

  // ---- gather programs
  {
    std::vector<std::vector<std::pair<int, int>>> gw(n), gr(n), gc(n);
    for (int r = 0; r < R; ++r)
      for (auto& kv : netmap[r])
        if (kv.second != 0) gw[kv.first].push_back({r, enc_nu(kv.second)});
    for (int e = 0; e < hm.nY; ++e) {
      gr[hm.entry_row[e]].push_back({e, hm.entry_col[e]});
      gc[hm.entry_col[e]].push_back({e, hm.entry_row[e]});
    }
    for (HostProg& P : hm.prog)
      if (!build_gather(gw, P.g_omega, err, P.width) || !build_gather(gr, P.g_row, err, P.width) ||
          !build_gather(gc, P.g_col, err, P.width))
        return CHEM_EUNSUPPORTED;
  }

  // ---- ordering (minimum degree, T last) and symbolic LU
  std::vector<std::vector<char>> full(m, std::vector<char>(m, 0));
  for (int row = 0; row < m; ++row)
    for (int col = 0; col < m; ++col) {
      bool in = (row == 0 || col == 0) ? true : Yp[row - 1][col - 1];
      full[row][col] = in;
    }
  std::vector<std::vector<char>> sym(m, std::vector<char>(m, 0));
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b)
      if (a != b && (full[a][b] || full[b][a])) sym[a][b] = 1;
  hm.perm = min_degree_order(m, sym, 0);
  hm.iperm.assign(m, 0);
  for (int p = 0; p < m; ++p) hm.iperm[hm.perm[p]] = p;
  std::vector<std::vector<char>> F(m, std::vector<char>(m, 0));
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q) F[p][q] = full[hm.perm[p]][hm.perm[q]];
  for (int p = 0; p < m; ++p) F[p][p] = 1;
  for (int k = 0; k < m; ++k)
    for (int i = k + 1; i < m; ++i) {
      if (!F[i][k]) continue;
      for (int j = k + 1; j < m; ++j) if (F[k][j]) F[i][j] = 1;
    }
  std::vector<std::vector<int>> slot(m, std::vector<int>(m, -1));
  hm.lu_rowptr.assign(m + 1, 0);
  for (int p = 0; p < m; ++p) {
    hm.lu_rowptr[p] = hm.nnz_LU;
    for (int q = 0; q < m; ++q)
      if (F[p][q]) { slot[p][q] = hm.nnz_LU++; hm.lu_col.push_back(q); }
  }
  hm.lu_rowptr[m] = hm.nnz_LU;
  if (hm.nnz_LU > 0xFFFE) { err = "factor too large for 16-bit program indices"; return CHEM_EUNSUPPORTED; }
  hm.lu_src.assign(hm.nnz_LU, -1);
  for (int p = 0; p < m; ++p)
    for (int q = 0; q < m; ++q)
      if (slot[p][q] >= 0 && full[hm.perm[p]][hm.perm[q]]) hm.lu_src[slot[p][q]] = s_index(hm.perm[p], hm.perm[q]);
  hm.lu_diag.assign(m, 0);
  for (int s = 0; s < m; ++s) hm.lu_diag[s] = slot[hm.iperm[s]][hm.iperm[s]];

  // ---- elimination program
  {
    std::vector<DagOp> ops;
    std::vector<std::vector<int>> upd_to(hm.nnz_LU);   // UPDATE ops writing each slot
    std::vector<int> recip(m), scale_of(hm.nnz_LU, -1);
    for (int k = 0; k < m; ++k) {
      recip[k] = (int)ops.size();
      ops.push_back(DagOp{K_RECIP, 1 << 20 | k, ElimOp{(uint16_t)k, (uint16_t)slot[k][k], 0, 0}, {}});
      for (int i = k + 1; i < m; ++i) {
        if (slot[i][k] < 0) continue;
        scale_of[slot[i][k]] = (int)ops.size();
        ops.push_back(DagOp{K_SCALE, slot[i][k], ElimOp{(uint16_t)slot[i][k], (uint16_t)k, 0, 0}, {}});
      }
      for (int i = k + 1; i < m; ++i) {
        if (slot[i][k] < 0) continue;
        for (int j = k + 1; j < m; ++j) {
          if (slot[k][j] < 0) continue;
          int t = slot[i][j];
          upd_to[t].push_back((int)ops.size());
          ops.push_back(DagOp{K_UPDATE, t, ElimOp{(uint16_t)t, (uint16_t)slot[i][k], (uint16_t)slot[k][j], 0}, {}});
          hm.lu_flops += 1;
        }
      }
    }
    // edges
    for (int k = 0; k < m; ++k) {
      for (int u : upd_to[slot[k][k]]) ops[u].succ.push_back(recip[k]);
      for (int i = k + 1; i < m; ++i) {
        if (slot[i][k] < 0) continue;
        int sc = scale_of[slot[i][k]];
        ops[recip[k]].succ.push_back(sc);
        for (int u : upd_to[slot[i][k]]) ops[u].succ.push_back(sc);
      }
    }
    for (size_t v = 0; v < ops.size(); ++v) {
      if (ops[v].kind != K_UPDATE) continue;
      int a = ops[v].enc.a, b = ops[v].enc.b;
      ops[scale_of[a]].succ.push_back((int)v);
      for (int u : upd_to[b]) ops[u].succ.push_back((int)v);
    }
    for (HostProg& P : hm.prog) {
      std::vector<DagOp> work = ops;
      if (!schedule(work, P.lu_ops, P.lu_kind, err, P.width)) return CHEM_EINVAL;
    }
  }
  // ---- substitution program (forward with unit L, backward with U and 1/diag), state-order indices
  {
    std::vector<DagOp> ops;
    std::vector<std::vector<int>> fw_w(m), fw_r(m), bw_w(m);
    std::vector<int> sc(m);
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < p; ++q)
        if (slot[p][q] >= 0) {
          int id = (int)ops.size();
          ops.push_back(DagOp{K_UPDATE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)slot[p][q], (uint16_t)hm.perm[q], 0}, {}});
          fw_w[p].push_back(id);
          fw_r[q].push_back(id);
        }
    for (int p = 0; p < m; ++p) {
      sc[p] = (int)ops.size();
      ops.push_back(DagOp{K_SCALE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)p, 0, 0}, {}});
    }
    std::vector<std::pair<int, int>> bw;   // (op id, q)
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q)
        if (slot[p][q] >= 0) {
          int id = (int)ops.size();
          ops.push_back(DagOp{K_UPDATE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)slot[p][q], (uint16_t)hm.perm[q], 0}, {}});
          bw_w[p].push_back(id);
          bw.push_back({id, q});
        }
    for (int p = 0; p < m; ++p) {
      for (int w : fw_w[p]) for (int r : fw_r[p]) ops[w].succ.push_back(r);     // RAW forward
      for (int w : fw_w[p]) ops[w].succ.push_back(sc[p]);
      for (int r : fw_r[p]) ops[r].succ.push_back(sc[p]);                       // WAR before scaling
      for (int w : bw_w[p]) {
        for (int f : fw_w[p]) ops[f].succ.push_back(w);                         // backward after forward
        for (int r : fw_r[p]) ops[r].succ.push_back(w);                         // WAR
        ops[w].succ.push_back(sc[p]);
      }
    }
    for (auto& pr : bw) ops[sc[pr.second]].succ.push_back(pr.first);           // RAW backward
    for (HostProg& P : hm.prog) {
      std::vector<DagOp> work = ops;
      if (!schedule(work, P.sv_ops, P.sv_kind, err, P.width)) return CHEM_EINVAL;
    }
  }
  // ---- transposed substitution (A^T x = b): forward with U^T (scaled by 1/diag), then backward with
  //      the unit L^T.  In factor positions: x_p -= U_qp x_q (q < p), x_p *= 1/U_pp; then x_p -= L_qp x_q
  //      (q > p).  Same op encoding, state-order vector indices.
  {
    std::vector<DagOp> ops;
    std::vector<std::vector<int>> f_w(m), f_r(m), b_w(m);
    std::vector<int> sc(m);
    for (int p = 0; p < m; ++p) {
      sc[p] = (int)ops.size();
      ops.push_back(DagOp{K_SCALE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)p, 0, 0}, {}});
    }
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < p; ++q)
        if (slot[q][p] >= 0) {   // U entry (q, p)
          int id = (int)ops.size();
          ops.push_back(DagOp{K_UPDATE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)slot[q][p], (uint16_t)hm.perm[q], 0}, {}});
          f_w[p].push_back(id);
          f_r[q].push_back(id);
          ops[sc[q]].succ.push_back(id);    // reads x_q after its scaling
          ops[id].succ.push_back(sc[p]);    // x_p scaled after all its updates
        }
    std::vector<std::pair<int, int>> bl;    // (op id, q)
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q)
        if (slot[q][p] >= 0) {   // L entry (q, p)
          int id = (int)ops.size();
          ops.push_back(DagOp{K_UPDATE, hm.perm[p], ElimOp{(uint16_t)hm.perm[p], (uint16_t)slot[q][p], (uint16_t)hm.perm[q], 0}, {}});
          b_w[p].push_back(id);
          bl.push_back({id, q});
          ops[sc[p]].succ.push_back(id);                       // backward phase after x_p's forward value
          for (int r : f_r[p]) ops[r].succ.push_back(id);      // WAR: forward readers of x_p first
        }
    for (auto& pr : bl) {
      const int q = pr.second;
      ops[sc[q]].succ.push_back(pr.first);                     // x_q forward-final
      for (int w : b_w[q]) ops[w].succ.push_back(pr.first);    // x_q backward-final
    }
    for (HostProg& P : hm.prog) {
      std::vector<DagOp> work = ops;
      if (!schedule(work, P.svT_ops, P.svT_kind, err, P.width)) return CHEM_EINVAL;
    }
  }

  // ---- Jacobian passes.  A reaction leaves one dq/dT value and one derivative slot per column species;
  // they are consumed by the pass's gather right after the pass.  Reactions are cut into P consecutive
  // ranges of about equal size, P the smallest count whose largest range fits the region the factor
  // and 1/diag take during a step (nnz_LU + m doubles), so the Jacobian needs no storage of its own.
  {
    std::vector<int> cost(R);
    long total = 0;
    for (int r = 0; r < R; ++r) { cost[r] = 1 + hm.rxi[(size_t)r * RX_I + 14]; total += cost[r]; }
    const long cap = hm.nnz_LU + m;
    std::vector<int> cut;   // first reaction of each pass, then R
    for (int P = std::max<long>(1, (total + cap - 1) / cap); ; ++P) {
      cut.assign(1, 0);
      long acc = 0, biggest = 0, cur = 0;
      for (int r = 0; r < R; ++r) {
        if (cur > 0 && (acc + cost[r]) * P > total * (long)cut.size() && (int)cut.size() < P) {
          cut.push_back(r);
          biggest = std::max(biggest, cur);
          cur = 0;
        }
        acc += cost[r];
        cur += cost[r];
      }
      biggest = std::max(biggest, cur);
      cut.push_back(R);
      hm.jreg = (int)std::max<long>(biggest, 1);
      if (biggest <= cap || P >= kMaxJPass || P >= R) break;
    }
    const int P = (int)cut.size() - 1;
    hm.jpass.clear();
    for (HostProg& Pg : hm.prog) Pg.g_jac.assign(P, HostGather());
    for (int p = 0; p < P; ++p) {
      const int rb = cut[p], re = cut[p + 1];
      const int sb = R > 0 && rb < R ? hm.rxi[(size_t)rb * RX_I + 13] : hm.n_dslot;
      const int cnt = re - rb;
      hm.jpass.insert(hm.jpass.end(), {rb, re, sb, cnt});
      std::vector<std::vector<std::pair<int, int>>> gj(hm.nY + n);
      for (int r = rb; r < re; ++r) {
        const int base = hm.rxi[(size_t)r * RX_I + 13];
        for (auto& kv : netmap[r]) {
          if (kv.second == 0) continue;
          const int nu = enc_nu(kv.second);
          gj[hm.nY + kv.first].push_back({r - rb, nu});
          for (size_t c = 0; c < slots_sp[r].size(); ++c)
            gj[eidx[kv.first][slots_sp[r][c]]].push_back({cnt + base + (int)c - sb, nu});
        }
      }
      for (HostProg& Pg : hm.prog)
        if (!build_gather(gj, Pg.g_jac[p], err, Pg.width, true)) return CHEM_EUNSUPPORTED;
    }
  }
  return CHEM_OK;
}

}  // namespace chemgb

// ------------------------------------------------------------------------ tabulated temperature functions
// Sec. 2.5 credits part of SpeedCHEM's speed to interpolating costly thermodynamic functions with
// polynomials of optimal degree.  Here the temperature functions that cost exponentials per evaluation are
// tabulated: exp(+-g_k) of every species (the factors of the equilibrium constants), every forward rate
// coefficient and every Troe centre.  Each is, on each of kTabIntervals equal intervals of u = 1/T, the
// polynomial through the Chebyshev points of the interval; one degree per class, the smallest in 1..8
// whose polynomials are within tol (relative) of the function at 17 equispaced points of every interval.
namespace chemgb {
namespace {

constexpr int kTabMaxDeg = 8;

// The function itself (double arithmetic, the same formulas as the exact device path).
double tab_function(const HostMech& hm, int cls, int f, double T) {
  const double lnT = std::log(T), invT = 1.0 / T;
  if (cls == TC_E || cls == TC_IE) {
    const double* s = &hm.sp[(size_t)f * SP_STRIDE];
    const double* c = s + 4 + (T < s[2] ? 0 : SP_RANGE);
    const double g = c[0] * (1.0 - lnT) + T * (c[9] + T * (c[10] + T * (c[11] + T * c[12]))) + c[13] * invT - c[14];
    return std::exp(cls == TC_E ? g : -g);
  }
  const double* D = &hm.rxd[(size_t)f * RX_D];
  if (cls == TC_KF) return std::exp(D[0] + D[1] * lnT - D[2] * invT);
  return D[6] * std::exp(-T * D[8]) + D[7] * std::exp(-T * D[9]) + (D[10] > 0.0 ? std::exp(-D[10] * invT) : 0.0);
}

// mono[d][k][i]: coefficient of tau^i in the Chebyshev polynomial T_k, for every degree bound d <= 8.
struct ChebToMono {
  double c[kTabMaxDeg + 1][kTabMaxDeg + 1];
  ChebToMono() {
    for (auto& row : c) for (double& x : row) x = 0.0;
    c[0][0] = 1.0;
    c[1][1] = 1.0;
    for (int k = 2; k <= kTabMaxDeg; ++k)
      for (int i = 0; i <= k; ++i) c[k][i] = (i > 0 ? 2.0 * c[k - 1][i - 1] : 0.0) - c[k - 2][i];
  }
};

}  // namespace

chem_status build_tables(const HostMech& hm, double tol, HostTables& t, std::string& err) {
  if (!(tol > 0.0 && tol < 1.0)) { err = "tab_tol must lie in (0, 1)"; return CHEM_EINVAL; }
  static const ChebToMono cm;
  const double kPi = 3.14159265358979323846;
  t = HostTables();
  t.tol = tol;
  t.u_lo = 1.0 / kTabThi;
  t.du = (1.0 / kTabTlo - 1.0 / kTabThi) / kTabIntervals;
  const int nf[kTabClasses] = {hm.n, hm.n, hm.R, hm.n_troe};
  for (int cls = 0; cls < kTabClasses; ++cls) {
    t.nfun[cls] = nf[cls];
    if (nf[cls] == 0) continue;
    for (int d = 1; d <= kTabMaxDeg && t.deg[cls] == 0; ++d) {
      std::vector<double> out((size_t)kTabIntervals * nf[cls] * (d + 1));
      double node[kTabMaxDeg + 1], val[kTabMaxDeg + 1], ch[kTabMaxDeg + 1];
      for (int i = 0; i <= d; ++i) node[i] = std::cos(kPi * (2 * i + 1) / (2.0 * (d + 1)));
      bool ok = true;
      for (int j = 0; j < kTabIntervals && ok; ++j) {
        const double u0 = t.u_lo + j * t.du;
        for (int f = 0; f < nf[cls] && ok; ++f) {
          for (int i = 0; i <= d; ++i) val[i] = tab_function(hm, cls, f, 1.0 / (u0 + 0.5 * (node[i] + 1.0) * t.du));
          // Chebyshev coefficients by discrete orthogonality at the nodes (T_k(node_i) = cos(k theta_i))
          for (int k = 0; k <= d; ++k) {
            double acc = 0.0;
            for (int i = 0; i <= d; ++i) acc += val[i] * std::cos(k * kPi * (2 * i + 1) / (2.0 * (d + 1)));
            ch[k] = acc * (k == 0 ? 1.0 : 2.0) / (d + 1);
          }
          double* mono = &out[((size_t)j * nf[cls] + f) * (d + 1)];
          for (int i = 0; i <= d; ++i) {
            double acc = 0.0;
            for (int k = i; k <= d; ++k) acc += ch[k] * cm.c[k][i];
            mono[i] = acc;
          }
          for (int q = 0; q <= 16 && ok; ++q) {
            const double tau = -1.0 + q / 8.0;
            double v = mono[d];
            for (int i = d - 1; i >= 0; --i) v = v * tau + mono[i];
            const double ex = tab_function(hm, cls, f, 1.0 / (u0 + 0.5 * (tau + 1.0) * t.du));
            ok = std::fabs(v - ex) <= tol * std::fabs(ex);
          }
        }
      }
      if (ok) {
        t.deg[cls] = d;
        t.coef[cls].swap(out);
      }
    }
  }
  return CHEM_OK;
}

}  // namespace chemgb

// ------------------------------------------------------------------------ mechanism description in JSON
namespace chemgb {
namespace {

struct JVal {
  enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
  double num = 0.0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
};

struct JParser {
  const char* p;
  const char* end;
  std::string err;
  int depth = 0;
  void ws() { while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p; }
  bool fail(const std::string& m) { if (err.empty()) err = m; return false; }
  bool lit(const char* s) {
    const size_t n = std::strlen(s);
    if ((size_t)(end - p) < n || std::strncmp(p, s, n) != 0) return false;
    p += n;
    return true;
  }
  bool string(std::string& out) {
    if (p >= end || *p != '"') return fail("string expected");
    ++p;
    while (p < end && *p != '"') {
      if (*p == '\\') {
        if (++p >= end) return fail("unterminated escape");
        const char c = *p++;
        switch (c) {
          case 'n': out += '\n'; break;
          case 't': out += '\t'; break;
          case 'r': out += '\r'; break;
          case 'b': out += '\b'; break;
          case 'f': out += '\f'; break;
          case 'u': if (end - p < 4) return fail("bad \\u escape"); p += 4; out += '?'; break;
          default: out += c;
        }
      } else {
        out += *p++;
      }
    }
    if (p >= end) return fail("unterminated string");
    ++p;
    return true;
  }
  bool value(JVal& v) {
    if (++depth > 64) return fail("nesting too deep");
    ws();
    if (p >= end) return fail("unexpected end of text");
    bool ok = true;
    if (*p == '{') {
      v.kind = JVal::OBJ;
      ++p; ws();
      if (p < end && *p == '}') { ++p; }
      else {
        while (ok) {
          ws();
          std::string key;
          if (!string(key)) return false;
          ws();
          if (p >= end || *p != ':') return fail("':' expected");
          ++p;
          v.obj.emplace_back(key, JVal());
          if (!value(v.obj.back().second)) return false;
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == '}') { ++p; break; }
          return fail("',' or '}' expected");
        }
      }
    } else if (*p == '[') {
      v.kind = JVal::ARR;
      ++p; ws();
      if (p < end && *p == ']') { ++p; }
      else {
        while (true) {
          v.arr.emplace_back();
          if (!value(v.arr.back())) return false;
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == ']') { ++p; break; }
          return fail("',' or ']' expected");
        }
      }
    } else if (*p == '"') {
      v.kind = JVal::STR;
      ok = string(v.str);
    } else if (lit("true")) { v.kind = JVal::BOOL; v.num = 1.0; }
    else if (lit("false")) { v.kind = JVal::BOOL; v.num = 0.0; }
    else if (lit("null")) { v.kind = JVal::NUL; }
    else {
      char* q = nullptr;
      const std::string tok(p, std::min<size_t>(64, (size_t)(end - p)));
      const double d = std::strtod(tok.c_str(), &q);
      if (q == tok.c_str()) return fail("value expected");
      p += (q - tok.c_str());
      v.kind = JVal::NUM;
      v.num = d;
    }
    --depth;
    return ok;
  }
};

const JVal* jfind(const JVal& o, const char* key) {
  for (auto& kv : o.obj)
    if (kv.first == key) return &kv.second;
  return nullptr;
}

// Flattens a (possibly nested) numeric array; inner = length of the innermost rows (1 for a flat one).
bool jflat(const JVal& v, std::vector<double>& out, int& inner, std::string& err, const char* key) {
  inner = 1;
  if (v.kind != JVal::ARR) { err = std::string("\"") + key + "\" must be an array"; return false; }
  for (auto& e : v.arr) {
    if (e.kind == JVal::NUM || e.kind == JVal::BOOL) { out.push_back(e.num); continue; }
    if (e.kind == JVal::ARR) {
      if (out.empty() && inner == 1) inner = (int)e.arr.size();
      if ((int)e.arr.size() != inner) { err = std::string("rows of \"") + key + "\" differ in length"; return false; }
      for (auto& x : e.arr) {
        if (x.kind != JVal::NUM) { err = std::string("\"") + key + "\" must hold numbers"; return false; }
        out.push_back(x.num);
      }
      continue;
    }
    err = std::string("\"") + key + "\" must hold numbers";
    return false;
  }
  return true;
}

}  // namespace

chem_status parse_mech_json(const char* text, JsonMech& jm, std::string& err) {
  if (!text) { err = "json_text must not be NULL"; return CHEM_EINVAL; }
  JParser P{text, text + std::strlen(text), {}};
  JVal root;
  if (!P.value(root)) { err = "JSON: " + P.err; return CHEM_EINVAL; }
  P.ws();
  if (P.p != P.end) { err = "JSON: text after the top-level value"; return CHEM_EINVAL; }
  if (root.kind != JVal::OBJ) { err = "JSON: the description must be an object"; return CHEM_EINVAL; }
  auto getd = [&](const char* key, std::vector<double>& out, int& inner, bool required) -> bool {
    const JVal* v = jfind(root, key);
    if (!v || v->kind == JVal::NUL) {
      if (required) err = std::string("JSON: missing \"") + key + "\"";
      return !required;
    }
    return jflat(*v, out, inner, err, key);
  };
  auto geti = [&](const char* key, std::vector<int>& out, int& inner, bool required) -> bool {
    std::vector<double> tmp;
    if (!getd(key, tmp, inner, required)) return false;
    for (double x : tmp) {
      if (x != std::floor(x) || std::fabs(x) > 2147483647.0) { err = std::string("JSON: \"") + key + "\" must hold integers"; return false; }
      out.push_back((int)x);
    }
    return true;
  };
  int in = 1;
  if (!getd("W", jm.W, in, true) || !getd("T_mid", jm.T_mid, in, true) ||
      !getd("nasa_lo", jm.nasa_lo, in, true) || !getd("nasa_hi", jm.nasa_hi, in, true) ||
      !geti("reac_ptr", jm.reac_ptr, in, true) || !geti("reac_sp", jm.reac_sp, in, true) ||
      !geti("reac_nu", jm.reac_nu, in, true) || !geti("prod_ptr", jm.prod_ptr, in, true) ||
      !geti("prod_sp", jm.prod_sp, in, true) || !geti("prod_nu", jm.prod_nu, in, true) ||
      !getd("A", jm.A, in, true) || !getd("b", jm.b, in, true) || !getd("Ea", jm.Ea, in, true) ||
      !geti("rtype", jm.rtype, in, true) || !geti("reversible", jm.reversible, in, true) ||
      !geti("eff_ptr", jm.eff_ptr, in, true) || !geti("eff_sp", jm.eff_sp, in, true) ||
      !getd("eff_alpha", jm.eff_alpha, in, true) || !getd("troe", jm.troe, in, true) ||
      !getd("low", jm.low, in, true))
    return CHEM_EINVAL;
  int comp_inner = 0;
  if (!geti("comp", jm.comp, comp_inner, false)) return CHEM_EINVAL;
  const int n = (int)jm.W.size(), R = (int)jm.A.size();
  if (n < 1) { err = "JSON: \"W\" must list at least one species"; return CHEM_EINVAL; }
  auto need = [&](size_t have, size_t want, const char* key) {
    if (have == want) return true;
    err = std::string("JSON: \"") + key + "\" has " + std::to_string(have) + " values, expected " + std::to_string(want);
    return false;
  };
  if (!need(jm.T_mid.size(), n, "T_mid") || !need(jm.nasa_lo.size(), 7 * (size_t)n, "nasa_lo") ||
      !need(jm.nasa_hi.size(), 7 * (size_t)n, "nasa_hi") || !need(jm.b.size(), R, "b") ||
      !need(jm.Ea.size(), R, "Ea") || !need(jm.rtype.size(), R, "rtype") ||
      !need(jm.reversible.size(), R, "reversible") || !need(jm.reac_ptr.size(), R + 1, "reac_ptr") ||
      !need(jm.prod_ptr.size(), R + 1, "prod_ptr") || !need(jm.eff_ptr.size(), R + 1, "eff_ptr") ||
      !need(jm.troe.size(), 4 * (size_t)R, "troe") || !need(jm.low.size(), 3 * (size_t)R, "low") ||
      !need(jm.eff_alpha.size(), jm.eff_sp.size(), "eff_alpha"))
    return CHEM_EINVAL;
  jm.n_elements = 0;
  if (!jm.comp.empty()) {
    if (comp_inner < 1 || jm.comp.size() != (size_t)n * comp_inner) {
      err = "JSON: \"comp\" must be an n_species x n_elements array";
      return CHEM_EINVAL;
    }
    jm.n_elements = comp_inner;
  }
  chem_mech_desc& d = jm.desc;
  d.n_species = n; d.n_reactions = R; d.n_elements = jm.n_elements;
  d.W = jm.W.data(); d.nasa_lo = jm.nasa_lo.data(); d.nasa_hi = jm.nasa_hi.data(); d.T_mid = jm.T_mid.data();
  d.comp = jm.comp.empty() ? nullptr : jm.comp.data();
  d.reac_ptr = jm.reac_ptr.data(); d.reac_sp = jm.reac_sp.data(); d.reac_nu = jm.reac_nu.data();
  d.prod_ptr = jm.prod_ptr.data(); d.prod_sp = jm.prod_sp.data(); d.prod_nu = jm.prod_nu.data();
  d.A = jm.A.data(); d.b = jm.b.data(); d.Ea = jm.Ea.data(); d.rtype = jm.rtype.data();
  d.reversible = jm.reversible.data(); d.eff_ptr = jm.eff_ptr.data(); d.eff_sp = jm.eff_sp.data();
  d.eff_alpha = jm.eff_alpha.data(); d.troe = jm.troe.data(); d.low = jm.low.data();
  return CHEM_OK;
}

}  // namespace chemgb
