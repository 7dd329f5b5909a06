/*
 * chem.h -- C ABI of the GB300 stiff-chemistry library.
 *
 * The method (Yang et al., "Development of a Chemistry Dynamic Load Balancing Solver with Sparse
 * Analytical Jacobian Approach ...", Sec. 1 and Sec. 2.5): every CFD cell is an independent homogeneous
 * gas-phase reactor whose species equations are advanced over the cell's flow time step by a stiff ODE
 * solver driven by a sparse analytical Jacobian (SpeedCHEM-style), with the chemistry load balanced
 * across workers (DLB) and per-cell time steps (LTS).  The paper names these techniques without
 * formulas; this library implements them as:
 *   - a constant-pressure adiabatic reactor, state y = (T, Y_1..Y_n);
 *   - NASA-7 thermo, modified Arrhenius, third-body and Troe fall-off rates, reverse rates from Kc;
 *   - an exact Jacobian J = S + u v^T whose sparse part S has a pattern fixed per mechanism (the rank-one
 *     term is the constant-pressure density coupling, v_i = Wbar / W_i);
 *   - the L-stable Rosenbrock method RODAS3 (or, by option, ROS2 or RODAS4) with a sparse LU whose
 *     fill-reducing ordering and symbolic factorisation are fixed once per mechanism, one warp (or two)
 *     per cell;
 *   - load balancing between processes as a host-side plan (chem_balance_plan).
 *
 * Conventions for every entry point below.
 *   - Array arguments of the compute calls are DEVICE pointers (cudaMalloc / torch tensors on the
 *     handle's device), FP64 unless stated, caller-owned, and must stay valid until the work queued on
 *     `stream` completes.  Cell arrays are structure-of-arrays with leading dimension N: species k of
 *     cell c is Y[k*N + c].
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Calls are asynchronous.
 *   - Return value: CHEM_OK, or an error code for argument, launch or CUDA errors; chem_last_error()
 *     returns the message of the last failure on the calling thread.  Per-cell numerical failures never
 *     fail the call: they are reported in the per-cell status array.
 *   - No call aborts, traps or prints.  A handle may be used from one host thread at a time.
 *   - Calls that take a handle run on the handle's device: they make it current for the call and put the
 *     caller's current device back before returning (chem_create likewise for its `device`).
 *   - Units: SI (K, Pa, kg/mol, mol/m^3, J/mol, s).
 */
#ifndef CHEM_H_
#define CHEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chem_handle_s* chem_handle;
typedef struct CUstream_st* chem_stream; /* identical to cudaStream_t */

typedef enum {
  CHEM_OK = 0,
  CHEM_EINVAL = 1,       /* invalid argument or mechanism description */
  CHEM_ENOMEM = 2,       /* device or host allocation failed */
  CHEM_ECUDA = 3,        /* a CUDA runtime call failed */
  CHEM_EUNSUPPORTED = 4  /* valid but outside the library's limits (e.g. shared memory per cell) */
} chem_status;

/* Per-cell status codes written by chem_integrate. */
enum {
  CHEM_CELL_OK = 0,
  CHEM_CELL_MAXSTEPS = 1,  /* max_substeps attempts reached before t = dt */
  CHEM_CELL_HMIN = 2,      /* step size fell below h_min */
  CHEM_CELL_NONFINITE = 3, /* max_nonfinite consecutive attempts produced non-finite values */
  CHEM_CELL_BADINPUT = 4,  /* T <= 0, p <= 0, dt < 0, non-finite input, or sum(Y/W) <= 0 */
  CHEM_CELL_TIMEOUT = 5,   /* the call's time budget ran out before this cell finished */
  CHEM_CELL_NOTAPE = 6     /* chem_adjoint: the forward pass took more accepted steps than the tape holds;
                              the cell's gradients are reported as zero (as for a failed forward pass,
                              which keeps its own status) */
};

/* Mechanism description (host memory, copied by chem_create; the caller keeps ownership).
   Reactions are reversible unless reversible[r] == 0.  rtype: 0 elementary, 1 third-body
   (rate multiplied by [M]), 2 Troe fall-off (k = k_inf Pr/(1+Pr) F, no [M] multiplier).
   Participants: CSR lists by reaction, species index and stoichiometric coefficient (1..3), at most 3
   distinct species and total order 3 per side.  Efficiencies: CSR list by reaction of species whose
   third-body efficiency differs from 1 (ignored for elementary reactions).  Arrhenius: k = A T^b
   exp(-Ea/(Ru T)), A in SI units of the reaction's order; for Troe, A/b/Ea are the high-pressure limit
   and low[3r..3r+2] = (A0, b0, Ea0) the low-pressure limit; troe[4r..4r+3] = (alpha, T3, T1, T2), with
   T2 <= 0 meaning the T2 term is absent.  NASA-7: nasa_lo/nasa_hi [7n], low set used for T < T_mid[k].
   comp (nullable): element counts [n*n_elements], enabling the element-balance check. */
typedef struct {
  int n_species;
  int n_reactions;
  int n_elements;
  const double* W;         /* [n] molar masses, kg/mol, > 0 */
  const double* nasa_lo;   /* [7n] */
  const double* nasa_hi;   /* [7n] */
  const double* T_mid;     /* [n] */
  const int* comp;         /* [n*n_elements] or NULL */
  const int* reac_ptr;     /* [R+1] */
  const int* reac_sp;
  const int* reac_nu;
  const int* prod_ptr;     /* [R+1] */
  const int* prod_sp;
  const int* prod_nu;
  const double* A;         /* [R] */
  const double* b;         /* [R] */
  const double* Ea;        /* [R] J/mol */
  const int* rtype;        /* [R] */
  const int* reversible;   /* [R] */
  const int* eff_ptr;      /* [R+1] */
  const int* eff_sp;
  const double* eff_alpha;
  const double* troe;      /* [4R] */
  const double* low;       /* [3R] */
} chem_mech_desc;

/* Sizes of a compiled mechanism. */
typedef struct {
  int n_species;
  int n_reactions;
  int n_state;        /* m = n_species + 1 */
  int nnz_S;          /* entries of the static Jacobian pattern (T row and column included) */
  int nnz_LU;         /* entries of the factor after fill (fill-reducing ordering, T last) */
  int lu_steps;       /* warp-wide steps of the precomputed elimination program */
  int solve_steps;    /* warp-wide steps of one forward+backward solve */
  int smem_per_cell;  /* bytes of shared memory one cell needs in the integrator */
  int n_dslots;       /* per-reaction derivative slots used by the Jacobian */
  int jac_passes;     /* passes of the Jacobian's reaction loop (their scratch shares the factor's space) */
  int smem_adjoint_per_cell;  /* bytes of shared memory one cell needs in chem_adjoint's reverse pass
                                 (checkpoint interval 16) */
  /* launch limits on the handle's device (0 for host-only handles), per lane group [one warp per cell,
     two warps per cell, two cells per warp]: the largest block in cells, the most cells resident per SM,
     and the library's automatic choices */
  int max_block_cells[3];
  int resident_cells[3];
  int auto_warps_per_cell;
  int auto_cells_per_warp;
} chem_info_t;

/* Options of chem_integrate (zero-initialise, then set; zero/negative fields take the defaults). */
typedef struct {
  double rtol;            /* default 1e-6 */
  double atol;            /* default 1e-12 (applies to T too) */
  double h_init;          /* default first step when h_io[c] <= 0: 1e-7 s */
  double h_min;           /* default 1e-20 s */
  double time_budget_s;   /* wall-clock budget of the call on the device; 0: none */
  int max_substeps;       /* default 100000 attempts per cell */
  int max_nonfinite;      /* default 10 consecutive non-finite attempts (each divides h by 10) */
  int mode;               /* 0: plain launch, one lane group per cell in index order (reference form);
                             1: persistent work-queue kernel over cells sorted by their previous
                             substep count */
  int block_cells;        /* cells in flight per block (each takes warps_per_cell warps); 0: automatic;
                             larger requests are reduced to the largest block that launches */
  int chunk;              /* cells taken per queue pull in mode 1; 0: automatic (1).  Values above an even
                             share of the cells over the resident lane groups, ceil(N / groups), are
                             reduced to that share (a larger pull only leaves lane groups idle); results
                             do not depend on it */
  int* naccept;           /* optional DEVICE array [N]: accepted steps per cell (NULL: not written) */
  double* trace;          /* optional DEVICE array [trace_cap*N]: attempt i of cell c at trace[i*N + c],
                             +h if accepted, -h if rejected, 0 after the last attempt (NULL: off) */
  int trace_cap;          /* attempts recorded per cell */
  int ckpt_every;         /* chem_adjoint: accepted steps between checkpoints (default 16, at most 64) */
  int tape_steps;         /* chem_adjoint: accepted steps the tape holds per cell (default 4096) */
  int warps_per_cell;     /* chem_integrate and chem_integrate_noalloc: lanes of one cell, 1 (one warp) or
                             2 (two warps of a block; wider reaction and species loops and more warps in
                             flight for mechanisms whose cells fill shared memory); 0: automatic (two when
                             one-warp cells leave fewer than 6 per SM, see chem_info).  Results of the two
                             choices agree to rounding, not bit for bit (different summation orders).
                             chem_adjoint uses one warp per cell. */
  int method;             /* Rosenbrock method: 0 RODAS3 (Sandu et al. 1997; order 3, embedded order 2,
                             L-stable; the default and the only one chem_adjoint differentiates),
                             1 ROS2 (Verwer et al. 1999; order 2, embedded order 1, L-stable,
                             gamma = 1 + 1/sqrt(2)), 2 RODAS4 (Hairer and Wanner, Sec. VI.4; 6 stages,
                             order 4, embedded order 3, stiffly accurate, L-stable, gamma = 1/4; same
                             shared memory per cell as RODAS3).  Other values: CHEM_EINVAL. */
  int cells_per_warp;     /* chem_integrate and chem_integrate_noalloc: 2 = two cells share a warp, 16 lanes
                             each (for mechanisms with few species, whose loops and sparse programs leave
                             most of a warp idle; needs warps_per_cell 0 or 1; block_cells is rounded to
                             an even count; in mode 1 the two halves of a warp take consecutive cells of the
                             sorted queue); 1 = one cell per warp (or per two warps); 0: automatic (see
                             chem_info: two for mechanisms of at most 16 species when half-warp blocks
                             keep at least as many cells resident per SM, else one).  Results agree with
                             one warp per cell to rounding. */
  int tabulate;           /* chem_integrate, chem_integrate_noalloc, chem_integrate_mapped: 1 = evaluate the
                             costly temperature functions from tables (an approximation; Sec. 2.5: SpeedCHEM
                             interpolates costly thermodynamic functions with polynomials of optimal
                             degree): every species' exp(+-g_k), g_k = h_k/(Ru T) - s_k/Ru, every forward rate
                             coefficient (the high-pressure limit of a fall-off reaction) and every Troe centre
                             F_cent, for 250 K <= T < 4000 K, as polynomials in 1/T on 640 equal intervals of
                             1/T, one degree per class of functions (the smallest up to 8 that keeps every
                             function within tab_tol, relative, at 17 points of every interval).  Outside
                             that range, the fall-off ratio k_0 [M] / k_inf, all other quantities and the
                             Jacobian's derivatives stay exact.  The tables are built on the host and kept
                             in the handle at the first call with a new tab_tol (about a second for 53
                             species / 325 reactions); chem_integrate_noalloc uses tables built before and
                             returns CHEM_EINVAL otherwise.  The tables hold the description's parameters:
                             CHEM_EINVAL after chem_set_params shifted them.  0: exact (default). */
  double tab_tol;         /* relative error bound of the tables; 0: 1e-10 */
  int specialized;        /* chem_integrate and chem_integrate_noalloc: 1 = run the mechanism-specialised
                             one-warp-per-cell kernels that chem_specialize compiled for this handle
                             (CHEM_EINVAL before that, or with warps_per_cell or cells_per_warp 2);
                             results agree with the library's own one-warp kernels to rounding (the
                             compiler may contract or order floating-point operations differently).
                             0: the library's kernels (default). */
} chem_integrate_opts;

/* Compile a mechanism for `device`: validation (indices, positive W and A, finite parameters,
   element balance when comp is given), reaction reordering by type, the static Jacobian pattern, a
   minimum-degree ordering with T last, the symbolic LU and its warp elimination program, and upload of
   all tables.  On success *out owns device memory until chem_destroy. */
chem_status chem_create(const chem_mech_desc* desc, int device, chem_handle* out);
/* device == -1 compiles on the host only (no GPU needed): chem_info, chem_jacobian_pattern and
   chem_export_plan work, compute calls return CHEM_EINVAL. */
/* chem_create from the JSON form of the description: an object whose keys are the field names of
   chem_mech_desc ("W", "nasa_lo", "nasa_hi", "T_mid", "comp", "reac_ptr", ..., "troe", "low"); the
   sizes follow from "W" (species) and "A" (reactions); two-dimensional fields (nasa_lo/hi [n][7],
   comp [n][elements], troe [R][4], low [R][3]) may be nested rows or flat arrays; "comp" may be absent
   or null (no element-balance check); other keys are ignored.  json_text is NUL-terminated host
   memory, read during the call only.  CHEM_EINVAL with a message for malformed JSON, missing keys or
   inconsistent lengths; then as chem_create. */
chem_status chem_create_from_json(const char* json_text, int device, chem_handle* out);
chem_status chem_destroy(chem_handle h);

/* Mechanism-specialised integration kernels (opt-in).  The one-warp-per-cell integration kernels (plain
   and persistent form) are compiled again at run time (NVRTC, loaded with dlopen) with this mechanism's
   sizes (species, reactions, nonzeros of S and of the factor, steps of the elimination and substitution
   programs) and the cell's shared-memory offsets as compile-time constants, so that the compiler folds
   the trip counts and addresses of the sparse-analytical evaluation into the code (Sec. 2.5: SpeedCHEM
   manages the mechanism's sparse algebra internally).  The tables and
   programs stay in device memory; only sizes and offsets become constants.  The kernels are loaded into
   the handle's device and used by calls with chem_integrate_opts.specialized = 1 until chem_destroy.
   Compiled code is cached on disk (directory CHEM_RTC_CACHE, else rtc_cache beside the library), keyed
   by the source, the headers, the options and the compiler's version; a second handle of the same
   mechanism loads it from there.  *compile_s (optional) receives the compile time in seconds (0 when
   both kernels came from the cache or the handle holds them already).  CHEM_EUNSUPPORTED when
   libnvrtc.so.13 cannot be loaded; CHEM_ECUDA with the compiler's log when compiling or loading fails.
   Calling it again on the same handle does nothing.  On a host-only handle (device -1) it compiles into
   the cache and loads nothing (no GPU needed), e.g. to fill the cache ahead of a run. */
chem_status chem_specialize(chem_handle h, double* compile_s);
/* The generated source of chem_specialize (the views with constant members; it includes the library's
   device headers).  buf: host memory of *len bytes, or NULL to query; on return *len = bytes needed
   (terminating NUL included); CHEM_EINVAL when buf is too small.  Works on host-only handles. */
chem_status chem_specialized_source(chem_handle h, char* buf, int* len);

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char* chem_last_error(void);

chem_status chem_info(chem_handle h, chem_info_t* info);

/* The static pattern of S in natural state order (0 = T, 1 + k = Y_k), CSR, HOST arrays:
   row_ptr [m+1], col_idx [nnz_S]. Entry e of chem_jacobian's S_vals is (row of e, col_idx[e]). */
chem_status chem_jacobian_pattern(chem_handle h, int* row_ptr, int* col_idx);

/* Host copy of a compiled plan, for inspection and CPU-side checks.  which:
     0 elimination program, 1 substitution program: 4 ints per lane-op (kind, t, a, b), 32 per step,
       t = 65535 marks an idle lane; kinds 0 reciprocal, 1 scale, 2 update (see the device code);
     2 ordering: perm[p] = state index at factor position p (m ints);
     3 factor pattern: row_ptr (m+1) then col (nnz_LU), factor positions;
     4 factor slot sources: S entry (internal order) feeding each factor slot, -1 for fill (nnz_LU);
     5 internal S entry -> CSR position of chem_jacobian_pattern (nnz_S);
     6 transposed substitution program (A^T x = b), same encoding as 1;
     7 compiled reaction order: description index of each compiled reaction (R);
     8, 9, 10 the programs of 0, 1 and 6 for two warps per cell: 64 lane-ops per step;
     11, 12, 13 the programs of 0, 1 and 6 for two cells per warp: 16 lane-ops per step.
   With out == NULL only *count is written.  *count: number of ints. */
chem_status chem_export_plan(chem_handle h, int which, int* out, int* count);

/* Right-hand side of the reactor ODE for N cells (each cell a homogeneous reactor, Sec. 1 and Sec. 2.5):
   dTdt [N] = -sum_k H_k w_k / (rho c_p), dYdt [n*N] = W_k w_k / rho, wdot [n*N] (nullable) = net molar
   production rates w_k in mol/(m^3 s).  Inputs T [N], p [N], Y [n*N]. */
chem_status chem_rates(chem_handle h, int N, const double* T, const double* p, const double* Y,
                       double* dTdt, double* dYdt, double* wdot, chem_stream stream);

/* Exact Jacobian of chem_rates' right-hand side, J = S + u v^T, for N cells (the sparse analytical
   Jacobian of Sec. 2.5; S in the static pattern of chem_jacobian_pattern):
   S_vals [nnz_S*N] (entry-major: entry e of cell c at S_vals[e*N + c], entries in the CSR order of
   chem_jacobian_pattern), u [m*N], v [m*N] (v_0 = 0, v_{1+k} = Wbar / W_k). */
chem_status chem_jacobian(chem_handle h, int N, const double* T, const double* p, const double* Y,
                          double* S_vals, double* u, double* v, chem_stream stream);

/* Advance N cells over their own step dt[c] (Sec. 2.5: every cell integrated over its flow time step, with
   its own step under local time stepping) by the Rosenbrock method of opts->method (RODAS3 by
   default) with error control.
   In/out: T [N], Y [n*N]; h_io [N] (in: first step, <= 0 takes h_init; out: next proposed step);
   nsub [N] (in: previous substep counts, the sort key of mode 1; out: attempts taken in this call);
   status [N] (out: CHEM_CELL_*).  In: p [N], dt [N].  opts may be NULL (defaults).
   Scratch for mode 1 (sorting and the queue) is held by the handle and grows on demand. */
chem_status chem_integrate(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                           double* h_io, int* nsub, int* status, const chem_integrate_opts* opts,
                           chem_stream stream);

/* Shift the Arrhenius parameters of every reaction relative to the description given to chem_create:
   ln A_j -> ln A_j + dlnA[j], Ea_j -> Ea_j + dEa[j] (DEVICE arrays [R] in description order, either may
   be NULL for zero).  For Troe reactions both limits shift together (the fall-off shape is unchanged and
   k_f, k_r scale exactly by exp(dlnA) exp(-dEa/(Ru T))).  Stream-ordered; later calls see the new
   parameters.  Calling it with two NULLs restores the description's values. */
chem_status chem_set_params(chem_handle h, const double* dlnA, const double* dEa, chem_stream stream);

/* Discrete adjoint of chem_integrate (the paper computes no sensitivities; this is the standard discrete
   adjoint of the Rosenbrock steps).  With the accepted step sizes of the forward integration frozen,
   for the objective L = sum_c (gT[c] T_c(dt) +
   sum_k gY[k*N+c] Y_k,c(dt)) it returns
     grad_lnA [R], grad_Ea [R] (DEVICE, description order, summed over cells; J/mol units for Ea),
     grad_cell [2R*N] (nullable; entry j*N + c for ln A_j, (R + j)*N + c for Ea_j, per cell),
     gT0 [N], gY0 [n*N] (nullable; dL/d initial T and Y).
   T [N] and Y [n*N] are the initial state in and the final state out, as in chem_integrate (same
   results).  The forward pass records the accepted step sizes and a checkpoint every
   opts->ckpt_every accepted steps (tape of opts->tape_steps accepted steps per cell, handle scratch);
   the reverse pass recomputes each segment from its checkpoint.  status [N] as chem_integrate, plus
   CHEM_CELL_NOTAPE.  opts: tolerances and limits as for chem_integrate (mode is ignored). */
chem_status chem_adjoint(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                         const double* gT, const double* gY, double* grad_lnA, double* grad_Ea, double* grad_cell,
                         double* gT0, double* gY0, int* status, const chem_integrate_opts* opts, chem_stream stream);

/* chem_integrate without any device allocation.  (The paper has no counterpart: this is a calling
   convenience of this library.)
   Some callers cannot allocate device memory at the point where they integrate chemistry: a CFD code
   whose memory pool has taken the device's memory at start-up, a time loop that must not pay the
   implicit device synchronisation cudaMalloc/cudaFree can cause, or a plug-in that may not grow its
   footprint after initialisation.  This entry point runs the same sorted work-queue integration as
   chem_integrate with mode 1 (results are identical) but takes its scratch (sort counters, queue
   head, time stamp, the cell permutation) from a fixed array in the library's static device memory
   instead of handle-owned memory, and calls no allocating routine.  The handle itself must already
   exist (chem_create allocates the mechanism tables once).
   Limits and rules:
   - at most 1,048,576 cells per call (larger N returns CHEM_EINVAL before anything is launched); the
     array takes 4 MiB + 512 bytes on every GPU that loads the library, until the process exits;
   - the first call on a device looks up the array's device address (once per device, with that
     device current) -- make that first call before any stream capture;
   - all calls share the one array and each call clears its counters first: calls whose GPU work
     overlaps (different streams, or different host threads without ordering) race and must not be
     issued; put them on one stream or synchronise between them;
   - opts as for chem_integrate; opts.mode is ignored (always the sorted work queue).
   Arguments, layouts and per-cell status as for chem_integrate. */
chem_status chem_integrate_noalloc(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                                   double* h_io, int* nsub, int* status, const chem_integrate_opts* opts,
                                   chem_stream stream);

/* Diagnostic: evaluates an elementary function of the device code on N doubles (device pointers x, y,
   y[i] = f(x[i])): fn 0 = the library's table-driven exponential (used for every rate constant,
   equilibrium constant and fall-off factor), fn 1 = the CUDA math library's exp, fn 2 = the
   library's table-driven logarithm (ln T, ln [M] and ln F_cent of the fall-off), fn 3 = the CUDA math
   library's log.  It has no counterpart in the paper; it exists so that the library's functions can be
   checked against CUDA's.  Runs on the current device.  CHEM_EINVAL for fn outside {0, 1, 2, 3},
   N < 0 or null pointers with N > 0. */
chem_status chem_eval_elementary(int fn, int N, const double* x, double* y, chem_stream stream);

/* Zonal reference-cell mapping (Sec. 2.5: for regions of low reactivity the chemistry solution is taken
   from a reference cell instead of being integrated).  Options of chem_integrate_mapped:
     T_max       cells with T >= T_max, a non-finite key value, p or dt, or a key quotient (below) of
                 magnitude 2^62 or more are never mapped (NaN: CHEM_EINVAL);
     dT          temperature bin width (> 0, finite);
     n_species   number of mass fractions in the zone key, 0..8;
     species     their indices (0-based, distinct, < n_species of the mechanism);
     dY          their bin widths (> 0, finite).
   A candidate cell (T < T_max) belongs to the zone given by the integers floor(T/dT), floor(Y_s/dY_s)
   for the listed species s, and the exact values of p and dt: cells of one zone differ by less than dT
   in T and dY_s in each listed Y_s and share p and dt. */
typedef struct {
  double T_max;
  double dT;
  int n_species;
  int species[8];
  double dY[8];
} chem_map_opts;

/* chem_integrate with zonal reference-cell mapping.  In every zone with more than one cell, the cell of
   lowest index is the zone's reference: it is integrated, and every other member takes over its change,
     T_c <- T_c + (T_ref(dt) - T_ref(0)),  Y_k,c <- Y_k,c + (Y_k,ref(dt) - Y_k,ref(0)) for all k,
   with status_c = status_ref, nsub_c = 0 (no substep of its own, the cost key of the next call) and h_io_c
   unchanged.  All other cells are integrated exactly as by chem_integrate.  The mapping keeps sum(Y)
   to rounding; it does not keep every Y_k >= 0 (the bins bound the error, the caller chooses them).
     map            host struct; NULL: no mapping (every cell integrated, results as chem_integrate);
     ref            DEVICE [N], out: the reference of each cell (the cell itself when it was integrated);
     n_integrated   HOST, out (nullable): the number of cells integrated.
   Other arguments as for chem_integrate; opts->trace and opts->naccept must be NULL; N <= 2^29.  The call waits
   once on `stream` (for the number of cells to integrate) and keeps scratch in the handle (about
   (n + 14) * 8 bytes per cell).  CHEM_EINVAL for invalid options. */
chem_status chem_integrate_mapped(chem_handle h, int N, double* T, const double* p, double* Y, const double* dt,
                                  double* h_io, int* nsub, int* status, const chem_integrate_opts* opts,
                                  const chem_map_opts* map, int* ref, int* n_integrated, chem_stream stream);

/* Load balancing between processes (Sec. 2.5: the chemistry work is redistributed between MPI ranks so
   that every rank carries about the same load).  A pure host computation, no handle and no device: every
   rank calls it on the same all-gathered input and obtains the same plan.
     world   number of ranks, >= 1.
     counts  HOST [world]: cells held by each rank (>= 0).
     costs   HOST [sum counts]: each cell's expected cost (its previous substep count, or 1 when none is
             known), rank 0's cells first, each rank's in its local order; finite and >= 0.
     dest    HOST [sum counts], out: the rank that integrates each cell (same order as costs).
   Rule: target = total cost / world.  Each rank keeps its cheapest cells (ascending cost, ties by local
   index) while their running sum stays within the target; the remaining cells are dealt in descending
   cost (ties by rank, then local index) to the rank with the least current load (ties to the lowest
   rank).  Hence no rank ends above target + the largest single cost, a rank at or below the target
   keeps all its cells, and a rank above it sends away the fewest cells the target allows.
   CHEM_EINVAL for world < 1, a negative count, a negative or non-finite cost, or NULL arrays with cells
   present; dest is then unspecified. */
chem_status chem_balance_plan(int world, const int64_t* counts, const double* costs, int32_t* dest);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H_ */
