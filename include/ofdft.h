/*
 * ofdft.h -- C ABI of the GB300 orbital-free DFT energy/potential library.
 *
 * The library evaluates, for an electron density rho on a periodic 3-D grid,
 * the energy E[rho] = T_TF + T_vW + T_NL + E_H + E_PP and its functional
 * derivative V = dE/drho (arXiv:2002.02985, Sec. 1 Eqs. efunc and euler),
 * the ionic forces of the electron-ion term, and the psi = sqrt(rho) density
 * optimisation of Sec. 2.4 (Eq. euler2).  T_NL is the density-dependent-kernel
 * nonlocal KEDF (LWT) evaluated with linear splines over a set of kF knots,
 * steps s1-s4 of Sec. 2.3 (Eqs. nl2, WT and the G_NL definition).
 *
 * Conventions (all entry points)
 *   - Units: Hartree atomic units; lengths in bohr, energies in Ha.
 *   - Cell: cell[9] holds the lattice vectors a_0, a_1, a_2 as rows (bohr),
 *     row-major.  Grid shape[3] = {n0, n1, n2}; fields are contiguous C-order
 *     arrays [n0][n1][n2] (n2 fastest) of float (OFDFT_FP32_MIXED) or double
 *     (OFDFT_FP64) in DEVICE memory owned by the caller.  Each n_a must be
 *     of the form 2^a 3^b 5^c with 2 <= n_a <= 1024.
 *   - Fourier convention: f_hat(G) = (1/N) sum_r f(r) e^{-iG.r}; the integer
 *     frequency of index k on an axis of n points is k for k <= n/2, else k-n.
 *   - V is the functional derivative in Ha/e: dE/drho_r = V_r * Omega/N.
 *   - All device work is enqueued on the stream given to ofdft_grid_create.
 *     Calls that return host values synchronise that stream.
 *
 * Ownership: the caller owns every density/potential buffer.  The library
 * owns the grid handle and its workspace (allocated with cudaMalloc on first
 * use for a precision and freed by ofdft_grid_destroy).  Nothing returned
 * needs freeing except the handle.  A handle must not be used from two host
 * threads at once.
 *
 * Errors: every entry point returns an int status; 0 = OFDFT_OK.  On error the
 * handle keeps a message readable with ofdft_last_error().  No C++ exception
 * crosses the ABI.
 */
#ifndef OFDFT_H
#define OFDFT_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define OFDFT_OK                    0
#define OFDFT_ERR_INVALID_ARG      -1  /* null pointer, bad shape, singular cell, bad knot count */
#define OFDFT_ERR_UNSUPPORTED_SIZE -2  /* a grid dimension not 2^a3^b5^c or outside [2, 1024] */
#define OFDFT_ERR_BAD_DENSITY      -3  /* NaN/Inf or negative density found */
#define OFDFT_ERR_OOM              -4  /* cudaMalloc failed */
#define OFDFT_ERR_CUDA             -5  /* any other CUDA error (message kept in the handle) */
#define OFDFT_ERR_NOT_CONVERGED    -6  /* optimiser reached max_iter */
#define OFDFT_ERR_NO_IONS          -7  /* a call needs ions but ofdft_set_ions was not called */
#define OFDFT_ERR_TIMEOUT          -8  /* a bounded device-side wait expired (the results are not valid) */

/* ---- functional description ----------------------------------------- */
#define OFDFT_TERM_TF       1u   /* Thomas-Fermi  C_TF int rho^(5/3)             */
#define OFDFT_TERM_VW       2u   /* von Weizsaecker, psi = sqrt(rho) form          */
#define OFDFT_TERM_NL       4u   /* nonlocal KEDF (LWT spline or global-kF WT)    */
#define OFDFT_TERM_HARTREE  8u   /* Hartree, G = 0 dropped                        */
#define OFDFT_TERM_PP      16u   /* local pseudopotential of the ions             */
#define OFDFT_TERM_XC      32u   /* LDA exchange-correlation: Dirac exchange and the
                                    Perdew-Zunger (1981) correlation the paper's
                                    benchmarks use (Sec. 3.1)                      */
#define OFDFT_TERMS_ALL    31u   /* the kinetic + electrostatic functional (no xc)   */
#define OFDFT_TERMS_VALID  63u   /* every defined term bit                          */

/* Energies returned by the evaluation calls, in this order (Ha). */
#define OFDFT_N_ENERGIES 7      /* total, TF, vW, NL, H, PP, XC */

#define OFDFT_KNOTS_LOG     0    /* geometric progression of kF knots (s1)        */
#define OFDFT_KNOTS_ARITH   1    /* arithmetic progression                        */

#define OFDFT_NLPOT_EXACT   0    /* V = exact derivative of the spline energy     */
#define OFDFT_NLPOT_INTERP  1    /* V = 2 alpha rho^(alpha-1) Phi (s3->s4 blend)  */

#define OFDFT_KERNEL_LWT        0  /* kernel at the local kF(r) via the knots      */
#define OFDFT_KERNEL_WT_GLOBAL  1  /* one WT kernel at kF(N_e/Omega)               */

#define OFDFT_FP64        0      /* fields double, all arithmetic FP64            */
#define OFDFT_FP32_MIXED  1      /* fields float, FFT/pointwise FP32, energies,
                                    knots and optimiser scalars FP64             */

typedef struct {
    unsigned terms;        /* OR of OFDFT_TERM_* */
    double alpha, beta;    /* exponents of Eq. nl2 (5/6, 5/6) */
    int n_knots;           /* M >= 2, <= 64 */
    int knot_spacing;      /* OFDFT_KNOTS_LOG | OFDFT_KNOTS_ARITH */
    const double *knots;   /* optional HOST array of n_knots frozen knots (ascending);
                              NULL = recompute from min/max rho on every call (s1) */
    int nl_potential;      /* OFDFT_NLPOT_EXACT | OFDFT_NLPOT_INTERP (needs alpha == beta) */
    int kernel;            /* OFDFT_KERNEL_LWT | OFDFT_KERNEL_WT_GLOBAL */
    int precision;         /* OFDFT_FP64 | OFDFT_FP32_MIXED */
    double rho_floor;      /* guard for rho^(alpha-1), 1/psi, kF (<= 0 means 1e-20) */
    double mgp_x;          /* Eq. MGP's x: 0 = the Wang-Teter kernel of Eq. WT (LWT / global WT);
                              MGP and MGPG 1, MGPA 1/2 (with LWT: LMGP/A/G).  |x| <= 10 */
    double mgp_y;          /* Eq. MGP's y, used when mgp_x != 0: MGP/MGPA 5/6, MGPG 5/3; (0, 10].
                              Reading: eta(q,t) = q/(2 k_F t^(1/3)), k_F of the scaled density
                              t rho.  The correction is tabulated once per grid and y (2^20 + 1
                              points in eta/(1+eta), FP64 quadrature on the GPU) and interpolated
                              linearly per G and knot */
} ofdft_functional;

/* Analytic local pseudopotential per species: v(q) = -4 pi Z exp(-(q rc)^2/4) / q^2,
 * i.e. -Z erf(r/rc)/r in real space; the q = 0 term is pi Z rc^2. */
typedef struct {
    int n_species;
    const double *Z;       /* [n_species] valence charge */
    const double *rc;      /* [n_species] core radius, bohr */
} ofdft_species;

typedef struct {
    int n;                 /* number of ions */
    const double *pos;     /* HOST [n][3] Cartesian positions, bohr */
    const int *species;    /* HOST [n] species index */
} ofdft_ions;

typedef struct {
    int iterations;        /* CG iterations done */
    int evaluations;       /* energy/potential evaluations done */
    double energy;         /* final total energy, Ha */
    double energies[OFDFT_N_ENERGIES];    /* total, TF, vW, NL, H, PP, XC */
    double mu;             /* chemical potential int rho V / N_e */
    double residual;       /* || (V - mu) psi ||_2 (with dV weight) at the end */
    double last_dE;        /* |E_k - E_{k-1}| of the last iteration */
} ofdft_opt_report;

typedef struct ofdft_grid ofdft_grid;   /* opaque */

/* Create a grid for the periodic cell (cell[9], rows = lattice vectors, bohr)
 * sampled on shape[3] points; work is enqueued on cuda_stream (a cudaStream_t,
 * NULL = legacy default stream) of the current device.  No device memory is
 * allocated until the first call that needs it.  Defines the Grid of Sec. 2.1. */
int ofdft_grid_create(const double cell[9], const int shape[3], void *cuda_stream, ofdft_grid **out);
int ofdft_grid_destroy(ofdft_grid *g);

/* Set the ions and build the external potential V_ext(G) = (1/Omega) sum_I
 * v(|G|) e^{-iG.R_I} on the half spectrum by the direct structure factor
 * (Sec. 2.5).  Copies the host arrays; may be called again for new positions. */
int ofdft_set_ions(ofdft_grid *g, const ofdft_ions *ions, const ofdft_species *sp);

/* Same as ofdft_set_ions, but the structure factor is the smooth particle-mesh
 * Ewald approximation of even B-spline order `order` (4..16), as the paper uses
 * for more than ~1000 ions (Sec. 2.5; Essmann et al. 1995):
 *   S(G) ~ prod_a conj(b_a(m_a)) sum_k Q(k) e^{-iG.r_k},  Q(k) = sum_I prod_a M_p(u_aI - k_a),
 * spread with fixed-point atomics (bit-reproducible).  Forces are then the exact
 * derivative of the PME energy (B-spline gather).  Needs every n_a >= order. */
int ofdft_set_ions_pme(ofdft_grid *g, const ofdft_ions *ions, const ofdft_species *sp, int order);

/* One energy + potential evaluation (Eq. efunc; Eq. euler for V; Sec. 2.3 s1-s4).
 * rho_dev: device [N] float/double (precision of f), >= 0.
 * E_out:   HOST double[OFDFT_N_ENERGIES] = {total, TF, vW, NL, H, PP, XC} (Ha); may be NULL.
 * V_dev:   device [N] output potential (Ha/e), same precision; may be NULL.
 * Synchronises the stream when E_out is not NULL. */
int ofdft_energy_potential(ofdft_grid *g, const void *rho_dev, const ofdft_functional *f,
                           double *E_out, void *V_dev);

/* Same evaluation, fully asynchronous: energies are written to E_dev (DEVICE
 * double[OFDFT_N_ENERGIES]) on the stream; nothing is synchronised and no host memory is
 * touched, so the call can be captured in a CUDA graph once the workspace
 * exists (make one ordinary call first). */
int ofdft_energy_potential_async(ofdft_grid *g, const void *rho_dev, const ofdft_functional *f,
                                 double *E_dev, void *V_dev);

/* Ionic forces F_I = -dE/dR_I of the electron-ion term (the only term of
 * Eq. efunc that depends on R_I): F_I = -sum_G G v(|G|) Im[conj(rho_hat) e^{-iG.R_I}].
 * F_out: HOST double[n_ions][3] (Ha/bohr).  precision selects the rho dtype. */
int ofdft_forces(ofdft_grid *g, const void *rho_dev, int precision, double *F_out);

/* Ion-ion electrostatic energy and forces of the ions given to ofdft_set_ions or
 * ofdft_set_ions_pme: point charges Z_s in a uniform neutralising background, by
 * Ewald summation.  The paper's Eq. efunc has no ion-ion term; with it (and
 * OFDFT_TERM_XC) the energy becomes a total energy for structures and forces.
 * The reciprocal sum runs over the grid's G vectors (the split parameter is set
 * from the grid so that the neglected terms are below 1e-16; with
 * ofdft_set_ions_pme the structure factor is the PME one), the real-space sum
 * over a cell list; FP64 throughout.  Independent of the density.
 * E_out: HOST double[1] (Ha) or NULL; F_out: HOST double[n][3] (Ha/bohr) or NULL
 * (not both NULL).  Synchronises the handle's stream.
 * Errors: OFDFT_ERR_NO_IONS, OFDFT_ERR_INVALID_ARG, OFDFT_ERR_OOM, OFDFT_ERR_CUDA. */
int ofdft_ewald(ofdft_grid *g, double *E_out, double *F_out);

/* psi = sqrt(rho) density optimisation (Sec. 2.4, Eq. euler2) by preconditioned CG
 * (ofdft_optimize_density_ex below offers TN and L-BFGS):
 * psi_dev (device [N], precision of f) holds the initial psi and receives the
 * result; int psi^2 = N_e is imposed first and then conserved by the
 * psi cos(l) + p sin(l) update.  Stops when |E_k - E_{k-1}| < tol_E_per_atom *
 * n_ions for 3 consecutive iterations (returns OFDFT_OK) or after max_iter
 * iterations (returns OFDFT_ERR_NOT_CONVERGED with the report filled).
 * rep may be NULL. */
int ofdft_optimize_density(ofdft_grid *g, void *psi_dev, const ofdft_functional *f,
                           double N_e, double tol_E_per_atom, int max_iter,
                           ofdft_opt_report *rep);

/* Search-direction methods of the density optimiser (Sec. 2.4, step 1: the paper names
 * nonlinear CG, L-BFGS and truncated Newton). */
#define OFDFT_OPT_CG 0      /* Polak-Ribiere+ conjugate gradient (the default) */
#define OFDFT_OPT_TN 1      /* truncated Newton: inner CG on the Newton equation */
#define OFDFT_OPT_LBFGS 2   /* limited-memory BFGS */

typedef struct {
    int method;         /* OFDFT_OPT_CG | OFDFT_OPT_TN | OFDFT_OPT_LBFGS */
    int precondition;   /* nonzero: the model-Hessian preconditioner a G^2/(G^4 + a G^2 + b)
                           (a from the local terms, b from Hartree at the mean density)
                           on the gradient (CG, TN's inner CG, L-BFGS's initial inverse Hessian) */
    int max_inner;      /* TN: at most this many inner CG steps (each one evaluation) per
                           outer iteration; 0 = 10; at most 100 */
    int lbfgs_m;        /* L-BFGS: correction pairs kept (2 fields each); 0 = 5; at most 32 */
    int update;         /* step (3): OFDFT_UPDATE_ROTATE psi cos(l) + p sin(l), p orthogonal to psi
                           (default), or OFDFT_UPDATE_SCALE psi + t p renormalised to N_e, p not
                           orthogonalised (the paper's scaling scheme, "not always stable") */
    int objective;      /* OFDFT_OBJECTIVE_ENERGY: the line search minimises E (strong Wolfe, default);
                           OFDFT_OBJECTIVE_RESIDUAL: the step lowers the norm of the residual of
                           Eq. euler2, |2 psi (V - mu) dV| (backtracking by halves from the first
                           trial until it falls by 1e-4 relative) - the paper's second way */
} ofdft_opt_options;

#define OFDFT_OBJECTIVE_ENERGY 0
#define OFDFT_OBJECTIVE_RESIDUAL 1

#define OFDFT_UPDATE_ROTATE 0
#define OFDFT_UPDATE_SCALE 1

/* ofdft_optimize_density with a choice of direction method (opt NULL = CG, preconditioned).
 * TN: the Newton equation H x = -g of the Lagrangian E - mu (int psi^2 - N_e) is solved in
 * the tangent space of the constraint by preconditioned CG, stopped when the residual
 * falls below min(0.5, sqrt(res)) |g| (res = RMS Euler-Lagrange residual per electron) or
 * curvature turns non-positive; H q is a forward difference of the gradient 2 psi V dV
 * (one E+V evaluation at psi + e q, |e q| = 1e-3 |psi| in FP32-mixed, 1e-6 in FP64).
 * L-BFGS: two-loop recursion over the last lbfgs_m pairs (step of psi, change of the
 * projected gradient), initial inverse Hessian gamma P.  Both start the line search at the
 * length of their step.  Allocates 4 (TN) or 2 lbfgs_m (L-BFGS) more device fields of N
 * elements, kept with the grid.  Errors: as ofdft_optimize_density, OFDFT_ERR_INVALID_ARG
 * for options out of range. */
int ofdft_optimize_density_ex(ofdft_grid *g, void *psi_dev, const ofdft_functional *f,
                              double N_e, double tol_E_per_atom, int max_iter,
                              const ofdft_opt_options *opt, ofdft_opt_report *rep);

/* Fourier (band-limited) interpolation of a real periodic field between two grids of
 * one cell, the step that carries a converged density to a finer grid in the paper's
 * multi-step optimisation (Sec. 2.4).  Frequencies present on both grids are copied;
 * a Nyquist term of the smaller grid is shared between +-n/2 of the larger (so the
 * interpolant passes through the coarse samples) or, going down, formed from both.
 * src_dev: DEVICE [from's N], dst_dev: DEVICE [to's N], both float (OFDFT_FP32_MIXED)
 * or double (OFDFT_FP64).  Runs on the grids' streams and synchronises `to`'s stream.
 * Errors: OFDFT_ERR_INVALID_ARG (NULL, different cells, unknown precision), OFDFT_ERR_CUDA. */
int ofdft_interpolate(ofdft_grid *from, const void *src_dev, ofdft_grid *to, void *dst_dev, int precision);

/* Multi-step density optimisation (Sec. 2.4): grids[0..n_levels-1] share one cell,
 * coarsest first; psi_dev (DEVICE, on the finest grid, grids[n_levels-1]) holds the
 * initial psi and receives the result.  The initial psi is interpolated to the coarsest
 * grid and optimised there (as ofdft_optimize_density, max_iter iterations at most per
 * level); each level's result is interpolated to the next finer grid and optimised
 * again.  Each grid needs its ions when f has the PP term.  rep (may be NULL) describes
 * the finest level; a coarse level that stops at max_iter still seeds the next.
 * Allocates one psi buffer per coarse level for the duration of the call. */
int ofdft_optimize_density_multistep(int n_levels, ofdft_grid *const *grids, void *psi_dev,
                                     const ofdft_functional *f, double N_e, double tol_E_per_atom,
                                     int max_iter, ofdft_opt_report *rep);

/* ---- Real-time TD-OFDFT (Sec. "Time-Dependent OFDFT", Eq. cn).  A complex collective
 * orbital psi = sqrt(rho) e^{iS}, held as two real device fields (re, im; precision of f),
 * obeys i dpsi/dt = H psi, H psi = -lap psi / 2 + v_eff[rho] psi with v_eff = d(E - T_vW)/drho
 * for the functional f (its von Weizsaecker term becomes the Laplacian; adiabatic: v_eff at
 * the instantaneous density).  Positions r are cell-centred, r = A^T (f - 1/2) for the
 * fractional grid coordinates f. */
typedef struct {
    double dt;              /* time step (a.u. of time); negative propagates backwards */
    int n_steps;            /* steps to take (>= 0) */
    int n_corrector;        /* corrector passes per step (0..16): each solves the step again
                               from psi(t) with (v_eff(t) + v_eff(t+dt)) / 2 of the last pass */
    double solver_tol;      /* relative residual of each Crank-Nicolson solve; 0 = 1e-11 (FP64)
                               or 1e-5 (FP32-mixed) */
    int max_solver_iter;    /* CG iterations per solve; 0 = 200 */
} ofdft_td_options;

typedef struct {
    int steps;              /* steps taken */
    int evaluations;        /* v_eff evaluations */
    int solver_iterations;  /* CG iterations over all solves */
    double max_residual;    /* largest final relative residual of a solve */
} ofdft_td_report;

/* psi <- psi exp(i k.r) (the laser kick of the TD-OFDFT section, with this library's sign,
 * see ofdft_td_propagate; k HOST double[3], 1/bohr).  psi_re, psi_im: DEVICE [N] of the
 * precision given (OFDFT_FP32_MIXED: float, OFDFT_FP64: double).  Enqueued on the handle's
 * stream.  Errors: OFDFT_ERR_INVALID_ARG (NULL pointer, unknown precision), OFDFT_ERR_CUDA. */
int ofdft_td_kick(ofdft_grid *g, void *psi_re, void *psi_im, const double k[3], int precision);

/* Propagate psi (DEVICE re/im, in place) by n_steps Crank-Nicolson steps
 * (1 + i dt/2 H) psi(t+dt) = (1 - i dt/2 H) psi(t) — the form that integrates i dpsi/dt = H psi;
 * the paper prints the two signs exchanged, which with its kick exp(-ikx) is the complex
 * conjugate of this scheme under exp(+ikx): the same density, dipole and spectrum.
 * Each step is a predictor (v_eff at rho(t)) and n_corrector passes.  Each linear system is
 * solved through its normal equations (1 + dt^2/4 H^2) x = (1 - i dt/2 H)^2 psi(t), real and
 * imaginary parts by preconditioned CG (M = 1/(1 + dt^2/4 (G^2/2 + vbar)^2)).
 * rho0: DEVICE [N] reference density for the dipole, or NULL (0).  dipole: HOST
 * double[n_steps + 1][3] receiving delta mu(t_n) = sum_r r (|psi|^2 - rho0) dV, or NULL.
 * Allocates 19 device fields of N elements (kept with the grid).  Returns
 * OFDFT_ERR_NOT_CONVERGED (after all steps, report filled) if a solve reached max_solver_iter;
 * otherwise as ofdft_energy_potential (the functional's PP term needs ions). */
int ofdft_td_propagate(ofdft_grid *g, void *psi_re, void *psi_im, const void *rho0, const ofdft_functional *f,
                       const ofdft_td_options *opt, double *dipole, ofdft_td_report *rep);

/* Oscillator strength sigma(w) = w Im[delta mu~(w)] with delta mu~(w) = sum_n dmu_n
 * e^{(i w - gamma) t_n} dt, t_n = n dt (HOST arrays: dmu[n], omega[n_omega] -> sigma[n_omega];
 * dmu is the dipole component along the kick; gamma >= 0 damps the finite record).  Host
 * arithmetic only (no device, no handle).  Errors: OFDFT_ERR_INVALID_ARG (NULL pointer,
 * n < 1, n_omega < 0, dt = 0, gamma < 0). */
int ofdft_td_spectrum(const double *dmu, int n, double dt, double gamma, int n_omega, const double *omega,
                      double *sigma);

/* Batched evaluation of n independent grids (snapshots), possibly of different
 * shapes (Sec. 3.2: many independent OFDFT problems farmed out at once): E_out HOST
 * [n][OFDFT_N_ENERGIES]; V_dev[i] and F_out[i] may be NULL (F_out needs ions).  All grids
 * must share one stream, and one grid may appear only once.  Snapshots whose evaluations
 * share a launch geometry (same shape, same compiled kernels) are grouped: each pass of the
 * evaluation is ONE launch over up to 32 of them, every snapshot keeping the blocks and
 * reduction order of its single evaluation (results bit-identical to single calls); groups
 * run concurrently on internal streams forked from and joined into the grids' stream, and
 * the whole batch is captured once into a CUDA graph and replayed while the arguments are
 * unchanged (OFDFT_OPTION_BATCH_GRAPH, OFDFT_OPTION_BATCH_GROUPED of the first grid; by
 * default the first call times grouped and one-launch-per-snapshot enqueueing and keeps the
 * faster).
 * Synchronises once.  Allocates, per distinct batch, the device copy of the evaluations'
 * arguments (a few KB per snapshot, kept with the cached plan; at most 16 plans). */
int ofdft_energy_potential_batched(int n, ofdft_grid *const *grids, const void *const *rho_dev,
                                   const ofdft_functional *f, double *E_out,
                                   void *const *V_dev, double *const *F_out);

/* The plan of the last batched call whose first grid was g: its launch groups (shape and
 * snapshot count each) and the kernel launches of the batch's evaluations; "" before any.
 * The string stays valid until the next batched call with g first (or g's destruction). */
const char *ofdft_batch_report(const ofdft_grid *g);

/* Per-kernel device timing of the evaluation pipeline (tracing aid, results
 * unchanged).  While enabled, every kernel launch of an evaluation is bracketed
 * by two CUDA events on the grid's stream.  ofdft_profile_read synchronises
 * the stream, folds the finished events into running totals and returns, for
 * kernel index idx in [0, 8), its name, launch count and total time in ms
 * (OFDFT_ERR_INVALID_ARG for other idx).  ofdft_profile_reset zeroes the totals. */
int ofdft_profile_enable(ofdft_grid *g, int enable);
int ofdft_profile_reset(ofdft_grid *g);
int ofdft_profile_read(ofdft_grid *g, int idx, const char **name, int *launches, double *total_ms);

/* Options of a grid for tests, diagnostics and callers with special needs.  None
 * changes what is computed (kernel choices agree to floating-point rounding).
 *   OFDFT_OPTION_KERNELS      OFDFT_KERNELS_AUTO (default): size-specialised kernels where
 *                             compiled, their launch shapes picked by the autotuner at the first
 *                             evaluation; OFDFT_KERNELS_GENERIC: the runtime-size kernels only;
 *                             OFDFT_KERNELS_TILE_RECIP: the default configuration of every role
 *                             with the column-tile reciprocal-space kernel in place of the
 *                             persistent register-resident one, no autotuning;
 *                             OFDFT_KERNELS_PER_CHANNEL_ROWS: the same with the rows transformed
 *                             one channel at a time.  A change drops the grid's
 *                             workspaces (synchronising its stream); they are rebuilt on next use.
 *   OFDFT_OPTION_BATCH_GRAPH  1 (default): a batched call whose first grid is g is captured once
 *                             into a CUDA graph and replayed; 0: enqueued directly on every call.
 *   OFDFT_OPTION_BATCH_GROUPED -1 (default): the first batched call of a batch whose first grid
 *                             is g runs it both ways (each once untimed, once timed with CUDA
 *                             events) and later calls with the same arguments use the faster;
 *                             1: each pass launched once per group of snapshots with one launch
 *                             geometry; 0: one launch per snapshot and pass (the same results).
 *   OFDFT_OPTION_WAIT_POLLS   polls of the bounded device-side wait for bulk (TMA) copies before
 *                             it gives up (default 4194304; 0 makes it give up at once, so that
 *                             the evaluation returns OFDFT_ERR_TIMEOUT: a test of that path; the
 *                             kernel still lets its copies land before it exits).
 *   OFDFT_OPTION_ALLOC_CAP    bytes of device memory the grid may allocate from now on (0: no cap);
 *                             an allocation past the cap fails with OFDFT_ERR_OOM.
 *   OFDFT_OPTION_EXACT_SUMS   1: in FP32-mixed evaluations and optimiser dot products every term of
 *                             every energy sum (and every FP32 product of a dot product) is added
 *                             in FP64; 0 (default): terms are summed in FP32 over short runs (at
 *                             most 16 terms: a thread's grid points or tile elements of one
 *                             channel, 8 products of a dot product), the runs in FP64, except the
 *                             density sums of the first kernel, whose per-thread partials are
 *                             added across each warp in FP32.  For tests that bound the error of
 *                             that grouping: evaluations then run the runtime-size kernels (the
 *                             same as OFDFT_KERNELS_GENERIC apart from the sums); slower.  A change
 *                             drops the grid's workspaces like OFDFT_OPTION_KERNELS.
 *   OFDFT_OPTION_PICK_ROWS, _PICK_PENCIL, _PICK_RECIP
 *                             index of the compiled configuration of that kernel role to use
 *                             (the order of ofdft_tuning_report; -1, the default: the autotuner
 *                             picks; an index past the list keeps the role's default).  A change
 *                             drops the grid's workspaces like OFDFT_OPTION_KERNELS.
 * Errors: OFDFT_ERR_INVALID_ARG (NULL, unknown option or value). */
#define OFDFT_OPTION_KERNELS      1
#define OFDFT_OPTION_BATCH_GRAPH  2
#define OFDFT_OPTION_WAIT_POLLS   3
#define OFDFT_OPTION_ALLOC_CAP    4
#define OFDFT_OPTION_PICK_ROWS    5
#define OFDFT_OPTION_PICK_PENCIL  6
#define OFDFT_OPTION_PICK_RECIP   7
#define OFDFT_OPTION_EXACT_SUMS   8
#define OFDFT_OPTION_BATCH_GROUPED 9
#define OFDFT_KERNELS_AUTO              0
#define OFDFT_KERNELS_GENERIC           1
#define OFDFT_KERNELS_PER_CHANNEL_ROWS  2
#define OFDFT_KERNELS_TILE_RECIP        3
int ofdft_set_option(ofdft_grid *g, int option, long long value);

/* The autotuner's record for the grid's workspace of the given precision: for each tuned
 * kernel role (the reciprocal-space pass, the n1 pencils, the n2 rows) every compiled
 * configuration with its measured time per evaluation (CUDA events, whole evaluations of
 * the first call's density) and the one picked; "(cached)" when an earlier grid of the same
 * shape was timed.  Empty before the first evaluation, or when nothing had to be chosen.
 * The string stays valid until the grid's next evaluation or destruction. */
const char *ofdft_tuning_report(const ofdft_grid *g, int precision);

/* Thomas-Fermi energy and potential that allocates no device memory.
 * The paper has no counterpart: this exists for callers that cannot let a
 * library call cudaMalloc -- a host application whose own allocator owns all
 * device memory (a pool sized up front, or memory shared with another runtime),
 * or code that must not pay for cudaMalloc's device-wide synchronisation.
 * Computes E_TF = C_TF sum_r rho^(5/3) dV into E_dev (DEVICE double[1]) and,
 * when V_dev is not NULL, V_TF = (5/3) C_TF rho^(2/3) into V_dev (DEVICE [n],
 * same precision as rho), asynchronously on cuda_stream.  The reduction
 * partials live in a static device array sized for OFDFT_NOALLOC_MAX_POINTS
 * points, held by every GPU that loads the library until the process exits;
 * n above that limit returns OFDFT_ERR_INVALID_ARG without touching the GPU.
 * The first call on each device looks up the array's device address (make it
 * before any stream capture).  All calls share the array, so calls that
 * overlap on the GPU race; order them on one stream.  Matches
 * ofdft_energy_potential with terms = OFDFT_TERM_TF, except on a bad density:
 * NaN, Inf or negative values give E = NaN (the regular call returns
 * OFDFT_ERR_BAD_DENSITY, which needs a synchronisation this call does not make);
 * V is then (5/3) C_TF max(rho, 0)^(2/3) as in the regular call. */
#define OFDFT_NOALLOC_MAX_POINTS 8388608LL   /* 4096 blocks x 2048 points */
int ofdft_tf_energy_potential_noalloc(const void *rho_dev, long long n, double dV, int precision,
                                      double *E_dev, void *V_dev, void *cuda_stream);

/* Measured FP64 fused multiply-add throughput of the current device, GFLOP/s (2 per FMA):
 * 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, three timed launches
 * (CUDA events) after a warm-up on cuda_stream.  A diagnostic: the roof of the FP64
 * evaluation path, whose kernels do all their arithmetic in FP64.  The paper has no
 * counterpart.  Synchronises the stream; allocates 8 bytes of device memory for the call.
 * Errors: OFDFT_ERR_INVALID_ARG (NULL), OFDFT_ERR_OOM, OFDFT_ERR_CUDA. */
int ofdft_fp64_fma_rate(void *cuda_stream, double *gflops);

/* Human-readable text of a status code, and the handle's last error message. */
const char *ofdft_status_string(int status);
const char *ofdft_last_error(const ofdft_grid *g);

/* Library version string. */
const char *ofdft_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OFDFT_H */
