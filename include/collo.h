/*
 * collo.h -- C ABI of the GB300 Radau-collocation interior-point Newton step.
 *
 * The library solves the parameter-estimation problem of the paper's Eq. 1
 * (min Phi(z, theta) s.t. dz/dt = f(z, theta), z(0) = x0, theta_lo <= theta
 * <= theta_hi) by the simultaneous method of Eq. 2: the states are kept as
 * NLP variables on a collocation mesh of N elements with K + 1 interpolation
 * points each, and the ODE becomes the collocation equations of Eq. 3.
 * Two sets of interpolation points, both with tau_0 = 0 (collo_mesh.scheme):
 * right Radau (Radau IIA) roots with K = 3, whose continuity weights in
 * Eq. 2c are b_j = delta_jK, and the paper's own Gauss-Legendre roots with
 * K = 4 (section "Collocation equation with condition independence";
 * "Optimization framework configurations"), whose continuity goes through the
 * extrapolated end value, b_j = l_j(1).  One experiment (N_c = 1 in Eq. 1d /
 * 2e) unless the problem is created with collo_problem_create_conditions.
 *
 * ---- Layouts (all arrays are C-contiguous, 0-based) ----------------------
 *   n species, r reactions, p estimated parameters, N elements, K = 3 or 4,
 *   n_x = n N (K+1) + p primal unknowns, n_c = n N (K+1) constraints.
 *   x      = [ z[N][K+1][n], theta[p] ]       (z[i][j][s]: element i, point j)
 *   lambda = c = [N][K+1][n]:
 *            c[i][0][s]  continuity z[i][0][s] - sum_j b_j z[i-1][j][s]
 *                        (Eq. 2c; Radau: z[i][0][s] - z[i-1][K][s]), or
 *                        the initial condition z[0][0][s] - x0[s]  (Eq. 2d);
 *            c[i][k][s]  collocation sum_j D[k][j] z[i][j][s] - h f_s(z[i][k], theta)
 *                        for k = 1..K  (Eq. 3), h = T / N.
 *   KKT vectors (rhs, solution) are [ x-part (n_x), lambda-part (n_c) ].
 *
 * ---- Memory ----------------------------------------------------------------
 *   Every array argument may be host memory (pageable or pinned) or device
 *   memory of the problem's GPU; the library copies with cudaMemcpyDefault.
 *   Arguments are caller-owned and only read / written during the call.
 *   collo_problem_create deep-copies its inputs; the problem owns all device
 *   memory it allocates and collo_problem_destroy frees it.
 *   Calls on one problem are not thread-safe; distinct problems may be used
 *   concurrently from different threads (each has its own CUDA stream).
 *
 * ---- Errors ----------------------------------------------------------------
 *   Every call returns a collo_status and never aborts; on failure
 *   collo_last_error() returns a thread-local message.
 */
#ifndef COLLO_H
#define COLLO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int collo_status;
enum {
  COLLO_OK = 0,                 /* solved to tol ("0" in the paper's Table 1) */
  COLLO_ACCEPTABLE = 1,         /* solved to the acceptable level ("0A")      */
  COLLO_ERR_INVALID_ARG = -1,   /* bad size, pointer, NaN input               */
  COLLO_ERR_OOM = -2,           /* device allocation failed / over budget     */
  COLLO_ERR_NUMERIC = -3,       /* non-finite values in an iterate            */
  COLLO_ERR_INERTIA = -4,       /* inertia correction failed (delta_w > max)  */
  COLLO_ERR_MAXITER = -5,       /* iteration cap                              */
  COLLO_ERR_TIMEOUT = -6,       /* wall-time cap ("T")                        */
  COLLO_ERR_LINESEARCH = -7,    /* step below alpha_min; no restoration ("R") */
  COLLO_ERR_NOT_FACTORED = -8,  /* collo_kkt_solve before collo_kkt_factor    */
  COLLO_ERR_DEVICE = -9,        /* CUDA runtime error                         */
  COLLO_ERR_NOT_EVALUATED = -10, /* collo_kkt_factor before collo_eval        */
  COLLO_PENDING = 2              /* collo_server_poll: not finished yet        */
};

/* Arithmetic of the KKT factorization and solve. */
enum {
  COLLO_PRECISION_FP64 = 0,  /* everything in FP64 (the plain path)            */
  COLLO_PRECISION_MIXED = 1  /* element blocks and block cyclic reduction in
                                FP32, parameter Schur complement, residuals and
                                refinement in FP64                              */
};

/* Mass-action reaction network: f_s(z, theta) = sum_r nu[s][r] k_r prod_{a in R_r} z_a,
 * nu[s][r] = (#s among products of r) - (#s among reactants of r).
 * Paper Eq. 1b (right-hand side f) and Eq. 1c (z(0) = x0, not theta-dependent). */
typedef struct collo_network {
  int n_species;              /* n >= 1                                        */
  int n_reactions;            /* r >= 1                                        */
  const int* reactants;       /* [r][2] species index or -1; 1 or 2 used slots;
                                 a repeated index means stoichiometry 2         */
  const int* products;        /* [r][2] species index or -1                    */
  const int* param_index;     /* [r] estimated parameter driving k_r, or -1    */
  const double* k_fixed;      /* [r] rate constant used when param_index = -1  */
  int log10_params;           /* 1: k_r = 10^theta_q; 0: k_r = theta_q         */
  const double* x0;           /* [n] initial state                             */
  int n_params;               /* p >= 0                                        */
  const double* theta_lo;     /* [p] lower bounds (finite), Eq. 1a             */
  const double* theta_hi;     /* [p] upper bounds (finite), theta_lo < theta_hi */
} collo_network;

/* Linear observables: observable o measures species species[o]. */
typedef struct collo_observables {
  int n_observables;
  const int* species;         /* [n_observables] */
} collo_observables;

/* Measurements (t_m, observable o_m, y_m, sigma_m), m = 0..M-1.
 * Objective Phi = 1/2 sum_m ((yhat_m - y_m) / sigma_m)^2, Eq. 2a, with
 * yhat_m = sum_j l_j(tau_m) z[i_m][j][s(o_m)]; i_m = ceil(t_m N / T) - 1
 * clamped to [0, N-1], tau_m = t_m N / T - i_m (a boundary time belongs to the
 * left element). */
typedef struct collo_data {
  int n_obs;                  /* M >= 0 */
  const double* t;            /* [M] in [0, T] */
  const int* observable;      /* [M] */
  const double* y;            /* [M] */
  const double* sigma;        /* [M] > 0 */
} collo_data;

/* Interpolation points of an element (collo_mesh.scheme). */
enum {
  COLLO_SCHEME_RADAU = 0,     /* Radau IIA roots, K = 3 */
  COLLO_SCHEME_GAUSS = 1      /* Gauss-Legendre roots, K = 4 (the paper's choice) */
};

/* Uniform collocation mesh, paper "collocation mesh t_ij = t_(i-1)0 + h_i tau_j".
 * A zero-initialised scheme is Radau.  INVALID_ARG for another (scheme, K). */
typedef struct collo_mesh {
  double T;                   /* horizon > 0 */
  int N;                      /* elements >= 1 */
  int K;                      /* collocation points: 3 (Radau) or 4 (Gauss) */
  int scheme;                 /* COLLO_SCHEME_* */
} collo_mesh;

/* Experimental conditions (paper Eq. 1d / 2e: c = 1..N_c, each with its own
 * state profile z^c and initial condition z^c(0), Eq. 1c / 2d; all share
 * theta).  The condition-dependent variables p^c of Eq. 3 are lifted to inputs
 * of the right-hand side: condition c multiplies each rate constant k_r by
 * rate_scale[c][r], so f(z, theta; p^c) keeps one expression per species.
 * Layout: the conditions' meshes one after another, z[c N + i][j][s] for
 * condition c, element i of its N (mesh->N), and c[c N + i][0] is
 * condition c's initial condition when i = 0, else continuity. */
typedef struct collo_conditions {
  int n_conditions;           /* N_c >= 1                                        */
  const double* x0;           /* [N_c][n] initial state of each condition        */
  const double* rate_scale;   /* [N_c][r] finite, > 0 (NULL: all 1)               */
  const int* obs_condition;   /* [M] condition of each measurement (NULL: all 0) */
} collo_conditions;

typedef struct collo_problem_options {
  int precision;              /* COLLO_PRECISION_*, default for factor/solve */
  void* stream;               /* cudaStream_t to run on, or NULL for an own stream */
  int device;                 /* CUDA device ordinal (default 0) */
  int launch_mode;            /* 0: each factorization / solve is one persistent
                                 cooperative kernel (levels separated by a bounded
                                 grid barrier); 1: one kernel launch per level.
                                 Both give bitwise-identical results. */
  int reserved[6];
} collo_problem_options;

typedef struct collo_problem collo_problem;

typedef struct collo_sizes {
  int n, r, p, N, K, M;       /* N: elements of all conditions (N_c x mesh->N) */
  int64_t n_x, n_c;
  int levels;                 /* block cyclic reduction levels */
  int64_t device_bytes;       /* device memory held by the problem */
  int n_conditions;           /* N_c */
  int elements_per_condition; /* mesh->N */
} collo_sizes;

/* Outputs of collo_eval.  Any pointer may be NULL (not wanted).
 * Jacobian of c (Eq. 2c, 2d, 3): the constant parts (D[k][j] I, +-I) are
 * implied; the variable blocks are
 *   jac_z[i][k-1][s][t]   = d c[i][k][s] / d z[i][k][t] - D[k][k] delta_st = -h df_s/dz_t
 *   jac_theta[i][k-1][s][q] = d c[i][k][s] / d theta_q                      = -h df_s/dtheta_q
 * Lagrangian Hessian W = obj_factor grad^2 Phi + sum lambda_c grad^2 c:
 *   hess_zz[i][k-1][s][t], hess_ztheta[i][k-1][s][q]  (node k = 1..K),
 *   hess_thth[q] (the theta-theta block is diagonal for mass action),
 *   hess_obj[i][s][j][l]  = obj_factor d^2 Phi / d z[i][j][s] d z[i][l][s]. */
typedef struct collo_eval_out {
  double* phi;                /* [1]  Phi (without obj_factor) */
  double* c;                  /* [n_c] */
  double* grad;               /* [n_x] obj_factor * grad Phi */
  double* jac_z;              /* [N][K][n][n] */
  double* jac_theta;          /* [N][K][n][p] */
  double* hess_zz;            /* [N][K][n][n] */
  double* hess_ztheta;        /* [N][K][n][p] */
  double* hess_thth;          /* [p] */
  double* hess_obj;           /* [N][n][K+1][K+1] */
} collo_eval_out;

typedef struct collo_inertia {
  int64_t n_pos, n_neg, n_zero;
} collo_inertia;

typedef struct collo_solve_info {
  int refinement_sweeps;      /* iterative-refinement sweeps performed */
  double residual;            /* final ||b - K x||_inf / max(1, ||b||_inf) */
} collo_solve_info;

typedef struct collo_ipm_options {
  double tol;                 /* scaled KKT error, default 1e-6 (paper)            */
  double acceptable_tol;      /* default 1e-4 (paper)                              */
  int acceptable_iter;        /* default 15 (paper)                                */
  int max_iter;               /* default 3000                                      */
  double max_wall_time;       /* seconds, default 3600 (paper's 1 h cap)          */
  int precision;              /* COLLO_PRECISION_*                                 */
  double mixed_mu_switch;     /* MIXED: use FP64 factorization once mu < this
                                 (default 0 = never by mu).  Independently, a MIXED
                                 solve whose refinement fails (relative residual
                                 above 1e-6 after refine_max sweeps, or no longer
                                 halving above it) redoes that step with an FP64
                                 factorization and factors in FP64 for the next
                                 2, 4, 8, ... iterations (doubling per failure)  */
  int refine_max;             /* max iterative-refinement sweeps (default 10)      */
  double refine_tol;          /* stop refining at ||r||/||b|| <= this (1e-10)       */
  int verbose;                /* print an iteration log to stdout                  */
  int reserved[8];
} collo_ipm_options;

typedef struct collo_result {
  collo_status status;
  int iterations;             /* Newton steps taken */
  int factorizations;         /* KKT factorizations (inertia corrections included,
                                 the speculative second candidates too)          */
  int line_search_trials;
  int refinement_sweeps;      /* FP64 iterative-refinement sweeps over all steps */
  int fp64_factorizations;    /* of the factorizations, those in FP64 (MIXED: after a
                                 mu switch or a refinement failure)              */
  double phi;                 /* objective at the final iterate */
  double kkt_error;           /* scaled optimality error E_0 at the final iterate */
  double mu;                  /* final barrier parameter */
  double wall_seconds;
  double* theta;              /* [p]   out (may be NULL) */
  double* x;                  /* [n_x] out (may be NULL) */
  double* lambda;             /* [n_c] out (may be NULL) */
} collo_result;

/* Build a problem: validates and deep-copies the inputs to device memory,
 * precomputes observation elements and interpolation weights.
 * Returns INVALID_ARG on bad sizes, indices, K != 3, non-finite inputs or
 * sigma <= 0; OOM / DEVICE on CUDA failure.  On success *out owns the
 * device memory. */
collo_status collo_problem_create(const collo_network* net, const collo_observables* obs,
                                  const collo_data* data, const collo_mesh* mesh,
                                  const collo_problem_options* opts, collo_problem** out);

/* collo_problem_create for N_c experimental conditions (above); net->x0 is
 * not used (each condition has its own).  conds = NULL or n_conditions = 1
 * with the network's x0 is collo_problem_create.  INVALID_ARG on a bad
 * condition index, non-finite initial states or scales <= 0. */
collo_status collo_problem_create_conditions(const collo_network* net,
                                             const collo_observables* obs, const collo_data* data,
                                             const collo_mesh* mesh, const collo_conditions* conds,
                                             const collo_problem_options* opts,
                                             collo_problem** out);

/* Wait for the problem's stream, free its device memory (and its stream when
 * the library created it).  NULL is a no-op. */
void collo_problem_destroy(collo_problem* prob);

/* Sizes of a created problem (n, r, p, N, K, M, n_x, n_c, the number of
 * cyclic-reduction levels, device bytes held).  INVALID_ARG on NULL. */
collo_status collo_problem_sizes(const collo_problem* prob, collo_sizes* out);

/* The problem's CUDA stream (cudaStream_t), for callers that time or order work. */
void* collo_problem_stream(const collo_problem* prob);

/* Device bytes the problem holds while an interior-point solve in `precision`
 * (COLLO_PRECISION_*) runs on it: its own arrays plus the factorization
 * stores (FP64 and its spare; with MIXED also the FP32 pair) that the solve
 * allocates, counted exactly as they would be allocated.  The server admits
 * by this figure.  INVALID_ARG on NULL or a bad precision. */
collo_status collo_problem_solve_bytes(const collo_problem* prob, int precision, int64_t* bytes);

/* Grid-barrier waits of this problem's own calls (collo_kkt_factor,
 * collo_kkt_solve, collo_ipm_solve; not batches or servers).  The persistent
 * kernels separate the phases of the elimination tree by grid barriers whose
 * waits are bounded: after max_polls polls (0: the default, about 1-2 s) a
 * wait gives up and the call returns COLLO_ERR_TIMEOUT, the paper's status
 * "T", with the device still usable.  unreachable != 0 is a failure-test
 * switch: every barrier then waits for one arrival more than the grid makes,
 * so every wait runs out (results of such a call are meaningless); set it back
 * to 0 for normal use.  INVALID_ARG on NULL or max_polls < 0. */
collo_status collo_problem_set_wait_limit(collo_problem* prob, long long max_polls,
                                          int unreachable);

/* Evaluate objective, constraints, constraint Jacobian and Lagrangian Hessian
 * at (x, lambda) on every (element, node) pair (the paper's SIMD evaluation of
 * Eq. 3 and its first and second derivatives, Introduction and Section
 * "Constructing GPU kernels").  x [n_x], lambda [n_c] (lambda may be NULL:
 * zero multipliers).  The derivatives are also kept inside the problem for
 * the next collo_kkt_factor.  Returns NUMERIC if a value is non-finite. */
collo_status collo_eval(collo_problem* prob, const double* x, const double* lambda,
                        double obj_factor, collo_eval_out* out);

/* collo_eval for callers that cannot allocate device memory while they run:
 * real-time loops that allocate everything before they start, so that no
 * step can fail or stall on an allocation, and processes whose device memory
 * is owned by another runtime or pool.  The paper has no counterpart.  It
 * evaluates what collo_eval evaluates and allocates nothing: no cudaMalloc,
 * cudaFree or allocating library call.
 * x [n_x] and lambda [n_c] (lambda may be NULL) and every pointer of *out
 * (all must be set; hess_thth may be NULL only when p = 0) are DEVICE
 * pointers of the problem's GPU, in the collo_eval layouts; a host pointer
 * (pinned or pageable) or memory of another GPU is refused with
 * COLLO_ERR_INVALID_ARG (checked by cudaPointerGetAttributes, which allocates
 * nothing).  The kernels are queued on `stream` (a cudaStream_t; NULL: the
 * problem's stream) and the call returns without waiting; *out is valid once
 * the stream reaches it.  Because it does not wait, it cannot report
 * non-finite values as collo_eval does (COLLO_ERR_NUMERIC): check *out->phi
 * and the constraint values after synchronising.  The caller's current
 * device is restored before the call returns.
 * Its scratch (per-element partial sums, N (4 + p) + 8 doubles) is a fixed
 * 4 MiB device array of the library (2^19 doubles), held by every GPU that
 * loads the library until the process exits; larger problems are rejected
 * with COLLO_ERR_INVALID_ARG.  The scratch needs no clearing (each call
 * overwrites all of it), but every call shares it: calls whose kernels
 * overlap on the GPU race, so issue them on one stream or order them.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) once, so make that first call before any stream
 * capture begins on that device.  The problem's derivative buffers are not
 * touched, so it does not replace collo_eval before collo_kkt_factor. */
collo_status collo_eval_noalloc(collo_problem* prob, const double* x, const double* lambda,
                                double obj_factor, const collo_eval_out* out, void* stream);

/* Factor the regularised KKT matrix of the most recent collo_eval:
 *   [ W + diag(sigma) + delta_w I    J^T       ]
 *   [ J                            -delta_c I  ]
 * sigma [n_x] (host or device).  Element blocks are condensed onto their
 * interface, the interface chain is reduced by block cyclic reduction, and
 * the p x p parameter Schur complement is factored in FP64; every pivot is a
 * static (state, multiplier) 2x2 block, so no pivoting is data dependent.
 * *out receives the inertia from Sylvester's law (counts of pivot-block
 * eigenvalue signs); the factorization does NOT correct it.
 * precision: COLLO_PRECISION_* or -1 for the problem default.
 * Returns NOT_EVALUATED if collo_eval has not run. */
collo_status collo_kkt_factor(collo_problem* prob, const double* sigma, double delta_w,
                              double delta_c, int precision, collo_inertia* out);

/* Solve K sol = rhs with the last factorization, refining in FP64 with the
 * exact KKT matrix until ||r||_inf <= refine_tol max(1, ||rhs||_inf) or
 * refine_max sweeps.  rhs, sol: [n_x + n_c]; may alias.  info may be NULL.
 * Returns NOT_FACTORED without a factorization. */
collo_status collo_kkt_solve(collo_problem* prob, const double* rhs, double* sol,
                             int refine_max, double refine_tol, collo_solve_info* info);

/* Lifted (relaxed-equality) condensed-space KKT form of the paper's solver
 * configuration (Section "Optimization framework configurations": MadNLP's
 * LiftedKKT; Introduction: a KKT form that factorizes without pivoting).
 * With the equalities relaxed to -r <= c(x) <= r through slacks s, the
 * Newton system in (dx, ds, dlam) is
 *   [ W + diag(sigma_x) + delta_w I   0              J^T ] [dx  ]   [r_x]
 *   [ 0                               diag(d)        -I  ] [ds  ] = [r_s]
 *   [ J                               -I              0  ] [dlam]   [r_c]
 * with d = sigma_s + delta_w; it condenses to the primal matrix
 *   Kc = W + diag(sigma_x) + delta_w I + J^T diag(d) J,
 * which is positive definite exactly when the system has the inertia
 * (n_x + n_c, n_c, 0) an interior-point step needs.
 *
 * collo_lifted_factor factors Kc of the most recent collo_eval by Cholesky
 * without pivoting, FP64 throughout: each element's interior points, then the
 * chain of n x n blocks over the elements' first points by block cyclic
 * reduction, then the p x p parameter block.  sigma_x [n_x] (host or device;
 * NULL: zero), sigma_s [n_c] (host or device, the slacks' barrier diagonal,
 * > 0).  *positive_definite (may be NULL) receives 1 when every pivot was
 * positive, else 0 (then Kc is not positive definite, or not numerically so:
 * raise delta_w).  The first call allocates the factorization's storage
 * (about N (Kn + 2n + p)^2 / 2 doubles); it stays with the problem.  Returns
 * NOT_EVALUATED before collo_eval, INVALID_ARG for a negative or non-finite
 * delta_w, OOM when the storage cannot be allocated. */
collo_status collo_lifted_factor(collo_problem* prob, const double* sigma_x,
                                 const double* sigma_s, double delta_w, int* positive_definite);

/* Solve the system above with the last positive-definite collo_lifted_factor
 * of the current evaluation: dx = Kc^-1 (r_x + J^T (d r_c + r_s)),
 * ds = J dx - r_c, dlam = d ds - r_s, refined in FP64 against the unreduced
 * system until its residual max-norm is <= refine_tol max(1, max|b|) or
 * refine_max sweeps.  r_x, dx: [n_x]; r_s, r_c, ds, dlam: [n_c]; host or
 * device; outputs may not alias inputs.  info may be NULL.  Returns
 * NOT_FACTORED without such a factorization (none, not positive definite, or
 * made before the last evaluation), NUMERIC for a non-finite residual. */
collo_status collo_lifted_solve(collo_problem* prob, const double* r_x, const double* r_s,
                                const double* r_c, double* dx, double* ds, double* dlam,
                                int refine_max, double refine_tol, collo_solve_info* info);

/* Solve the estimation problem in the lifted form: the filter line-search
 * interior-point method of collo_ipm_solve (same constants, barrier update,
 * inertia-correction schedule and line search, Waechter & Biegler 2006) on
 * the relaxed problem -relax <= c(x) <= relax, with the slacks and their bound
 * duals as bounded variables (constraint violation measured as
 * ||c(x) - s||_1), each Newton step from collo_lifted_factor /
 * collo_lifted_solve (FP64, refined to 1e-12 in at most 20 sweeps; a
 * non-positive Cholesky pivot triggers the inertia correction).  States start
 * from the collocation forward sweep at theta0 pushed into its bounds; slacks
 * from c(x0) pushed into [-relax, relax]; multipliers 0, bound duals 1.
 * relax > 0 (1e-8 in the library's reading of the paper's configuration).
 * opts: tol, acceptable_tol, acceptable_iter, max_iter, max_wall_time and
 * verbose are honoured (precision and refinement settings are not: the
 * lifted form is FP64).  The iterate is left in the problem; result as for
 * collo_ipm_solve (fp64_factorizations = factorizations).  Returns the
 * solver status, or INVALID_ARG / OOM / DEVICE before the solve starts. */
collo_status collo_lifted_ipm_solve(collo_problem* prob, const double* theta0, double relax,
                                    const collo_ipm_options* opts, collo_result* result);

/* Defaults: the paper's tolerances (relative KKT error 1e-6, acceptable 1e-4
 * for 15 iterations; Section "Optimization framework configurations"), 3000
 * iterations, a 3600 s wall cap, FP64 precision, refinement to 1e-10 in at
 * most 10 sweeps, no log.  NULL is a no-op. */
void collo_ipm_options_default(collo_ipm_options* opts);

/* Solve the estimation problem from theta0 [p] with the filter line-search
 * primal-dual interior-point method (paper Introduction; Waechter & Biegler
 * 2006), all iterates resident on the device.  States start from a
 * collocation forward sweep at theta0.  opts may be NULL (defaults).
 * result->status is the solver outcome; the return value is the same.  A call
 * that fails before the solve starts (INVALID_ARG, OOM, DEVICE) returns its
 * error and leaves *result unwritten. */
collo_status collo_ipm_solve(collo_problem* prob, const double* theta0,
                             const collo_ipm_options* opts, collo_result* result);

/* Solve `count` independent problems (e.g. the starts of a multistart run,
 * or instances of different networks and sizes) together: every phase of
 * every Newton step runs as one launch over all unfinished problems
 * (element-level grids, one cooperative kernel for all factorizations /
 * solves), and each problem follows exactly the iterates it would follow
 * alone.  probs: [count] problems created on the same device; theta0[i]:
 * [p_i] start of problem i; results[i] as for collo_ipm_solve (its theta / x /
 * lambda pointers are honoured).  The batch runs on the first problem's
 * CUDA stream.  The call returns COLLO_OK when every problem has a final
 * status in results[i].status. */
collo_status collo_batch_solve(collo_problem* const* probs, int count, const double* const* theta0,
                               const collo_ipm_options* opts, collo_result* results);

/* Measurement hook for batches: re-runs one batched phase of `count`
 * problems (phase 1 factorization in `precision` with each problem's last
 * regularisation, 2 solve without refinement, 3 evaluation with derivatives at
 * each problem's current iterate, 4 the element-condensation part of phase 1
 * alone, 5 the rest of phase 1: cyclic reduction and parameter Schur
 * complement, 6 the condensation of element blocks above 124 rows alone,
 * 7 that of the smaller, register-tiled element blocks alone) reps times
 * between CUDA events and returns the average milliseconds per launch.
 * Problems must have been evaluated (e.g. by a solve). */
collo_status collo_batch_time_phase(collo_problem* const* probs, int count, int phase,
                                    int precision, int reps, double* ms_per_launch);

/* Continuous-batching server.  Problems are submitted at any time; each
 * collo_server_step admits waiting problems, in submission order, into free
 * slots while the device memory held by admitted problems stays within
 * budget_bytes (0: no limit), initialises them, advances every admitted
 * problem by one Newton step in batched launches, and retires finished ones.
 * The forward sweeps (initial states) of an admitted group run on a second
 * stream of the server beside the other problems' Newton steps, one block per
 * problem (meanwhile the cooperative kernels of the steps leave that many SMs
 * free); the group takes its first Newton step at the first collo_server_step
 * after its sweeps have finished.  One group sweeps at a time; into an idle
 * server a group is swept on the main stream at once.
 * A problem's footprint is collo_problem_solve_bytes: its factorization
 * stores are allocated when it is admitted and freed (stream-ordered) when it
 * retires, so a retired problem is left unfactored; a problem larger than the
 * whole budget is not run and its result has status COLLO_ERR_OOM.  Their
 * state (x, lambda, bound duals, barrier parameter, filter) stays on the
 * device between steps.  A problem may be submitted again once its previous
 * ticket is done.
 * collo_server_poll returns COLLO_PENDING until the ticket's solve ended,
 * then COLLO_OK with the result (theta copied if result->theta is set).
 * Submitted problems must stay alive until polled as done. */
typedef struct collo_server collo_server;
/* create: max_slots >= 1 slots on `device`, opts as for collo_ipm_solve (NULL:
 * defaults); INVALID_ARG / DEVICE / OOM.  submit: theta0 [p] is copied;
 * INVALID_ARG on NULL arguments.  step: INVALID_ARG on NULL; OOM when an
 * admitted problem's storage cannot be allocated; DEVICE on a CUDA error (a
 * solve's own outcome goes to its result, not to the step's status);
 * n_active / n_waiting report the slots in use and the queue. */
collo_status collo_server_create(int max_slots, int64_t budget_bytes,
                                 const collo_ipm_options* opts, int device, collo_server** out);
collo_status collo_server_submit(collo_server* server, collo_problem* prob, const double* theta0,
                                 long long* ticket);
collo_status collo_server_step(collo_server* server, int* n_active, int* n_waiting);
collo_status collo_server_poll(collo_server* server, long long ticket, collo_result* result);
/* Admission grouping: collo_server_step admits waiting problems only when at
 * least min_free_slots slots are free (or no slot is busy) and no earlier
 * group is still sweeping; default 1.  Each group's forward sweeps take as
 * long as its slowest problem's, so grouping trades idle slots for fewer
 * rounds.  INVALID_ARG if < 1. */
collo_status collo_server_set_admission(collo_server* server, int min_free_slots);
/* The CUDA stream (cudaStream_t) the server's Newton steps are queued on
 * (the forward sweeps of admitted groups run on a second stream of its own). */
void* collo_server_stream(collo_server* server);
/* Device bytes held by the admitted problems now and the most held at once
 * since the server was created (either pointer may be NULL). */
collo_status collo_server_memory(collo_server* server, int64_t* active_bytes, int64_t* peak_bytes);
/* Totals since the server was created: Newton steps taken by all jobs, jobs
 * that reached a final status, and of those the ones solved (COLLO_OK or
 * COLLO_ACCEPTABLE).  Any pointer may be NULL. */
collo_status collo_server_counters(collo_server* server, long long* newton_steps,
                                   long long* finished, long long* converged);

/* Measurement hook: with the environment variable COLLO_PROFILE=1 set before
 * the first solve, the IPM driver synchronises its stream at each phase
 * boundary and accumulates host wall milliseconds per phase (0 derivatives
 * and optimality measures, 1 right-hand sides, 2 factorizations with inertia
 * correction, 3 solves with refinement, 4 step sizes, 5 line search,
 * 6 step update, 7 server admission) and the rounds of phases 2, 3, 5 and 7.
 * Copies min(n, 8) entries into ms / rounds (either may be NULL), zeroes the
 * totals if reset != 0, and returns 8 when profiling is on, else 0. */
int collo_phase_profile(double* ms, long long* rounds, int n, int reset);
void collo_server_destroy(collo_server* server);

/* ---- Mesh refinement (paper Section "Static collocation mesh limitations"
 * and Conclusion: a mesh fixed at the nominal parameters may be too coarse
 * near the optimum; refine the interval width in an outer loop).  The loop
 * here is batched on the GPU. */

/* A new problem with coarse's network, observables and data on a uniform
 * mesh of N elements (same horizon and collocation scheme).  The caller owns *out. */
collo_status collo_problem_create_refined(const collo_problem* coarse, int N,
                                          collo_problem** out);

/* Collocation defect of x [n_x] (host or device): for element i, the
 * collocation polynomial z_i(tau) = sum_j l_j(tau) z_ij leaves at the
 * midpoints tau*_m = (tau_(m-1) + tau_m) / 2, m = 1..K, of consecutive
 * interpolation points the residual d_ims = sum_j l_j'(tau*_m) z_ijs
 * - h f_s(z_i(tau*_m), theta) (h times the ODE residual); per_element [N]
 * (host or device, may be NULL) receives max_{m,s} |d_ims| and *max_defect
 * (may be NULL) the maximum over elements. */
collo_status collo_defect(collo_problem* prob, const double* x, double* per_element,
                          double* max_defect);

/* Interpolates the coarse solution x_coarse [n_x of coarse] onto fine's mesh:
 * the states at fine's interpolation points t = (i + tau_j) h_f from the
 * coarse collocation polynomial of the element holding t (a time on a coarse
 * element boundary from the left element, t = 0 from the first), theta
 * copied; x_fine [n_x of fine].  Both problems must differ only in their
 * meshes, with fine at least half as many elements as coarse. */
collo_status collo_interpolate(collo_problem* coarse, const double* x_coarse,
                               collo_problem* fine, double* x_fine);

/* Warm start: the next interior-point solve of prob (collo_ipm_solve,
 * collo_batch_solve or the server) starts from x [n_x] (states and theta,
 * theta pushed into its bounds as a theta0 would be) and lambda [n_c] (NULL:
 * zero) instead of the forward sweep at theta0, whose theta0 argument is then
 * ignored; bound duals and the barrier parameter start as usual.  The start
 * is consumed by that solve; x = NULL clears it. */
collo_status collo_problem_set_start(collo_problem* prob, const double* x, const double* lambda);

/* Batched refinement: solves probs from theta0 as collo_batch_solve does;
 * then, up to max_levels times, every problem whose last solve ended in
 * COLLO_OK or COLLO_ACCEPTABLE with a defect (collo_defect of its solution)
 * above defect_tol is re-created on twice as many elements (at most
 * max_elements; 0: no limit), warm-started from its interpolated solution,
 * and all of them are solved again together.  finals[i] is the problem of
 * problem i's last solve: probs[i] or a problem this call created, which the
 * caller then destroys (intermediate ones are destroyed here); results[i] its
 * result (theta honoured at every level, x and lambda only when no refinement
 * happened); levels[i] how many times it was refined. */
collo_status collo_refine_solve(collo_problem* const* probs, int count, const double* const* theta0,
                                const collo_ipm_options* opts, double defect_tol, int max_levels,
                                int max_elements, collo_problem** finals, collo_result* results,
                                int* levels);

/* Collocation forward sweep at theta (the IPM's initial states): writes
 * z [N][K+1][n] into x_out [n_x] (theta copied into its tail).  Returns the
 * number of elements whose Newton iteration failed in *failures. */
collo_status collo_initial_states(collo_problem* prob, const double* theta, double* x_out,
                                  int* failures);

/* Measurement hooks (used by the benchmark's roofline report).
 * collo_time_phase re-launches one phase reps times between CUDA events on
 * the problem's stream and returns the average milliseconds per launch:
 *   phase 0: element condensation kernel alone (needs collo_eval; uses the
 *            sigma and regularisation of the last collo_kkt_factor), leaves
 *            the problem unfactored;
 *   phase 1: whole factorization (element condensation, cyclic reduction,
 *            parameter Schur complement);
 *   phase 2: one solve without refinement (needs a factorization in
 *            `precision`), on the last right-hand side;
 *   phase 3: evaluation with derivatives at the solver's current iterate;
 *   phase 4: collocation forward sweep at the current theta;
 *   phase 5: the lifted factorization's element kernel alone, phase 6 all of
 *            its kernels, phase 7 one lifted solve without refinement on the
 *            last right-hand side of collo_lifted_solve (each needs a
 *            positive-definite collo_lifted_factor of the current evaluation
 *            and leaves it intact; `precision` is ignored: FP64).
 * Returns NOT_EVALUATED / NOT_FACTORED when its input state is missing. */
collo_status collo_time_phase(collo_problem* prob, int phase, int precision, int reps,
                              double* ms_per_launch);

/* Launch schedule of the batched kernels, process-wide (the paper has no
 * counterpart; it sets how the work is laid out on the GPU, not what is
 * computed).  Results are bitwise reproducible for a fixed schedule;
 * slab_pairs changes the rounding order of element and reduction blocks held
 * in the global slab.  Change it only while no solve is running. */
typedef struct collo_schedule {
  int big_threads;            /* threads per block of the condensation of element
                                 blocks above 124 rows: 512 (one block per SM, the
                                 default) or 256 (two blocks per SM where their
                                 shared memory fits) */
  int slab_pairs;             /* pairs per panel of blocks whose packed triangle is
                                 held in the global slab: 8 or 16 (default 16) */
  int solve_top_blocks;       /* the batched solve runs the reduction levels with
                                 at most this many blocks per instance in one CUDA
                                 block per instance (default 8) */
  int solve_elems_per_block;  /* elements per 8-warp block of the solve's grid
                                 (default 8) */
  int reserved[4];
} collo_schedule;
collo_status collo_get_schedule(collo_schedule* out);
/* INVALID_ARG when a field is outside the values above (1..4096 for
 * solve_top_blocks, 1..1024 for solve_elems_per_block). */
collo_status collo_set_schedule(const collo_schedule* s);
/* Autotuner: on `count` evaluated problems (as for collo_batch_time_phase),
 * times the large-element condensation (phase 6) for each (big_threads,
 * slab_pairs) and then the solve (phase 2) for each (solve_top_blocks in
 * 2..32, solve_elems_per_block in 4..32), reps launches each between CUDA
 * events, keeps the fastest of each, sets it as the schedule and returns it
 * in *best, with the two phases' milliseconds per launch under the schedule
 * it started from and under the chosen one (either pointer may be NULL).  On
 * error the schedule it started from is restored. */
collo_status collo_autotune(collo_problem* const* probs, int count, int precision, int reps,
                            collo_schedule* best, double* ms_before, double* ms_after);

/* Fused multiply-add throughput of the current device in TFLOP/s (2 flops
 * per FMA), for precision COLLO_PRECISION_FP64 (DFMA) or _MIXED (FFMA):
 * the arithmetic roof of the element factorization.  Allocates a small
 * buffer and runs about a millisecond. */
collo_status collo_alu_peak(int precision, double* tflops);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all problems, all threads); a monotone counter for launch accounting. */
long long collo_launch_count(void);

const char* collo_last_error(void);

/* Library version string. */
const char* collo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* COLLO_H */
