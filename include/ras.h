/*
 * ras.h - C ABI of the GB300 multilevel restricted-additive-Schwarz
 * Newton-Krylov solver for compressible gas flow with the Peng-Robinson EOS
 * (Li, Yang, Yang, arXiv 2007.13966).
 *
 * Conventions (every entry point):
 *  - Arrays are DEVICE pointers owned by the caller unless stated otherwise;
 *    FP64; cell n = i + nx*(j + ny*k) (x fastest). The library never frees
 *    them and never keeps them past the call, except where a create function
 *    says it copies them.
 *  - Handles (ras_problem, ras_precond) own their device workspaces; they are
 *    created by *_create / ras_setup and released by *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream unless they return a convergence
 *    result (gmres_solve, newton_step, ras_factor's pivot check), which
 *    synchronise it.
 *  - Return value: RAS_OK (0); > 0 did not converge; < 0 error. No exception
 *    crosses the ABI. ras_status_string() describes a code.
 */
#ifndef RAS_H
#define RAS_H

#ifdef __cplusplus
extern "C" {
#endif

enum ras_status {
    RAS_OK = 0,
    RAS_GMRES_MAXIT = 1,       /* linear solve hit maxit without Eq. equ:linear_stop */
    RAS_NEWTON_MAXIT = 2,      /* Newton hit maxit without Eq. equ:nonlinear_stop   */
    RAS_LINESEARCH_FAIL = 3,   /* step length fell below ls_min_lambda               */
    RAS_EINVAL = -1,           /* invalid argument (NULL, size, option out of range) */
    RAS_ECUDA = -2,            /* a CUDA runtime call failed                         */
    RAS_ENOMEM = -3,           /* device allocation failed                           */
    RAS_ENAN = -4,             /* NaN/Inf in a norm                                  */
    RAS_EZEROPIVOT = -5,       /* zero or non-finite ILU / LU pivot                  */
    RAS_ENOROOT = -6,          /* no admissible EOS root                             */
    RAS_ETIMEOUT = -7          /* a bounded device wait gave up                      */
};

/* Structured cell-centred grid (Section 2; Fig. 1). nz = 1 for 2D
 * (the thickness hz is then the cell depth). Spacing in metres. */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    double gz;             /* gravitational acceleration (m/s^2) along the z axis, depth
                              increasing with the z index (Eq. gover_sys's rho g grad h
                              term, rho = pW/(ZRT) of Eq. equ:density, arithmetic mean
                              over a face); 0 = no gravity. Fixed-pressure connections
                              are at their cell's depth. */
    int upwind;            /* face mobility: 0 = arithmetic mean of the two cells (default);
                              1 = the upstream cell's, by the sign of the face potential
                              (fixed-pressure connections alike; the density of the
                              gravity term stays the mean) */
    int conservative;      /* accumulation term: 0 = Eq. gover_sys's V phi c(p) D_t p
                              (default); 1 = the conservative form V phi D_t (p/Z) of the
                              time derivative of phi rho (Eq. mass conservation / (W/RT)),
                              with the same BDF weights on p/Z at the three levels;
                              Jacobian V phi c(p) dD_t/dp */
} ras_grid;

/* Fluid (Section 2, Eq. attrfactor and the m(omega), omega(T_br) fits;
 * constants of Section 4). SI units: K, Pa, J/(mol K), kg/mol, Pa s.
 * If omega_from_Tb != 0, omega is computed from Tb by the Section 2
 * correlation; otherwise `omega` is used. */
typedef struct {
    double Tc, pc, omega, Tb;
    int omega_from_Tb;
    double T, R, W, mu;
} ras_eos;

/* Rock and fixed-pressure connections. kx, ky, kz (m^2) and phi are device
 * arrays of N cells. Connections (wells and Dirichlet faces) join cell
 * conn_cell[q] to pressure conn_p[q] (Pa) through geometric transmissibility
 * conn_T[q] (m^3); they must be sorted by cell (several per cell allowed).
 * conn_* are device arrays of nconn entries. ras_problem_create copies all of
 * it; the caller may free these arrays afterwards. */
typedef struct {
    const double *kx, *ky, *kz, *phi;
    int nconn;
    const int *conn_cell;
    const double *conn_p, *conn_T;
    const double *rate_Q;  /* NULL, or device [N]: fixed injection rates (the paper's Case-2
                              fixed injection velocity), the Darcy volume rate Q_n (m^3/s,
                              positive into the cell) through boundary faces of cell n;
                              the injected gas carries the cell's own p/Z:
                              F_n -= (p_n/Z_n) Q_n, dF_n/dp_n -= c(p_n) Q_n */
} ras_rock;

/* Jacobian (or any 7-point operator) as seven device arrays of N entries:
 * c[0] centre, c[1] -x, c[2] +x, c[3] -y, c[4] +y, c[5] -z, c[6] +z;
 * c[s][n] = dF_n / dp_{neighbour s of n}, zero where the neighbour is absent. */
typedef struct {
    double *c[7];
} ras_stencil;

/* Schwarz preconditioner options (Sections 3.1-3.2). */
typedef struct {
    int px, py, pz;        /* subdomain counts per axis (Omega_i, Fig. 1)             */
    int overlap;           /* delta >= 0 (cells per side, cut at the boundary)       */
    int ras_type;          /* fine-level combination of the subdomain solves:
                              0 = AS, Eq. equ:as-class (sum over overlapped boxes),
                              1 = left-RAS, Eq. equ:as-left (owned cells, default),
                              2 = right-RAS, Eq. equ:as-right (owned-cell input,
                              sum over overlapped boxes); 0 and 2 sum the boxes
                              covering a cell in ascending box order            */
    int ilu_k;             /* level of fill k of the ILU(k) subdomain solver (natural
                              order in each box, no pivoting; Section 4's ILU(k)
                              variants): 0 = ILU(0); 1, 2 = ILU(1), ILU(2) (the fill
                              of larger k leaves the 5x5x5 neighbourhood:
                              RAS_EINVAL); k > 0 requires ras_type = 1           */
    int factor_prec;       /* 64 = FP64 factors and solves; 32 = FP32 factors, FP32
                              solves; 16 = BF16-stored factors, FP32 solves          */
    int nlevels;           /* 1 = one-level; 2 = two-level (Eq. equ:v-cycle);
                              3 = three-level V-cycle (Algorithm 1, mu = nu = 1)     */
    int coarsen[3];        /* coarse:fine ratio per axis of each coarsening (Table 7:
                              2 to 16). A coarse cell's interpolation support is
                              about 2 r fine cells per axis; the Galerkin product
                              stages it in shared memory whole or in slabs of
                              z-planes, and set-up returns RAS_EINVAL when even one
                              x-y plane of it does not fit (x and y ratios beyond
                              about 25 with FP64 coarse arithmetic, 31 with FP32)
                              or its x extent reaches 256 cells (x ratio > 127)   */
    int interp_order;      /* 2 = (bi/tri)linear, Eq. equ:inter-second; 1 = nearest
                              coarse centre, Eq. equ:inter-frist (order 3 couples
                              coarse cells up to four apart, beyond the 125-point
                              coarse operator: not supported)                     */
    int mlevel_type;       /* 0 = V-cycle, 1 = left-Kaskade, 2 = right-Kaskade,
                              3 = additive, 4 = coarse-only (Eqs. equ:v-cycle ..
                              equ:coarse-level)                                      */
    int coarse_prec;       /* 64 or 32: precision of the dense block coarse LU        */
    int coarse_overlap;    /* nlevels = 3: overlap delta_c of the middle-level Schwarz
                              smoother (px x py x pz subdomains, ILU(0) on the
                              Galerkin operator's nonzero pattern, factor_prec);
                              coarse_solver = 1: overlap of the coarse-grid
                              Schwarz preconditioner                                */
    int coarse_solver;     /* nlevels = 2: 0 = exact dense block LU; 1 = FGMRES(30)
                              on the Galerkin coarse operator preconditioned by
                              left-RAS(ILU(0)) on the coarse grid (min(p, coarse
                              cells) subdomains per axis, overlap coarse_overlap,
                              coarse_prec factors), stopped at coarse_rtol
                              (Remark 2, Section 4: 0.2)                          */
    double coarse_rtol;    /* relative tolerance of the coarse FGMRES (> 0)           */
} ras_opts;

typedef struct {
    int restart;           /* GMRES(m) restart length (30 in Section 4)              */
    int maxit;             /* total iteration cap                                     */
    double rtol, atol;     /* Eq. equ:linear_stop, read as max(rtol ||b||, atol)      */
} ras_krylov_opts;

typedef struct {
    int iters;             /* FGMRES iterations done                                  */
    int converged;         /* 1 if the stop test was met                              */
    double r0, rfinal;     /* ||b|| and the final true residual norm                  */
    double *history;       /* HOST buffer (may be NULL): residual estimates, one per
                              iteration plus the initial and each restart's value    */
    int history_cap;       /* capacity of history                                     */
    int history_len;       /* entries written                                         */
} ras_krylov_stats;

typedef struct {
    int maxit;             /* Newton iteration cap (50)                               */
    double rtol, atol;     /* Eq. equ:nonlinear_stop: eps_r, eps_a                    */
    double ls_alpha;       /* sufficient-decrease alpha (1e-4, Section 3)             */
    double ls_min_lambda;  /* smallest step length before failure (1e-8)              */
    ras_krylov_opts lin;   /* inner FGMRES options                                    */
} ras_newton_opts;

typedef struct {
    int iters;             /* Newton iterations                                       */
    int lin_iters;         /* FGMRES iterations summed over the Newton iterations     */
    int residual_evals;    /* residual evaluations (incl. line-search trials)         */
    double f0, ffinal;     /* ||F(X^0)|| and the final ||F||                          */
    double *fhistory;      /* HOST buffer (may be NULL): ||F|| after each iteration   */
    int fhistory_cap, fhistory_len;
    int *lin_history;      /* HOST buffer (may be NULL): FGMRES iterations per Newton */
    int lin_history_cap;
    double *lambdas;       /* HOST buffer (may be NULL): accepted step lengths        */
} ras_newton_stats;

typedef struct ras_problem ras_problem;
typedef struct ras_precond ras_precond;

/* Creates the discrete problem: computes the PR constants a, b
 * (Eq. attrfactor), the harmonic-average face transmissibilities of the
 * two-point flux scheme (Section 2, CCFD) and copies phi and the connections.
 * The grid must have nx, ny >= 1, nz >= 1 and positive spacings; N = nx*ny*nz
 * must fit in int32. Returns RAS_EINVAL on bad arguments, RAS_ENOROOT if a
 * fixed connection pressure has no admissible root (see residual_eval). */
int ras_problem_create(const ras_grid *grid, const ras_eos *eos, const ras_rock *rock,
                       void *stream, ras_problem **out);
void ras_problem_destroy(ras_problem *prob);

/* Residual of Eq. implicit-method-bdf1 (bdf_order = 1) or
 * Eq. implicit-method-bdf2 (bdf_order = 2) integrated over each cell:
 *   F_n = V phi_n c(p_n) D_t p_n + sum_faces T_f mbar_f (p_n - p_m)
 *         + sum_conns T_q mbar_q (p_n - p_q),
 * c(p) = (p/Z)(1/p - Z'/Z) (Eq. gover_sys), m = p/(mu Z), mbar the arithmetic
 * mean of the two sides; Z is the largest real root of Eq. equ:PR, Z' the
 * closed form under Eq. gover_sys. p, p_l, p_lm1: device [N] (p_lm1 unused
 * for bdf_order 1). F: device [N] output. J: if non-NULL, its seven arrays
 * (device [N] each) receive the exact Jacobian. normF: if non-NULL, HOST
 * pointer that receives ||F||_2 (the call then synchronises the stream).
 * Root selection (the paper defers it to its references): Z is the largest
 * real root, chosen in FP64; a cell whose root is not admissible (Z not finite,
 * Z <= B, or a multiple root where dZ/dp is unbounded) gets F_n = NaN and sets
 * the problem's no-root flag, which this call reports as RAS_ENOROOT when
 * normF is requested (the flag is then cleared), else the next synchronising
 * call on the problem does. */
int residual_eval(ras_problem *prob, const double *p, const double *p_l, const double *p_lm1,
                  double dt, int bdf_order, double *F, const ras_stencil *J, double *normF,
                  void *stream);

/* y = J x for a 7-point operator (the Jacobian-vector product of the Krylov
 * solve, Eq. jacobian). x, y: device [N], must not alias; J's seven arrays are
 * read, not kept. Asynchronous on `stream`. RAS_EINVAL for a NULL pointer or
 * array, or x == y. */
int ras_stencil_matvec(const ras_problem *prob, const ras_stencil *J, const double *x,
                       double *y, void *stream);

/* Symbolic set-up, once per grid: the P_x x P_y x P_z partition with overlap
 * (Section 3.1, Fig. 1), per-subdomain boxes, the wavefront (level) schedule of
 * the natural-order ILU(0) triangular solves, factor storage, and for
 * nlevels = 2 the interpolation (Eq. equ:inter-second), the coarse grid and the
 * dense block-LU layout; for nlevels = 3 also the middle grid (fine grid
 * coarsened by coarsen[]) with its own partition (overlap coarse_overlap) and
 * the coarsest grid (middle grid coarsened by coarsen[]) with its block-LU
 * layout. Returns RAS_EINVAL for unsupported options (nlevels = 3 requires
 * mlevel_type = 0). */
int ras_setup(const ras_problem *prob, const ras_opts *opts, ras_precond **out);
void ras_precond_destroy(ras_precond *pc);

/* Numeric factorisation, once per Newton iteration: A_i = R_i^delta J
 * (R_i^delta)^T (Eq. equ:as-class), ILU(0) without pivoting in natural order
 * inside each overlapped subdomain, stored at factor_prec; for nlevels = 2 also
 * the Galerkin coarse operator R J P (R = P^T) and its dense block LU; for
 * nlevels = 3 the middle operator A_1 = P_1^T J P_1 (FP64), the ILU(0) factors
 * of its subdomains (on A_1's nonzero pattern) and the block LU of
 * A_0 = P_0^T A_1 P_0. The multilevel preconditioners also keep a private copy
 * of J for the fine-level residuals, so J may be freed after the call.
 * Synchronises the stream to check pivots: RAS_EZEROPIVOT on a zero or
 * non-finite pivot. */
int ras_factor(ras_precond *pc, const ras_stencil *J, void *stream);

/* z = M^{-1} r. One level: left-RAS, Eq. equ:as-left,
 *   z = sum_i (R_i^0)^T (L_i U_i)^{-1} R_i^delta r
 * (or AS / right-RAS by ras_type, which then also serves as M in the
 * multilevel combinations).
 * Two levels: the configured two-level combination (Eq. equ:v-cycle by
 * default). Three levels: Algorithm 1 with one RAS-Richardson pre- and
 * post-smoothing step on the fine and middle levels and the exact block-LU
 * solve on the coarsest. r, z: device [N], must not alias. Requires a prior
 * ras_factor. */
int ras_apply(ras_precond *pc, const double *r, double *z, void *stream);

/* Right-preconditioned flexible GMRES(m) (Section 3, Eq. jacobian, Remark 2)
 * for J x = b from x = 0, classical Gram-Schmidt applied twice, Givens
 * rotations; stops when the residual estimate satisfies
 * ||b - J x|| <= max(rtol ||b||, atol). b, x: device [N]. stats may be NULL.
 * Returns RAS_OK or RAS_GMRES_MAXIT (x then holds the last iterate). */
int gmres_solve(ras_problem *prob, const ras_stencil *J, ras_precond *pc, const double *b,
                double *x, const ras_krylov_opts *opts, ras_krylov_stats *stats, void *stream);

/* One implicit time step (Sections 2-3): inexact Newton X^{k+1} = X^k +
 * lambda s^k (Eq. newton_iterate) from X^0 = p (normally p_l), J s = -F by
 * gmres_solve with pc refactored every iteration, cubic backtracking line
 * search with sufficient decrease ||F(X + lambda s)|| <= (1 - alpha lambda)||F||,
 * stop on Eq. equ:nonlinear_stop. p: device [N], in: initial guess, out:
 * p^{l+1}. stats may be NULL. A starting state with a cell without an
 * admissible EOS root returns RAS_ENOROOT; a line-search trial state without
 * one is treated as a failed trial (the step is shortened). */
int newton_step(ras_problem *prob, ras_precond *pc, double *p, const double *p_l,
                const double *p_lm1, double dt, int bdf_order, const ras_newton_opts *opts,
                ras_newton_stats *stats, void *stream);

/* ------------------------------------------------------------------------
 * Batches of independent reservoirs (the paper treats one reservoir; several
 * unrelated reservoirs solved together on one GPU are this library's
 * extension). A batch references n existing problem handles and their
 * preconditioners -- one-level left-RAS (nlevels 1, ras_type 1, ilu_k 0), all
 * with the same factor_prec, each problem in the batch once -- and owns one set
 * of Krylov vectors for all of them (the reservoirs' vectors concatenated,
 * (2 restart + 1) x sum of N doubles plus five more vectors). Every FGMRES
 * operation runs for all reservoirs in one launch: the subdomain solves of all
 * reservoirs' boxes, their 7-point operators, the Arnoldi dot products and
 * updates; each reservoir keeps its own Krylov scalars, stop test and Newton
 * line search, evaluated on the host after one synchronisation per Arnoldi step
 * for the whole batch. A reservoir whose solve has finished does no further
 * work. Results equal the single-reservoir routines' up to the order of the
 * floating-point sums (each reduction is still deterministic). The handles must
 * outlive the batch; a batch must not be used concurrently from several host
 * threads. All pointer arrays below are HOST arrays of n entries (the vectors
 * they point to are device vectors of each reservoir's N). */
typedef struct ras_batch ras_batch;

/* Returns RAS_EINVAL if n < 1, a pointer is NULL, a preconditioner is not of the
 * kind above or does not belong to its problem, a problem appears twice, or the
 * total padded length exceeds 2^31 - 1; RAS_ENOMEM if device memory runs out. */
int ras_batch_create(int n, ras_problem *const *problems, ras_precond *const *preconds,
                     ras_batch **out);
void ras_batch_destroy(ras_batch *batch);

/* FGMRES on every reservoir: J[i] x[i] = rhs[i] right-preconditioned by the
 * reservoir's current factors (ras_factor first), the single-reservoir
 * gmres_solve's iteration per reservoir. J: host array of n stencils (device
 * coefficient arrays); rhs, x: host arrays of n device pointers; stats: host
 * array of n (or NULL). Returns RAS_OK, or RAS_GMRES_MAXIT if some reservoir
 * stopped at maxit (its stats say which). */
int ras_batch_gmres(ras_batch *batch, const ras_stencil *J, const double *const *rhs,
                    double *const *x, const ras_krylov_opts *opts, ras_krylov_stats *stats,
                    void *stream);

/* One implicit time step of every reservoir: newton_step's iteration per
 * reservoir (factor, batched FGMRES, cubic backtracking), the reservoirs'
 * residual evaluations launched together before each synchronisation.
 * p[i]: device [N_i], in: initial guess, out: p^{l+1}; p_l, p_lm1 (bdf_order 2):
 * host arrays of device pointers; dt: host array of n step sizes; stats: host
 * array of n (or NULL). Returns RAS_OK, or the status of the first reservoir (in
 * batch order) that did not meet its Newton test. */
int ras_batch_newton_step(ras_batch *batch, double *const *p, const double *const *p_l,
                          const double *const *p_lm1, const double *dt, int bdf_order,
                          const ras_newton_opts *opts, ras_newton_stats *stats, void *stream);

/* Human-readable description of a status code (static storage). */
const char *ras_status_string(int status);

/* ||x||_2 of a device vector, written to the DEVICE scalar *result, without
 * allocating any memory. The paper has no counterpart: this is library
 * plumbing for callers that cannot allocate device memory at call time (a
 * framework that owns all device memory through its own pool, where a raw
 * cudaMalloc behind its back fragments memory or breaks its budget; a
 * latency-critical loop that cannot afford an allocation, its implicit
 * synchronisation or its failure). It computes the same deterministic
 * reduction as the norm of residual_eval (bit for bit), with its partial sums
 * (608 doubles, 4.75 KB) in a static device array inside the library that
 * every device which loads the library keeps until the process exits.
 * x: device [n], 0 <= n <= 2^31 - 1 (larger n or n < 0: RAS_EINVAL, checked
 * before any CUDA call). Asynchronous on `stream`. The first call in a
 * device's context looks up that array's device address (once per device
 * and context, with the device current; a context created after
 * cudaDeviceReset looks it up again); make that first call before any
 * stream capture. All calls share the one array: calls that overlap on the
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller. Nothing in the array needs clearing: every call
 * overwrites all of it before reading it. */
int ras_norm2_noalloc(const double *x, long long n, double *result, void *stream);

/* ----------------------------------------------------------------------------
 * Discrete adjoint of the time loop. The paper computes no sensitivities;
 * these calls give the pieces of the adjoint of the residual of Section 2
 * (Eq. gover_sys with Eqs. implicit-method-bdf1 / -bdf2) with respect to
 * per-cell log-permeability multipliers theta (k_{a,i} = k0_{a,i} exp(theta_i)
 * on every axis; the transmissibility of a cell's fixed-pressure connections
 * scales with its permeability). For a time loop with objective Phi(p^1..p^L):
 *   J_l^T lambda^l = -dPhi/dp^l + (2/dt) s(p^{l+1}) lambda^{l+1}
 *                    - (1/(2 dt)) s(p^{l+2}) lambda^{l+2},
 *   dPhi/dtheta = sum_l (dF^l/dtheta)^T lambda^l,
 * with s(p) = V phi c(p) and the history terms of the BDF2 steps.
 * All arrays are device [N] FP64 unless stated; asynchronous on `stream`.
 * ------------------------------------------------------------------------- */

/* JT = J^T as a 7-point operator: JT->c[s][n] = J->c[opp(s)][neighbour s of n]
 * (e.g. JT -x of cell n = J +x of cell n - 1), zero where the neighbour is
 * absent. J and JT must not share arrays (RAS_EINVAL). */
int ras_stencil_transpose(const ras_problem *prob, const ras_stencil *J, ras_stencil *JT,
                          void *stream);

/* rhs = -dphi + c1 s(p1) lam1 + c2 s(p2) lam2, s(p) = V phi c(p) per cell; a
 * term whose state (p1 or p2) is NULL is absent, dphi NULL reads as 0. In the
 * backward sweep over a BDF2 time loop (Eq. implicit-method-bdf2) c1 = 2/dt and
 * c2 = -1/(2 dt), the weights with which p^l enters the residuals of steps l+1
 * and l+2; p1, p2 are the states where those residuals take s (p^{l+1}, p^{l+2},
 * or p^l itself in the conservative form). */
int ras_adjoint_rhs(const ras_problem *prob, const double *dphi, const double *p1,
                    const double *lam1, double c1, const double *p2, const double *lam2,
                    double c2, double *rhs, void *stream);

/* grad += (dF/dtheta)^T lam at the state p: per face (lam_i - lam_j) T mbar
 * (p_i - p_j) k_j / (k_i + k_j) to cell i (and symmetrically to j), per
 * connection lam_i T_c mbar (p_i - p_c). Uses the problem's per-cell mobility
 * scratch (do not overlap with residual_eval of the same problem on another
 * stream). */
int ras_grad_logk(ras_problem *prob, const double *p, const double *lam, double *grad,
                  void *stream);

/* Text of the last CUDA runtime failure seen by the library (static storage,
 * empty if none); diagnostic only. */
const char *ras_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded. */
long long ras_kernel_launches(void);

/* Per-kernel-class device timing of ras_apply's subdomain-solve kernel:
 * when enabled, every launch is bracketed by CUDA events on its stream;
 * ras_timing_read returns the summed milliseconds and the launch count since
 * the last reset (synchronises the events). */
int ras_timing_enable(ras_precond *pc, int enable);
int ras_timing_read(ras_precond *pc, double *total_ms, long long *launches, int reset);

/* Algorithmic bytes of one subdomain-solve launch of ras_apply (factors read
 * once, r read over the overlapped boxes, z written once), for roofline
 * reporting. */
double ras_apply_bytes(const ras_precond *pc);

/* Level schedule of the fine-level subdomain solves (a performance setting; the
 * preconditioner's values do not depend on it): consecutive wavefront levels are
 * staged into shared memory in chunks of at most chunk_cells cells (at least the
 * widest level), and each box is solved by `threads` threads (a multiple of 32,
 * <= 512). 0 keeps the default of that argument (1024 cells, 384 for FP64
 * factors; the widest level rounded up to a warp). Smaller chunks use less shared
 * memory per box, so more boxes run per SM: worth it when there are many more
 * boxes than SMs. Synchronous; no apply of this handle may be in flight; a batch
 * created before the call keeps the old launch settings (create it again).
 * RAS_EINVAL for ILU(k > 0) handles, negative or invalid values, or a schedule
 * whose shared memory exceeds the per-block limit (the old schedule stays). */
int ras_set_apply_schedule(ras_precond *pc, int chunk_cells, int threads);
/* The current schedule (chunk_cells after raising it to the widest level). */
int ras_get_apply_schedule(const ras_precond *pc, int *chunk_cells, int *threads);

/* Kernel of the fine-level subdomain solves of Eq. equ:as-left (a performance
 * setting: both give the same values, bit for bit, in the same arithmetic order,
 * from the same factor records; the switch takes effect at the next ras_apply).
 * 0 (the default): level-scheduled, every wavefront level i + j + k of a box
 * separated by a CTA barrier, each thread looking its cell up in the level's
 * table (the schedule above applies), each owned z written as soon as the
 * backward sweep has it. 1: pencil-wavefront: each thread owns an x-pencil
 * (j, k) of a box and advances one cell per level, its -x neighbour kept in a
 * register, its positions following from the pencil and the level with no table
 * look-up; pencils numbered by anti-diagonal j + k; the records are staged in
 * chunks of levels (the schedule's chunk size) and z is written as soon as it is
 * final. Allowed for left-RAS (ras_type 1) ILU(0) with FP32 or BF16 factors when
 * no overlapped box has more than 1024 x-pencils (RAS_EINVAL otherwise). */
int ras_set_apply_kernel(ras_precond *pc, int kernel);
/* The current kernel of the subdomain solves (0 or 1, as above). */
int ras_get_apply_kernel(const ras_precond *pc, int *kernel);

/* Dense FP32 product C = alpha A B + beta C on the tcgen05 tensor cores, the
 * building block of the dense coarse-level block elimination (Section 3.2: the
 * exact coarse solve of the two-level methods). FP32 accuracy from the TF32 tensor
 * path by the three-term split A B ~ Ah Bh + Ah Bl + Al Bh (h: rounded to TF32,
 * l: the FP32 remainder), accumulated in FP32. Row-major device arrays: A m x k
 * (lda), B k x n (ldb), C m x n (ldc). m and n multiples of 128, k a positive
 * multiple of 32, leading dimensions multiples of 4 (>= the row length), 16-byte
 * aligned bases; else RAS_EINVAL. Synchronises the stream; RAS_ETIMEOUT if a
 * bounded wait for the tensor core gave up. */
int ras_gemm_f32(int m, int n, int k, float alpha, const float *A, int lda, const float *B, int ldb,
                 float beta, float *C, int ldc, void *stream);

/* The cyclic-reduction schedule of the coarse block-tridiagonal system (the opt-in
 * elimination order of the exact coarse solve, Section 3.2, RAS_COARSE_CR=1 at
 * set-up) as the library builds it for nb diagonal blocks, for inspection and
 * host-side checks: host only, no CUDA call. Matrix slots: s < nb is diagonal
 * block s (inverted in place when eliminated); nb + k and 2 nb + k hold the
 * couplings L(k) = A(k, k-1) and U(k) = A(k, k+1); higher slots are products
 * (*nslot slots beyond the nb diagonal blocks). fac: nround, last; then per round
 * nE and the nE blocks it inverts, followed by two phases, each a task count n and
 * n tasks of 8 ints {out, acc, sign, a1, b1, a2, b2, 0} meaning
 * out = (acc ? out : 0) + sign (a1 b1 [+ a2 b2]) (a2 < 0: one term); after the
 * rounds block `last` is inverted. sol: a phase count, then per phase a task count
 * n and n tasks of 8 ints {out, 0, sub, m1, v1, m2, v2, 0} on block vectors (bit
 * 16 set: the solution x, clear: the right-hand side g; low 16 bits: the block)
 * meaning out = (sub ? out - t : t), t = m1 v1 [+ m2 v2] (m2 < 0: one term). The
 * tasks of one phase are independent of each other. The lengths go to *fac_len and
 * *sol_len even when fac_cap or sol_cap is too small (then RAS_EINVAL); RAS_EINVAL
 * also for nb < 1, nb > 65535 or a NULL pointer. */
int ras_coarse_cr_schedule(int nb, int *fac, int fac_cap, int *sol, int sol_cap, int *fac_len, int *sol_len,
                           int *nslot);

#ifdef __cplusplus
}
#endif
#endif /* RAS_H */
