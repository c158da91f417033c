/*
 * dd_nls -- optimized Schwarz time stepping for the 2D nonlinear Schroedinger and
 * Gross-Pitaevskii equations on one GPU (sm_103a).
 *
 * Method: C. Besse, F. Xing, "Domain decomposition algorithms for the two dimensional
 * nonlinear Schroedinger equation and simulation of Bose-Einstein condensates",
 * arXiv:1603.05110.  Section / equation labels below are the paper's.
 *
 * Problem (eq. Sch, BC): on Omega = (xl,xr) x (yb,yu),
 *     i u_t + lap * Lap u + V(x,y) u + kappa |u|^2 u = 0,
 * homogeneous Neumann on y = yb, yu and the transmission operator S-bar (Robin -ip,
 * eq. TCSRobin, or S_pade^m, eq. TCS) on x = xl, xr (or Neumann there, see `bc`).
 * The GPE of eq. (GPE_Trans) is this form with lap = 1/2, V = -V_trap, kappa = -beta.
 * Time: the midpoint scheme of eq. (CNS); one step solves L_x v = (2i/dt) u_{n-1} for
 * v = (u_n + u_{n-1})/2 and commits u_n = 2v - u_{n-1}.
 * Space: Q1 finite elements on a uniform mesh of nx x ny cells (Sec. 2.2).
 * Domain decomposition: n_strips equal x-strips without overlap (Sec. 2.1); the interface
 * vector g = (r_1, l_2, r_2, ..., l_N) (Sec. 2.3) is iterated by the classical algorithm
 * (eq. algo_d) or the preconditioned algorithm (eq. algo_pd, P = I - L_h of eq. Lmpi).
 *
 * Conventions (all entry points):
 *  - Complex arrays are interleaved (re, im) doubles.
 *  - A nodal field is (ny+1) rows of (nx+1) nodes, x fastest: element (iy, ix) at
 *    index iy*(nx+1) + ix.
 *  - An interface vector g is 2*(n_strips-1) traces of ny+1 nodes in the order
 *    (r_1, l_2, r_2, l_3, ..., r_{N-1}, l_N) of Sec. 2.3, i.e. trace 2i is the right
 *    datum of strip i and trace 2i+1 the left datum of strip i+1 (0-based strips).
 *  - ptr_kind says whether caller pointers are host (DD_NLS_PTR_HOST, any pageable or
 *    pinned memory) or device (DD_NLS_PTR_DEVICE) memory; any other value is DD_NLS_EINVAL.
 *    Pointers are only used during the call; the library keeps no reference to caller memory.
 *  - The handle owns all device memory it uses (allocated in dd_nls_create, released in
 *    dd_nls_destroy).  All GPU work is issued on the stream given to dd_nls_create
 *    (NULL: the legacy default stream); calls return after that work has finished.
 *  - Errors are returned as dd_nls_status codes; the GPU is never trapped.  After an
 *    error, dd_nls_last_error() describes it.  A handle is not thread safe.
 *  - Parameters are checked before any device work (DD_NLS_EINVAL): sizes (nx a multiple of
 *    n_strips; ny + 1 and nx / n_strips + 1 at most 2^20 nodes, a strip at most 2^30), every
 *    enum field one of its values, every real field finite, xr > xl, yu > yb, dt > 0,
 *    lap > 0, Robin p > 0, Pade m in 1..96; tolerances, nl_adapt, trap_gx, trap_gy and
 *    wait_limit_ms >= 0.
 */
#ifndef DD_NLS_H
#define DD_NLS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_nls dd_nls;   /* opaque, library-owned */

typedef enum {
    DD_NLS_OK = 0,
    DD_NLS_EINVAL = 1,       /* invalid argument or parameter combination */
    DD_NLS_ENOMEM = 2,       /* device or host allocation failed */
    DD_NLS_ECUDA = 3,        /* a CUDA runtime call failed */
    DD_NLS_ENOCONV = 4,      /* an iteration hit its cap; the step is not committed */
    DD_NLS_ENONFINITE = 5,   /* NaN/Inf in an input or an iterate; the step is not committed */
    DD_NLS_ETIMEOUT = 6,     /* a bounded device-side wait gave up; the step is not committed */
    DD_NLS_EBREAKDOWN = 7    /* Krylov breakdown (p^T A p = 0); the step is not committed */
} dd_nls_status;

enum { DD_NLS_TC_ROBIN = 0, DD_NLS_TC_PADE = 1 };          /* eq. TCSRobin / eq. TCS */
enum { DD_NLS_BC_SAME = 0, DD_NLS_BC_NEUMANN = 1 };        /* physical x-edges */
enum { DD_NLS_CLASSICAL = 0, DD_NLS_PRECONDITIONED = 1 };  /* eq. algo_d / eq. algo_pd */
/* Arithmetic of the strip solves: FP64 throughout; FP32 inner Krylov with the FP64 nonlinear
 * residual; or FP32 inner Krylov with the residual in double-word arithmetic (pairs of FP32
 * numbers, about 48 significant bits, on the FP32 pipe; with S_pade the auxiliary phi rows
 * and their coupling to the edge nodes keep the FP64 residual).  Interface vectors, the
 * Schwarz test, u_n and the diagnostics are FP64 in every mode.  In the double-word mode a strip whose tolerance is below
 * 1e-12 finishes with the FP64 residual; while all strip tolerances of a step are 1e-12 or
 * looser the strip state travels between that step's launches in double-word form and u_n is
 * rebuilt from it (rounded to ~48 bits) at the end of the step. */
enum { DD_NLS_FP64 = 0, DD_NLS_FP32_INNER = 1, DD_NLS_FP32_DW = 2 };
enum { DD_NLS_GUESS_ZERO = 0, DD_NLS_GUESS_PREVIOUS = 1 }; /* g_n^0 (Sec. 5) */
enum { DD_NLS_PTR_HOST = 0, DD_NLS_PTR_DEVICE = 1 };
/* How P x = y of eq. (algo_pd) is solved: GMRES on the assembled L_h blocks (Sec. 4.2), or
 * exactly in the cosine basis that diagonalises every block of L_h (uniform mesh, Neumann
 * data on y = yb, yu); both apply the same P. */
enum { DD_NLS_PSOLVE_GMRES = 0, DD_NLS_PSOLVE_MODAL = 1 };

typedef struct {
    /* Omega, mesh and strips (Sec. 2.1-2.2); nx must be a multiple of n_strips */
    double xl, xr, yb, yu;
    int nx, ny, n_strips;
    /* equation (Sch) and time step (CNS) */
    double dt, lap, kappa;
    /* transmission operator S-bar: Robin parameter p, or Pade order m and rotation theta */
    int tc;
    double p;
    int pade_m;
    double pade_theta;
    int bc;           /* DD_NLS_BC_SAME: S-bar with zero data on x = xl, xr; or Neumann */
    int algorithm;    /* DD_NLS_CLASSICAL or DD_NLS_PRECONDITIONED */
    int precision;    /* DD_NLS_FP64, DD_NLS_FP32_INNER (FP32 Krylov + FP64 residual) or
                         DD_NLS_FP32_DW (FP32 Krylov + double-word residual) */
    int guess;        /* interface guess for each step when dd_nls_step is called */
    /* stopping tests */
    double tol;          /* ||R(g)-g|| <= tol*||R(g)|| (or <= tol if tol_absolute) */
    int tol_absolute;
    int max_schwarz;
    double nl_tol;       /* strip solves: ||b - A(zeta) zeta|| <= tol_k * ||b||; tol_k = nl_tol
                            unless nl_adapt is set (see below) */
    int max_nl;
    double inner_tol;    /* Krylov: residual reduction per correction */
    int max_inner;
    double gmres_tol;    /* P x = y (eq. algo_pd): relative residual */
    int gmres_restart;
    int gmres_max;
    int psolve;          /* DD_NLS_PSOLVE_MODAL (default) or DD_NLS_PSOLVE_GMRES */
    double nl_relax;     /* first relaxation factor of the strip fixed point (1: eq. localpbrobin
                            as printed); a correction that does not cut the residual by 10%
                            multiplies it by 0.6 (down to 0.25).  Same limit, safer path.
                            Values outside (0, 1] act as 1. */
    int nl_picard;       /* operator of each strip correction: 0 (default) the complex-linear part
                            of the Jacobian, diag(w(W + 2 kappa|zeta|^2)); 1 the frozen operator
                            of the fixed point of eq. localpbrobin, diag(w(W + kappa|zeta|^2)).
                            The residual is exact either way, so the limit is the same. */
    double nl_adapt;     /* 0 (default): strip solves always to nl_tol.  > 0, preconditioned
                            algorithm with two or more strips only: tol_k = nl_adapt x the last
                            relative interface residual (at most 1e-6, never below nl_tol), and
                            a step converges only once tol_k <= max(nl_tol, nl_adapt x tol).
                            Same fixed point, cheaper early Schwarz iterations.  A Schwarz
                            iteration that does not cut the relative interface residual by 4x
                            ends the inexact solves for the rest of the step. */
    /* Rotating frame of the GPE (Sec. 5.2.1, eq. x1Ax, GPE_Trans, u1u).  The solve runs in the
     * coordinates x~ = A(t)^T x, A(t) the rotation by omega_rot t, where the rotation term of
     * eq. (GPE) is absent and the trap becomes time dependent. */
    double omega_rot;    /* omega of eq. (GPE): the angle of A(t) and the -omega <u, L_z u> term of
                            the energy (stats.energy_lab) */
    double trap_gx, trap_gy; /* either > 0: the trap V_trap = (gx^2 x^2 + gy^2 y^2)/2 of eq. (GPE) taken
                            at (x, y) = A(t_n) x~ is added to the potential (eq. Sch sign: V - V_trap),
                            and step n solves with W_n = (V_n + V_{n-1})/2 of eq. (CNS), t_n = n dt
                            (n counts committed steps, see dd_nls_set_state).  0, 0: no trap term */
    int psolve_modes;    /* modal P solve: only the lowest psolve_modes cosine modes are solved with
                            (I - L_h); the others take P = I (a partially constructed I - L_h, the
                            paper's closing suggestion).  0 (default): all modes, the exact P */
    double wait_limit_ms;  /* bound of every device-side wait between blocks of a strip; on expiry the
                            call returns DD_NLS_ETIMEOUT and commits nothing.  0 (default): 2000 ms */
    int solver_layout;   /* 0 (default) and 2: FP32 Robin strips whose rows, split over a cluster of 16
                            CTAs, fit in their shared memory are solved one strip per thread-block
                            cluster (inner Krylov state on chip, partial sums through distributed shared
                            memory, double-word scalar recurrences); everything else as in 1.
                            1: one cooperative launch over all strips, blocks split among strips by
                            expected work, global-memory barriers.  The converged step is the same
                            either way. */
} dd_nls_params;

typedef struct {
    int steps;                    /* steps committed by this call */
    int schwarz_iterations;       /* Schwarz iterations, summed over the call's steps */
    int last_schwarz_iterations;  /* of the last step */
    long long nl_iterations;      /* strip nonlinear iterations, summed over strips */
    long long krylov_iterations;  /* inner Krylov iterations, summed over strips */
    long long gmres_iterations;   /* GMRES iterations on P x = y */
    double residual;              /* last relative interface residual ||R(g)-g||/||R(g)|| */
    double residual_abs;          /* last absolute interface residual ||R(g)-g|| */
    double mass;                  /* u_n^H M u_n of the last committed step */
    double energy;                /* u^H S u - u^H M_W u - (kappa/2lap) sum w|u|^4, scaled by 1/lap, with
                                     W = V(t_n)/lap the potential at the time of u_n */
    double setup_ms;              /* L_h construction (preconditioned), at create */
    double lz;                    /* <u_n, L_z u_n>, L_z = -i (x d_y - y d_x) (Sec. 5.2.1): nodal
                                     quadrature, central differences (one-sided on the boundary) */
    double energy_lab;            /* the energy of eq. (GPE) (its Hamiltonian), lap u^H S u
                                     - sum w V(t_n)|u|^2 - (kappa/2) sum w |u|^4 - omega_rot lz; for the
                                     GPE (lap = 1/2, V = -V_trap, kappa = -beta) this is
                                     int 1/2|grad u|^2 + V_trap|u|^2 + beta/2 |u|^4 - omega u* L_z u */
} dd_nls_stats;

/* Device time of the library's kernels, accumulated while profiling is on. */
typedef struct {
    double strip_solve_ms;        /* the batched strip solver (Krylov + stencil) */
    long long strip_solve_launches;
    double strip_solve_bytes;     /* algorithmic bytes moved by those launches */
    double strip_solve_flops;
    double interface_ms;          /* traces, residuals, GMRES, L_h products */
    double other_ms;              /* right sides, commit, diagnostics */
    long long kernel_launches;    /* all kernels this handle launched while profiling was on */
    double phase_cycles[5];       /* strip solver, SM cycles per block (averaged over blocks, summed
                                     over launches): FP64 residual, Krylov stencil phase, Krylov
                                     update phase, correction commit, waits at barriers/reductions */
} dd_nls_profile;

/* Fill *p with defaults: NLS (lap=1, kappa=1), Robin p=1, classical, FP64, previous-step
 * guess, tol 1e-10, nl_tol 1e-13 (max_nl 300), inner_tol 1e-6, GMRES restart 30 / tol 1e-10,
 * modal P solve on all modes, no rotation and no trap, 2 s device wait limit. */
void dd_nls_default_params(dd_nls_params* p);

/* Create a solver.  V: real nodal potential (ny+1)*(nx+1) in the sign of eq. (Sch), or
 * NULL for V = 0.  u0: complex nodal initial datum.  stream: a cudaStream_t or NULL.
 * Builds L_h (eq. Lmpi) when algorithm is PRECONDITIONED (2(ny+1) strip solves, Sec. 4.2).
 * Errors: EINVAL (bad sizes / parameters / NULL out or u0), ENOMEM, ECUDA. */
int dd_nls_create(const dd_nls_params* p, const double* V, const double* u0, int ptr_kind,
                  void* stream, dd_nls** out);

/* Advance nsteps time steps (eq. CNS), each by the Schwarz iteration to `tol`.
 * u_out (nullable): receives u_n after the last step.  stats (nullable).
 * A step whose iteration fails is not committed and the error is returned. */
int dd_nls_step(dd_nls* h, int nsteps, double* u_out, int ptr_kind, dd_nls_stats* stats);

/* Run the Schwarz iteration of the current step (u_{n-1} = current state) from the
 * interface guess g0 (nullable: the `guess` policy) without committing; g_out (nullable)
 * receives the converged R(g); v_out (nullable) the nodal v = (u_n + u_{n-1})/2. */
int dd_nls_solve_interface(dd_nls* h, const double* g0, double* g_out, double* v_out,
                           int ptr_kind, dd_nls_stats* stats);

/* One time step like dd_nls_step(h, 1, ...) but started from the interface guess g0
 * (instead of the `guess` policy), e.g. a learned guess from dd_cnn_guess. */
int dd_nls_step_guess(dd_nls* h, const double* g0, double* u_out, int ptr_kind, dd_nls_stats* stats);

/* Checkpoint: u (complex nodal, nullable) and g (interface vector used as the previous-
 * step guess, nullable).  set_state also sets the step counter to `step`. */
int dd_nls_get_state(dd_nls* h, double* u, double* g, int* step, int ptr_kind);
int dd_nls_set_state(dd_nls* h, const double* u, const double* g, int step, int ptr_kind);

/* Copy the L_h blocks X^{j,1..4} (Props 3.1/3.2) of strip j into x (4 row-major
 * (ny+1)x(ny+1) complex matrices, X1 X2 X3 X4).  EINVAL unless PRECONDITIONED with GMRES.
 * dd_nls_get_modal copies the diagonal of the blocks in the cosine basis instead: 4 vectors
 * of ny+1 complex values (x1 x2 x3 x4); EINVAL unless PRECONDITIONED with MODAL. */
int dd_nls_get_blocks(dd_nls* h, int strip, double* x, int ptr_kind);
int dd_nls_get_modal(dd_nls* h, int strip, double* x, int ptr_kind);

/* The lab-frame field u(t_n, x, y) = u~(t_n, A(t_n)^T (x, y)) of eq. (u1u), t_n = n dt the time of
 * the current state, on the valid zone (xl/sqrt2, xr/sqrt2) x (yb/sqrt2, yu/sqrt2) of Sec. 5.2.1
 * (inside every rotated copy A(t) Omega of a square domain centred at the origin): out receives
 * (ny_out+1) rows of (nx_out+1) complex values, x fastest, the Q1 interpolant of the computed u~
 * at the rotated points.  Errors: EINVAL for nx_out or ny_out outside 1 .. 2^30-1 or a NULL out. */
int dd_nls_lab_frame(dd_nls* h, int nx_out, int ny_out, double* out, int ptr_kind);

int dd_nls_set_profiling(dd_nls* h, int on);
int dd_nls_get_profile(dd_nls* h, dd_nls_profile* prof);

/* One time step (eq. CNS) without allocating device memory.  The paper has no counterpart:
 * this entry point is for callers that cannot call cudaMalloc when they step -- code inside
 * a memory pool or arena that owns the device, a process that must not change the
 * allocation state of a context it shares, a path where cudaMalloc's implicit
 * synchronisation is not allowed.  All working memory comes from one fixed 64 MiB device
 * array inside the library (held on every GPU that loads the library until the process
 * exits); a problem that needs more is rejected with DD_NLS_EINVAL, as are more than 64
 * strips.  Only the classical algorithm with the Robin condition (FP64 or FP32 inner).
 * V (nullable), u (in: u_{n-1}, out: u_n), g0 (nullable: zero guess) and g_out (nullable:
 * the converged R(g), the next step's guess) are DEVICE pointers in the layouts above;
 * stream may be NULL.  Every call uses the same array: calls that overlap on the GPU race.
 * The first call on a device looks up the array's address (with that device current); make
 * it before any stream capture.  That address is kept until the process exits, so after a
 * cudaDeviceReset of the device this entry point must not be called again in that process.
 * The call waits for its stream once per Schwarz iteration (the host decides convergence).
 * Errors: dd_nls_last_error(NULL) describes them (one message buffer per host thread). */
int dd_nls_step_noalloc(const dd_nls_params* p, const double* V, double* u, const double* g0,
                        double* g_out, void* stream, dd_nls_stats* stats);

/* Batched instances (many independent problems stepped together).  Every Schwarz
 * iteration solves the strips of all instances that have not yet converged in one
 * persistent launch, then updates every instance's interface vector (eq. fluxlr) in one
 * launch; each instance stops at its own `tol`.  Instances may differ in the domain, mesh,
 * strips, dt, lap, kappa, Robin p, bc, algorithm, tol, tol_absolute, nl_tol, max_schwarz,
 * guess, nl_adapt and psolve_modes.  precision (DD_NLS_FP64, DD_NLS_FP32_INNER or
 * DD_NLS_FP32_DW; the latter needs nl_tol >= 1e-12), inner_tol, max_nl, max_inner, nl_relax
 * and nl_picard must agree across instances.  V is static: trap_gx = trap_gy = 0; omega_rot,
 * solver_layout, wait_limit_ms and the GMRES fields are not used (no per-step diagnostics,
 * cooperative layout).  Each uses Robin transmission and either the classical
 * algorithm (eq. algo_d) or the preconditioned one (eq. algo_pd) with psolve =
 * DD_NLS_PSOLVE_MODAL (the exact P^-1 on cosine modes, one set of factors per instance, built
 * at create; nl_adapt and psolve_modes apply as in dd_nls_step).  An autotuner picks the
 * strip solver's block size and block count for the batch shape the first time a shape is
 * stepped (timed on the first Schwarz iteration).
 * params, V (nullable, or entries NULL) and u0 are arrays of n entries; pointers are host or
 * device per ptr_kind.  Errors: dd_nls_batch_last_error(). */
typedef struct dd_nls_batch dd_nls_batch;
int dd_nls_batch_create(int n, const dd_nls_params* params, const double* const* V,
                        const double* const* u0, int ptr_kind, void* stream, dd_nls_batch** out);
/* nsteps steps of every instance; stats (nullable) receives n entries. */
int dd_nls_batch_step(dd_nls_batch* b, int nsteps, dd_nls_stats* stats);
/* u_n of instance i, nodal layout above. */
int dd_nls_batch_get_u(dd_nls_batch* b, int i, double* u, int ptr_kind);
/* Replace the state u_{n-1} of instance i (nodal layout above); the interface guess of the next
 * step is kept.  Host pointers go through a staging buffer the batch owns. */
int dd_nls_batch_set_u(dd_nls_batch* b, int i, const double* u, int ptr_kind);
/* The autotuner's choice: threads per block and blocks per launch (0 before the first step). */
int dd_nls_batch_tuning(dd_nls_batch* b, int* block_size, int* blocks);
int dd_nls_batch_set_profiling(dd_nls_batch* b, int on);
int dd_nls_batch_get_profile(dd_nls_batch* b, dd_nls_profile* prof);
const char* dd_nls_batch_last_error(const dd_nls_batch* b);
void dd_nls_batch_destroy(dd_nls_batch* b);

/* Learned interface guess (no counterpart in the paper, which starts each step from the
 * previous converged vector, Sec. 5).  A 4-layer CNN (3x3 convolutions 6->32->32->32->2, ReLU,
 * BF16 operands with FP32 accumulation on the tensor cores) maps the last three converged
 * interface vectors of a problem with n_traces = 2(N-1) traces of nodes_per_trace = ny+1
 * nodes to a correction of a base guess:
 *     g0 = g1 + e (g1 - g2) + s1 * net(g1/s0, (g1-g2)/s1, (g2-g3)/s1),
 * s0 = rms(g1), s1 = rms(g1-g2) (g1 the most recent), e = 1 (linear extrapolation, the default)
 * or e = 0 (the paper's previous-step vector), chosen by dd_cnn_set_base (EINVAL otherwise).
 * n_traces x nodes_per_trace is at most 2^28.  Interface vectors are DEVICE pointers in the
 * ABI layout.  Parameters: one FP32 array of dd_cnn_num_params() values, per layer the
 * weights [Cout][Cin][3][3] then the biases [Cout]; the caller supplies the initial values.
 * dd_cnn_train_step: one Adam step (lr, betas 0.9/0.999) on the squared error of the
 * correction for the target vector gt; loss (nullable) receives the mean squared error.
 * dd_cnn_loss_grad: the same loss and its gradient (host or device per ptr_kind), no update. */
typedef struct dd_cnn dd_cnn;
enum { DD_CNN_BASE_PREVIOUS = 0, DD_CNN_BASE_EXTRAPOLATE = 1 };
int dd_cnn_create(int n_traces, int nodes_per_trace, void* stream, dd_cnn** out);
int dd_cnn_set_base(dd_cnn* c, int base);
long long dd_cnn_num_params(const dd_cnn* c);
int dd_cnn_set_params(dd_cnn* c, const float* w, int ptr_kind);
int dd_cnn_get_params(dd_cnn* c, float* w, int ptr_kind);
int dd_cnn_guess(dd_cnn* c, const double* g1, const double* g2, const double* g3, double* g0);
int dd_cnn_train_step(dd_cnn* c, const double* g1, const double* g2, const double* g3, const double* gt,
                      float lr, double* loss);
int dd_cnn_loss_grad(dd_cnn* c, const double* g1, const double* g2, const double* g3, const double* gt,
                     float* grad, double* loss, int ptr_kind);
const char* dd_cnn_last_error(const dd_cnn* c);
void dd_cnn_destroy(dd_cnn* c);

/* Release everything the handle owns.  NULL is ignored. */
void dd_nls_destroy(dd_nls* h);

/* Text of the last error on this handle (or of the last failed create when h is NULL). */
const char* dd_nls_last_error(const dd_nls* h);

#ifdef __cplusplus
}
#endif
#endif /* DD_NLS_H */
