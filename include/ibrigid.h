/*
 * ibrigid.h -- C ABI of the GB300 (sm_103a) rigid-body immersed-boundary solver.
 *
 * The library solves the rigidly constrained Stokes saddle-point system of
 * Kallemov, Bhalla, Griffith, Donev, "An Immersed Boundary Method for Rigid
 * Bodies" (arXiv:1505.07865), Sec. III.B, Eq. constrained_Stokes
 *
 *     [ A   G  -S~ ] [v     ]   [g]
 *     [-D   0   0  ] [pi    ] = [h]        A = rho/dt I - eta h^-2 Lap (Eq. A_def)
 *     [-J   0   0  ] [Lambda]   [W]        W = -K U  (rigid no-slip, Sec. II)
 *
 * with S~ = S - vol^-1 1^T for periodic steady Stokes (Sec. III.D, Eq.
 * constrained_periodic, together with <v> = 0), by flexible GMRES (Sec. V)
 * right-preconditioned with the Schur-complement preconditioner of Sec. V.A:
 * an inner GMRES(N_s) Stokes solve preconditioned by the projection
 * preconditioner P_S (Sec. V.B, Eq. P1_practical) built from geometric
 * multigrid V-cycles, followed by the approximate mobility solve
 * M~ Lambda = dU (Eq. mob_subproblem) with the dense analytic M~ of Sec. IV
 * (Eq. M_tilde_ij), factorised once per geometry (Sec. V.C).
 *
 * Conventions (all entry points):
 *  - Every function returns IBR_OK (0) or a negative IBR_E* code and never
 *    throws; ibr_last_error() gives a thread-local message for the last
 *    failure on the calling thread.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Output
 *    buffers are caller-allocated.  The library owns all device memory of a
 *    grid and frees it in ibr_destroy_grid.
 *  - Pointers documented as "device" must point to memory of the CUDA device
 *    that was current when the grid was created; "host" means pageable or
 *    pinned host memory.
 *  - Work is issued on the grid's stream (the cuda_stream given to
 *    ibr_create_grid, or a library-created stream when NULL).  Entry points
 *    that return host data synchronise that stream; the op-level entry points
 *    on device data (ibr_apply_*, ibr_op_*) are asynchronous on that stream.
 *  - Grid layout: a cell-centred scalar is n[0]*n[1](*n[2]) doubles, x index
 *    fastest.  Velocity component alpha is stored on the faces normal to
 *    axis alpha, entry (i,j,k) being the lower face of cell (i,j,k), i.e. at
 *    (i + 1/2 - delta_{alpha,0}/2, ...) h.  A system vector is
 *    [v_0 | ... | v_{d-1} | pi | Lambda], Lambda marker-major (i*d + alpha),
 *    markers in the order bodies were added and, within a body, the order
 *    given to ibr_set_markers.
 *  - Sign convention (Sec. III.B): Lambda is the force of the markers on the
 *    fluid (it enters the momentum equation as +S Lambda); the force and
 *    torque of a body on the fluid is K^T Lambda, the drag on the body is its
 *    negative.
 */
#ifndef IBRIGID_H
#define IBRIGID_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define IBR_OK        0
#define IBR_EINVAL   -1   /* bad argument (size, pointer, option)                 */
#define IBR_ENOMEM   -2   /* device or host allocation failed                     */
#define IBR_ENOTCONV -3   /* FGMRES hit max_iters; results are still readable     */
#define IBR_ETIMEOUT -4   /* time_cap_ms exceeded; results are still readable     */
#define IBR_ENUMERIC -5   /* NaN/Inf in data, or M~ not made SPD by any shift     */
#define IBR_ECUDA    -6   /* a CUDA runtime call failed                           */
#define IBR_ESTATE   -7   /* call out of order (e.g. solve before markers)        */
#define IBR_EPENDING -8   /* ibr_server_poll: the request has not finished yet    */

/* ---- boundary conditions per axis side (bc[axis][0]=low, [1]=high) -------- */
#define IBR_PERIODIC 0
#define IBR_NOSLIP   1
#define IBR_VELOCITY 2

/* ---- kernels, precisions, kinematics, preconditioner variants ------------- */
#define IBR_KERNEL_PESKIN4 4   /* 4-point Peskin kernel (Sec. III.A)            */
#define IBR_KERNEL_BKP6    6   /* six-point kernel of Bao, Kaye and Peskin, the
                                  kernel the paper uses (Sec. III.A): support 6
                                  nodes per axis, three continuous derivatives;
                                  periodic boxes only                           */
#define IBR_FP64  0            /* every step in float64                           */
#define IBR_MIXED 1            /* FP64 outer FGMRES / matvec / true residual;     */
                               /* FP32 preconditioner (MG, P_S, inner GMRES,      */
                               /* spread/interp inside it, M~^-1)                 */
#define IBR_PRESCRIBED 0       /* body velocity given (Sec. II)                   */
#define IBR_FREE       1       /* body force and torque given, velocity unknown   */
#define IBR_PC_LOWER 0         /* lower block-triangular Schur preconditioner     */
#define IBR_PC_FULL  1         /* full Schur preconditioner (steps 1-4, Sec. V.A) */
#define IBR_MOB_AUTO  0        /* RPY (3-D) / App. B steady form (2-D)            */
#define IBR_MOB_RPY   1        /* Eq. RPYTensor (+ periodic correction, App. A)   */
#define IBR_MOB_FIT2D 2        /* App. B Eq. fg_steady_2d                          */
                               /* (analytic forms: one dense block per body,
                                  the block-diagonal form of Sec. IX, bodies
                                  not coupled; see IBR_MOB_COUPLED)              */
#define IBR_MOB_COUPLED 16     /* OR-ed with IBR_MOB_AUTO / RPY / FIT2D: one dense
                                  block of all markers (M~_ij for every pair,
                                  Sec. IV.B; minimum-image displacements on
                                  periodic axes) while dim N <= 6144, else one
                                  block per body.  The analytic far field is
                                  not the periodic one: on crowded periodic 2-D
                                  problems coupling raised FGMRES iterations
                                  several-fold, hence off by default          */
#define IBR_MOB_TRUE  3        /* the true mobility M0 = J L^-1 S of all markers,
                                  one dense block, built in the set-up from
                                  N*dim Stokes solves (Sec. V.C, VII.F: for
                                  fixed geometries)                             */
#define IBR_MOB_PAIR  4        /* periodic grids: M~_ij = the grid's own pair
                                  mobility at displacement q_i - q_j, from a
                                  table of 2 x dim Stokes solves (unit forces at
                                  two off-node source points) built once per
                                  grid, symmetrised and averaged over the
                                  sources (Sec. IV's translation-invariant pair
                                  mobility, tabulated instead of fitted); one
                                  dense block for all markers while dim N <=
                                  6144 (bodies coupled), else one per body      */

typedef struct ibr_grid ibr_grid;   /* opaque */

typedef struct ibr_solve_opts {
    double tol;            /* relative residual ||b - A x||_2 / ||b||_2 (true)   */
    int    restart;        /* FGMRES restart length m                           */
    int    max_iters;      /* cap on outer iterations (all restarts)            */
    int    n_s;            /* inner Stokes GMRES iterations N_s (Sec. V.A);
                              0: 2 on periodic grids, 4 with walls             */
    int    variant;        /* IBR_PC_LOWER or IBR_PC_FULL                       */
    int    mg_pre;         /* pre-smoothing sweeps per V-cycle level            */
    int    mg_post;        /* post-smoothing sweeps per V-cycle level           */
    int    mob_model;      /* IBR_MOB_*                                          */
    double mob_a_over_h;   /* marker radius a/h in M~; 0: the grid kernel's value */
                           /* (ibr_mobility_defaults: 1.25 / 1.47 in 3-D, Sec.    */
                           /* IV.A; in 2-D the fitted App. B self-mobility radius) */
    double mob_coef[9];    /* App. B coefficients a0..a4, b0..b3 (2-D steady);   */
                           /* all zero: the grid kernel's fitted set             */
    double time_cap_ms;    /* <= 0: none                                         */
} ibr_solve_opts;

typedef struct ibr_solve_info {
    int    status;         /* same as the return code of ibr_solve_coupled      */
    int    iters;          /* outer FGMRES iterations                            */
    int    restarts;       /* completed restart cycles                           */
    int    ps_applications;/* applications of P_S (the paper's cost unit)      */
    double rel_res_est;    /* Givens estimate at exit                            */
    double rel_res_true;   /* recomputed ||b - A x|| / ||b|| in FP64             */
    double ms_setup;       /* marker binning + M~ build/factor, wall ms          */
    double ms_solve;       /* FGMRES, wall ms                                    */
} ibr_solve_info;

typedef struct ibr_step_info {
    int    status;         /* same as the return code of ibr_advance             */
    int    steps;          /* time steps taken                                   */
    int    iters_total;    /* outer FGMRES iterations over all steps             */
    int    iters_last;     /* outer FGMRES iterations of the last step           */
    double change;         /* ||v^{n+1} - v^n|| / ||v^{n+1}|| of the last step   */
    double rel_res_last;   /* true relative residual of the last step's solve    */
    double ms;             /* wall ms of the call                                */
} ibr_step_info;

/* Fills opts with the defaults: tol 1e-8, restart 50, max_iters 1000, N_s 0 (automatic),
 * IBR_PC_LOWER, mg 2/2, IBR_MOB_AUTO, a/h 0 and coefficients 0 (the grid
 * kernel's defaults, ibr_mobility_defaults), no time cap. */
int ibr_solve_opts_default(ibr_solve_opts* opts);

/* The library's default parameters of the analytic M~ for a kernel
 * (IBR_KERNEL_PESKIN4 / IBR_KERNEL_BKP6) in dim 2 or 3: the marker radius a/h
 * and, in 2-D, the coefficients a0..a4, b0..b3 of App. B's steady forms
 * (Eq. fg_steady_2d; zeros in 3-D, where M~ is the RPY tensor, Eq. RPYTensor).
 * 3-D radii are the paper's (Sec. IV.A: 1.25 h and 1.47 h).  The paper does
 * not print its 2-D coefficients; these are fitted by its procedure (Sec.
 * IV.B, App. B) to the library's own periodic pair mobility of each kernel
 * (paper_1505_07865_gb300/fit_mobility_2d.py, output mobility_fit_2d.json).
 * Either output may be NULL.  Needs no GPU. */
int ibr_mobility_defaults(int dim, int kernel, double* a_over_h, double* coef9);

/* Creates a uniform MAC grid (Sec. III).  dim in {2,3}; n[0..dim-1] cells per
 * axis (each even, >= 4); L[0..dim-1] box lengths (cubic cells: L[a]/n[a]
 * equal for all a).  bc[2a + s] (s = 0 low, 1 high end of axis a): both
 * IBR_PERIODIC, or both walls, IBR_NOSLIP (zero velocity) or IBR_VELOCITY
 * (velocity given by ibr_set_boundary_velocity, zero until then).  Walls
 * follow App. D: fields are extended beyond a wall by linear extrapolation
 * through the wall value, and the same extension gives interpolation and
 * spreading near the wall.  On a wall axis the velocity component normal to
 * the wall stores faces 0..n-1 of its n+1 faces: face 0 lies on the low wall
 * (its equation is v = wall value, and it holds that value in the solution),
 * the high wall face is not stored.
 * eta > 0 viscosity; rho, dt >= 0 (rho == 0 or dt == 0: steady Stokes, A =
 * -eta h^-2 Lap).  kernel: IBR_KERNEL_PESKIN4, or IBR_KERNEL_BKP6 on a
 * periodic box (the analytic M~ then takes a = 1.47 h in 3-D, Sec. IV.A).
 * precision: IBR_FP64 or
 * IBR_MIXED.  cuda_stream: a cudaStream_t, or NULL for a library-created
 * blocking stream (ordered with the legacy default stream).  On success *out owns the
 * grid's device memory.  Errors: IBR_EINVAL, IBR_ENOMEM, IBR_ECUDA. */
int ibr_create_grid(ibr_grid** out, int dim, const int* n, const double* L,
                    const int* bc /* dim*2 */, double eta, double rho, double dt,
                    int kernel, int precision, void* cuda_stream);

/* Adds a rigid body with reference point x_c[dim] and orientation quat[4]
 * (w,x,y,z; unit; 2-D uses the rotation about z it describes).  kinematics:
 * IBR_PRESCRIBED (velocity given) or IBR_FREE (force and torque given; the
 * rigid velocity becomes an unknown: the markers satisfy J v = K U and the
 * force balance K^T Lambda = F is added, Sec. II; the preconditioner adds the
 * body block N = (K^T M~^-1 K)^-1 in FP64, Sec. VIII).  Writes the body index
 * (0,1,...) to *body_id. */
int ibr_add_body(ibr_grid* g, const double* x_c, const double* quat, int kinematics, int* body_id);

/* Sets the N markers of a body from body-frame offsets r_body[N*dim] (host).
 * Lab positions q_i = x_c + Q(quat) r_i are wrapped into [0, L) on periodic
 * axes and must lie in [0, L] on wall axes (IBR_EINVAL at set-up).  Marks the geometry dirty: the next solve (or ibr_prepare) rebins the
 * markers and rebuilds and refactors M~.  N >= 1.  M~ is factorised by
 * Cholesky; a block that is not positive definite (the analytic M~ need not
 * be, Sec. V.C) is factorised as M~ + delta I with the smallest delta in
 * 1e-3 f(0) * 2^k that succeeds (IBR_ENUMERIC if none up to k = 40). */
int ibr_set_markers(ibr_grid* g, int body_id, const double* r_body, int N);

/* Velocity on the wall face = 2a + s (an IBR_VELOCITY side): values[dim][P]
 * (host, copied), P = cells of the other axes (lower axis fastest); values[a]
 * is the normal velocity at the wall's normal faces, values[b] (b != a) the
 * tangential velocity at the wall positions of component b's faces.  The
 * data enters the right-hand side (the lifted App. D extension); the net
 * flux through all walls must vanish (checked at solve time: IBR_EINVAL),
 * and markers must stay 2h away from walls with nonzero data (checked in the
 * set-up: IBR_EINVAL).  IBR_EINVAL for other faces. */
int ibr_set_boundary_velocity(ibr_grid* g, int face, const double* values);

/* Runs the geometry set-up now (marker lab positions, kernel weights, the
 * sorted face-gather lists of S, M~ build and factorisation) with the
 * mobility options of opts (NULL: defaults). */
int ibr_prepare(ibr_grid* g, const ibr_solve_opts* opts);

/* Solves the constrained system for body_UO[B*(dim+rot)] (host; per body U
 * then Omega for a prescribed body, applied force F then torque T for a free
 * one; rot = 1 in 2-D, 3 in 3-D) with momentum forcing g (NULL: zero; else dim face arrays laid out as
 * above, on the device if g_on_device != 0, else on the host; for periodic
 * steady Stokes each component must have zero mean) and h = 0.  FGMRES starts
 * from x0 = 0 and stops when the true relative residual is <= opts->tol.
 * The solution stays resident (ibr_get_forces / ibr_get_fields / ibr_get_solution).
 * Returns IBR_OK, IBR_ENOTCONV, IBR_ETIMEOUT (results readable), or an error. */
int ibr_solve_coupled(ibr_grid* g, const double* body_UO, const double* gforce, int g_on_device,
                      const ibr_solve_opts* opts, ibr_solve_info* info);

/* Time stepping (Sec. VII.F; the nozzle flow).  Advances the fluid state v^n
 * (the last solution's velocity; at rest with the wall values if there is
 * none) by up to nsteps steps of size dt: each step solves the constrained
 * system with the backward-Euler operator A = rho/dt I - eta h^-2 Lap and
 *     g = (rho/dt) v^n - rho (3/2 N(v^n) - 1/2 N(v^{n-1})) + f
 * (the first step of a history uses N(v^n) alone), N(v) = div(v v) in the
 * centred second-order flux form on the MAC grid with the same wall
 * extension as the fluid operators; FGMRES starts from the previous step's
 * solution.  Stops early when ||v^{n+1} - v^n|| <= steady_tol ||v^{n+1}||
 * (steady state; 0: never).  body_UO as in ibr_solve_coupled (fixed for all
 * steps); gforce: a constant body force f (dim face arrays, device if
 * g_on_device, else host) or NULL.  Needs rho > 0 and dt > 0 (IBR_EINVAL).
 * A step whose solve does not converge stops the march with its status. */
int ibr_advance(ibr_grid* g, const double* body_UO, const double* gforce, int g_on_device, int nsteps,
                double steady_tol, const ibr_solve_opts* opts, ibr_step_info* info);

/* Sets the fluid velocity state v (dim face arrays; device if on_device, else
 * host) that ibr_advance starts from (pressure and Lambda zero; the wall
 * faces take the wall values); restarts the AB2 history.  Runs the geometry
 * set-up if needed. */
int ibr_set_velocity(ibr_grid* g, const double* v, int on_device);

/* Copies the marker forces Lambda[N*dim] (may be NULL) and the per-body
 * K^T Lambda = [force; torque] of each body on the fluid, body_FT[B*(dim+rot)]
 * (may be NULL), of the last solve to host memory. */
int ibr_get_forces(ibr_grid* g, double* Lambda, double* body_FT);

/* Rigid velocities [B*(dim+rot)] after a solve: body_UO (the array given to the
 * solve) with the rows of free bodies replaced by their computed U, Omega. */
int ibr_get_body_velocities(ibr_grid* g, const double* body_UO, double* out);

/* Copies the velocity (dim face arrays, concatenated) and pressure of the last
 * solve.  to_device != 0: v and p are device pointers; else host. */
int ibr_get_fields(ibr_grid* g, double* v, double* p, int to_device);

/* Total length of a system vector, (dim+1)*cells + dim*N + (dim+rot)*(free
 * bodies) (the free bodies' velocities come last), and the marker and body
 * counts (any output pointer may be NULL). */
int ibr_sizes(const ibr_grid* g, long long* system_len, int* n_markers, int* n_bodies);

/* ---- op-level entry points (device pointers, FP64, asynchronous) ----------
 * These expose each step of the hot path separately so each can be checked
 * against an independent implementation.  They require ibr_prepare (or a
 * solve) after the last ibr_set_markers. */

/* y = (system matrix) x for the full constrained operator above, x and y of
 * length ibr_sizes().system_len (Sec. III.B / III.D). */
int ibr_apply_system(ibr_grid* g, const double* x, double* y);

/* f = S~ Lambda (Sec. III.A Eq. S_unweighted; minus vol^-1 sum Lambda for
 * periodic steady Stokes, Sec. III.D).  lam[N*dim], f: dim face arrays. */
int ibr_op_spread(ibr_grid* g, const double* lam, double* f);

/* U = J v (Sec. III.A).  v: dim face arrays, U[N*dim]. */
int ibr_op_interp(ibr_grid* g, const double* v, double* U);

/* V = K UO (marker velocities [N*dim]) and FT = K^T Lambda ([B*(dim+rot)]). */
int ibr_op_rigid(ibr_grid* g, const double* UO, double* V);
int ibr_op_rigid_T(ibr_grid* g, const double* lam, double* FT);

/* Copies dense mobility block b into out (row-major): the single block of all
 * markers ((dim N)^2 doubles, b = 0) with IBR_MOB_TRUE (M0), and for one body or
 * several bodies while dim N <= 6144 (Eq. M_tilde_ij for every marker pair);
 * else the M~ block of body b ((dim N_b)^2 doubles). */
int ibr_op_mtilde(ibr_grid* g, int body, double* out);

/* out = M~^-1 rhs (block diagonal over bodies, [N*dim]) with the factorised
 * M~ in the grid's preconditioner precision.  The mixed path factorises on the
 * tensor cores: blocked Cholesky (128-blocks), triangular inverse and
 * M~^-1 = L^-T L^-1, their products in split TF32 (ibr_op_gemm_tf32x3). */
int ibr_op_mtilde_solve(ibr_grid* g, const double* rhs, double* out);

/* One application z = P_S^-1 r of the Stokes preconditioner (Sec. V.B,
 * Eq. P1_practical) in the preconditioner precision, r and z of length
 * (dim+1)*cells (velocity then pressure). */
int ibr_op_stokes_pc(ibr_grid* g, const double* r, double* z);

/* C = beta C + alpha A B^T on the tensor cores: the dense product of the
 * mixed-precision M~ factorisation (Sec. V.C), exposed for parity checks.
 * A [M][lda], B [N][ldb], C [M][ldc] row-major FP32 device arrays (A and B
 * 16-byte aligned, lda and ldb multiples of 4); M and N multiples of 128, K
 * a positive multiple of 32 (else IBR_EINVAL).  Each operand is split into two TF32 parts, the
 * three leading products are accumulated in FP32 (close to FP32 accuracy).
 * Issued on cuda_stream (NULL: legacy default stream) and waited for. */
int ibr_op_gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                       float alpha, float beta, void* cuda_stream);

/* N = div(v v) (the advection term of ibr_advance: centred flux form, the
 * wall extension with the wall data), v and N device arrays of dim face
 * arrays (FP64). */
int ibr_op_advect(ibr_grid* g, const double* v, double* N);

/* k V-cycles of the scalar multigrid for (sigma I - kappa Delta_h) u = f on the
 * cell grid, starting from u (in/out); on wall axes the cell-centred
 * homogeneous Neumann rule of the pressure.  sigma = 0 requires mean-zero f
 * and returns mean-zero u. */
int ibr_op_vcycle(ibr_grid* g, double sigma, double kappa, const double* f, double* u, int k);

/* The V-cycles of ibr_op_vcycle (FP64, the grid's default 2/2 sweeps when
 * pre = post = 2) for callers that cannot allocate device memory: code running
 * inside an application that gives all device memory to its own pool
 * allocator, a plug-in inside a host program that owns the CUDA context, or
 * any caller that must not trigger the allocator's device-wide
 * synchronisation.  The paper has no counterpart; this is an interface
 * service.  No grid handle: dim, n[dim] (even, >= 4), L[dim] describe the
 * periodic cell grid; f (right-hand side) and u (initial guess in, result out)
 * are device arrays of n[0]*...*n[dim-1] doubles owned by the caller; k
 * V-cycles of pre/post red-black sweeps are issued on cuda_stream (NULL: the
 * legacy default stream); asynchronous.  The coarse-level buffers live in one
 * 4 MiB file-scope device array (524288 doubles, enough for grids up to 96^3
 * or 1024x512); a grid whose coarse levels need more returns IBR_EINVAL with
 * a message.  Nothing is allocated or freed.  The first call on each device
 * looks up the array's device address (make that first call before any stream
 * capture).  Every call shares the array: calls that overlap on the GPU race,
 * and the array keeps the last call's contents. */
int ibr_op_vcycle_noalloc(int dim, const int* n, const double* L, double sigma, double kappa,
                          const double* f, double* u, int k, int pre, int post, void* cuda_stream);

/* Device bytes a periodic grid of cells n[0..dim-1] holds through a solve
 * with n_bodies prescribed bodies of n_markers[b] markers, FGMRES restart
 * `restart`, inner iterations n_s (0: 2) in `precision` with mobility model
 * mob_model: the outer Krylov workspace, the preconditioner (multigrid levels,
 * inner basis, P_S work), the marker data, the dense mobility blocks (and for
 * IBR_MOB_PAIR its table and the solves that build it; in IBR_MIXED the
 * tensor-core factorisation's padded copies and packed operands), each allocation of >= 1 MiB
 * rounded up to the allocator's 2 MiB pages.  Used by the serving engine's
 * admission control; an upper estimate of the growth of device memory in use. */
int ibr_estimate_device_bytes(int dim, const int* n, int n_bodies, const int* n_markers, int restart, int n_s,
                              int precision, int mob_model, long long* bytes);

/* ---- serving engine (continuous batching of independent solves) -----------
 * A request is one constrained solve on a periodic box from x0 = 0 (steady
 * Stokes, prescribed or free rigid bodies), the problem of ibr_solve_coupled.
 * The engine runs `slots` worker threads, each on its own non-blocking CUDA
 * stream of the device current at ibr_server_create, so requests that run at
 * the same time overlap on the GPU.  Requests start in arrival order when a
 * slot is free and the device bytes they need (ibr_estimate_device_bytes)
 * fit next to those of the running requests and of the resident grids under
 * hbm_budget_bytes; the oldest waiting request evicts idle resident grids
 * (least recently used first) to make room; younger requests that fit may
 * start ahead of it, at most 8 in a row.  A request that could never fit
 * finishes at once with IBR_ENOMEM.  Grids stay resident after a request
 * (multigrid hierarchy, Krylov workspace, marker data, factorised mobility,
 * captured preconditioner graph): a later request of the same grid shape
 * (dim, n, L, eta, precision) reuses one, and a request with the same
 * geometry (bodies, markers, mobility options) also skips the set-up.
 * Each request's result is the one ibr_solve_coupled gives for it alone:
 * every kernel of the library reduces in a fixed order, so the mix changes
 * timing only.  Thread safety: submit, poll and get_stats may be called from
 * any thread. */
#define IBR_SERVER_AUTOTUNE 1  /* flags: tune the schedule per grid shape: the
                                  first request of a shape whose opts are NULL
                                  or leave N_s automatic (n_s = 0) is solved
                                  with N_s in {1,2,3} x multigrid
                                  sweeps in {1/1, 2/2} and the fastest
                                  schedule is used for that shape from then
                                  on (requests of the shape wait for it)      */
#define IBR_RUNNING 1          /* ibr_result.status of a started request      */
#define IBR_QUEUED  2          /* ibr_result.status of a waiting request      */

typedef struct ibr_server ibr_server;  /* opaque */

typedef struct ibr_request {
    int    dim;                /* 2 or 3                                          */
    int    n[3];               /* cells per axis (even, >= 4; periodic box)        */
    double L[3];               /* box lengths, cubic cells                         */
    double eta;                /* viscosity (steady Stokes)                        */
    int    precision;          /* IBR_MIXED or IBR_FP64                            */
    int    n_bodies;           /* >= 1                                             */
    const double* x_c;         /* [n_bodies*dim] reference points (host)           */
    const double* quat;        /* [n_bodies*4] orientations (w,x,y,z), or NULL     */
    const int*    kinematics;  /* [n_bodies] IBR_PRESCRIBED / IBR_FREE, or NULL    */
    const int*    n_markers;   /* [n_bodies]                                       */
    const double* r_body;      /* [sum n_markers * dim] body-frame offsets, body
                                  after body                                      */
    const double* body_UO;     /* [n_bodies*(dim+rot)] as in ibr_solve_coupled     */
    const ibr_solve_opts* opts;/* NULL: defaults; n_s = 0 lets the autotuner pick
                                  N_s and the multigrid sweeps                    */
    int    want_fields;        /* 1: keep v and pi for ibr_server_poll             */
} ibr_request;

typedef struct ibr_result {
    int    status;             /* ibr_solve_coupled's code, IBR_ENOMEM (never fits),
                                  or IBR_RUNNING / IBR_QUEUED while pending       */
    int    iters;              /* outer FGMRES iterations                          */
    double rel_res_true;       /* true relative residual at exit                   */
    double ms_setup, ms_solve; /* as in ibr_solve_info                             */
    double t_submit_ms;        /* server clock (ms since ibr_server_create)        */
    double t_start_ms;         /* admitted to a slot                               */
    double t_end_ms;           /* result on the host                               */
    long long reserved_bytes;  /* device bytes reserved for the request's grid     */
    int    slot;               /* worker that ran it                               */
    int    reused_grid;        /* a resident grid of the same shape was reused     */
    int    reused_geometry;    /* ... with the same geometry: no set-up            */
    int    tuned;              /* this request ran the schedule autotuner          */
    int    n_s, mg_pre, mg_post; /* schedule used                                  */
    int    n_markers, n_bodies;
} ibr_result;

typedef struct ibr_server_stats {
    long long submitted, completed, rejected, queued, running;
    long long reserved_bytes, peak_reserved_bytes, budget_bytes;
    long long grids_created, grids_reused, geometry_reused, evictions, resident_grids;
    long long tuned_shapes;
} ibr_server_stats;

/* Starts the engine: slots in [1, 64] workers, hbm_budget_bytes > 0, flags 0 or
 * IBR_SERVER_AUTOTUNE. */
int ibr_server_create(ibr_server** out, int slots, long long hbm_budget_bytes, int flags);
/* Queues a request (all arrays copied; never waits for the GPU) and writes
 * its ticket.  IBR_EINVAL for malformed requests. */
int ibr_server_submit(ibr_server* s, const ibr_request* req, long long* ticket);
/* Waits up to timeout_ms (< 0: without limit, 0: no wait) for the ticket.  If
 * it has finished: copies the result (res) and, for each non-NULL pointer,
 * Lambda [N*dim], body_FT [B*(dim+rot)] (K^T Lambda per body) and, if the
 * request wanted them, v [dim*cells] and p [cells] to host memory, releases
 * the ticket and returns the request's status (ibr_last_error() gives its
 * message).  If not: IBR_EPENDING (res, if non-NULL, gets its current state);
 * IBR_EINVAL for an unknown or already collected ticket. */
int ibr_server_poll(ibr_server* s, long long ticket, double timeout_ms, ibr_result* res, double* Lambda,
                    double* body_FT, double* v, double* p);
/* Counters of the engine since ibr_server_create (requests submitted /
 * completed / rejected, queued and running now, device bytes reserved now and
 * at most, the budget, grids created / reused, geometry reuses, evictions,
 * resident grids, tuned shapes). */
int ibr_server_get_stats(ibr_server* s, ibr_server_stats* out);
/* Stops the engine: requests not yet started are dropped, running ones
 * finish, resident grids and uncollected results are freed. NULL accepted. */
int ibr_server_destroy(ibr_server* s);

/* ---- instrumentation (measurement support; the paper has no counterpart) ---
 * Process-wide.  ibr_launch_count: kernels launched by the library since it
 * was loaded.  ibr_profile_enable(1): from then on every launch is bracketed
 * by CUDA events on its own stream; ibr_profile_read(idx, ...) returns, for
 * entry idx (IBR_EINVAL past the end), a kernel-class name, launches, summed
 * event time in ms, summed algorithmic bytes (each array read or written
 * once) and summed tensor-core FLOPs (executed TF32 products; 0 for the
 * other classes; any output may be NULL); the first half of the entries count every launch of a class, the
 * second half ("<name>@large") only its launches that move >= 32 MiB.  It
 * synchronises on the recorded events.  ibr_profile_reset clears the sums.
 * While profiling is on the preconditioner runs without CUDA graphs. */
long long ibr_launch_count(void);
int ibr_profile_enable(int on);
int ibr_profile_reset(void);
int ibr_profile_read(int idx, char* name, int name_len, long long* launches, double* ms, double* bytes,
                     double* flops);

/* The smoother tiles picked by the library's autotuner: the red-black half
 * sweep of a periodic 3-D multigrid level runs 32 x by threads per block,
 * each on a column of kz cells; the first multigrid set-up of each level
 * shape times the candidates (by in {4, 8}, kz in {2..32}) on scratch arrays
 * and keeps the fastest (IBR_TUNE=0 in the environment: a fixed heuristic).
 * Entry idx: shape_c_esz[5] = n0, n1, n2, stacked fields, element bytes; by;
 * kz (any pointer may be NULL).  IBR_EINVAL past the last entry. */
int ibr_tuned_smoother_tile(int idx, int* shape_c_esz, int* by, int* kz);

/* The V-cycle schedules picked by the library's autotuner (measurement
 * support; the paper leaves the multigrid to the implementer, Sec. V.B).  On
 * a periodic 3-D grid the coarse levels of a V-cycle can run in one launch:
 * one thread-block cluster of 8 CTAs per stacked field, the levels split into
 * z-slabs held in the CTAs' shared memory (neighbouring slabs read through
 * distributed shared memory), the smallest levels in the first CTA.  The
 * first multigrid set-up of each hierarchy shape times one V-cycle with the
 * per-level kernels and with the cluster kernel taking over at each feasible
 * level, and keeps the fastest (the V-cycle's result is the same for every
 * schedule; IBR_TUNE=0 in the environment: a fixed rule, the cluster kernel
 * from the finest level of at most 32768 cells; IBR_MG_CLUSTER=0: never;
 * IBR_MG_CLUSTER_LEVEL=<l>: from level l wherever that is feasible).
 * Entry idx: shape_l_c_esz[6] = n0, n1, n2 of the finest level, levels,
 * stacked fields, element bytes; cluster_level = the level the cluster kernel
 * starts at, -2 for none (any pointer may be NULL).  IBR_EINVAL past the last
 * entry. */
int ibr_tuned_vcycle_schedule(int idx, int* shape_l_c_esz, int* cluster_level);

/* Destroys the grid and frees its device memory. NULL is accepted. */
int ibr_destroy_grid(ibr_grid* g);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* ibr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IBRIGID_H */
