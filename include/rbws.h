/*
 * rbws.h -- C ABI of librbws, a GB300 (sm_103a) implementation of the online
 * hot path of the reduced basis warm-start (RBWS) iterative method
 * (Hou, Chen & Xia, arXiv 2311.13862).
 *
 * The library solves, for a batch of parameters mu, the parametrised system of
 * Eq. (1), A(mu) u = f, where A(mu) = sum_q mu_q A_q is the 7-point finite
 * difference discretisation of -div(kappa grad u) on the unit cube with zero
 * Dirichlet data (the diffusion model of Sec. 4), kappa piecewise constant on
 * Q block subdomains (kappa = mu_q on subdomain q).  The interior grid has
 * nx*ny*nz nodes, h = 1/(n+1) per axis, the face coefficient between two nodes
 * is the arithmetic mean of their kappa (a boundary face takes the interior
 * node's kappa), and the 1/h^2 scaling is part of A.
 *
 * Conventions for every call:
 *  - Vectors on the grid are planar: instance b, node (i,j,k) is element
 *    b*n_dof + (k*ny + j)*nx + i (x fastest), n_dof = nx*ny*nz.
 *  - Parameter arrays are host arrays, row-major [B][Q], float64, copied by
 *    the call.
 *  - "device" pointers are CUDA device pointers on the problem's device
 *    (e.g. a torch tensor's data_ptr()); the caller owns them.  The library
 *    owns the problem, its reduced basis and surrogate network, and its own
 *    workspace (allocated lazily, kept until rbws_problem_destroy).
 *  - Calls are synchronous: they return after their GPU work is complete.
 *  - Negative status = error, nothing usable was produced; positive = result
 *    usable with a warning.  rbws_last_error() gives a message (thread-local).
 *    No C++ exception crosses this interface.
 *  - A problem handle must not be used by two threads at once.
 */
#ifndef RBWS_H
#define RBWS_H
#include <stdint.h>

#if defined(__GNUC__)
#define RBWS_API __attribute__((visibility("default")))
#else
#define RBWS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbws_problem_s* rbws_problem; /* opaque, library-owned */

typedef enum {
  RBWS_OK = 0,
  RBWS_WARN_NOT_CONVERGED = 1, /* some instances hit max_iters or broke down */
  RBWS_ERR_INVALID_ARG = -1,
  RBWS_ERR_OOM = -2,
  RBWS_ERR_CUDA = -3,
  RBWS_ERR_NO_BASIS = -4,      /* a reduced basis / surrogate is required first */
  RBWS_ERR_NOT_SPD = -5,       /* a reduced matrix failed its Cholesky factorisation */
  RBWS_ERR_DEVICE_TIMEOUT = -6, /* a bounded device-side wait ran out (no result) */
  RBWS_ERR_STATE = -7,
  RBWS_ERR_UNSUPPORTED = -8
} rbws_status;

/* Initial value of the online solve (Algorithm 4, line 2). */
typedef enum {
  RBWS_WARM_ZERO = 0,               /* u0 = 0 (the zero-start baseline)           */
  RBWS_WARM_GALERKIN = 1,           /* u0 = W A_N(mu)^{-1} W^T f (Sec. 2.3)       */
  RBWS_WARM_LEARNED = 2,            /* u0 = W c_net(mu), surrogate network          */
  RBWS_WARM_LEARNED_CORRECTED = 3,  /* c_net plus one reduced CG step on A_N c = f_N */
  RBWS_WARM_L1ROC = 4               /* u0 = W c, c = argmin ||P (f - A(mu) W c)||_2 over
                                       the collocation nodes of rbws_offline_l1roc
                                       (Sec. 3.1, the paper's RBWS initial value)     */
} rbws_warm_mode;

/* Preconditioner P of Algorithm 1. */
typedef enum {
  RBWS_PREC_NONE = 0,   /* plain CG                                           */
  RBWS_PREC_JACOBI = 1, /* P(r) = D^{-1} r, D = diag(A(mu))                      */
  RBWS_PREC_MSRB = 2,   /* Algorithm 3: one Jacobi sweep + RB correction (W)     */
  RBWS_PREC_MG = 3      /* Algorithm 2: one multigrid V-cycle (MGCG).  Levels:
                           each axis coarsened to n // 2 nodes (the even fine
                           nodes) while the level has more than 64 unknowns and
                           every axis at least 2 nodes; linear interpolation P
                           per axis; Galerkin coarse operators P^T A P; damped
                           Jacobi smoothing (omega = 2/3), 2 pre- and 2 post-
                           steps; exact solve on the coarsest level.  FP64, or
                           FP32 inside RBWS_FP32_IR (the inner iteration's
                           V-cycle in FP32, coarsest inverse formed in FP64)  */
} rbws_precond;

typedef enum {
  RBWS_FP64 = 0,    /* all CG arithmetic in FP64                                */
  RBWS_FP32_IR = 1  /* PCG in FP32 inside FP64 iterative refinement: the FP32
                       correction is folded into the FP64 solution and the
                       FP64 residual f - A u replaces the FP32 one every
                       inner_tol reduction (reliable updates); the search
                       direction is kept; convergence is decided on the FP64
                       residual                                                 */
} rbws_precision;

typedef struct { int32_t nx, ny, nz; } rbws_grid;   /* interior nodes per axis */
typedef struct { int32_t bx, by, bz; } rbws_blocks; /* block rule, Q = bx*by*bz */

/* Axes of the mixed boundary value problem (the shape of the paper's Example 2,
 * Sec. 4: diffusion tensor K = kappa diag(1, 1, 1e-2), homogeneous Neumann
 * face x = 1, homogeneous Dirichlet data elsewhere).  kappa_scale[a]: the
 * tensor's diagonal entry for axis a (> 0).  neumann_hi[a] = 1: the face at
 * coordinate 1 of axis a is a homogeneous Neumann face; the axis then has
 * h = 1/n with nodes at i/n (i = 1..n, the last one on the face) instead of
 * h = 1/(n+1).  The operator is the node-centred finite-volume form: face
 * coefficient kappa_scale[a] (kappa_i + kappa_j)/2 / h_a^2 times the face's
 * area relative to a full cell, where a node on a Neumann face has half a
 * control volume (its faces across the other axes have half the area), so A
 * stays symmetric; the matching right-hand side of a source s is s times the
 * node's relative control volume (1, 1/2 on a Neumann face, 1/4 on an edge of
 * two).  All ones / zeros: the Sec. 4 model problem of rbws_problem_create. */
typedef struct {
  double kappa_scale[3];
  int32_t neumann_hi[3];
  int32_t reserved;      /* 0 */
} rbws_axes;

/* Optional measurement record filled by rbws_solve_batch (options.profile).
 * With profiling on, iterations are launched one by one instead of as a
 * captured CUDA graph, and the first iteration of every block of check_every
 * iterations is bracketed by CUDA events on the work stream. */
typedef struct {
  int64_t launches;    /* kernels launched by the call (graph nodes included)        */
  int64_t samples;     /* iterations whose two phase kernels were timed              */
  double stencil_ms;   /* summed durations of the sampled stencil-phase launches     */
  double update_ms;    /* summed durations of the sampled update-phase launches      */
  double active_dofs;  /* summed (active instances x n_dof) over the sampled launches */
  int32_t elem_bytes;  /* 8: FP64 CG kernels were sampled; 4: FP32 inner kernels     */
  int32_t schedule;    /* FP32 kernels: -1 one node per thread, else the autotuner's
                          schedule (0..3, see rbws_autotune); -1 for FP64            */
  double precond_ms;   /* FP32_IR with RBWS_PREC_MG: summed durations of the V-cycles
                          of the sampled iterations (after the update phase)         */
  double mg_fine_ms[4]; /* ... and of their finest-level steps: two smoothing steps
                          from zero, residual, prolongation pass + one smoothing
                          step, last smoothing step + rho partials                  */
  double mg_prolong_ms; /* ... of the prolongation pass alone (part of mg_fine_ms[2]) */
} rbws_profile;

typedef struct {
  int32_t max_iters;    /* L_max of Algorithm 1 (counted over all restarts)     */
  int32_t precond;      /* rbws_precond                                          */
  int32_t precision;    /* rbws_precision                                        */
  int32_t max_restarts; /* true-residual restarts of Algorithm 4 (default 3)     */
  double inner_tol;     /* FP32_IR: an FP64 refinement step (reliable update) is
                           taken each time an instance's FP32 residual has
                           fallen by this factor since its last one (0 = auto:
                           1e-2)                                                  */
  int32_t max_outer;    /* reserved (10)                                         */
  int32_t check_every;  /* iterations between host convergence polls and, in
                           FP32_IR, reliable-update tests (0 = auto: 8, or 2
                           for FP32_IR with RBWS_PREC_MG)                      */
  void* stream;         /* cudaStream_t: all GPU work of the call is issued on it;
                           NULL = an internal stream ordered after the legacy
                           default stream                                         */
  rbws_profile* profile; /* NULL = off; else zeroed and filled by the call        */
  double* relres_hist;  /* NULL = off.  FP64 precision, rbws_solve_batch only:
                           host [B][hist_len]; entry k of instance b = ||r_k||/||f||
                           once A has been applied to k search directions (the
                           recursive residual of Algorithm 1; at a true-residual
                           check of Algorithm 4 the true residual replaces it).
                           Entry 0 is the initial residual of u0.  Entries past
                           the last iteration, or past hist_len, are NaN /
                           not written.                                          */
  int32_t hist_len;     /* entries per instance (>= 1 when relres_hist is set)   */
  int64_t wait_cycles;  /* bound of each device-side wait of the TMA-fed FP32
                           kernels (an mbarrier wait for a staged plane), in SM
                           clock cycles; 0 = the default, 4e9 (about 2 s at
                           2 GHz).  When a wait runs out the kernel flags it,
                           lets its copies in flight land and returns, and the
                           call returns RBWS_ERR_DEVICE_TIMEOUT with no result;
                           the problem stays usable.  A small value is a test
                           knob that makes the waits run out on purpose.  < 0
                           returns RBWS_ERR_INVALID_ARG.                       */
  int32_t ru_mode;      /* FP32_IR reliable updates: 0 = auto (float-float where
                           the grid takes the 4-node kernels, nx % 4 == 0, else
                           FP64), 1 = FP64 (u += d, r = f - A u in FP64), 2 =
                           float-float: the solution and the true residual are
                           kept as pairs of floats (about 48 bits) and updated
                           as r -= A d, u += d on the FP32 pipe; an instance
                           whose residual meets tol is converted to FP64 and
                           its FP64 residual decides (if it fails, the tracked
                           residual is reset from it).  2 falls back to FP64
                           where the 4-node kernels do not apply.             */
  int32_t persistent;   /* 1: an FP64 solve with the Jacobi preconditioner or none
                           runs as ONE persistent cooperative kernel: start,
                           iterations, true-residual checks and restarts, with
                           the convergence loop on the device (no host polling,
                           no graph); its grid barriers are bounded by
                           wait_cycles (RBWS_ERR_DEVICE_TIMEOUT when one runs
                           out).  rbws_solve_requests then solves the batches of
                           every grid in that one launch.  0 (default): captured
                           CUDA graphs of the phase kernels, polled by the host
                           between blocks of check_every iterations.  Ignored
                           for other precisions and preconditioners.          */
} rbws_options;

/* Fills *opt with the defaults listed above (max_iters 20000, Jacobi, FP64,
 * no profile, no residual history). */
RBWS_API void rbws_options_default(rbws_options* opt);

/* Creates a problem on CUDA device `device` (Eq. 1; kappa = mu_q on
 * subdomain q).  Exactly one of `blocks` / `subdomain_map` is non-NULL:
 *  - blocks: the block rule.  Along an axis with n nodes and b blocks, node i
 *    (1..n) lies in block min(floor(b*i/(n+1)), b-1); id = (kz*by+ky)*bx+kx;
 *    1 <= b <= 16 per axis and Q must equal bx*by*bz.
 *  - subdomain_map: host [nz][ny][nx] uint8, values < Q (copied), 1 <= Q <= 64.
 *    The grid planes across which the map changes anywhere cut each axis into
 *    segments; the map is constant on every box between them.  Supported up
 *    to 64 segments per axis and 65536 coefficient classes (a node's class is
 *    its own and its two neighbours' segments along each axis, so a segment
 *    yields up to 3 classes per axis); larger maps return
 *    RBWS_ERR_UNSUPPORTED, a value >= Q returns RBWS_ERR_INVALID_ARG.  Both
 *    checks run before any device is touched.
 * f_host: host [n_dof] right-hand side, or NULL for f = 1 at every interior
 * node (copied).  Each axis needs 2 <= n <= 1024. */
RBWS_API rbws_status rbws_problem_create(const rbws_grid* grid, const rbws_blocks* blocks,
                                const uint8_t* subdomain_map, int32_t Q, const double* f_host,
                                int device, rbws_problem* out);
/* rbws_problem_create with the axes of a mixed boundary value problem (see
 * rbws_axes; NULL = rbws_problem_create).  Blocks follow the block rule by
 * coordinate: on an axis with a Neumann face node i (at i/n) lies in block
 * min(floor(b*i/n), b-1).  f_host NULL: a unit source, i.e. the right-hand
 * side holds each node's relative control volume.  RBWS_ERR_INVALID_ARG for a
 * kappa_scale that is not positive and finite or a neumann_hi other than 0/1.
 * The multigrid preconditioner coarsens a Neumann axis like any other (n // 2
 * nodes at the even fine nodes); with n even its last coarse node lies on the
 * face. */
RBWS_API rbws_status rbws_problem_create_ex(const rbws_grid* grid, const rbws_blocks* blocks,
                                            const uint8_t* subdomain_map, int32_t Q, const double* f_host,
                                            const rbws_axes* axes, int device, rbws_problem* out);
RBWS_API void rbws_problem_destroy(rbws_problem p);
/* A problem whose coefficient varies from node to node: A(mu) = sum_q mu_q A_q with A_q
 * the 7-point operator of a diffusion coefficient kappa_q(x) given at the cell faces
 * (the paper's Example 1, Sec. 4: kappa = 1 + mu_1 g(x), i.e. Q = 2, kappa_0 = 1,
 * kappa_1 = g, mu = (1, mu_1)).  Dirichlet data on the whole boundary, h = 1/(n+1) per
 * axis, node (i, j, k) (0-based) at ((i+1) hx, (j+1) hy, (k+1) hz).
 *  - kfx: host [Q][nz][ny][nx+1], kappa_q on the x faces: face f (0..nx) of row (j, k)
 *    lies between nodes f-1 and f, faces 0 and nx touch the boundary;
 *  - kfy: host [Q][nz][ny+1][nx], kfz: host [Q][nz+1][ny][nx], likewise (all copied).
 * The face coefficient is kappa_face / h_a^2; a boundary face adds it to the diagonal and
 * its boundary value reaches the right-hand side through rbws_dirichlet_lift.  Every
 * value must be finite and >= 0, and every node needs a positive diagonal for the
 * coefficients mu the caller will pass (mu_q >= 0 with sum_q mu_q kappa_q > 0 keeps A(mu)
 * symmetric positive definite); a node whose six faces are zero in every term is
 * rejected (RBWS_ERR_INVALID_ARG).  f_host: host [n] or NULL for f = 1.  Each axis needs
 * 2 <= n <= 256 (each node is its own coefficient class, 8-bit per axis); 1 <= Q <= 64.
 * The solvers, warm starts, the greedy, L1ROC and the multigrid preconditioner (Galerkin
 * coarse operators of every term, one coefficient row per coarse node) all apply; the
 * per-instance coefficient tables take n x 8 values per instance.  Not supported:
 * rbws_apply_operator_static (RBWS_ERR_UNSUPPORTED). */
RBWS_API rbws_status rbws_problem_create_field(const rbws_grid* grid, int32_t Q, const double* kfx,
                                               const double* kfy, const double* kfz, const double* f_host,
                                               int device, rbws_problem* out);
/* The Dirichlet lift of a problem made by rbws_problem_create_field: lift_out (device
 * [Q][n] FP64, caller-owned) gets, per term q, the right-hand side that boundary data g
 * adds through A_q: sum over a node's boundary faces of kappa_q(face) / h_a^2 times g at
 * the boundary point across that face (the elimination of the boundary values from
 * -div(kappa grad u) = f).  g_host: host values on the six boundary planes, concatenated:
 * x = 0 and x = 1 ([nz][ny] each, at (0 or 1, y_j, z_k)), y = 0 and y = 1 ([nz][nx]),
 * z = 0 and z = 1 ([ny][nx]), 2 (nz ny + nz nx + ny nx) values.  The right-hand side of
 * A(mu) u = f + sum_q mu_q lift_q then holds affine data g(mu) = sum_k t_k(mu) G_k by
 * linearity (rbws_affine_sources).  RBWS_ERR_UNSUPPORTED on other problems. */
RBWS_API rbws_status rbws_dirichlet_lift(rbws_problem p, const double* g_host, void* lift_out);
/* f_out[b] = sum_k theta[b][k] F[k] for B instances: F device [K][n] FP64, theta host
 * [B][K], f_out device [B][n] FP64 (caller-owned; it must not overlap F).  1 <= K <= 64.
 * Affine right-hand sides (a source plus Dirichlet lifts, Example 1 of Sec. 4) for
 * rbws_solve_batch_rhs and rbws_offline_greedy_rhs. */
RBWS_API rbws_status rbws_affine_sources(rbws_problem p, const void* F, int32_t K, const double* theta,
                                         int32_t B, void* f_out);


/* Problem sizes: n_dof, Q and the current reduced basis dimension N (0 if
 * none).  Any pointer may be NULL. */
RBWS_API rbws_status rbws_problem_info(rbws_problem p, int64_t* n_dof, int32_t* Q, int32_t* N);

/* y[b] = A(mu[b]) x[b] for B instances (the stencil of Eq. 1 applied
 * matrix-free).  x, y: device [B][n_dof], float64 (RBWS_FP64) or float32
 * (RBWS_FP32_IR selects the FP32 kernel).  stream: cudaStream_t or NULL. */
RBWS_API rbws_status rbws_apply_operator(rbws_problem p, const double* mu, int32_t B, const void* x,
                                void* y, int32_t precision, void* stream);

/* rbws_apply_operator in the mu-interleaved layout: x, y device [nz][ny][nx][B]
 * (element (node, b) at node*B + b, node = (k*ny + j)*nx + i), float64 or float32
 * (RBWS_FP32_IR).  A warp takes 32 consecutive instances of one node.  The layout is an
 * alternative for the autotuner (rbws_autotune_layout); the solvers keep the planar one.
 * Synchronous; allocates an interleaved copy of the coefficient tables in
 * library-owned scratch. */
RBWS_API rbws_status rbws_apply_operator_interleaved(rbws_problem p, const double* mu, int32_t B, const void* x,
                                                     void* y, int32_t precision, void* stream);
/* Times y = A x for B instances in the planar layout (the z-march of the solvers) and in
 * the mu-interleaved one (rbws_apply_operator_interleaved), best of three launches each
 * after a warm-up, with CUDA events; planar_ms / interleaved_ms (may be NULL) receive the
 * times and layout_out (may be NULL) 0 for planar, 1 for interleaved, the faster one. */
RBWS_API rbws_status rbws_autotune_layout(rbws_problem p, int32_t B, int32_t precision, double* planar_ms,
                                          double* interleaved_ms, int32_t* layout_out);

/* y[b] = P(mu[b]) x[b]: the preconditioner of Algorithm 1 applied to B
 * vectors (device [B][n_dof] FP64; x and y distinct, x unchanged).  precond:
 * RBWS_PREC_JACOBI (D^{-1} x) or RBWS_PREC_MG (one V-cycle of Algorithm 2 from
 * a zero initial value, the operator RBWS_PREC_MG uses inside PCG).  Other
 * preconditioners return RBWS_ERR_UNSUPPORTED, as does RBWS_PREC_MG on a grid
 * whose coarsest level would exceed 1024 unknowns.  stream: cudaStream_t or
 * NULL; returns after the work completed. */
RBWS_API rbws_status rbws_apply_preconditioner(rbws_problem p, const double* mu, int32_t B, int32_t precond,
                                               const void* x, void* y, void* stream);

/* One FP32 multigrid V-cycle y = MG(x) (Algorithm 2) exactly as the mixed-precision
 * iteration applies it (finest level on the 4-node tiles with TMA-fed steps where the grid
 * allows): x, y device [B][n] FP32, x != y.  A test and analysis entry point; allocates
 * the FP32 iteration's buffers for B instances in library-owned scratch.  Synchronous on
 * stream (NULL: the problem's own).  RBWS_ERR_DEVICE_TIMEOUT if a stage wait ran out. */
RBWS_API rbws_status rbws_apply_mg32(rbws_problem p, const double* mu, int32_t B, const void* x, void* y,
                                     void* stream);

/* One reliable update of the mixed-precision iteration (the FP32 iteration
 * inside FP64 refinement, RBWS_FP32_IR) in float-float arithmetic, exactly as
 * rbws_solve_batch applies it with ru_mode 0 or 2 (a test entry point: it pins
 * the float-float arithmetic against an FP64 residual).  The solution and the
 * true residual are carried as pairs of floats (hi + lo); the call starts from
 * u = u0, r = f - A(mu) u0 (u0 taken at FP32 precision, as the mixed-precision
 * starts provide it) and applies one update with the correction d:
 *   r <- r - A(mu) d,   u <- u + d,
 * with the coefficients split into float pairs, Knuth's TwoSum for the sums and
 * the fused multiply-add for the exact product error.  u0: device [B][n] FP64
 * (values representable in FP32); d: device [B][n] FP32; u_out, r_out: device
 * [B][n] FP64 = hi + lo of u and r.  Needs nx % 4 == 0 (else
 * RBWS_ERR_UNSUPPORTED).  Synchronous; library-owned scratch. */
RBWS_API rbws_status rbws_update_ff(rbws_problem p, const double* mu, int32_t B, const void* u0, const void* d,
                                    void* u_out, void* r_out);

/* rbws_apply_operator for callers that cannot allocate device memory after
 * start-up: services that run inside a fixed device-memory budget shared with
 * another framework's caching allocator, or latency-sensitive code that
 * cannot accept the implicit device synchronisation cudaMalloc / cudaFree may
 * perform.  The paper has no counterpart; this is a deployment variant.
 * Same arguments and result as rbws_apply_operator, but the call allocates
 * nothing: its scratch (the device copy of mu and the per-instance
 * coefficient tables) lives in one static 4 MiB device array that every GPU
 * loading the library holds until the process exits.  A call needs
 * 8*B*Q + 64*B*C bytes (+ 32*B*C for float32), each part rounded up to 256,
 * where C is the number of coefficient classes of the grid (at most
 * (3*bx+2)*(3*by+2)*(3*bz+2)); larger requests return RBWS_ERR_INVALID_ARG
 * with the sizes in the message.  The first call on a device (and the first
 * after the caller reset that device's context) sets up the array's device
 * address with cudaGetSymbolAddress.  All calls share the array and it keeps the last call's contents;
 * every call overwrites what it reads, so nothing needs to start at zero.
 * Calls whose GPU work overlaps (from two threads, two problems on one
 * device, or two streams) race on the array.  Synchronous: the call returns
 * after its GPU work has completed. */
RBWS_API rbws_status rbws_apply_operator_static(rbws_problem p, const double* mu, int32_t B,
                                                const void* x, void* y, int32_t precision,
                                                void* stream);

/* Offline L1ROC (Sec. 3.1, Algorithm 5): the RB space and the collocation nodes
 * X^m = X_s u X_r of the over-collocation online solve.
 *  - First parameter mu_train[0]; each snapshot by Jacobi-PCG to snapshot_tol.
 *  - DEIM on the snapshots: with the k current vectors and their points, c solves
 *    W[points] c = u[points]; rho = u - W c; the new point is argmax |rho| (ties:
 *    the smaller node index) and the new vector rho / rho[point].  The space stops
 *    growing when max |rho| <= 1e-10 max |u|.
 *  - From the second snapshot on, DEIM also runs on the RB residual
 *    f - A(mu) W c(mu) of the new parameter (c from the current online solve),
 *    adding one residual point; a point already present is kept once.
 *  - The next parameter maximises the L1 indicator ||T^-1 c(mu)||_1 over the
 *    training points not yet selected, T upper triangular with U = W T (U the
 *    snapshots): the L1 norm of the coefficients in the snapshot basis.
 * The basis (not orthonormal) replaces any previous one; its Galerkin data
 * (W^T A_q W, W^T f) are formed too, so every warm mode can use it.  n_max <= 64.
 * selected_out / eta_hist_out: host [n_max] or NULL (eta_hist_out[k] = largest
 * indicator once the basis has k+1 vectors, NaN if none); n_out: final N. */
RBWS_API rbws_status rbws_offline_l1roc(rbws_problem p, const double* mu_train, int32_t n_train, int32_t n_max,
                                        double snapshot_tol, int32_t* selected_out, double* eta_hist_out,
                                        int32_t* n_out);

/* Per-instance right-hand sides (a non-affine source f(mu), the shape of the paper's
 * Example 2, Sec. 4).  The library does not store them: the caller passes device arrays.
 *
 * rbws_gaussian_source: f_out (device [B][n] FP64, caller-owned) = exp(-|x - c_b|^2 /
 * (2 s_b^2)) at the interior nodes x = ((i+1)/(nx+1), (j+1)/(ny+1), (k+1)/(nz+1)), with
 * params (host [B][4]) = (c_x, c_y, c_z, s_b).  RBWS_ERR_INVALID_ARG if s_b <= 0.  On a
 * problem with a Neumann face (rbws_problem_create_ex) the node coordinates and control-volume
 * weights of rbws_gaussian_source_ex apply. */
RBWS_API rbws_status rbws_gaussian_source(rbws_problem p, const double* params, int32_t B, void* f_out);
/* The general form: f_out[b] = (offset + amplitude exp(-|x - c_b|^2 / width))
 * times each node's relative control volume (rbws_axes), params host [B][6] =
 * (c_x, c_y, c_z, width, amplitude, offset), node coordinates i/(n+1), or i/n
 * on an axis with a Neumann face.  The paper's Example 2 source mu7 +
 * exp(-|x - (mu4, mu5, mu6)|^2 / mu7) / mu7 is (mu4, mu5, mu6, mu7, 1/mu7, mu7).
 * rbws_gaussian_source is (c, 2 s^2, 1, 0).  RBWS_ERR_INVALID_ARG if a width is
 * not positive or a parameter not finite. */
RBWS_API rbws_status rbws_gaussian_source_ex(rbws_problem p, const double* params, int32_t B, void* f_out);

/* rbws_solve_batch with right-hand side f_b (device [B][n] FP64, row b) for instance b
 * instead of the problem's f.  The relative residuals are against ||f_b||.  Warm starts:
 * RBWS_WARM_ZERO and RBWS_WARM_GALERKIN (c_b from A_N(mu_b) c_b = W^T f_b; W^T f_b formed
 * on the device: in FP64 by dot products for RBWS_FP64, and for RBWS_FP32_IR in one pass
 * over the sources with the FP32 copy of W that the mixed-precision lift also uses, FP32
 * products summed in FP64, so the start matches the FP64 one to FP32 rounding while
 * convergence is still decided on the FP64 residual); preconditioners other than MSRB.
 * Others return RBWS_ERR_UNSUPPORTED; a zero f_b RBWS_ERR_INVALID_ARG. */
RBWS_API rbws_status rbws_solve_batch_rhs(rbws_problem p, const double* mu, int32_t B, const void* f,
                                          double tol, int32_t warm, const rbws_options* opt, void* u_out,
                                          int32_t* iters_out, double* relres_out, int32_t* status_out);

/* rbws_offline_greedy (residual indicator) with a right-hand side f_t per training
 * parameter (f_train: device [n_train][n] FP64): the snapshot of mu_t solves A(mu_t) u = f_t
 * and the indicator is ||f_t - A(mu_t) W c_t|| / ||f_t|| with A_N(mu_t) c_t = W^T f_t.
 * The basis then serves rbws_solve_batch_rhs (and rbws_solve_batch, whose reduced right-hand
 * side stays W^T f for the problem's f).  Scratch: n_train x n_max doubles besides the
 * greedy's own. */
RBWS_API rbws_status rbws_offline_greedy_rhs(rbws_problem p, const double* mu_train, const void* f_train,
                                             int32_t n_train, int32_t n_max, double greedy_tol,
                                             double snapshot_tol, int32_t* selected_out,
                                             double* indicator_hist_out, int32_t* n_out);

/* Accuracy of the RB space as a function of its dimension (the r_N-versus-N view
 * of Sec. 5's offline-cost discussion, and the Galerkin RB method of Sec. 2.3):
 * relres_out[b] (host [B]) = ||f - A(mu_b) W_n c_n(mu_b)||_2 / ||f||_2, with
 * W_n the first n_use vectors of the current basis and c_n the Galerkin
 * coefficients (W_n^T A(mu_b) W_n) c_n = W_n^T f from the leading n_use x n_use
 * blocks of the reduced matrices.  mu: host [B][Q].  1 <= n_use <= N, else
 * RBWS_ERR_INVALID_ARG; RBWS_ERR_NO_BASIS without a Galerkin basis;
 * RBWS_ERR_NOT_SPD if a reduced matrix is not positive definite.  Synchronous;
 * allocates B FP64 vectors of the grid in library-owned scratch. */
RBWS_API rbws_status rbws_rb_residuals(rbws_problem p, const double* mu, int32_t B, int32_t n_use,
                                       double* relres_out);

/* The collocation data of the L1ROC basis: M_out = number of nodes; points_out
 * (host [M] or NULL) = their node indices ((z*ny + y)*nx + x) in the order they
 * were added; T_out (host [N][N] row-major or NULL) = T with U = W T.
 * RBWS_ERR_NO_BASIS without an L1ROC basis. */
RBWS_API rbws_status rbws_l1roc_info(rbws_problem p, int32_t* M_out, int64_t* points_out, double* T_out);

/* Online L1ROC solve: c_out (host [B][N]) = argmin ||P (f - A(mu_b) W c)||_2, by
 * Householder QR on the device.  RBWS_ERR_NO_BASIS without an L1ROC basis,
 * RBWS_ERR_STATE if a collocation matrix is rank deficient. */
RBWS_API rbws_status rbws_l1roc_coefficients(rbws_problem p, const double* mu, int32_t B, double* c_out);

/* Error indicators of the offline greedy. */
typedef enum {
  RBWS_INDICATOR_RESIDUAL = 0, /* eta(mu) = ||f - A(mu) W c(mu)|| / ||f|| (full-order residual) */
  RBWS_INDICATOR_L1 = 1        /* ||R^{-1} c(mu)||_1: the L1 norm of the RB coefficients with
                                  respect to the unorthogonalised snapshots (Sec. 3.1), R the
                                  Gram-Schmidt factor (u_k = sum_j R[j][k] w_j)               */
} rbws_indicator;

/* Offline greedy (Algorithm 5's loop with the Galerkin RB of Sec. 2.3 and the
 * chosen indicator): first parameter = mu_train[0]; snapshot solves by
 * Jacobi-PCG to snapshot_tol (a snapshot that stalls above snapshot_tol at
 * the rounding floor of the FP64 residual is used if its true relative
 * residual is below 1e-9); Gram-Schmidt applied twice; the next parameter
 * maximises the indicator over the training points not yet selected (ties:
 * smallest index).  Stops at n_max, when max indicator <
 * greedy_tol, or when a snapshot adds no new direction (||w|| < 1e-10 ||u||).
 * Replaces any previous basis; 1 <= n_max <= 160.  selected_out [n_max], eta_hist_out [n_max]
 * (eta_hist[k] = max eta once the basis has k+1 vectors) may be NULL. */
RBWS_API rbws_status rbws_offline_greedy(rbws_problem p, const double* mu_train, int32_t n_train,
                                int32_t n_max, double greedy_tol, double snapshot_tol,
                                int32_t indicator, int32_t* selected_out, double* eta_hist_out,
                                int32_t* n_out);

/* Installs a reduced basis computed elsewhere: W host [N][n_dof] (orthonormal
 * columns stored one after another), ANq host [Q][N][N] = W^T A_q W,
 * fN host [N] = W^T f, 1 <= N <= 160.  Copied. */
RBWS_API rbws_status rbws_set_basis(rbws_problem p, int32_t N, const double* W, const double* ANq,
                           const double* fN);
/* Copies the basis out: W host [N][n_dof], ANq host [Q][N][N], fN host [N];
 * any pointer may be NULL. */
RBWS_API rbws_status rbws_get_basis(rbws_problem p, double* W, double* ANq, double* fN);

/* Reduced Galerkin solve only: c[b] = A_N(mu[b])^{-1} f_N, host out [B][N]. */
RBWS_API rbws_status rbws_reduced_solve(rbws_problem p, const double* mu, int32_t B, double* c_out);

/* ---- learned warm start (a production pattern on top of the paper) -------
 * A fully connected network x(mu) -> p -> H -> H -> H -> N with GELU (erf
 * form) after the hidden layers predicts the reduced coefficients c(mu) of
 * the current basis (N = basis dimension, p = Q); the warm start is u0 = W c
 * (Algorithm 4, line 2, with the network in place of the RB solver).  Inputs
 * x_q = 2 (log mu_q - log mu_lo) / (log mu_hi - log mu_lo) - 1; outputs are
 * scaled by per-coefficient RMS factors of the training targets.  Weights are
 * BF16 tensor-core operands with FP32 accumulation and FP32 master copies.
 * Parameter layout (float): W1[H][p] b1[H] W2[H][H] b2[H] W3[H][H] b3[H]
 * W4[N][H] b4[N], W_l row-major [out][in]. */

/* Trains the network on the GPU: targets host [n][N] (NULL = the reduced
 * Galerkin coefficients of the n parameters, computed on the device), loss =
 * mean squared error of the scaled coefficients, Adam (beta 0.9/0.999, eps
 * 1e-8) with learning rate lr, minibatches of `batch` in the given order
 * (the remainder n % batch is unused), `epochs` passes.
 *  - Coefficient scales: scale_j = sqrt(mean_b c[b][j]^2) over the n targets
 *    (1 where that is 0), rounded to FP32; the network fits c[b][j] / scale_j.
 *  - Initial parameters, U(-1/sqrt(fan_in), 1/sqrt(fan_in)): parameter i
 *    (0-based, in the layout above) takes the (i+1)-th output z of splitmix64
 *    started from state `seed` (Steele, Lea & Flood 2014), u = (z >> 11) 2^-53,
 *    and the value (2u - 1) b rounded to FP32, with b = 1/sqrt(fan_in) rounded
 *    to FP32 and fan_in the layer's input width (p for W1 and b1, H for the
 *    others).  epochs = 0 installs these parameters untrained.
 *  - Adam (Kingma & Ba 2015, Algorithm 1), per minibatch step t = 1, 2, ...:
 *    m = 0.9 m + 0.1 g, v = 0.999 v + 0.001 g^2,
 *    w -= lr (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8), in FP32.
 * final_loss_out: mean minibatch loss of the last epoch (NaN if epochs = 0).
 * Needs a basis; replaces any previous network. */
RBWS_API rbws_status rbws_train_surrogate(rbws_problem p, const double* mu, int32_t n,
                                          const double* targets, int32_t hidden, int32_t epochs,
                                          int32_t batch, double lr, double mu_lo, double mu_hi,
                                          uint64_t seed, double* final_loss_out);
/* Installs network parameters (host float, layout above) and coefficient
 * scales (host [N] or NULL = ones) for the current basis dimension N. */
RBWS_API rbws_status rbws_surrogate_set_params(rbws_problem p, int32_t hidden, const float* params,
                                               const float* coef_scale, double mu_lo, double mu_hi);
/* Copies the network out (any pointer may be NULL). */
RBWS_API rbws_status rbws_surrogate_get_params(rbws_problem p, int32_t* hidden, float* params,
                                               float* coef_scale);
/* Predicted coefficients c[b] (host [B][N]) for B parameters; corrected != 0
 * adds one reduced CG step on A_N(mu) c = f_N from the prediction. */
RBWS_API rbws_status rbws_surrogate_forward(rbws_problem p, const double* mu, int32_t B,
                                            int32_t corrected, double* c_out);
/* Loss and gradient of the current network on given inputs x (host [B][p],
 * already normalised) and scaled targets t (host [B][N]); grad_out host [P]
 * (layout above) may be NULL.  For gradient checks. */
RBWS_API rbws_status rbws_surrogate_loss_grad(rbws_problem p, const float* x, const float* t,
                                              int32_t B, double* loss_out, float* grad_out);

/* Online batched solve: Algorithm 4 with the chosen initial value and
 * preconditioner for B parameters.  Stopping test ||r||_2/||f||_2 < tol on
 * the recursive residual, then a true-residual check with restarts.
 * u_out: device [B][n_dof] float64.  iters_out (host [B]) = applications of
 * A to a search direction (inner iterations for FP32_IR), 0 if the initial
 * value already meets tol.  relres_out (host [B], may be NULL) = final true
 * relative residual.  status_out (host [B], may be NULL): 0 converged,
 * 1 max_iters, 2 breakdown.  opt may be NULL (defaults).  Returns RBWS_OK,
 * RBWS_WARN_NOT_CONVERGED, or an error. */
RBWS_API rbws_status rbws_solve_batch(rbws_problem p, const double* mu, int32_t B, double tol,
                             int32_t warm, const rbws_options* opt, void* u_out,
                             int32_t* iters_out, double* relres_out, int32_t* status_out);

/* Autotuner of the FP32 PCG phase kernels for batches of B instances on this
 * problem's grid (needs nx % 4 == 0): times each candidate tile (4*tx x ty
 * nodes, tx in {32,16,8,4}, 64..256 threads), z-chunk (8..64 planes) and
 * iteration schedule (0: 44 bytes per DoF with s and A p stored; 1: 32 bytes,
 * s formed on the fly and A p recomputed; 2: schedule 0 with its stencil
 * phase fed by TMA; 3: 32 bytes with s = D^{-1} r stored and both phases fed
 * by TMA) on the GPU with CUDA events, and
 * keeps the fastest for later FP32_IR solves with B instances.  cache_path
 * (may be NULL): a text file of "grid/B/fp32 tx ty zc ms schedule" lines; a
 * matching line is used without timing, a new choice is appended.  Outputs
 * (may be NULL): the chosen tile, chunk and the mean time in ms of one
 * stencil-phase plus update-phase pair. */
RBWS_API rbws_status rbws_autotune(rbws_problem p, int32_t B, const char* cache_path, int32_t* tx_out,
                                   int32_t* ty_out, int32_t* zc_out, int32_t* schedule_out,
                                   double* ms_out);

/* Solves n_req single-parameter requests that may live on different grids
 * (problems) in one call: the requests of each problem form one batch, and
 * the batches of different problems run concurrently, each on its problem's
 * own stream.  mu[r]: host [Q of probs[r]]; u_out[r]: device [n_dof of
 * probs[r]] float64.  iters_out (host [n_req]); relres_out, status_out and
 * latency_ms_out (host [n_req]) may be NULL.  latency_ms_out[r] = time from
 * the start of the earliest batch to the moment request r reached its final
 * status, from the GPU's global timer.  opt->stream, opt->profile and
 * opt->relres_hist must be NULL.  A problem must not be used by another call
 * meanwhile. */
RBWS_API rbws_status rbws_solve_requests(int32_t n_req, const rbws_problem* probs,
                                         const double* const* mu, void* const* u_out, double tol,
                                         int32_t warm, const rbws_options* opt, int32_t* iters_out,
                                         double* relres_out, int32_t* status_out,
                                         double* latency_ms_out);

/* Checkpoint of the offline stage (the paper's offline/online split): writes
 * the problem description (grid, blocks, map or face fields, axes, f), the
 * reduced basis W, A_N^q, f_N and the surrogate network (if any) to `path` in a
 * versioned binary format (version 3, or 4 for a face-field problem; rbws_load
 * also reads version 2, written before the axes existed) with an FNV-1a
 * checksum.  Synchronous; the problem is unchanged. */
RBWS_API rbws_status rbws_save(rbws_problem p, const char* path);
/* Creates a problem on `device` from a checkpoint written by rbws_save.
 * Returns RBWS_ERR_STATE with a message if the file is not a checkpoint, has
 * another version, is truncated, or fails its checksum. */
RBWS_API rbws_status rbws_load(const char* path, int device, rbws_problem* out);

/* Thread-local message for the last error (never NULL). */
RBWS_API const char* rbws_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
