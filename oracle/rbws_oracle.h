/*
 * rbws_oracle.h -- plain, slow CPU FP64 oracle for the reduced basis
 * warm-start (RBWS) method of Hou, Chen & Xia, arXiv 2311.13862.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it
 * is not part of the product.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header, table or
 * helper with the CUDA library: the operator is assembled as an explicit CSR
 * matrix here, whereas the CUDA path applies it matrix-free.
 *
 * Every function follows one passage of the paper (section / equation /
 * algorithm) and is written to be checked by eye against it.  Parallelism:
 * only the loop over independent parameter instances in orc_solve_batch and
 * orc_greedy's indicator sweep uses OpenMP; each solve itself is serial.
 *
 * Parity status: every function below is pinned by CPU tests (closed forms,
 * invariants, library cross-checks) except the trained network weights
 * produced by orc_mlp_* + an optimiser, which are "parity unpinned": only the
 * forward/backward passes are pinned (finite differences).
 */
#ifndef RBWS_ORACLE_H
#define RBWS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- O1: operator, Eq. (1) and the diffusion model of Sec. 4 ------------ */

/* Subdomain id of every interior node under the block rule: along an axis with
 * n interior nodes split into b blocks, node i (1..n) belongs to block
 * min(floor(b*i/(n+1)), b-1).  id = (kz*by + ky)*bx + kx.  map: [nz][ny][nx]. */
void orc_block_map(int nx, int ny, int nz, int bx, int by, int bz, uint8_t* map);
/* The same by coordinate on axes with a Neumann face (node i at i/n there):
 * block min(floor(b*i/n), b-1) on such an axis. */
void orc_block_map_ex(int nx, int ny, int nz, int bx, int by, int bz, const int* neumann, uint8_t* map);

/* Number of nonzeros of the 7-point pattern on an nx*ny*nz interior grid. */
int64_t orc_csr_nnz(int nx, int ny, int nz);

/* Explicit CSR of the Q affine terms A_q (kappa = e_q), all sharing one
 * pattern (row_ptr[n+1], col[nnz], sorted columns).  vals is [Q][nnz].
 * Face coefficient = arithmetic mean of the two nodes' kappa (boundary faces
 * take the interior node's kappa), scaled by 1/h^2 per axis, h = 1/(n+1).
 * Returns 0, or -1 if a map entry is >= Q. */
int orc_assemble_affine(int nx, int ny, int nz, const uint8_t* map, int Q,
                        int64_t* row_ptr, int32_t* col, double* vals);

/* The general form of orc_assemble_affine: diffusion tensor diag(kscale) times
 * kappa, and per axis either Dirichlet data at both ends (neumann[a] = 0:
 * h = 1/(n+1), nodes i*h, i = 1..n) or a homogeneous Neumann face at coordinate
 * 1 (neumann[a] = 1: h = 1/n, the last node on the face).  Node-centred finite
 * volumes: a node on a Neumann face has half a control volume, so its face
 * areas across the other axes and its right-hand side weight are halved (the
 * rows stay symmetric).  Face coefficient kscale[a] (kappa_i + kappa_j)/2 / h_a^2,
 * times the face's relative area.  (The mixed boundary value problem of the
 * paper's Example 2, Sec. 4: K = nu diag(1, 1, 1e-2), Neumann face x = 1.) */
int orc_assemble_ex(int nx, int ny, int nz, const uint8_t* map, int Q, const double* kscale,
                    const int* neumann, int64_t* row_ptr, int32_t* col, double* vals);
/* Relative control volume of each node (1, 1/2 on a Neumann face, 1/4 on an
 * edge of two): the weight of the source term in the right-hand side. */
/* The Q affine terms of an operator whose coefficient is given at the cell faces
 * (kappa_q(x) varying from node to node, as in the paper's Example 1, Sec. 4, where
 * kappa = 1 + mu_1 g(x)): Dirichlet data on the whole boundary, h = 1/(n+1), node
 * (i, j, k) at ((i+1) hx, (j+1) hy, (k+1) hz).  kfx [Q][nz][ny][nx+1] holds kappa_q on the
 * x faces (face f between nodes f-1 and f; faces 0 and nx touch the boundary), kfy
 * [Q][nz][ny+1][nx], kfz [Q][nz+1][ny][nx] likewise.  Face coefficient kappa_face / h_a^2;
 * the pattern and column order are those of orc_assemble_affine.  Returns 0. */
int orc_assemble_field(int nx, int ny, int nz, int Q, const double* kfx, const double* kfy,
                       const double* kfz, int64_t* row_ptr, int32_t* col, double* vals);
/* The Dirichlet lift of the same operator: lift [Q][n], the part of the right-hand side that
 * boundary data g gives through each term, sum over a node's boundary faces of
 * kappa_q(face) / h_a^2 times g at the boundary point across that face.  gb holds g on the six
 * boundary planes, concatenated: x = 0 and x = 1 ([nz][ny] each), y = 0 and y = 1 ([nz][nx]),
 * z = 0 and z = 1 ([ny][nx]). */
void orc_dirichlet_lift(int nx, int ny, int nz, int Q, const double* kfx, const double* kfy,
                        const double* kfz, const double* gb, double* lift);
void orc_node_weights(int nx, int ny, int nz, const int* neumann, double* w);

/* CSR of A(mu) for one parameter, assembled directly from kappa = mu[map]
 * (Eq. 1; the same face rule as above, so A(mu) = sum_q mu_q A_q up to
 * rounding).  One value array instead of Q: the memory-light form for large
 * grids with many subdomains.  Returns 0, or -1 if a map entry is >= Q. */
int orc_assemble_mu(int nx, int ny, int nz, const uint8_t* map, int Q, const double* mu,
                    int64_t* row_ptr, int32_t* col, double* vals);

/* vals_out[e] = sum_q mu[q] * vals_q[q][e]  (A(mu) = sum_q mu_q A_q). */
void orc_csr_combine(int64_t nnz, int Q, const double* vals_q, const double* mu, double* vals_out);

/* y = A x for CSR A (n rows). */
void orc_csr_matvec(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    const double* x, double* y);

/* ---- dense helpers (Cholesky), used by the reduced solves --------------- */

/* In-place lower Cholesky of the symmetric positive definite N x N matrix a
 * (row-major; only the lower triangle is read).  Returns 0, or -1 if a pivot
 * is not positive. */
int orc_cholesky(int N, double* a);
/* Solve L L^T x = b with the factor from orc_cholesky; b overwritten by x. */
void orc_cholesky_solve(int N, const double* l, double* b);

/* ---- reduced Galerkin solve, Sec. 2.3 (RB system) ----------------------- */

/* c = A_N(mu)^{-1} f_N with A_N(mu) = sum_q mu_q A_N^q.  ANq: [Q][Nmax][Nmax]
 * row-major, of which the leading N x N block is used.  Returns 0 or -1. */
int orc_rb_solve(int N, int Nmax, int Q, const double* ANq, const double* fN, const double* mu,
                 double* c);

/* ---- O2: PCG, Algorithm 1, and its restart wrapper, Algorithm 4 ---------- */

enum { ORC_PREC_NONE = 0, ORC_PREC_JACOBI = 1, ORC_PREC_MSRB = 2 };
enum { ORC_CONVERGED = 0, ORC_MAX_ITERS = 1, ORC_BREAKDOWN = 2 };

/* RB data the MSRB preconditioner (Algorithm 3) needs.  W: [N][n] (basis
 * vectors stored one after another), chol_AN: Cholesky factor of A_N(mu). */
typedef struct {
  int N;
  int64_t n;
  const double* W;
  const double* chol_AN;
} orc_msrb;

/* Solve A u = f from the initial value in u (overwritten by the result).
 * Stopping test: ||r_k||_2 / ||f||_2 < tol on the recursively updated
 * residual; on exit the true residual f - A u is formed and, if it fails the
 * test, PCG restarts from u (at most max_restarts times).  iters counts
 * applications of A to a search direction, over all restarts.  relres_hist,
 * if not NULL, receives ||r_k||/||f|| for k = 0..iters (size max_iters+1).
 * Returns the status (ORC_CONVERGED / ORC_MAX_ITERS / ORC_BREAKDOWN). */
int orc_pcg(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
            const double* f, double* u, int precond, const orc_msrb* msrb, double tol,
            int max_iters, int max_restarts, int* iters, double* relres, double* relres_hist);

/* ---- O3: greedy reduced basis, Algorithm 5 skeleton with Galerkin RB ----- */

/* Builds W (n x N, stored [N][n]) greedily over the training set mu_train
 * [n_train][Q]: first parameter = index 0; snapshot by Jacobi-PCG to
 * snapshot_tol; classical Gram-Schmidt applied twice; stop on breakdown
 * (||w|| < 1e-10 ||u||), at n_max, or when max eta < greedy_tol; next
 * parameter = argmax over not-yet-selected training points of the indicator
 * (ties: smallest index): indicator 0 = residual eta(mu) = ||f - A(mu) W c(mu)||
 * / ||f||; indicator 1 = the L1 norm of the RB coefficients with respect to the
 * unorthogonalised snapshots (Sec. 3.1), ||R^{-1} c(mu)||_1 with U = W R from
 * the Gram-Schmidt steps.
 * Outputs: W [n_max][n], ANq [Q][n_max][n_max], fN [n_max], selected [n_max],
 * eta_hist [n_max] (eta_hist[k] = max eta over the unselected training set
 * once the basis has k+1 vectors; NaN if that set is empty),
 * n_out = final N.  Returns 0 or a negative error. */
int orc_greedy(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q, int Q,
               int64_t nnz, const double* f, const double* mu_train, int n_train, int n_max,
               double greedy_tol, double snapshot_tol, int indicator, double* W, double* ANq,
               double* fN, int32_t* selected, double* eta_hist, int* n_out);

/* Residual indicator for one mu with a given basis (see orc_greedy). */
double orc_rb_indicator(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q,
                        int Q, int64_t nnz, const double* f, const double* W, int N, int Nmax,
                        const double* ANq, const double* fN, const double* mu);

/* ---- O4/O5: online batch, Algorithm 4 (RBI-PCG) -------------------------- */

enum { ORC_WARM_ZERO = 0, ORC_WARM_GALERKIN = 1, ORC_WARM_GIVEN = 2 };

/* For each of B parameters (OpenMP over instances): u0 = 0 (zero), W c with
 * c the reduced Galerkin solution (galerkin), or W c_given[b] (given, for
 * learned coefficients); then PCG with the chosen preconditioner (MSRB uses
 * the same W and A_N(mu)).  u_out: [B][n].  relres0_out: initial ||r||/||f||.
 * Returns the number of threads used (> 0), or a negative error. */
int orc_solve_batch(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q,
                    int Q, int64_t nnz, const double* f, const double* mu, int B, int warm,
                    const double* c_given, int N, int Nmax, const double* W, const double* ANq,
                    const double* fN, int precond, double tol, int max_iters, int max_restarts,
                    double* u_out, int32_t* iters_out, double* relres_out, double* relres0_out,
                    int32_t* status_out, int n_threads);

/* ---- O7: learned warm start network ------------------------------------- */

/* Fully connected p -> H -> H -> H -> N with GELU(x) = x/2 (1 + erf(x/sqrt 2))
 * after the three hidden layers.  Parameters, row-major, W_l is [out][in]:
 * W1[H][p] b1[H] W2[H][H] b2[H] W3[H][H] b3[H] W4[N][H] b4[N], concatenated.
 * x: [B][p] inputs, y: [B][N] outputs. */
int64_t orc_mlp_param_count(int p, int H, int N);
void orc_mlp_forward(int p, int H, int N, const double* params, int B, const double* x, double* y);
/* Loss L = (1/(B*N)) sum (y - t)^2 and its gradient w.r.t. every parameter
 * (grad: same layout as params).  Returns L. */
double orc_mlp_loss_grad(int p, int H, int N, const double* params, int B, const double* x,
                         const double* t, double* grad);

#ifdef __cplusplus
}
#endif
#endif
