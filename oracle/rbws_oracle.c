/*
 * rbws_oracle.c -- plain CPU FP64 oracle of the RBWS method (arXiv 2311.13862).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Straight loops,
 * explicit CSR, textbook algorithms; no blocking or fusion.  See the header
 * for what each function computes and which passage it follows.
 */
#include "rbws_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* O1. Operator (Eq. 1; diffusion model of Sec. 4 discretised by 7-point FD) */
/* ------------------------------------------------------------------------ */

static int block_of(int i, int n, int b) {
  /* node i in 1..n of an axis with n interior nodes, cut into b blocks */
  int k = (int)(((int64_t)b * i) / (n + 1));
  return k < b - 1 ? k : b - 1;
}

void orc_block_map(int nx, int ny, int nz, int bx, int by, int bz, uint8_t* map) {
  for (int k = 1; k <= nz; k++)
    for (int j = 1; j <= ny; j++)
      for (int i = 1; i <= nx; i++) {
        int id = (block_of(k, nz, bz) * by + block_of(j, ny, by)) * bx + block_of(i, nx, bx);
        map[((int64_t)(k - 1) * ny + (j - 1)) * nx + (i - 1)] = (uint8_t)id;
      }
}

void orc_block_map_ex(int nx, int ny, int nz, int bx, int by, int bz, const int* neumann, uint8_t* map) {
  for (int k = 1; k <= nz; k++)
    for (int j = 1; j <= ny; j++)
      for (int i = 1; i <= nx; i++) {
        /* node i of an axis sits at i/(n+1), or at i/n on an axis with a Neumann face */
        const int kx = block_of(i, neumann[0] ? nx - 1 : nx, bx);
        const int ky = block_of(j, neumann[1] ? ny - 1 : ny, by);
        const int kz = block_of(k, neumann[2] ? nz - 1 : nz, bz);
        map[((int64_t)(k - 1) * ny + (j - 1)) * nx + (i - 1)] = (uint8_t)((kz * by + ky) * bx + kx);
      }
}

int64_t orc_csr_nnz(int nx, int ny, int nz) {
  int64_t n = (int64_t)nx * ny * nz;
  /* diagonal + one entry per interior-interior face, counted from both ends */
  int64_t faces = (int64_t)(nx - 1) * ny * nz + (int64_t)nx * (ny - 1) * nz +
                  (int64_t)nx * ny * (nz - 1);
  return n + 2 * faces;
}

int orc_assemble_ex(int nx, int ny, int nz, const uint8_t* map, int Q, const double* kscale,
                    const int* neumann, int64_t* row_ptr, int32_t* col, double* vals) {
  /* Node-centred finite volumes on the unit cube.  Along axis a with n nodes:
   * Dirichlet at both ends, h = 1/(n+1), nodes at i*h (i = 1..n); or, with a
   * homogeneous Neumann face at coordinate 1, h = 1/n and the last node lies on
   * that face with a half control volume.  The flux through a face is
   * kf * (u_self - u_nb) / h_a^2 times the face's area relative to a full cell;
   * kf = kscale[a] * (kappa_self + kappa_nb) / 2, a Dirichlet boundary face taking
   * kappa_self.  With no Neumann face and kscale = 1 this is the 7-point FD
   * operator of the Sec. 4 diffusion model. */
  const int n3[3] = {nx, ny, nz};
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t nnz = orc_csr_nnz(nx, ny, nz);
  double inv_h2[3];
  for (int a = 0; a < 3; a++) {
    const double cells = neumann[a] ? (double)n3[a] : (double)(n3[a] + 1);
    inv_h2[a] = 1.0 / ((1.0 / cells) * (1.0 / cells));
  }
  for (int64_t e = 0; e < n; e++)
    if (map[e] >= Q) return -1;
  memset(vals, 0, sizeof(double) * (size_t)Q * (size_t)nnz);

  int64_t pos = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        const int64_t row = ((int64_t)k * ny + j) * nx + i;
        const int q_self = map[row];
        const int idx[3] = {i, j, k};
        /* relative width of the control volume along each axis: 1/2 on a Neumann face */
        double wid[3];
        for (int a = 0; a < 3; a++) wid[a] = (neumann[a] && idx[a] == n3[a] - 1) ? 0.5 : 1.0;
        row_ptr[row] = pos;
        /* the six neighbours: (di,dj,dk) and the axis of each */
        const int di[6] = {0, 0, 0, 0, -1, 1};
        const int dj[6] = {0, 0, -1, 1, 0, 0};
        const int dk[6] = {-1, 1, 0, 0, 0, 0};
        const int ax[6] = {2, 2, 1, 1, 0, 0};
        /* Columns in increasing order: z-1, y-1, x-1, self, x+1, y+1, z+1. */
        const int order[7] = {0, 2, 4, -1, 5, 3, 1};
        int64_t diag_pos = -1;
        for (int t = 0; t < 7; t++) {
          int f = order[t];
          if (f < 0) {
            diag_pos = pos;
            col[pos] = (int32_t)row;
            pos++;
            continue;
          }
          int ii = i + di[f], jj = j + dj[f], kk = k + dk[f];
          int interior = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
          if (!interior) continue;
          col[pos] = (int32_t)(((int64_t)kk * ny + jj) * nx + ii);
          pos++;
        }
        int64_t p = row_ptr[row];
        for (int t = 0; t < 7; t++) {
          int f = order[t];
          if (f < 0) { p++; continue; }
          const int a = ax[f];
          int ii = i + di[f], jj = j + dj[f], kk = k + dk[f];
          int interior = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
          /* past the last node of a Neumann axis there is no face at all */
          const int step = a == 0 ? di[f] : (a == 1 ? dj[f] : dk[f]);
          if (!interior && neumann[a] && step > 0) continue;
          /* area of the face relative to a full cell face: the widths across it */
          const double area = wid[(a + 1) % 3] * wid[(a + 2) % 3];
          int q_nb = interior ? map[((int64_t)kk * ny + jj) * nx + ii] : q_self;
          for (int q = 0; q < Q; q++) {
            double kap_self = (q == q_self) ? 1.0 : 0.0;
            double kap_nb = (q == q_nb) ? 1.0 : 0.0;
            double kf = 0.5 * (kap_self + kap_nb) * kscale[a] * inv_h2[a] * area;
            vals[(int64_t)q * nnz + diag_pos] += kf;
            if (interior) vals[(int64_t)q * nnz + p] -= kf;
          }
          if (interior) p++;
        }
      }
  row_ptr[n] = pos;
  return pos == nnz ? 0 : -2;
}

/* The diffusion coefficient given at the cell faces (a coefficient that varies from node to
 * node, as in the paper's Example 1, Sec. 4).  Node (i, j, k), 0-based, sits at
 * ((i+1) hx, (j+1) hy, (k+1) hz) with h = 1/(n+1) per axis and Dirichlet data on the whole
 * boundary.  The x face f (0..nx) of row (j, k) lies between nodes f-1 and f (node -1 and
 * node nx being boundary points); kfx[q][k][j][f] is kappa_q there, and likewise
 * kfy[q][k][f][i] (f = 0..ny) and kfz[q][f][j][i] (f = 0..nz).  The flux through a face is
 * kappa_face (u_self - u_nb) / h_a^2; a boundary face adds kappa_face / h_a^2 to the
 * diagonal (its boundary value goes to the right-hand side, orc_dirichlet_lift). */
static double field_face(int nx, int ny, int nz, int q, const double* kfx, const double* kfy,
                         const double* kfz, int i, int j, int k, int dir) {
  /* dir: 0 west, 1 east, 2 south, 3 north, 4 down, 5 up */
  switch (dir) {
    case 0: return kfx[(((int64_t)q * nz + k) * ny + j) * (nx + 1) + i];
    case 1: return kfx[(((int64_t)q * nz + k) * ny + j) * (nx + 1) + i + 1];
    case 2: return kfy[(((int64_t)q * nz + k) * (ny + 1) + j) * nx + i];
    case 3: return kfy[(((int64_t)q * nz + k) * (ny + 1) + j + 1) * nx + i];
    case 4: return kfz[(((int64_t)q * (nz + 1) + k) * ny + j) * nx + i];
    default: return kfz[(((int64_t)q * (nz + 1) + k + 1) * ny + j) * nx + i];
  }
}

int orc_assemble_field(int nx, int ny, int nz, int Q, const double* kfx, const double* kfy,
                       const double* kfz, int64_t* row_ptr, int32_t* col, double* vals) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t nnz = orc_csr_nnz(nx, ny, nz);
  const double inv_h2[3] = {(double)(nx + 1) * (nx + 1), (double)(ny + 1) * (ny + 1),
                            (double)(nz + 1) * (nz + 1)};
  memset(vals, 0, sizeof(double) * (size_t)Q * (size_t)nnz);
  int64_t pos = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        const int64_t row = ((int64_t)k * ny + j) * nx + i;
        row_ptr[row] = pos;
        /* the neighbour through each face, in increasing column order:
         * down (z-1), south (y-1), west (x-1), self, east (x+1), north (y+1), up (z+1) */
        const int dirs[7] = {4, 2, 0, -1, 1, 3, 5};
        const int ddx[6] = {-1, 1, 0, 0, 0, 0}, ddy[6] = {0, 0, -1, 1, 0, 0}, ddz[6] = {0, 0, 0, 0, -1, 1};
        const int axis[6] = {0, 0, 1, 1, 2, 2};
        int64_t diag = -1;
        for (int t = 0; t < 7; t++) {
          const int d = dirs[t];
          if (d < 0) {
            diag = pos;
            col[pos++] = (int32_t)row;
            continue;
          }
          const int ii = i + ddx[d], jj = j + ddy[d], kk = k + ddz[d];
          if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
          col[pos++] = (int32_t)(((int64_t)kk * ny + jj) * nx + ii);
        }
        /* values: every face adds to the diagonal; an interior face also gives -coef */
        int64_t p = row_ptr[row];
        for (int t = 0; t < 7; t++) {
          const int d = dirs[t];
          if (d < 0) { p++; continue; }
          const int ii = i + ddx[d], jj = j + ddy[d], kk = k + ddz[d];
          const int interior = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
          for (int q = 0; q < Q; q++) {
            const double c = field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, d) * inv_h2[axis[d]];
            vals[(int64_t)q * nnz + diag] += c;
            if (interior) vals[(int64_t)q * nnz + p] -= c;
          }
          if (interior) p++;
        }
      }
  row_ptr[n] = pos;
  return pos == nnz ? 0 : -2;
}

void orc_dirichlet_lift(int nx, int ny, int nz, int Q, const double* kfx, const double* kfy,
                        const double* kfz, const double* gb, double* lift) {
  /* gb: the Dirichlet data on the six boundary planes, concatenated:
   * x = 0 [nz][ny], x = 1 [nz][ny], y = 0 [nz][nx], y = 1 [nz][nx], z = 0 [ny][nx], z = 1 [ny][nx],
   * each value at the boundary point facing an interior node across one face.
   * lift[q][node] = sum over the node's boundary faces of kappa_q(face) / h_a^2 * g. */
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t ox0 = 0, ox1 = (int64_t)nz * ny, oy0 = 2 * (int64_t)nz * ny, oy1 = oy0 + (int64_t)nz * nx,
                oz0 = oy1 + (int64_t)nz * nx, oz1 = oz0 + (int64_t)ny * nx;
  const double ihx = (double)(nx + 1) * (nx + 1), ihy = (double)(ny + 1) * (ny + 1),
               ihz = (double)(nz + 1) * (nz + 1);
  for (int q = 0; q < Q; q++)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          double v = 0.0;
          if (i == 0) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 0) * ihx * gb[ox0 + (int64_t)k * ny + j];
          if (i == nx - 1) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 1) * ihx * gb[ox1 + (int64_t)k * ny + j];
          if (j == 0) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 2) * ihy * gb[oy0 + (int64_t)k * nx + i];
          if (j == ny - 1) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 3) * ihy * gb[oy1 + (int64_t)k * nx + i];
          if (k == 0) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 4) * ihz * gb[oz0 + (int64_t)j * nx + i];
          if (k == nz - 1) v += field_face(nx, ny, nz, q, kfx, kfy, kfz, i, j, k, 5) * ihz * gb[oz1 + (int64_t)j * nx + i];
          lift[(int64_t)q * n + ((int64_t)k * ny + j) * nx + i] = v;
        }
}

void orc_node_weights(int nx, int ny, int nz, const int* neumann, double* w) {
  /* volume of each node's control volume relative to a full cell */
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double v = 1.0;
        if (neumann[0] && i == nx - 1) v *= 0.5;
        if (neumann[1] && j == ny - 1) v *= 0.5;
        if (neumann[2] && k == nz - 1) v *= 0.5;
        w[((int64_t)k * ny + j) * nx + i] = v;
      }
}

int orc_assemble_affine(int nx, int ny, int nz, const uint8_t* map, int Q,
                        int64_t* row_ptr, int32_t* col, double* vals) {
  const double one[3] = {1.0, 1.0, 1.0};
  const int none[3] = {0, 0, 0};
  return orc_assemble_ex(nx, ny, nz, map, Q, one, none, row_ptr, col, vals);
}

int orc_assemble_mu(int nx, int ny, int nz, const uint8_t* map, int Q, const double* mu,
                    int64_t* row_ptr, int32_t* col, double* vals) {
  /* Eq. (1) for one parameter, written out directly: kappa(node) = mu[map(node)],
   * face coefficient (kappa_self + kappa_nb)/2 (a boundary face: kappa_self),
   * scaled by 1/h^2 of its axis; the face adds to the diagonal and its negative
   * goes to the neighbour's column.  Same sparsity pattern and column order as
   * orc_assemble_affine. */
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t nnz = orc_csr_nnz(nx, ny, nz);
  const double sx = (double)(nx + 1) * (nx + 1);
  const double sy = (double)(ny + 1) * (ny + 1);
  const double sz = (double)(nz + 1) * (nz + 1);
  for (int64_t e = 0; e < n; e++)
    if (map[e] >= Q) return -1;
  int64_t pos = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        const int64_t row = ((int64_t)k * ny + j) * nx + i;
        const double kap = mu[map[row]];
        /* neighbours in increasing column order: z-1, y-1, x-1, (self), x+1, y+1, z+1 */
        const int di[6] = {0, 0, -1, 1, 0, 0};
        const int dj[6] = {0, -1, 0, 0, 1, 0};
        const int dk[6] = {-1, 0, 0, 0, 0, 1};
        const double sc[6] = {sz, sy, sx, sx, sy, sz};
        row_ptr[row] = pos;
        double diag = 0.0;
        int64_t diag_pos = -1;
        for (int t = 0; t < 6; t++) {
          if (t == 3) { /* the diagonal sits between x-1 and x+1 */
            diag_pos = pos;
            col[pos++] = (int32_t)row;
          }
          const int ii = i + di[t], jj = j + dj[t], kk = k + dk[t];
          const int interior = ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz;
          const int64_t nb = ((int64_t)kk * ny + jj) * nx + ii;
          const double kf = interior ? 0.5 * (kap + mu[map[nb]]) * sc[t] : kap * sc[t];
          diag += kf;
          if (interior) {
            col[pos] = (int32_t)nb;
            vals[pos] = -kf;
            pos++;
          }
        }
        vals[diag_pos] = diag;
      }
  row_ptr[n] = pos;
  return pos == nnz ? 0 : -2;
}

void orc_csr_combine(int64_t nnz, int Q, const double* vals_q, const double* mu, double* vals_out) {
  for (int64_t e = 0; e < nnz; e++) {
    double s = 0.0;
    for (int q = 0; q < Q; q++) s += mu[q] * vals_q[(int64_t)q * nnz + e];
    vals_out[e] = s;
  }
}

void orc_csr_matvec(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                    const double* x, double* y) {
  for (int64_t r = 0; r < n; r++) {
    double s = 0.0;
    for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; e++) s += val[e] * x[col[e]];
    y[r] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Vector and dense helpers                                                  */
/* ------------------------------------------------------------------------ */

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

static double norm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

int orc_cholesky(int N, double* a) {
  for (int j = 0; j < N; j++) {
    double d = a[j * N + j];
    for (int k = 0; k < j; k++) d -= a[j * N + k] * a[j * N + k];
    if (!(d > 0.0)) return -1;
    double ljj = sqrt(d);
    a[j * N + j] = ljj;
    for (int i = j + 1; i < N; i++) {
      double s = a[i * N + j];
      for (int k = 0; k < j; k++) s -= a[i * N + k] * a[j * N + k];
      a[i * N + j] = s / ljj;
    }
    for (int i = 0; i < j; i++) a[i * N + j] = 0.0; /* clear the upper triangle */
  }
  return 0;
}

void orc_cholesky_solve(int N, const double* l, double* b) {
  for (int i = 0; i < N; i++) { /* L y = b */
    double s = b[i];
    for (int k = 0; k < i; k++) s -= l[i * N + k] * b[k];
    b[i] = s / l[i * N + i];
  }
  for (int i = N - 1; i >= 0; i--) { /* L^T x = y */
    double s = b[i];
    for (int k = i + 1; k < N; k++) s -= l[k * N + i] * b[k];
    b[i] = s / l[i * N + i];
  }
}

/* A_N(mu) = sum_q mu_q A_N^q (leading N x N block of Nmax x Nmax terms). */
static void reduced_matrix(int N, int Nmax, int Q, const double* ANq, const double* mu, double* a) {
  for (int i = 0; i < N; i++)
    for (int j = 0; j < N; j++) {
      double s = 0.0;
      for (int q = 0; q < Q; q++) s += mu[q] * ANq[((int64_t)q * Nmax + i) * Nmax + j];
      a[i * N + j] = s;
    }
}

int orc_rb_solve(int N, int Nmax, int Q, const double* ANq, const double* fN, const double* mu,
                 double* c) {
  double* a = (double*)malloc(sizeof(double) * (size_t)N * N + 1);
  reduced_matrix(N, Nmax, Q, ANq, mu, a);
  int rc = orc_cholesky(N, a);
  if (rc == 0) {
    for (int i = 0; i < N; i++) c[i] = fN[i];
    orc_cholesky_solve(N, a, c);
  }
  free(a);
  return rc;
}

/* u = W c with W stored [N][n]. */
static void lift(int64_t n, int N, const double* W, const double* c, double* u) {
  for (int64_t i = 0; i < n; i++) u[i] = 0.0;
  for (int j = 0; j < N; j++)
    for (int64_t i = 0; i < n; i++) u[i] += c[j] * W[(int64_t)j * n + i];
}

/* ------------------------------------------------------------------------ */
/* O2. PCG (Algorithm 1) with preconditioners P = I, D^{-1} (Jacobi), MSRB   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  int kind;
  const double* dinv;   /* Jacobi: 1 / diag(A) */
  const orc_msrb* msrb; /* MSRB: W and chol(A_N(mu)) */
  double* t1;           /* scratch, n */
  double* t2;           /* scratch, n */
} precond_ctx;

/* s = P(r).  MSRB, Algorithm 3 with one undamped Jacobi sweep from zero:
 *   u~ = D^{-1} b,  res = b - A u~,  u_rb = W A_N^{-1} W^T res,  s = u~ + u_rb. */
static void apply_precond(const precond_ctx* P, const double* r, double* s) {
  const int64_t n = P->n;
  if (P->kind == ORC_PREC_NONE) {
    for (int64_t i = 0; i < n; i++) s[i] = r[i];
    return;
  }
  for (int64_t i = 0; i < n; i++) s[i] = P->dinv[i] * r[i];
  if (P->kind == ORC_PREC_JACOBI) return;
  const orc_msrb* m = P->msrb;
  orc_csr_matvec(n, P->row_ptr, P->col, P->val, s, P->t1);
  for (int64_t i = 0; i < n; i++) P->t1[i] = r[i] - P->t1[i];
  double cN[512];
  for (int j = 0; j < m->N; j++) cN[j] = dot(n, m->W + (int64_t)j * n, P->t1);
  orc_cholesky_solve(m->N, m->chol_AN, cN);
  lift(n, m->N, m->W, cN, P->t2);
  for (int64_t i = 0; i < n; i++) s[i] += P->t2[i];
}

int orc_pcg(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
            const double* f, double* u, int precond, const orc_msrb* msrb, double tol,
            int max_iters, int max_restarts, int* iters, double* relres, double* relres_hist) {
  double* r = (double*)malloc(sizeof(double) * n);
  double* s = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  double* dinv = (double*)malloc(sizeof(double) * n);
  double* t1 = (double*)malloc(sizeof(double) * n);
  double* t2 = (double*)malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; i++) {
    double d = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
      if (col[e] == i) d = val[e];
    dinv[i] = 1.0 / d;
  }
  precond_ctx P = {n, row_ptr, col, val, precond, dinv, msrb, t1, t2};
  const double fnorm = norm2(n, f);
  int k = 0, status = ORC_CONVERGED;
  double rel = 0.0;

  for (int attempt = 0; attempt <= max_restarts; attempt++) {
    /* r_0 = f - A u_0, s_0 = P(r_0), p_0 = s_0 */
    orc_csr_matvec(n, row_ptr, col, val, u, q);
    for (int64_t i = 0; i < n; i++) r[i] = f[i] - q[i];
    rel = norm2(n, r) / fnorm;
    if (relres_hist && attempt == 0) relres_hist[0] = rel;
    if (rel < tol) { status = ORC_CONVERGED; break; } /* true residual meets the test */
    if (k >= max_iters) { status = ORC_MAX_ITERS; break; }
    apply_precond(&P, r, s);
    for (int64_t i = 0; i < n; i++) p[i] = s[i];
    double rs = dot(n, r, s);
    status = ORC_MAX_ITERS;
    /* continue while ||r_k||/||f|| >= tol and k < L_max (Alg. 1's loop test
     * read as "not yet converged") */
    while (rel >= tol && k < max_iters) {
      orc_csr_matvec(n, row_ptr, col, val, p, q);
      double pq = dot(n, p, q);
      if (!(pq > 0.0)) { status = ORC_BREAKDOWN; break; }
      double alpha = rs / pq;
      for (int64_t i = 0; i < n; i++) u[i] += alpha * p[i];
      for (int64_t i = 0; i < n; i++) r[i] -= alpha * q[i];
      apply_precond(&P, r, s);
      double rs_new = dot(n, r, s);
      double beta = rs_new / rs;
      rs = rs_new;
      for (int64_t i = 0; i < n; i++) p[i] = s[i] + beta * p[i];
      k++;
      rel = norm2(n, r) / fnorm;
      if (relres_hist) relres_hist[k] = rel;
    }
    if (status == ORC_BREAKDOWN) break;
    if (rel >= tol) { status = ORC_MAX_ITERS; break; }
    /* the recursive residual passed: check the true residual (Algorithm 4)
     * on the next pass of the attempt loop, restarting from u if needed */
    status = ORC_CONVERGED;
    if (attempt == max_restarts) {
      orc_csr_matvec(n, row_ptr, col, val, u, q);
      for (int64_t i = 0; i < n; i++) r[i] = f[i] - q[i];
      rel = norm2(n, r) / fnorm;
      if (rel >= tol) status = ORC_MAX_ITERS;
    }
  }
  *iters = k;
  *relres = rel;
  free(r); free(s); free(p); free(q); free(dinv); free(t1); free(t2);
  return status;
}

/* ------------------------------------------------------------------------ */
/* O3. Greedy RB (Algorithm 5 skeleton; Galerkin RB system of Sec. 2.3)      */
/* ------------------------------------------------------------------------ */

double orc_rb_indicator(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q,
                        int Q, int64_t nnz, const double* f, const double* W, int N, int Nmax,
                        const double* ANq, const double* fN, const double* mu) {
  double c[512];
  double* val = (double*)malloc(sizeof(double) * nnz);
  double* u = (double*)malloc(sizeof(double) * n);
  double* au = (double*)malloc(sizeof(double) * n);
  double eta = INFINITY;
  if (orc_rb_solve(N, Nmax, Q, ANq, fN, mu, c) == 0) {
    orc_csr_combine(nnz, Q, vals_q, mu, val);
    lift(n, N, W, c, u);
    orc_csr_matvec(n, row_ptr, col, val, u, au);
    for (int64_t i = 0; i < n; i++) au[i] = f[i] - au[i];
    eta = norm2(n, au) / norm2(n, f);
  }
  free(val); free(u); free(au);
  return eta;
}

/* L1 indicator: c w.r.t. W -> x = R^{-1} c w.r.t. the snapshots (U = W R,
 * R upper triangular [Nmax][Nmax]); returns sum |x_j|. */
static double l1_indicator(int N, int Nmax, const double* R, const double* c) {
  double x[512];
  for (int i = N - 1; i >= 0; i--) {
    double s = c[i];
    for (int k = i + 1; k < N; k++) s -= R[i * Nmax + k] * x[k];
    x[i] = s / R[i * Nmax + i];
  }
  double l1 = 0.0;
  for (int i = 0; i < N; i++) l1 += fabs(x[i]);
  return l1;
}

int orc_greedy(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q, int Q,
               int64_t nnz, const double* f, const double* mu_train, int n_train, int n_max,
               double greedy_tol, double snapshot_tol, int indicator, double* W, double* ANq,
               double* fN, int32_t* selected, double* eta_hist, int* n_out) {
  if (n_max < 1 || n_max > 512 || n_train < 1 || indicator < 0 || indicator > 1) return -1;
  double* R = (double*)calloc((size_t)n_max * n_max, sizeof(double));
  double* val = (double*)malloc(sizeof(double) * nnz);
  double* u = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* eta = (double*)malloc(sizeof(double) * n_train);
  char* taken = (char*)calloc((size_t)n_train, 1);
  double coef[512];
  int N = 0, rc = 0;
  int next = 0; /* first parameter: index 0 of the training set */
  memset(ANq, 0, sizeof(double) * (size_t)Q * n_max * n_max);
  for (int k = 0; k < n_max; k++) eta_hist[k] = NAN;

  while (N < n_max) {
    /* snapshot u(mu_next) by Jacobi-PCG from zero */
    const double* mu = mu_train + (int64_t)next * Q;
    orc_csr_combine(nnz, Q, vals_q, mu, val);
    for (int64_t i = 0; i < n; i++) u[i] = 0.0;
    int it;
    double rel;
    int st = orc_pcg(n, row_ptr, col, val, f, u, ORC_PREC_JACOBI, NULL, snapshot_tol, 100000, 3,
                     &it, &rel, NULL);
    if (st != ORC_CONVERGED) { rc = -2; break; }
    /* classical Gram-Schmidt, applied twice: w = (I - W W^T)^2 u; the
     * coefficients of both passes form column N of R (u = W R[:,N]) */
    for (int64_t i = 0; i < n; i++) w[i] = u[i];
    for (int j = 0; j < N; j++) R[j * n_max + N] = 0.0;
    for (int pass = 0; pass < 2; pass++) {
      for (int j = 0; j < N; j++) coef[j] = dot(n, W + (int64_t)j * n, w);
      for (int j = 0; j < N; j++) {
        R[j * n_max + N] += coef[j];
        for (int64_t i = 0; i < n; i++) w[i] -= coef[j] * W[(int64_t)j * n + i];
      }
    }
    double wn = norm2(n, w);
    if (wn < 1e-10 * norm2(n, u)) break; /* basis numerically complete */
    R[N * n_max + N] = wn;
    for (int64_t i = 0; i < n; i++) W[(int64_t)N * n + i] = w[i] / wn;
    selected[N] = next;
    taken[next] = 1;
    /* new row and column of A_N^q = W^T A_q W, and the new entry of W^T f */
    const double* wN = W + (int64_t)N * n;
    for (int q = 0; q < Q; q++) {
      orc_csr_matvec(n, row_ptr, col, vals_q + (int64_t)q * nnz, wN, v);
      for (int j = 0; j <= N; j++) {
        double a = dot(n, W + (int64_t)j * n, v); /* w_j^T A_q w_N */
        ANq[((int64_t)q * n_max + j) * n_max + N] = a;
        ANq[((int64_t)q * n_max + N) * n_max + j] = a;
      }
    }
    fN[N] = dot(n, wN, f);
    N++;
    /* residual indicator over the unselected training parameters */
    int any = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < n_train; t++) {
      if (taken[t]) {
        eta[t] = -1.0;
      } else if (indicator == 0) {
        eta[t] = orc_rb_indicator(n, row_ptr, col, vals_q, Q, nnz, f, W, N, n_max, ANq, fN,
                                  mu_train + (int64_t)t * Q);
      } else {
        double c[512];
        eta[t] = orc_rb_solve(N, n_max, Q, ANq, fN, mu_train + (int64_t)t * Q, c) == 0
                     ? l1_indicator(N, n_max, R, c)
                     : INFINITY;
      }
    }
    double best = -1.0;
    next = -1;
    for (int t = 0; t < n_train; t++)
      if (!taken[t]) {
        any = 1;
        if (eta[t] > best) { best = eta[t]; next = t; } /* strict: ties keep the smaller index */
      }
    eta_hist[N - 1] = any ? best : NAN;
    if (!any || best < greedy_tol) break;
  }
  *n_out = N;
  free(val); free(u); free(w); free(v); free(eta); free(taken); free(R);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* O4/O5. Online batch: RB warm start (Algorithm 4) + PCG / MSRBCG          */
/* ------------------------------------------------------------------------ */

int orc_solve_batch(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals_q,
                    int Q, int64_t nnz, const double* f, const double* mu, int B, int warm,
                    const double* c_given, int N, int Nmax, const double* W, const double* ANq,
                    const double* fN, int precond, double tol, int max_iters, int max_restarts,
                    double* u_out, int32_t* iters_out, double* relres_out, double* relres0_out,
                    int32_t* status_out, int n_threads) {
  int used = 1;
  int err = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
#pragma omp parallel
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
    double* val = (double*)malloc(sizeof(double) * nnz);
    double* tmp = (double*)malloc(sizeof(double) * n);
    double* chol = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * (N > 0 ? N : 1));
    double c[512];
#pragma omp for schedule(dynamic, 1)
    for (int b = 0; b < B; b++) {
      const double* m = mu + (int64_t)b * Q;
      double* u = u_out + (int64_t)b * n;
      orc_csr_combine(nnz, Q, vals_q, m, val);
      for (int64_t i = 0; i < n; i++) u[i] = 0.0;
      int need_chol = (warm == ORC_WARM_GALERKIN) || (precond == ORC_PREC_MSRB);
      if (need_chol) {
        reduced_matrix(N, Nmax, Q, ANq, m, chol);
        if (orc_cholesky(N, chol) != 0) {
#pragma omp atomic write
          err = -5;
          continue;
        }
      }
      if (warm == ORC_WARM_GALERKIN) {
        for (int j = 0; j < N; j++) c[j] = fN[j];
        orc_cholesky_solve(N, chol, c);
        lift(n, N, W, c, u);
      } else if (warm == ORC_WARM_GIVEN) {
        lift(n, N, W, c_given + (int64_t)b * N, u);
      }
      if (relres0_out) {
        orc_csr_matvec(n, row_ptr, col, val, u, tmp);
        for (int64_t i = 0; i < n; i++) tmp[i] = f[i] - tmp[i];
        relres0_out[b] = norm2(n, tmp) / norm2(n, f);
      }
      orc_msrb ms = {N, n, W, chol};
      int it;
      double rel;
      int st = orc_pcg(n, row_ptr, col, val, f, u, precond, &ms, tol, max_iters, max_restarts, &it,
                       &rel, NULL);
      iters_out[b] = it;
      if (relres_out) relres_out[b] = rel;
      if (status_out) status_out[b] = st;
    }
    free(val); free(tmp); free(chol);
  }
  return err ? err : used;
}

/* ------------------------------------------------------------------------ */
/* O7. Warm-start network: forward and backward in FP64                      */
/* ------------------------------------------------------------------------ */

int64_t orc_mlp_param_count(int p, int H, int N) {
  return (int64_t)H * p + H + 2 * ((int64_t)H * H + H) + (int64_t)N * H + N;
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_deriv(double x) {
  /* d/dx [x Phi(x)] = Phi(x) + x phi(x) */
  const double inv_sqrt_2pi = 0.39894228040143267794;
  return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * inv_sqrt_2pi * exp(-0.5 * x * x);
}

/* y[o] = b[o] + sum_i Wt[o][i] x[i] */
static void dense(int in, int out, const double* Wt, const double* b, const double* x, double* y) {
  for (int o = 0; o < out; o++) {
    double s = b[o];
    for (int i = 0; i < in; i++) s += Wt[(int64_t)o * in + i] * x[i];
    y[o] = s;
  }
}

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
} mlp_view;

static mlp_view mlp_split(int p, int H, int N, const double* params) {
  mlp_view v;
  const double* c = params;
  v.W1 = c; c += (int64_t)H * p;
  v.b1 = c; c += H;
  v.W2 = c; c += (int64_t)H * H;
  v.b2 = c; c += H;
  v.W3 = c; c += (int64_t)H * H;
  v.b3 = c; c += H;
  v.W4 = c; c += (int64_t)N * H;
  v.b4 = c;
  return v;
}

void orc_mlp_forward(int p, int H, int N, const double* params, int B, const double* x, double* y) {
  mlp_view v = mlp_split(p, H, N, params);
  double* z = (double*)malloc(sizeof(double) * H);
  double* a = (double*)malloc(sizeof(double) * H);
  for (int b = 0; b < B; b++) {
    dense(p, H, v.W1, v.b1, x + (int64_t)b * p, z);
    for (int i = 0; i < H; i++) a[i] = gelu(z[i]);
    dense(H, H, v.W2, v.b2, a, z);
    for (int i = 0; i < H; i++) a[i] = gelu(z[i]);
    dense(H, H, v.W3, v.b3, a, z);
    for (int i = 0; i < H; i++) a[i] = gelu(z[i]);
    dense(H, N, v.W4, v.b4, a, y + (int64_t)b * N);
  }
  free(z); free(a);
}

double orc_mlp_loss_grad(int p, int H, int N, const double* params, int B, const double* x,
                         const double* t, double* grad) {
  mlp_view v = mlp_split(p, H, N, params);
  mlp_view g = mlp_split(p, H, N, grad);
  int64_t np = orc_mlp_param_count(p, H, N);
  memset(grad, 0, sizeof(double) * np);
  double *z1 = malloc(sizeof(double) * H), *a1 = malloc(sizeof(double) * H);
  double *z2 = malloc(sizeof(double) * H), *a2 = malloc(sizeof(double) * H);
  double *z3 = malloc(sizeof(double) * H), *a3 = malloc(sizeof(double) * H);
  double *y = malloc(sizeof(double) * N), *dy = malloc(sizeof(double) * N);
  double *da = malloc(sizeof(double) * H), *dz = malloc(sizeof(double) * H);
  double loss = 0.0;
  const double scale = 1.0 / ((double)B * N);
  double* gW[4] = {(double*)g.W1, (double*)g.W2, (double*)g.W3, (double*)g.W4};
  double* gb[4] = {(double*)g.b1, (double*)g.b2, (double*)g.b3, (double*)g.b4};
  for (int b = 0; b < B; b++) {
    const double* xb = x + (int64_t)b * p;
    /* forward, keeping pre-activations */
    dense(p, H, v.W1, v.b1, xb, z1);
    for (int i = 0; i < H; i++) a1[i] = gelu(z1[i]);
    dense(H, H, v.W2, v.b2, a1, z2);
    for (int i = 0; i < H; i++) a2[i] = gelu(z2[i]);
    dense(H, H, v.W3, v.b3, a2, z3);
    for (int i = 0; i < H; i++) a3[i] = gelu(z3[i]);
    dense(H, N, v.W4, v.b4, a3, y);
    for (int o = 0; o < N; o++) {
      double e = y[o] - t[(int64_t)b * N + o];
      loss += e * e;
      dy[o] = 2.0 * e * scale;
    }
    /* backward through layer 4: dW4 = dy a3^T, db4 = dy, da3 = W4^T dy */
    for (int o = 0; o < N; o++) {
      gb[3][o] += dy[o];
      for (int i = 0; i < H; i++) gW[3][(int64_t)o * H + i] += dy[o] * a3[i];
    }
    for (int i = 0; i < H; i++) {
      double s = 0.0;
      for (int o = 0; o < N; o++) s += v.W4[(int64_t)o * H + i] * dy[o];
      da[i] = s;
    }
    /* layers 3, 2 (hidden -> hidden) */
    const double* zs[3] = {z1, z2, z3};
    const double* as_in[3] = {xb, a1, a2};
    const double* Wl[3] = {v.W1, v.W2, v.W3};
    for (int l = 2; l >= 0; l--) {
      int in = (l == 0) ? p : H;
      for (int i = 0; i < H; i++) dz[i] = da[i] * gelu_deriv(zs[l][i]);
      for (int o = 0; o < H; o++) {
        gb[l][o] += dz[o];
        for (int i = 0; i < in; i++) gW[l][(int64_t)o * in + i] += dz[o] * as_in[l][i];
      }
      if (l > 0) {
        for (int i = 0; i < H; i++) {
          double s = 0.0;
          for (int o = 0; o < H; o++) s += Wl[l][(int64_t)o * H + i] * dz[o];
          da[i] = s;
        }
      }
    }
  }
  free(z1); free(a1); free(z2); free(a2); free(z3); free(a3);
  free(y); free(dy); free(da); free(dz);
  return loss * scale;
}
