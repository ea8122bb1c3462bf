// field.cu -- problems whose coefficient varies from node to node (the paper's
// Example 1, Sec. 4: kappa = 1 + mu_1 g(x) on the unit cube with Dirichlet data).
//
// Such a problem makes every node its own coefficient class, so the solvers'
// class-indexed tables become per-node tables and every stencil, reliable-update
// and multigrid kernel runs unchanged.  What is specific to it lives here:
//   - k_field_tables: the per-instance tables, coef[b][node] = sum_q mu_q R_q[node]
//     from the scaled 7-point rows R_q of each affine term;
//   - k_dirichlet_lift: the right-hand side that boundary data adds through each
//     term (the boundary values eliminated from -div(kappa grad u) = f);
//   - k_affine_sources: f_b = sum_k theta_bk F_k, the affine right-hand sides
//     (a source plus lifts of affine boundary data).
#include <cuda_runtime.h>

#include "internal.h"

namespace rbws {

namespace {

// rows: [Q][n][7] = (-kW, -kE, -kS, -kN, -kD, -kU, D) per term, scaled by 1/h^2.
__global__ void k_field_tables(int Q, int64_t n, const double* __restrict__ rows, const double* __restrict__ mu,
                               int B, double* __restrict__ coef64, float* __restrict__ coef32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * B) return;
  const int b = (int)(t / n);
  const int64_t node = t - (int64_t)b * n;
  const double* m = mu + (int64_t)b * Q;
  double v[7];
#pragma unroll
  for (int k = 0; k < 7; k++) v[k] = 0.0;
  for (int q = 0; q < Q; q++) {
    const double mq = m[q];
    const double* r = rows + ((int64_t)q * n + node) * 7;
#pragma unroll
    for (int k = 0; k < 7; k++) v[k] = fma(mq, r[k], v[k]);
  }
  double* o64 = coef64 + t * kCoefStride;
#pragma unroll
  for (int k = 0; k < 7; k++) o64[k] = v[k];
  o64[7] = 1.0 / v[6];
  if (coef32) {
    float* o32 = coef32 + t * kCoefStride;
#pragma unroll
    for (int k = 0; k < 7; k++) o32[k] = (float)v[k];
    o32[7] = 1.0f / (float)v[6];
  }
}

// lift[q][node]: the boundary faces of the node in the order west, east, south, north,
// down, up; -rows[..][face] is the face's kappa_q / h^2.  gb planes: x = 0, x = 1
// ([nz][ny]), y = 0, y = 1 ([nz][nx]), z = 0, z = 1 ([ny][nx]).
__global__ void k_dirichlet_lift(Geo g, int Q, const double* __restrict__ rows, const double* __restrict__ gb,
                                 double* __restrict__ lift) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)Q * g.n) return;
  const int64_t node = t % g.n;
  const int i = (int)(node % g.nx), j = (int)((node / g.nx) % g.ny), k = (int)(node / ((int64_t)g.nx * g.ny));
  const int64_t ox1 = (int64_t)g.nz * g.ny, oy0 = 2 * ox1, oy1 = oy0 + (int64_t)g.nz * g.nx,
                oz0 = oy1 + (int64_t)g.nz * g.nx, oz1 = oz0 + (int64_t)g.ny * g.nx;
  const double* r = rows + t * 7;
  double v = 0.0;
  if (i == 0) v += -r[0] * gb[(int64_t)k * g.ny + j];
  if (i == g.nx - 1) v += -r[1] * gb[ox1 + (int64_t)k * g.ny + j];
  if (j == 0) v += -r[2] * gb[oy0 + (int64_t)k * g.nx + i];
  if (j == g.ny - 1) v += -r[3] * gb[oy1 + (int64_t)k * g.nx + i];
  if (k == 0) v += -r[4] * gb[oz0 + (int64_t)j * g.nx + i];
  if (k == g.nz - 1) v += -r[5] * gb[oz1 + (int64_t)j * g.nx + i];
  lift[t] = v;
}

__global__ void k_affine_sources(int64_t n, int K, const double* __restrict__ F, const double* __restrict__ theta,
                                 int B, double* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * B) return;
  const int b = (int)(t / n);
  const int64_t i = t - (int64_t)b * n;
  const double* th = theta + (int64_t)b * K;
  double v = 0.0;
  for (int k = 0; k < K; k++) v = fma(th[k], F[(int64_t)k * n + i], v);
  out[t] = v;
}

unsigned blocks_for(int64_t total, int threads) { return (unsigned)((total + threads - 1) / threads); }

}  // namespace

void launch_field_tables(int Q, int64_t n, const double* rows, const double* mu, int B, double* coef64,
                         float* coef32, cudaStream_t s) {
  k_field_tables<<<blocks_for(n * B, 256), 256, 0, s>>>(Q, n, rows, mu, B, coef64, coef32);
}

void launch_dirichlet_lift(const Geo& g, int Q, const double* rows, const double* gb, double* lift,
                           cudaStream_t s) {
  k_dirichlet_lift<<<blocks_for((int64_t)Q * g.n, 256), 256, 0, s>>>(g, Q, rows, gb, lift);
}

void launch_affine_sources(int64_t n, int K, const double* F, const double* theta, int B, double* out,
                           cudaStream_t s) {
  k_affine_sources<<<blocks_for(n * B, 256), 256, 0, s>>>(n, K, F, theta, B, out);
}

}  // namespace rbws
