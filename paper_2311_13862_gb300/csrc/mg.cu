// mg.cu -- multigrid V-cycle preconditioner (Algorithm 2) for the batched PCG.
//
// Grid hierarchy: along an axis with n nodes the next coarser level has
// m = n / 2 nodes, at the fine nodes 2, 4, ..., 2m (1-based); P_i is linear
// interpolation along each axis with the Dirichlet boundary as zero, and the
// coarse operators are the Galerkin products A^i = P_i^T A^{i+1} P_i.
//
// Every level's operator is kept in the class form of the finest one: the
// row of a node depends only on its class triple (x, y, z).  On the finest
// level a class is (own, lower, upper) segment along the axis.  On a coarse
// level the class of coarse node J along an axis is the tuple of fine classes
// at fine nodes 2J-2 .. 2J+2 ("outside" beyond the grid): the Galerkin row of
// J only involves fine rows 2J-1 .. 2J+1, their neighbours 2J-2 .. 2J+2 and
// the interpolation weights there, all fixed by that tuple.  So each level is
// a small table of 27-point rows per class, formed once per affine term on
// the host (A^i(mu) = sum_q mu_q A_q^i because P does not depend on mu), and
// combined per instance on the device.  The coarsest level (at most 64
// unknowns for cubes) is solved with an explicit inverse per instance.
//
// Smoothing is damped Jacobi, u <- u + omega D^-1 (b - A u) with omega = 2/3,
// two steps before and two after the coarse correction, the first from zero.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <vector>

#include "internal.h"

namespace rbws {

// ---------------------------------------------------------------------------
// Host: the hierarchy
// ---------------------------------------------------------------------------
namespace {

inline int off27(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

// Classes of the coarse axis from the fine axis classes.
void coarsen_axis(const std::vector<uint8_t>& fine, std::vector<uint8_t>& coarse, int* ncls) {
  const int n = (int)fine.size(), m = n / 2;
  coarse.assign(m, 0);
  std::map<std::vector<int>, int> ids;
  for (int J = 1; J <= m; J++) {
    std::vector<int> key(5);
    for (int t = 0; t < 5; t++) {
      const int i = 2 * J - 2 + t;  // 1-based fine node
      key[t] = (i >= 1 && i <= n) ? fine[i - 1] : -1;
    }
    auto it = ids.find(key);
    const int id = it == ids.end() ? (int)ids.size() : it->second;
    if (it == ids.end()) ids[key] = id;
    coarse[J - 1] = (uint8_t)std::min(id, 255);  // more than 256 classes is rejected by the caller
  }
  *ncls = (int)ids.size();
}

// Interpolation weights of fine node l (1-based) from the coarse nodes of an
// axis with m coarse nodes: (K, w) pairs, K 1-based.
int pweights(int l, int m, int K[2], double w[2]) {
  if (l % 2 == 0) {
    K[0] = l / 2;
    w[0] = 1.0;
    return 1;
  }
  int c = 0;
  if ((l - 1) / 2 >= 1) K[c] = (l - 1) / 2, w[c++] = 0.5;
  if ((l + 1) / 2 <= m) K[c] = (l + 1) / 2, w[c++] = 0.5;
  return c;
}

// First node (1-based) of each class along an axis.
std::vector<int> representatives(const std::vector<uint8_t>& cls, int ncls) {
  std::vector<int> rep(ncls, 0);
  for (int i = (int)cls.size(); i >= 1; i--) rep[cls[i - 1]] = i;
  return rep;
}

}  // namespace

std::vector<double> fine_rows_q(const AxisClasses& ax, const AxisClasses& ay, const AxisClasses& az, int bx, int by,
                                const uint8_t* segq, int Q, double sx, double sy, double sz) {
  const int ncx = ax.ncls(), ncy = ay.ncls(), ncz = az.ncls();
  std::vector<double> tq((size_t)Q * ncx * ncy * ncz * 27, 0.0);
  for (int q = 0; q < Q; q++)
    for (int czi = 0; czi < ncz; czi++)
      for (int cyi = 0; cyi < ncy; cyi++)
        for (int cxi = 0; cxi < ncx; cxi++) {
          const int ox = ax.key[3 * cxi], lx = ax.key[3 * cxi + 1], hx = ax.key[3 * cxi + 2];
          const int oy = ay.key[3 * cyi], ly = ay.key[3 * cyi + 1], hy = ay.key[3 * cyi + 2];
          const int oz = az.key[3 * czi], lz = az.key[3 * czi + 1], hz = az.key[3 * czi + 2];
          auto kap = [&](int a, int b, int c) {
            const int box = (c * by + b) * bx + a;
            return (segq ? segq[box] : box) == q ? 1.0 : 0.0;
          };
          const double kc = kap(ox, oy, oz);
          // the face rule of k_coef_tables: mean / Dirichlet boundary (-1) / none past a
          // Neumann face (-2), areas halved across the axes of a Neumann face
          auto face = [&](int nb, double knb, double s) {
            return nb >= 0 ? 0.5 * (kc + knb) * s : (nb == -1 ? kc * s : 0.0);
          };
          const double wx = hx == -2 ? 0.5 : 1.0, wy = hy == -2 ? 0.5 : 1.0, wz = hz == -2 ? 0.5 : 1.0;
          const double kW = face(lx, lx >= 0 ? kap(lx, oy, oz) : 0.0, sx) * (wy * wz);
          const double kE = face(hx, hx >= 0 ? kap(hx, oy, oz) : 0.0, sx) * (wy * wz);
          const double kS = face(ly, ly >= 0 ? kap(ox, ly, oz) : 0.0, sy) * (wx * wz);
          const double kN = face(hy, hy >= 0 ? kap(ox, hy, oz) : 0.0, sy) * (wx * wz);
          const double kD = face(lz, lz >= 0 ? kap(ox, oy, lz) : 0.0, sz) * (wx * wy);
          const double kU = face(hz, hz >= 0 ? kap(ox, oy, hz) : 0.0, sz) * (wx * wy);
          double* row = &tq[(((size_t)q * ncz + czi) * ncy + cyi) * ncx * 27 + (size_t)cxi * 27];
          row[off27(0, 0, 0)] = kW + kE + kS + kN + kD + kU;
          row[off27(-1, 0, 0)] = -kW;
          row[off27(1, 0, 0)] = -kE;
          row[off27(0, -1, 0)] = -kS;
          row[off27(0, 1, 0)] = -kN;
          row[off27(0, 0, -1)] = -kD;
          row[off27(0, 0, 1)] = -kU;
        }
  return tq;
}

MGPlan::~MGPlan() {
  for (auto p : d_cls) cudaFree(p);
  for (auto p : d_tq) cudaFree(p);
  cudaFree(d_a0q);
}

std::string mg_build_plan(const AxisClasses& ax, const AxisClasses& ay, const AxisClasses& az,
                          std::vector<double> fine_tq, int Q, MGPlan* plan) {
  // level grids, finest first
  std::vector<std::array<int, 3>> dims{{ax.n, ay.n, az.n}};
  for (;;) {
    const auto d = dims.back();
    if ((int64_t)d[0] * d[1] * d[2] <= kMGCoarsest || std::min({d[0], d[1], d[2]}) < 2) break;
    if ((int)dims.size() == kMGMaxLevels) return "multigrid: too many levels";
    dims.push_back({d[0] / 2, d[1] / 2, d[2] / 2});
  }
  const int L = (int)dims.size();
  plan->J = L - 1;
  plan->Q = Q;
  plan->lv.assign(L, {});
  const auto& d0 = dims.back();
  plan->n0 = d0[0] * d0[1] * d0[2];
  if (plan->n0 > kMGMaxDense) return "multigrid: the coarsest level would have more than 1024 unknowns";
  // finest level: the 7-point rows of each affine term (kappa = e_q) by class
  MGPlan::Level& F = plan->lv[plan->J];
  F.nx = ax.n, F.ny = ay.n, F.nz = az.n;
  F.n = (int64_t)F.nx * F.ny * F.nz;
  F.cx = ax.cls, F.cy = ay.cls, F.cz = az.cls;
  F.ncx = ax.ncls(), F.ncy = ay.ncls(), F.ncz = az.ncls();
  F.tq = std::move(fine_tq);
  // coarse levels: classes and Galerkin rows from the next finer level
  for (int i = plan->J - 1; i >= 0; i--) {
    const MGPlan::Level& f = plan->lv[i + 1];
    MGPlan::Level& c = plan->lv[i];
    c.nx = f.nx / 2, c.ny = f.ny / 2, c.nz = f.nz / 2;
    c.n = (int64_t)c.nx * c.ny * c.nz;
    coarsen_axis(f.cx, c.cx, &c.ncx);
    coarsen_axis(f.cy, c.cy, &c.ncy);
    coarsen_axis(f.cz, c.cz, &c.ncz);
    if (c.ncx > 255 || c.ncy > 255 || c.ncz > 255) return "multigrid: too many coarse classes along an axis";
    if ((int64_t)c.ncls() > (1 << 20)) return "multigrid: too many coarse classes";
    const std::vector<int> rx = representatives(c.cx, c.ncx), ry = representatives(c.cy, c.ncy),
                           rz = representatives(c.cz, c.ncz);
    c.tq.assign((size_t)Q * c.ncls() * 27, 0.0);
    for (int q = 0; q < Q; q++)
      for (int czi = 0; czi < c.ncz; czi++)
        for (int cyi = 0; cyi < c.ncy; cyi++)
          for (int cxi = 0; cxi < c.ncx; cxi++) {
            const int Jx = rx[cxi], Jy = ry[cyi], Jz = rz[czi];
            double* row = &c.tq[(((size_t)q * c.ncz + czi) * c.ncy + cyi) * c.ncx * 27 + (size_t)cxi * 27];
            // row J of P^T A P = sum_i P[i][J] sum_l A[i][l] P[l][K]
            for (int iz = 2 * Jz - 1; iz <= 2 * Jz + 1; iz++) {
              if (iz < 1 || iz > f.nz) continue;
              const double wz = iz == 2 * Jz ? 1.0 : 0.5;
              for (int iy = 2 * Jy - 1; iy <= 2 * Jy + 1; iy++) {
                if (iy < 1 || iy > f.ny) continue;
                const double wy = iy == 2 * Jy ? 1.0 : 0.5;
                for (int ix = 2 * Jx - 1; ix <= 2 * Jx + 1; ix++) {
                  if (ix < 1 || ix > f.nx) continue;
                  const double wi = (ix == 2 * Jx ? 1.0 : 0.5) * wy * wz;
                  const int fcls = (f.cz[iz - 1] * f.ncy + f.cy[iy - 1]) * f.ncx + f.cx[ix - 1];
                  const double* frow = &f.tq[((size_t)q * f.ncls() + fcls) * 27];
                  for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                      for (int dx = -1; dx <= 1; dx++) {
                        const double a = frow[off27(dx, dy, dz)];
                        const int lx = ix + dx, ly = iy + dy, lz = iz + dz;
                        if (a == 0.0 || lx < 1 || lx > f.nx || ly < 1 || ly > f.ny || lz < 1 || lz > f.nz) continue;
                        int Kx[2], Ky[2], Kz[2];
                        double wx_[2], wy_[2], wz_[2];
                        const int nkx = pweights(lx, c.nx, Kx, wx_), nky = pweights(ly, c.ny, Ky, wy_),
                                  nkz = pweights(lz, c.nz, Kz, wz_);
                        for (int a3 = 0; a3 < nkz; a3++)
                          for (int a2 = 0; a2 < nky; a2++)
                            for (int a1 = 0; a1 < nkx; a1++)
                              row[off27(Kx[a1] - Jx, Ky[a2] - Jy, Kz[a3] - Jz)] +=
                                  wi * a * wx_[a1] * wy_[a2] * wz_[a3];
                      }
                }
              }
            }
          }
  }
  // level 0 as dense matrices of the affine terms
  const MGPlan::Level& c0 = plan->lv[0];
  const int n0 = plan->n0;
  plan->a0q.assign((size_t)Q * n0 * n0, 0.0);
  for (int q = 0; q < Q; q++)
    for (int k = 0; k < c0.nz; k++)
      for (int j = 0; j < c0.ny; j++)
        for (int i = 0; i < c0.nx; i++) {
          const int row_id = (k * c0.ny + j) * c0.nx + i;
          const int cls = (c0.cz[k] * c0.ncy + c0.cy[j]) * c0.ncx + c0.cx[i];
          const double* r = &c0.tq[((size_t)q * c0.ncls() + cls) * 27];
          for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
              for (int dx = -1; dx <= 1; dx++) {
                const int x = i + dx, y = j + dy, z = k + dz;
                if (x < 0 || x >= c0.nx || y < 0 || y >= c0.ny || z < 0 || z >= c0.nz) continue;
                plan->a0q[((size_t)q * n0 + row_id) * n0 + (z * c0.ny + y) * c0.nx + x] += r[off27(dx, dy, dz)];
              }
        }
  // device copies (levels below the finest; the finest uses the solver's tables and Geo)
  for (int i = 0; i < plan->J; i++) {
    const MGPlan::Level& c = plan->lv[i];
    std::vector<uint8_t> cls(c.cx);
    cls.insert(cls.end(), c.cy.begin(), c.cy.end());
    cls.insert(cls.end(), c.cz.begin(), c.cz.end());
    if (cudaMalloc(&plan->d_cls[i], cls.size()) != cudaSuccess ||
        cudaMalloc(&plan->d_tq[i], sizeof(double) * c.tq.size()) != cudaSuccess)
      return "multigrid: out of device memory";
    cudaMemcpy(plan->d_cls[i], cls.data(), cls.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(plan->d_tq[i], c.tq.data(), sizeof(double) * c.tq.size(), cudaMemcpyHostToDevice);
  }
  if (cudaMalloc(&plan->d_a0q, sizeof(double) * plan->a0q.size()) != cudaSuccess)
    return "multigrid: out of device memory";
  cudaMemcpy(plan->d_a0q, plan->a0q.data(), sizeof(double) * plan->a0q.size(), cudaMemcpyHostToDevice);
  return "";
}

// ---------------------------------------------------------------------------
// Device: per-instance set-up
// ---------------------------------------------------------------------------
namespace {

// out[b][c][0..26] = sum_q mu[b][q] tq[q][c][..];  out[b][c][27] = 1 / diagonal.
template <typename T>
__global__ void k_mg_tables(int Q, int ncls, const double* __restrict__ tq, const double* __restrict__ mu,
                            int B, T* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * ncls) return;
  const int b = (int)(t / ncls), c = (int)(t % ncls);
  T* o = out + t * 28;
  double diag = 1.0;
  for (int k = 0; k < 27; k++) {
    double v = 0.0;
    for (int q = 0; q < Q; q++) v = fma(mu[(int64_t)b * Q + q], tq[((int64_t)q * ncls + c) * 27 + k], v);
    o[k] = (T)v;
    if (k == 13) diag = v;
  }
  o[27] = (T)(1.0 / diag);
}

// Level-0 matrix of one instance per CTA: A = sum_q mu_q A0_q, lower Cholesky
// in place, L^-1 column by column, then A^-1 = L^-T L^-1 (FP64; also rounded
// to FP32 when ai32 is set).
__global__ void k_mg_dense_setup(int Q, int n0, const double* __restrict__ a0q, const double* __restrict__ mu,
                                 double* __restrict__ A_all, double* __restrict__ Li_all,
                                 double* __restrict__ Ai_all, float* __restrict__ ai32, int* __restrict__ info) {
  const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int64_t nn = (int64_t)n0 * n0;
  double* A = A_all + b * nn;
  double* Li = Li_all + b * nn;
  double* Ai = Ai_all + b * nn;
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int64_t e = tid; e < nn; e += nt) {
    double v = 0.0;
    for (int q = 0; q < Q; q++) v = fma(mu[(int64_t)b * Q + q], a0q[q * nn + e], v);
    A[e] = v;
    Li[e] = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n0; k++) {
    if (tid == 0) {
      const double d = A[(int64_t)k * n0 + k];
      if (!(d > 0.0)) bad = 1;
      A[(int64_t)k * n0 + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = A[(int64_t)k * n0 + k];
    for (int i = k + 1 + tid; i < n0; i += nt) A[(int64_t)i * n0 + k] /= piv;
    __syncthreads();
    const int m = n0 - k - 1;  // trailing lower triangle (pairs i >= j)
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      if (j <= i) A[(int64_t)i * n0 + j] -= A[(int64_t)i * n0 + k] * A[(int64_t)j * n0 + k];
    }
    __syncthreads();
  }
  for (int j = tid; j < n0; j += nt) {  // column j of L^-1
    Li[(int64_t)j * n0 + j] = 1.0 / A[(int64_t)j * n0 + j];
    for (int i = j + 1; i < n0; i++) {
      double s = 0.0;
      for (int k = j; k < i; k++) s = fma(A[(int64_t)i * n0 + k], Li[(int64_t)k * n0 + j], s);
      Li[(int64_t)i * n0 + j] = -s / A[(int64_t)i * n0 + i];
    }
  }
  __syncthreads();
  for (int64_t e = tid; e < nn; e += nt) {
    const int i = (int)(e / n0), j = (int)(e % n0);
    double s = 0.0;
    for (int k = max(i, j); k < n0; k++) s = fma(Li[(int64_t)k * n0 + i], Li[(int64_t)k * n0 + j], s);
    Ai[e] = s;
    if (ai32) ai32[b * nn + e] = (float)s;
  }
  if (tid == 0) info[b] = bad;
}

}  // namespace

void mg_tail_prepare();  // kernel attributes of the one-kernel tail (below)

void launch_mg_setup(const MGPlan& plan, const double* mu, int B, int fp32, void* const* tables, double* dense_a,
                     double* dense_l, double* ainv64, float* ainv32, int* info, cudaStream_t s) {
  mg_tail_prepare();
  for (int i = 1; i < plan.J; i++) {
    const int ncls = plan.lv[i].ncls();
    const unsigned blocks = (unsigned)(((int64_t)B * ncls + 127) / 128);
    if (fp32)
      k_mg_tables<float><<<blocks, 128, 0, s>>>(plan.Q, ncls, plan.d_tq[i], mu, B, (float*)tables[i]);
    else
      k_mg_tables<double><<<blocks, 128, 0, s>>>(plan.Q, ncls, plan.d_tq[i], mu, B, (double*)tables[i]);
  }
  k_mg_dense_setup<<<B, 256, 0, s>>>(plan.Q, plan.n0, plan.d_a0q, mu, dense_a, dense_l, ainv64,
                                     fp32 ? ainv32 : nullptr, info);
}

// ---------------------------------------------------------------------------
// Device: the V-cycle
// ---------------------------------------------------------------------------
// The finest level with fused FP32 steps (two pre- and two post-smoothing
// steps): Y = S(0, r, 2) with the first step formed on the fly; R = r - A Y;
// restriction; coarse cycle e; X = Y + P e + omega D^-1 (r - A (Y + P e));
// out = X + omega D^-1 (r - A X) with the rho partials.
int vcycle_fine_fused(const MGBatch& m, const float* rhs, float* out, int slot, cudaStream_t s);

namespace {

__device__ __forceinline__ bool mg_skip(const InstState* st, const int* mask, int b) {
  return (st && st[b].status != ST_ACTIVE) || (mask && !mask[b]);
}

template <typename T, bool kSeven>
__device__ __forceinline__ T mg_row_apply(const T* __restrict__ row, const T* __restrict__ x, int i, int j, int k,
                                          int nx, int ny, int nz) {
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const int64_t c = ((int64_t)k * ny + j) * nx + i;
  if (kSeven) {  // -kW, -kE, -kS, -kN, -kD, -kU, D
    T v = row[6] * x[c];
    if (i > 0) v = fma(row[0], x[c - 1], v);
    if (i < nx - 1) v = fma(row[1], x[c + 1], v);
    if (j > 0) v = fma(row[2], x[c - sy], v);
    if (j < ny - 1) v = fma(row[3], x[c + sy], v);
    if (k > 0) v = fma(row[4], x[c - sz], v);
    if (k < nz - 1) v = fma(row[5], x[c + sz], v);
    return v;
  }
  T v = T(0);
#pragma unroll
  for (int dz = -1; dz <= 1; dz++) {
    if (k + dz < 0 || k + dz >= nz) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      if (j + dy < 0 || j + dy >= ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        if (i + dx < 0 || i + dx >= nx) continue;
        v = fma(row[(dz + 1) * 9 + (dy + 1) * 3 + dx + 1], x[c + dz * sz + dy * sy + dx], v);
      }
    }
  }
  return v;
}

// mode 0: out = omega D^-1 rhs (smoothing from zero)
// mode 1: out = x + omega D^-1 (rhs - A x)
// mode 2: out = rhs - A x (residual)
template <typename T, bool kSeven>
__global__ void __launch_bounds__(256) k_mg_level(MGLevel L, const InstState* __restrict__ st,
                                                  const int* __restrict__ mask, int mode,
                                                  const T* __restrict__ rhs, const T* __restrict__ x,
                                                  T* __restrict__ out, T omega) {
  const int b = blockIdx.y;
  if (mg_skip(st, mask, b)) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= L.n) return;
  const int i = (int)(t % L.nx), j = (int)((t / L.nx) % L.ny), k = (int)(t / ((int64_t)L.nx * L.ny));
  const int cls = (L.cz[k] * L.ncy + L.cy[j]) * L.ncx + L.cx[i];
  const T* row = (const T*)L.coef + ((int64_t)b * L.ncx * L.ncy * L.ncz + cls) * L.stride;
  const int64_t off = (int64_t)b * L.n;
  const T dinv = row[L.stride - 1];
  const T bv = rhs[off + t];
  if (mode == 0) {
    out[off + t] = omega * dinv * bv;
    return;
  }
  const T ax = mg_row_apply<T, kSeven>(row, x + off, i, j, k, L.nx, L.ny, L.nz);
  out[off + t] = mode == 1 ? fma(omega * dinv, bv - ax, x[off + t]) : bv - ax;
}

// rc = P^T rf (coarse node J gathers fine nodes 2J-1 .. 2J+1 per axis).
template <typename T>
__global__ void __launch_bounds__(256) k_mg_restrict(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                                                     const InstState* __restrict__ st, const int* __restrict__ mask,
                                                     const T* __restrict__ rf, T* __restrict__ rc) {
  const int b = blockIdx.y;
  if (mg_skip(st, mask, b)) return;
  const int64_t cn = (int64_t)cnx * cny * cnz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cn) return;
  const int I = (int)(t % cnx), Jy = (int)((t / cnx) % cny), K = (int)(t / ((int64_t)cnx * cny));
  const int64_t fn = (int64_t)fnx * fny * fnz;
  const T* r = rf + (int64_t)b * fn;
  T v = T(0);
  for (int dz = -1; dz <= 1; dz++) {
    const int z = 2 * K + 1 + dz;  // 0-based fine index of 1-based 2(K+1)+dz
    if (z < 0 || z >= fnz) continue;
    const T wz = dz == 0 ? T(1) : T(0.5);
    for (int dy = -1; dy <= 1; dy++) {
      const int y = 2 * Jy + 1 + dy;
      if (y < 0 || y >= fny) continue;
      const T wy = dy == 0 ? wz : T(0.5) * wz;
      for (int dx = -1; dx <= 1; dx++) {
        const int x = 2 * I + 1 + dx;
        if (x < 0 || x >= fnx) continue;
        v = fma(dx == 0 ? wy : T(0.5) * wy, r[((int64_t)z * fny + y) * fnx + x], v);
      }
    }
  }
  rc[(int64_t)b * cn + t] = v;
}

// uf += P ec (fine node i takes coarse i/2 if i is even, else half of each
// coarse neighbour (i-1)/2 and (i+1)/2 that exists; 1-based).
__device__ __forceinline__ int pw(int i0, int m, int K[2], float w[2]) {
  const int i = i0 + 1;
  if (i % 2 == 0) {
    K[0] = i / 2 - 1;
    w[0] = 1.f;
    return 1;
  }
  int c = 0;
  if ((i - 1) / 2 >= 1) K[c] = (i - 1) / 2 - 1, w[c++] = 0.5f;
  if ((i + 1) / 2 <= m) K[c] = (i + 1) / 2 - 1, w[c++] = 0.5f;
  return c;
}

template <typename T>
__global__ void __launch_bounds__(256) k_mg_prolong_add(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                                                        const InstState* __restrict__ st,
                                                        const int* __restrict__ mask, const T* __restrict__ ec,
                                                        T* __restrict__ uf) {
  const int b = blockIdx.y;
  if (mg_skip(st, mask, b)) return;
  const int64_t fn = (int64_t)fnx * fny * fnz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= fn) return;
  const int i = (int)(t % fnx), j = (int)((t / fnx) % fny), k = (int)(t / ((int64_t)fnx * fny));
  int Kx[2], Ky[2], Kz[2];
  float wx[2], wy[2], wz[2];  // 1 or 1/2: exact in either type
  const int nx_ = pw(i, cnx, Kx, wx), ny_ = pw(j, cny, Ky, wy), nz_ = pw(k, cnz, Kz, wz);
  const T* e = ec + (int64_t)b * cnx * cny * cnz;
  T v = T(0);
  for (int c = 0; c < nz_; c++)
    for (int bq = 0; bq < ny_; bq++)
      for (int a = 0; a < nx_; a++)
        v = fma((T)(wx[a] * wy[bq] * wz[c]), e[((int64_t)Kz[c] * cny + Ky[bq]) * cnx + Kx[a]], v);
  uf[(int64_t)b * fn + t] += v;
}

// x0 = A0^-1 b0 per instance (one CTA per instance).
template <typename T>
__global__ void k_mg_dense_apply(int n0, const T* __restrict__ ainv, const InstState* __restrict__ st,
                                 const int* __restrict__ mask, const T* __restrict__ rhs, T* __restrict__ out) {
  const int b = blockIdx.x;
  if (mg_skip(st, mask, b)) return;
  const T* Ai = ainv + (int64_t)b * n0 * n0;
  const T* r = rhs + (int64_t)b * n0;
  for (int i = threadIdx.x; i < n0; i += blockDim.x) {
    T v = T(0);
    for (int j = 0; j < n0; j++) v = fma(Ai[(int64_t)i * n0 + j], r[j], v);
    out[(int64_t)b * n0 + i] = v;
  }
}

// Coarse-level fused steps (27-point Galerkin rows): one thread per (x, y)
// column of a tile, marching through a chunk of z planes.  Every plane of the
// chunk (with its x/y halo and the planes either side) is staged in shared
// memory at once, so the loads of a whole chunk are in flight together; the
// march keeps the 3 x 3 neighbourhoods of three planes in registers.  The
// staged field is xin (kStage 0), omega D^-1 rhs (1) or xin + P e (2, e staged
// first over the chunk's coarse footprint); the output a damped Jacobi step
// (kOut 0) or the residual rhs - A x (kOut 1) -- as on the finest level.
using Pw = PRows;
__device__ __forceinline__ Pw pweight(int j, int m) { return prows(j, m); }

__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }

// Shared memory of one fused coarse step (elements): the staged planes z0-1 ..
// z1 with their x/y halo, the right-hand side of the own nodes, and (kStage 2)
// the coarse correction over the chunk's footprint.
__host__ __device__ inline int64_t coarse_smem_elems(int TX, int TY, int zc, bool with_e) {
  const int64_t st = (int64_t)(zc + 2) * (TX + 2) * (TY + 2) + (int64_t)zc * TX * TY;
  return st + (with_e ? (int64_t)(TX / 2 + 3) * (TY / 2 + 3) * (zc / 2 + 3) : 0);
}

template <typename T, int kStage, int kOut>
__global__ void __launch_bounds__(256) k_mg_coarse(MGLevel L, const InstState* __restrict__ st,
                                                   const int* __restrict__ mask, const T* __restrict__ rhs,
                                                   const T* __restrict__ xin, T* __restrict__ out,
                                                   const T* __restrict__ ec, int cnx, int cny, int cnz, T omega,
                                                   int tiles_x, int zc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.z;
  if (mg_skip(st, mask, b)) return;
  const int TX = blockDim.x, TY = blockDim.y, NT = TX * TY;
  const int tid = (int)threadIdx.y * TX + (int)threadIdx.x;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = blockIdx.y * zc, z1 = min(L.nz, z0 + zc), nzl = z1 - z0;
  const int PW = TX + 2, PS = PW * (TY + 2), NPL = nzl + 2;
  const int64_t plane = (int64_t)L.nx * L.ny, off = (int64_t)b * L.n;
  const int ncls = L.ncx * L.ncy * L.ncz;
  const T* tab = (const T*)L.coef + (int64_t)b * ncls * 28;
  const T* rb = rhs + off;
  T* srhs = sm + (int64_t)(zc + 2) * PS;  // [nzl][TY][TX]
  T* se = srhs + (int64_t)zc * TX * TY;   // kStage 2: e over the footprint
  // the footprint of e: fine i in [x0-1, x0+TX] uses coarse floor((i-1)/2) .. floor(i/2)
  const int ex_lo = floor_half(x0 - 2), ey_lo = floor_half(y0 - 2), ez_lo = floor_half(z0 - 2);
  const int EW = floor_half(x0 + TX) - ex_lo + 1, EH = floor_half(y0 + TY) - ey_lo + 1;
  const int ED = floor_half(z1) - ez_lo + 1;
  constexpr int KB = kStage == 2 ? 8 : 16;  // loads in flight per thread while staging
  if (kStage == 2) {
    const T* eb = ec + (int64_t)b * cnx * cny * cnz;
    const int ne = EW * EH * ED;
    for (int e0 = tid; e0 < ne; e0 += KB * NT) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; q++) {
        const int e = e0 + q * NT;
        v[q] = T(0);
        if (e < ne) {
          const int ix = e % EW, iy = (e / EW) % EH, iz = e / (EW * EH);
          const int cx = ex_lo + ix, cy = ey_lo + iy, cz = ez_lo + iz;
          if (cx >= 0 && cx < cnx && cy >= 0 && cy < cny && cz >= 0 && cz < cnz)
            v[q] = eb[((int64_t)cz * cny + cy) * cnx + cx];
        }
      }
#pragma unroll
      for (int q = 0; q < KB; q++)
        if (e0 + q * NT < ne) se[e0 + q * NT] = v[q];
    }
    __syncthreads();
  }
  // stage every plane of the chunk at once (zeros outside the grid): a thread
  // owns the cells (tx + c TX, ty + a TY) of each staged plane, c, a in {0, 1},
  // and issues the loads of PB planes before their stores
  const int i = x0 + (int)threadIdx.x, j = y0 + (int)threadIdx.y;
  const bool own = i < L.nx && j < L.ny;
  const int64_t col = (int64_t)j * L.nx + i;
  int cell_s[4], cell_cx[4], cell_cy[4];  // smem offset in a plane (-1: no cell); classes (kStage 1)
  int cell_col[4];                        // grid column j*nx + i, -1 outside the grid
  int cell_i[4], cell_j[4];               // grid position (kStage 2)
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const int hx = (int)threadIdx.x + (c & 1) * TX, hy = (int)threadIdx.y + (c >> 1) * TY;
    const bool cell = hx < TX + 2 && hy < TY + 2;
    const int ii = x0 + hx - 1, jj = y0 + hy - 1;
    const bool in = cell && ii >= 0 && ii < L.nx && jj >= 0 && jj < L.ny;
    cell_s[c] = cell ? hy * PW + hx : -1;
    cell_col[c] = in ? jj * L.nx + ii : -1;
    cell_cx[c] = in && kStage == 1 ? L.cx[ii] : 0;
    cell_cy[c] = in && kStage == 1 ? L.cy[jj] : 0;
    cell_i[c] = ii;
    cell_j[c] = jj;
  }
  constexpr int PB = kStage == 2 ? 2 : 4;
  T cell_od[4] = {T(0), T(0), T(0), T(0)};  // kStage 1: omega / D of each cell in z class cell_zc
  int cell_zc = -1;
  for (int p0 = 0; p0 < NPL; p0 += PB) {
    T v[PB][4];
#pragma unroll
    for (int q = 0; q < PB; q++) {
      const int z = z0 + p0 + q - 1;
      const bool zin = p0 + q < NPL && z >= 0 && z < L.nz;
      if (kStage == 1 && zin) {
        const int zcl = L.cz[z];
        if (zcl != cell_zc) {  // the table is read again only where the z class changes
          cell_zc = zcl;
#pragma unroll
          for (int c = 0; c < 4; c++)
            cell_od[c] = cell_col[c] >= 0
                             ? omega * tab[(int64_t)((zcl * L.ncy + cell_cy[c]) * L.ncx + cell_cx[c]) * 28 + 27]
                             : T(0);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; c++) {
        v[q][c] = T(0);
        if (zin && cell_col[c] >= 0) {
          const int64_t idx = (int64_t)z * plane + cell_col[c];
          if (kStage == 1) {
            v[q][c] = cell_od[c] * rb[idx];
          } else {
            v[q][c] = xin[off + idx];
            if (kStage == 2) {  // + (P e) from the staged footprint
              const Pw rz = pweight(z, cnz), rx = pweight(cell_i[c], cnx), ry = pweight(cell_j[c], cny);
              T pe = T(0);
#pragma unroll
              for (int cz = 0; cz < 2; cz++) {
                const int kz = cz ? rz.k1 : rz.k0;
                if (kz < 0) continue;
#pragma unroll
                for (int bq = 0; bq < 2; bq++) {
                  const int ky = bq ? ry.k1 : ry.k0;
                  if (ky < 0) continue;
                  const float wyz = (cz ? rz.w1 : rz.w0) * (bq ? ry.w1 : ry.w0);
                  const T* row = se + ((kz - ez_lo) * EH + (ky - ey_lo)) * EW - ex_lo;
                  if (rx.k0 >= 0) pe = fma((T)(wyz * rx.w0), row[rx.k0], pe);
                  if (rx.k1 >= 0) pe = fma((T)(wyz * rx.w1), row[rx.k1], pe);
                }
              }
              v[q][c] += pe;
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PB; q++)
      if (p0 + q < NPL)
#pragma unroll
        for (int c = 0; c < 4; c++)
          if (cell_s[c] >= 0) sm[(p0 + q) * PS + cell_s[c]] = v[q][c];
  }
  // the right-hand side of the own node, 16 planes of loads in flight
  if (own)
    for (int q0 = 0; q0 < nzl; q0 += 16) {
      T v[16];
#pragma unroll
      for (int q = 0; q < 16; q++) v[q] = q0 + q < nzl ? rb[(int64_t)(z0 + q0 + q) * plane + col] : T(0);
#pragma unroll
      for (int q = 0; q < 16; q++)
        if (q0 + q < nzl) srhs[(q0 + q) * NT + tid] = v[q];
    }
  __syncthreads();
  if (!own) return;
  // march in z with the 3 x 3 neighbourhoods of planes z-1, z, z+1 in registers
  const int oslot = ((int)threadIdx.y + 1) * PW + (int)threadIdx.x + 1;
  T w[3][9];
#pragma unroll
  for (int pz = 0; pz < 2; pz++)
#pragma unroll
    for (int q = 0; q < 9; q++) w[pz][q] = sm[pz * PS + oslot + (q / 3 - 1) * PW + (q % 3 - 1)];
  T c[27];
  T dinv = T(0);
  int zcls_cur = -1;
  const int cxy = L.cy[j] * L.ncx + L.cx[i];
  for (int z = z0; z < z1; ++z) {
    const T* Pn = sm + (z - z0 + 2) * PS + oslot;
#pragma unroll
    for (int q = 0; q < 9; q++) w[2][q] = Pn[(q / 3 - 1) * PW + (q % 3 - 1)];
    const int zcl = L.cz[z];
    if (zcl != zcls_cur) {
      zcls_cur = zcl;
      const T* row = tab + (int64_t)(zcl * L.ncy * L.ncx + cxy) * 28;
#pragma unroll
      for (int k = 0; k < 27; k++) c[k] = row[k];
      dinv = row[27];
    }
    T ax = T(0);
#pragma unroll
    for (int dz = 0; dz < 3; dz++)
#pragma unroll
      for (int q = 0; q < 9; q++) ax = fma(c[dz * 9 + q], w[dz][q], ax);
    const T bv = srhs[(z - z0) * NT + tid];
    const int64_t idx = off + (int64_t)z * plane + col;
    if (kOut == 1) out[idx] = bv - ax;
    else out[idx] = fma(omega * dinv, bv - ax, w[1][4]);
#pragma unroll
    for (int q = 0; q < 9; q++) {
      w[0][q] = w[1][q];
      w[1][q] = w[2][q];
    }
  }
}

// ---------------------------------------------------------------------------
// The small levels in one kernel: levels top .. 0 of the V-cycle (top has at
// most kMGTailMax unknowns), one CTA of 1024 threads per instance (its sweeps are
// latency-bound: 1024 threads halve each sweep's length; 512 measured 0.918 against
// 0.907 ms per V-cycle at 64^3 with 256 instances), every vector of those
// levels in shared memory: the same steps as the per-level kernels (two
// smoothing steps from zero, residual, restriction, the level below,
// prolongation, two smoothing steps), with a barrier between steps.
// ---------------------------------------------------------------------------
struct MGTail {
  int top;                    // highest level handled here (>= 1)
  MGLevel lv[kMGMaxLevels];   // views of levels 0 .. top (coef: 28-wide tables, level 0 unused)
  int off[kMGMaxLevels];      // shared-memory offset (elements) of level l's three vectors
  int n0;
  MGLevel up;                 // up.n > 0: add P (top solution) into up_x on this level (top + 1)
};

// Node t = (k ny + j) nx + i of a thread's strided sweep t = tid, tid + nt, ...,
// with (i, j, k) carried from one node to the next instead of divided out.
struct TailPos {
  int i, j, k, di, dj, dk, nx, ny;
  __device__ __forceinline__ TailPos(int t, int nt, int nx_, int ny_) : nx(nx_), ny(ny_) {
    i = t % nx;
    j = (t / nx) % ny;
    k = t / (nx * ny);
    di = nt % nx;
    dj = (nt / nx) % ny;
    dk = nt / (nx * ny);
  }
  __device__ __forceinline__ void next() {
    i += di;
    const int ci = i >= nx;
    if (ci) i -= nx;
    j += dj + ci;
    const int cj = j >= ny;
    if (cj) j -= ny;
    k += dk + cj;
  }
};

template <typename T>
__device__ __forceinline__ T tail_apply(const MGLevel& L, const T* __restrict__ tab, const T* x, int t, int i, int j,
                                        int k, T* dinv) {
  const int cls = (L.cz[k] * L.ncy + L.cy[j]) * L.ncx + L.cx[i];
  T v = T(0);
  if constexpr (sizeof(T) == 4) {
    // the class row in seven 16-byte loads (28 floats, 16-byte aligned); the same products
    // in the same order as the scalar loop below
    float c[28];
    const float4* r4 = reinterpret_cast<const float4*>(tab + (int64_t)cls * 28);
#pragma unroll
    for (int q = 0; q < 7; q++) {
      const float4 w = __ldg(r4 + q);
      c[4 * q] = w.x, c[4 * q + 1] = w.y, c[4 * q + 2] = w.z, c[4 * q + 3] = w.w;
    }
    *dinv = c[27];
#pragma unroll
    for (int dz = -1; dz <= 1; dz++) {
      if (k + dz < 0 || k + dz >= L.nz) continue;
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
        if (j + dy < 0 || j + dy >= L.ny) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
          if (i + dx < 0 || i + dx >= L.nx) continue;
          v = fma(c[(dz + 1) * 9 + (dy + 1) * 3 + dx + 1], x[t + (dz * L.ny + dy) * L.nx + dx], v);
        }
      }
    }
  } else {
    const T* row = tab + (int64_t)cls * 28;
    *dinv = row[27];
    for (int dz = -1; dz <= 1; dz++) {
      if (k + dz < 0 || k + dz >= L.nz) continue;
      for (int dy = -1; dy <= 1; dy++) {
        if (j + dy < 0 || j + dy >= L.ny) continue;
        for (int dx = -1; dx <= 1; dx++) {
          if (i + dx < 0 || i + dx >= L.nx) continue;
          v = fma(row[(dz + 1) * 9 + (dy + 1) * 3 + dx + 1], x[t + (dz * L.ny + dy) * L.nx + dx], v);
        }
      }
    }
  }
  return v;
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_mg_tail(MGTail tl, const InstState* __restrict__ st,
                                                 const int* __restrict__ mask, const T* __restrict__ rhs_top,
                                                 T* __restrict__ out_top, const T* __restrict__ ainv, T omega,
                                                 T* __restrict__ up_x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.x;
  if (mg_skip(st, mask, b)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto vb = [&](int l) { return sm + tl.off[l]; };                       // right-hand side
  auto vy = [&](int l) { return sm + tl.off[l] + tl.lv[l].n; };          // smoothed iterate / solution
  auto vt = [&](int l) { return sm + tl.off[l] + 2 * tl.lv[l].n; };      // scratch
  auto tab = [&](int l) { return (const T*)tl.lv[l].coef + (int64_t)b * tl.lv[l].ncx * tl.lv[l].ncy * tl.lv[l].ncz * 28; };
  // the right-hand side of the top level
  {
    const int n = (int)tl.lv[tl.top].n;
    for (int t = tid; t < n; t += nt) vb(tl.top)[t] = rhs_top[(int64_t)b * n + t];
  }
  __syncthreads();
  // down: smoothing, residual, restriction
  for (int l = tl.top; l >= 1; l--) {
    const MGLevel& L = tl.lv[l];
    const int n = (int)L.n;
    const T* tb = tab(l);
    T *bb = vb(l), *yy = vy(l), *tt = vt(l);
    {
      TailPos q(tid, nt, L.nx, L.ny);
      for (int t = tid; t < n; t += nt, q.next()) {  // tt = omega D^-1 b
        const T di = tb[(int64_t)((L.cz[q.k] * L.ncy + L.cy[q.j]) * L.ncx + L.cx[q.i]) * 28 + 27];
        tt[t] = omega * di * bb[t];
      }
    }
    __syncthreads();
    {
      TailPos q(tid, nt, L.nx, L.ny);
      for (int t = tid; t < n; t += nt, q.next()) {  // yy = tt + omega D^-1 (b - A tt)
        T di;
        const T ax = tail_apply<T>(L, tb, tt, t, q.i, q.j, q.k, &di);
        yy[t] = fma(omega * di, bb[t] - ax, tt[t]);
      }
    }
    __syncthreads();
    {
      TailPos q(tid, nt, L.nx, L.ny);
      for (int t = tid; t < n; t += nt, q.next()) {  // tt = b - A yy
        T di;
        tt[t] = bb[t] - tail_apply<T>(L, tb, yy, t, q.i, q.j, q.k, &di);
      }
    }
    __syncthreads();
    const MGLevel& C = tl.lv[l - 1];
    T* cb = vb(l - 1);
    TailPos qc(tid, nt, C.nx, C.ny);
    for (int t = tid; t < (int)C.n; t += nt, qc.next()) {  // b_{l-1} = P^T tt
      const int I = qc.i, J = qc.j, K = qc.k;
      T v = T(0);
      for (int dz = -1; dz <= 1; dz++) {
        const int z = 2 * K + 1 + dz;
        if (z < 0 || z >= L.nz) continue;
        for (int dy = -1; dy <= 1; dy++) {
          const int y = 2 * J + 1 + dy;
          if (y < 0 || y >= L.ny) continue;
          for (int dx = -1; dx <= 1; dx++) {
            const int x = 2 * I + 1 + dx;
            if (x < 0 || x >= L.nx) continue;
            const T w = (T)((dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f));
            v = fma(w, tt[(z * L.ny + y) * L.nx + x], v);
          }
        }
      }
      cb[t] = v;
    }
    __syncthreads();
  }
  // level 0: the explicit inverse
  {
    const int n0 = tl.n0;
    const T* Ai = ainv + (int64_t)b * n0 * n0;
    const T* b0 = vb(0);
    for (int i = tid; i < n0; i += nt) {
      T v = T(0);
      for (int j = 0; j < n0; j++) v = fma(Ai[(int64_t)i * n0 + j], b0[j], v);
      vy(0)[i] = v;
    }
    __syncthreads();
  }
  // up: prolongation, smoothing
  for (int l = 1; l <= tl.top; l++) {
    const MGLevel& L = tl.lv[l];
    const MGLevel& C = tl.lv[l - 1];
    const int n = (int)L.n;
    const T* tb = tab(l);
    T *bb = vb(l), *yy = vy(l), *tt = vt(l);
    const T* e = vy(l - 1);
    TailPos qp(tid, nt, L.nx, L.ny);
    for (int t = tid; t < n; t += nt, qp.next()) {  // yy += P e
      const Pw rx = pweight(qp.i, C.nx), ry = pweight(qp.j, C.ny), rz = pweight(qp.k, C.nz);
      T v = T(0);
      for (int c = 0; c < 2; c++) {
        const int kz = c ? rz.k1 : rz.k0;
        if (kz < 0) continue;
        for (int bq = 0; bq < 2; bq++) {
          const int ky = bq ? ry.k1 : ry.k0;
          if (ky < 0) continue;
          const float wyz = (c ? rz.w1 : rz.w0) * (bq ? ry.w1 : ry.w0);
          const T* row = e + (kz * C.ny + ky) * C.nx;
          if (rx.k0 >= 0) v = fma((T)(wyz * rx.w0), row[rx.k0], v);
          if (rx.k1 >= 0) v = fma((T)(wyz * rx.w1), row[rx.k1], v);
        }
      }
      yy[t] += v;
    }
    __syncthreads();
    {
      TailPos q(tid, nt, L.nx, L.ny);
      for (int t = tid; t < n; t += nt, q.next()) {  // tt = yy + omega D^-1 (b - A yy)
        T di;
        const T ax = tail_apply<T>(L, tb, yy, t, q.i, q.j, q.k, &di);
        tt[t] = fma(omega * di, bb[t] - ax, yy[t]);
      }
    }
    __syncthreads();
    T* dst = l == tl.top && tl.up.n == 0 ? out_top + (int64_t)b * n : yy;
    {
      TailPos q(tid, nt, L.nx, L.ny);
      for (int t = tid; t < n; t += nt, q.next()) {  // solution = tt + omega D^-1 (b - A tt)
        T di;
        const T ax = tail_apply<T>(L, tb, tt, t, q.i, q.j, q.k, &di);
        dst[t] = fma(omega * di, bb[t] - ax, tt[t]);
      }
    }
    __syncthreads();
  }
  if (tl.up.n > 0) {  // up_x += P e on the level above, e = the top solution (in shared memory)
    const MGLevel& U = tl.up;
    const MGLevel& C = tl.lv[tl.top];
    const T* e = vy(tl.top);
    T* ub = up_x + (int64_t)b * U.n;
    // threads over x (nt a multiple of U.nx: no divisions in the loop), rows and planes
    // stepped; the read-modify-writes of up_x go in batches of KB (loads first)
    const bool rows = nt % U.nx == 0;
    const int i0 = rows ? tid % U.nx : 0, rstep = rows ? nt / U.nx : 1, jfirst = rows ? tid / U.nx : 0;
    const Pw rx0 = pweight(i0, C.nx);
    constexpr int KB = 4;
    int k = 0, j = jfirst;  // next (plane, row) of this thread
    if (j >= U.ny) k = U.nz;
    while (rows && k < U.nz) {
      int kq[KB], jq[KB];
      T old[KB];
#pragma unroll
      for (int q = 0; q < KB; q++) {
        kq[q] = k;
        jq[q] = j;
        old[q] = k < U.nz ? ub[((int64_t)k * U.ny + j) * U.nx + i0] : T(0);
        if (k < U.nz) {
          j += rstep;
          if (j >= U.ny) {
            j = jfirst;
            k++;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < KB; q++) {
        if (kq[q] >= U.nz) continue;
        const Pw rz = pweight(kq[q], C.nz), ry = pweight(jq[q], C.ny);
        T v = T(0);
#pragma unroll
        for (int c = 0; c < 2; c++) {
          const int kz = c ? rz.k1 : rz.k0;
          if (kz < 0) continue;
#pragma unroll
          for (int bq = 0; bq < 2; bq++) {
            const int ky = bq ? ry.k1 : ry.k0;
            if (ky < 0) continue;
            const float wyz = (c ? rz.w1 : rz.w0) * (bq ? ry.w1 : ry.w0);
            const T* row = e + (kz * C.ny + ky) * C.nx;
            if (rx0.k0 >= 0) v = fma((T)(wyz * rx0.w0), row[rx0.k0], v);
            if (rx0.k1 >= 0) v = fma((T)(wyz * rx0.w1), row[rx0.k1], v);
          }
        }
        ub[((int64_t)kq[q] * U.ny + jq[q]) * U.nx + i0] = old[q] + v;
      }
    }
    if (!rows)
      for (int t = tid; t < (int)U.n; t += nt) {
        const int i = t % U.nx, j = (t / U.nx) % U.ny, k = t / (U.nx * U.ny);
        const Pw rx = pweight(i, C.nx), ry = pweight(j, C.ny), rz = pweight(k, C.nz);
        T v = T(0);
        for (int c = 0; c < 2; c++) {
          const int kz = c ? rz.k1 : rz.k0;
          if (kz < 0) continue;
          for (int bq = 0; bq < 2; bq++) {
            const int ky = bq ? ry.k1 : ry.k0;
            if (ky < 0) continue;
            const float wyz = (c ? rz.w1 : rz.w0) * (bq ? ry.w1 : ry.w0);
            const T* row = e + (kz * C.ny + ky) * C.nx;
            if (rx.k0 >= 0) v = fma((T)(wyz * rx.w0), row[rx.k0], v);
            if (rx.k1 >= 0) v = fma((T)(wyz * rx.w1), row[rx.k1], v);
          }
        }
        ub[t] += v;
      }
  }
}

}  // namespace

constexpr size_t kMGTailSmem = 200 * 1024;  // dynamic shared memory the tail may use

void mg_tail_prepare() {
  cudaFuncSetAttribute(k_mg_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMGTailSmem);
  cudaFuncSetAttribute(k_mg_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMGTailSmem);
}

namespace {

// Shared memory of the tail kernel for levels 0 .. top (elements).
inline int tail_elems(const MGPlan& P, int top, int* off) {
  int o = 0;
  for (int l = 0; l <= top; l++) {
    off[l] = o;
    o += 3 * (int)P.lv[l].n;
  }
  return o;
}

// uf += P ec on the finest FP32 level, 4G x-consecutive fine nodes per thread
// (fnx % 4G == 0, so cnx = fnx / 2): a group of four at i0 reads coarse columns
// i0/2 - 1 .. i0/2 + 1 of each coarse row it touches, and G = 2 groups share the
// middle column.  The G float4 loads of uf are issued before the coarse reads, so
// each thread keeps 16G bytes of the stream in flight.
template <int G>
__global__ void __launch_bounds__(256) k_mg_prolong_add4(int fnx, int fny, int fnz, int cnx, int cny, int cnz,
                                                         const InstState* __restrict__ st,
                                                         const int* __restrict__ mask, const float* __restrict__ ec,
                                                         float* __restrict__ uf) {
  const int b = blockIdx.y;
  if (mg_skip(st, mask, b)) return;
  const int gx = fnx / (4 * G);
  const int64_t ng = (int64_t)gx * fny * fnz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ng) return;
  float4* p = reinterpret_cast<float4*>(uf + (int64_t)b * fnx * fny * fnz) + G * t;
  float4 u[G];
#pragma unroll
  for (int q = 0; q < G; q++) u[q] = p[q];
  const int i0 = 4 * G * (int)(t % gx), j = (int)((t / gx) % fny), k = (int)(t / ((int64_t)gx * fny));
  const Pw ry = pweight(j, cny), rz = pweight(k, cnz);
  const float* e = ec + (int64_t)b * cnx * cny * cnz;
  const int c1 = i0 / 2;
#pragma unroll
  for (int c = 0; c < 2; c++) {
    const int kz = c ? rz.k1 : rz.k0;
    if (kz < 0) continue;
#pragma unroll
    for (int bq = 0; bq < 2; bq++) {
      const int ky = bq ? ry.k1 : ry.k0;
      if (ky < 0) continue;
      const float w = (c ? rz.w1 : rz.w0) * (bq ? ry.w1 : ry.w0);
      const float* row = e + ((int64_t)kz * cny + ky) * cnx + c1;
      float ev[2 * G + 1];
      ev[0] = c1 > 0 ? row[-1] : 0.f;
#pragma unroll
      for (int q = 1; q <= 2 * G; q++) ev[q] = row[q - 1];
#pragma unroll
      for (int q = 0; q < G; q++) {
        const float e0 = ev[2 * q], e1 = ev[2 * q + 1], e2 = ev[2 * q + 2];
        u[q].x = fmaf(w, 0.5f * (e0 + e1), u[q].x);
        u[q].y = fmaf(w, e1, u[q].y);
        u[q].z = fmaf(w, 0.5f * (e1 + e2), u[q].z);
        u[q].w = fmaf(w, e2, u[q].w);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < G; q++) p[q] = u[q];
}

inline dim3 level_grid(int64_t n, int B) { return dim3((unsigned)((n + 255) / 256), (unsigned)B); }

template <typename T>
int level_op(const MGBatch& m, int i, int mode, const T* rhs, const T* x, T* out, cudaStream_t s) {
  const MGLevel& L = m.lv[i];
  if (L.stride == 8)
    k_mg_level<T, true><<<level_grid(L.n, m.B), 256, 0, s>>>(L, m.st, m.mask, mode, rhs, x, out, (T)kMGOmega);
  else
    k_mg_level<T, false><<<level_grid(L.n, m.B), 256, 0, s>>>(L, m.st, m.mask, mode, rhs, x, out, (T)kMGOmega);
  return 1;
}

// Fused coarse-level step on level view L (27-point rows).
template <typename T>
void coarse_step(const MGBatch& m, const MGLevel& L, int stage, int outk, const T* rhs, const T* xin, T* out,
                 const T* ec, const MGLevel* C, cudaStream_t s) {
  const int TX = L.nx >= 32 ? 32 : (L.nx >= 16 ? 16 : 8);
  const int TY = std::max(1, std::min(256 / TX, L.ny));
  const int tiles_x = (L.nx + TX - 1) / TX, tiles_y = (L.ny + TY - 1) / TY;
  // z-chunks: at least two waves of 4 resident CTAs per SM where the level allows,
  // and the whole chunk's staging within 48 KB of shared memory
  int nzc = 1;
  while ((int64_t)tiles_x * tiles_y * nzc * m.B < 8 * 152 && nzc * 2 <= L.nz / 4) nzc *= 2;
  int zc = (L.nz + nzc - 1) / nzc;
  while (zc > 1 && sizeof(T) * coarse_smem_elems(TX, TY, zc, stage == 2) > 48 * 1024) zc = (zc + 1) / 2;
  nzc = (L.nz + zc - 1) / zc;
  const dim3 grid(tiles_x * tiles_y, nzc, m.B), block(TX, TY);
  const size_t smem = sizeof(T) * coarse_smem_elems(TX, TY, zc, stage == 2);
  const int cnx = C ? C->nx : 0, cny = C ? C->ny : 0, cnz = C ? C->nz : 0;
  const T om = (T)kMGOmega;
#define RBWS_MG_COARSE(S, O) \
  k_mg_coarse<T, S, O><<<grid, block, smem, s>>>(L, m.st, m.mask, rhs, xin, out, ec, cnx, cny, cnz, om, tiles_x, zc)
  if (stage == 1 && outk == 0) RBWS_MG_COARSE(1, 0);
  else if (stage == 0 && outk == 1) RBWS_MG_COARSE(0, 1);
  else if (stage == 2 && outk == 0) RBWS_MG_COARSE(2, 0);
  else RBWS_MG_COARSE(0, 0);
#undef RBWS_MG_COARSE
}

// out = MG(rhs, A^i, i).  With up (the iterate of level i + 1): where the small
// levels run in one kernel, that kernel adds P out into up itself, does not
// store out, and sets *added.
template <typename T>
int vcycle(const MGBatch& m, int i, const T* rhs, T* out, cudaStream_t s, T* up = nullptr,
           bool* added = nullptr) {
  const MGPlan& P = *m.plan;
  if (added) *added = false;
  if constexpr (sizeof(T) == 4) {
    if (i == P.J && i > 0 && m.fine_cg) return vcycle_fine_fused(m, rhs, out, -1, s);
  }
  if (i > 0 && i < P.J && P.lv[i].n <= kMGTailMax) {
    MGTail tl;
    tl.top = i;
    tl.n0 = P.n0;
    for (int l = 0; l <= i; l++) tl.lv[l] = m.lv[l];
    tl.up = m.lv[i + 1];
    if (!up) tl.up.n = 0;
    const size_t smem = sizeof(T) * (size_t)tail_elems(P, i, tl.off);
    if (smem <= kMGTailSmem) {
      k_mg_tail<T><<<m.B, 1024, smem, s>>>(tl, m.st, m.mask, rhs, out, (const T*)m.ainv, (T)kMGOmega, up);
      if (added) *added = up != nullptr;
      return 1;
    }
  }
  if (i > 0 && i < P.J) {
    // coarse level with fused 27-point steps (kMGNu = 2): Y = S(0, rhs, 2);
    // W = rhs - A Y; restriction; coarse cycle e; W = step from Y + P e; out = step from W
    static_assert(kMGNu == 2, "the fused levels do two pre- and two post-smoothing steps");
    const MGLevel& F = m.lv[i];
    const MGLevel& C = m.lv[i - 1];
    T* Y = (T*)m.w1[i];
    T* W = (T*)m.w2[i];
    T* crhs = (T*)m.rhs[i - 1];
    T* csol = (T*)m.sol[i - 1];
    coarse_step<T>(m, F, 1, 0, rhs, nullptr, Y, nullptr, nullptr, s);
    coarse_step<T>(m, F, 0, 1, rhs, Y, W, nullptr, nullptr, s);
    k_mg_restrict<T><<<level_grid(C.n, m.B), 256, 0, s>>>(F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask, W,
                                                          crhs);
    bool added = false;
    int launches = 3 + vcycle<T>(m, i - 1, crhs, csol, s, Y, &added);
    if (added) coarse_step<T>(m, F, 0, 0, rhs, Y, W, nullptr, nullptr, s);  // Y holds Y + P e already
    else coarse_step<T>(m, F, 2, 0, rhs, Y, W, csol, &C, s);                 // W = step from Y + P e
    coarse_step<T>(m, F, 0, 0, rhs, W, out, nullptr, nullptr, s);
    return launches + 2;
  }
  if (i == 0) {
    k_mg_dense_apply<T><<<m.B, 128, 0, s>>>(P.n0, (const T*)m.ainv, m.st, m.mask, rhs, out);
    return 1;
  }
  int launches = 0;
  T* cur = (T*)m.w1[i];
  T* nxt = (T*)m.w2[i];
  launches += level_op<T>(m, i, 0, rhs, nullptr, cur, s);  // pre-smoothing from zero
  for (int k = 1; k < kMGNu; k++) {
    launches += level_op<T>(m, i, 1, rhs, cur, nxt, s);
    std::swap(cur, nxt);
  }
  launches += level_op<T>(m, i, 2, rhs, cur, nxt, s);       // residual into the free buffer
  const MGLevel& F = m.lv[i];
  const MGLevel& C = m.lv[i - 1];
  T* crhs = (T*)m.rhs[i - 1];
  T* csol = (T*)m.sol[i - 1];
  k_mg_restrict<T><<<level_grid(C.n, m.B), 256, 0, s>>>(F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask, nxt,
                                                        crhs);
  launches += 1;
  launches += vcycle<T>(m, i - 1, crhs, csol, s);
  k_mg_prolong_add<T><<<level_grid(F.n, m.B), 256, 0, s>>>(F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask,
                                                           csol, cur);
  launches += 1;
  for (int k = 1; k <= kMGNu; k++) {                         // post-smoothing
    T* dst = k == kMGNu ? out : nxt;
    launches += level_op<T>(m, i, 1, rhs, cur, dst, s);
    if (k < kMGNu) std::swap(cur, nxt);
  }
  return launches;
}

}  // namespace

int vcycle_fine_fused(const MGBatch& m, const float* rhs, float* out, int slot, cudaStream_t s) {
  static_assert(kMGNu == 2, "the fused finest level does two pre- and two post-smoothing steps");
  const int J = m.plan->J;
  const MGLevel& F = m.lv[J];
  const MGLevel& C = m.lv[J - 1];
  float* Y = (float*)m.w1[J];
  float* W = (float*)m.w2[J];
  float* crhs = (float*)m.rhs[J - 1];
  float* csol = (float*)m.sol[J - 1];
  MGFineArgs fa{rhs, nullptr, Y, C.nx, C.ny, C.nz, m.mask, (float)kMGOmega, slot, m.od};
  // the steps that write no partials run on wider tiles (less halo); the last,
  // with the rho partials, on the iteration's own tiling
  CGArgs<float> am = *m.fine_cg;
  if (m.mg_tile.tx > 0) {
    am.tiles_x = m.mg_tiles_x;
    am.tiles_y = m.mg_tiles_y;
    am.zc = m.mg_zc;
    am.nzc = m.mg_nzc;
  }
  const Tile tm = m.mg_tile.tx > 0 ? m.mg_tile : m.fine_tile;
  auto fine = [&](int k, int stage, int outk, bool open = true) {  // k: step index for the optional events
    if (m.ev && open) cudaEventRecord(m.ev[2 * k], s);
    if (outk == 2) launch_mg_fine_v4(*m.fine_cg, m.fine_tile, stage, outk, fa, s);
    else launch_mg_fine_v4(am, tm, stage, outk, fa, s);
    if (m.ev) cudaEventRecord(m.ev[2 * k + 1], s);
  };
  fine(0, 1, 0);  // Y = two smoothing steps from zero
  fa.xin = Y;
  int launches = 2;
  // coarse right-hand side P^T (r - A Y) in one pass where the tiling allows
  fa.out = crhs;
  if (m.ev) cudaEventRecord(m.ev[2], s);
  const bool fused_rr = launch_mg_fine_v4(am, tm, 0, 3, fa, s) == 0;
  if (!fused_rr) {
    fa.out = W;
    launch_mg_fine_v4(am, tm, 0, 1, fa, s);  // W = r - A Y
    k_mg_restrict<float><<<level_grid(C.n, m.B), 256, 0, s>>>(F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask, W,
                                                              crhs);
    launches += 1;
  }
  if (m.ev) cudaEventRecord(m.ev[3], s);
  launches += vcycle<float>(m, J - 1, crhs, csol, s);
  // Y += P e (a streaming pass), then W = one smoothing step from Y (timed together).  Forming
  // Y + P e where the step stages its planes (the coarse footprint staged per chunk) measured
  // no faster than the separate streaming pass.
  if (m.ev) cudaEventRecord(m.ev[4], s);
  if (F.nx % 8 == 0)
    k_mg_prolong_add4<2><<<dim3((unsigned)((F.n / 8 + 255) / 256), (unsigned)m.B), 256, 0, s>>>(
        F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask, csol, Y);
  else
    k_mg_prolong_add4<1><<<dim3((unsigned)((F.n / 4 + 255) / 256), (unsigned)m.B), 256, 0, s>>>(
        F.nx, F.ny, F.nz, C.nx, C.ny, C.nz, m.st, m.mask, csol, Y);
  launches += 1;
  if (m.ev) cudaEventRecord(m.ev[8], s);  // the prolongation pass ends here
  fa.xin = Y;
  fa.out = W;
  fine(2, 0, 0, false);  // W = smoothing step from Y
  fa.xin = W;
  fa.out = out;
  fine(3, 0, slot >= 0 ? 2 : 0);  // out = last step (+ rho)
  return launches + 2;
}

int launch_mg_vcycle(const MGBatch& m, const void* rhs, void* out, int slot, cudaStream_t s) {
  if (m.fp32) {
    if (m.fine_cg && m.plan->J > 0) return vcycle_fine_fused(m, (const float*)rhs, (float*)out, slot, s);
    return vcycle<float>(m, m.plan->J, (const float*)rhs, (float*)out, s);
  }
  return vcycle<double>(m, m.plan->J, (const double*)rhs, (double*)out, s);
}

void launch_diag_inverse(const MGLevel& L, int B, const double* x, double* y, cudaStream_t s) {
  if (L.stride == 8)
    k_mg_level<double, true><<<level_grid(L.n, B), 256, 0, s>>>(L, nullptr, nullptr, 0, x, nullptr, y, 1.0);
  else
    k_mg_level<double, false><<<level_grid(L.n, B), 256, 0, s>>>(L, nullptr, nullptr, 0, x, nullptr, y, 1.0);
}

}  // namespace rbws
