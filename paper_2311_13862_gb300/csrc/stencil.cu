// stencil.cu -- matrix-free affine 7-point operator and the fused Jacobi-PCG
// phase kernels (Algorithm 1) for sm_103a.
//
// Layout: planar [B][nz][ny][nx], x fastest.  Every stencil kernel marches a
// CTA tile of TX x TY columns through a chunk of z planes.  Plane z (with a
// one-node halo in x and y) is staged in a 3-slot shared-memory ring; the
// z-1 / z+1 values of a thread's own column stay in registers, so each plane
// is read from memory once per tile.  One __syncthreads per plane.
//
// Coefficients come from a per-instance class table (see internal.h): a
// thread caches its column's 8-value row and reloads it only when the z class
// changes, so the FP64 stencil costs 1 DMUL + 6 DFMA per node.  GB300 runs
// FP64 at ~1/60 of its FP32 rate, so the FP64 kernels are written to minimise
// FP64 instructions, not bytes.
//
// Reductions are deterministic: each CTA reduces its threads in a fixed tree
// and writes one partial; consumers sum an instance's partials in index order
// with a fixed shuffle tree, so every CTA of an instance (and every rerun)
// sees bit-identical scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace rbws {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_down(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;  // valid in lane 0
}

// Deterministic block sum of two values; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  a = warp_sum_down(a);
  b = warp_sum_down(b);
  __syncthreads();  // red may still be in use by an earlier reduction
  if (lane == 0) {
    red[warp] = a;
    red[32 + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    double x = lane < nw ? red[lane] : 0.0;
    double y = lane < nw ? red[32 + lane] : 0.0;
    a = warp_sum_down(x);
    b = warp_sum_down(y);
  }
}

// Sum of an instance's partials in a fixed order (called by a full warp);
// result valid in lane 0.
__device__ __forceinline__ double sum_partials(const double* part, int P, int lane) {
  double s = 0.0;
  for (int c = lane; c < P; c += 32) s += part[c];
  return warp_sum_down(s);
}
__device__ __forceinline__ double2 sum_partials2(const double2* part, int P, int lane) {
  double x = 0.0, y = 0.0;
  for (int c = lane; c < P; c += 32) {
    double2 v = part[c];
    x += v.x;
    y += v.y;
  }
  return make_double2(warp_sum_down(x), warp_sum_down(y));
}

// Column geometry of the calling thread inside its CTA tile.
struct Column {
  int i, j;
  bool own;
  int64_t col;  // j*nx + i
  int xy;       // class index (cy*ncx + cx) of the column
};

__device__ __forceinline__ Column make_column(const Geo& g, int x0, int y0) {
  Column c;
  c.i = x0 + (int)threadIdx.x;
  c.j = y0 + (int)threadIdx.y;
  c.own = c.i < g.nx && c.j < g.ny;
  c.col = (int64_t)c.j * g.nx + c.i;
  c.xy = c.own ? (int)g.cy[c.j] * g.ncx + (int)g.cx[c.i] : 0;
  return c;
}

// The z-marching stencil skeleton.  load(idx) returns the staged field at an
// in-domain node (idx = z*nx*ny + j*nx + i); consume(idx, x_c, y, dinv) gets
// y = (A x)(node) for each owned node of planes [z0, z1), or with kResid
// y = base(idx) - (A x)(node) (the terms subtracted in the same FMA chain).
struct ZNoBase {
  __device__ __forceinline__ double operator()(int64_t) const { return 0.0; }
};
template <typename T, bool kResid = false, class Load, class Consume, class Base = ZNoBase>
__device__ __forceinline__ void zmarch(const Geo& g, const T* __restrict__ coef_b, int x0, int y0,
                                       int z0, int z1, T* sm, Load load, Consume consume, Base base = Base()) {
  const int TX = blockDim.x, TY = blockDim.y;
  const int tid = threadIdx.y * TX + threadIdx.x;
  const Column cl = make_column(g, x0, y0);
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int PW = TX + 2, PS = PW * (TY + 2);
  const int nh = 2 * TX + 2 * TY;
  int hi, hj;
  if (tid < TX) {
    hi = tid; hj = -1;
  } else if (tid < 2 * TX) {
    hi = tid - TX; hj = TY;
  } else if (tid < 2 * TX + TY) {
    hi = -1; hj = tid - 2 * TX;
  } else {
    hi = TX; hj = tid - 2 * TX - TY;
  }
  const int gi = x0 + hi, gj = y0 + hj;
  const bool has_halo = tid < nh;
  const bool hin = has_halo && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
  const int64_t hcol = (int64_t)gj * g.nx + gi;
  const int hslot = (hj + 1) * PW + hi + 1;
  const int oslot = ((int)threadIdx.y + 1) * PW + (int)threadIdx.x + 1;

  auto stage = [&](int z, T* Pl) -> T {
    T v = T(0);
    const bool zin = z >= 0 && z < g.nz;
    if (zin && cl.own) v = load((int64_t)z * plane + cl.col);
    Pl[oslot] = v;
    if (has_halo) {
      T hv = T(0);
      if (zin && hin) hv = load((int64_t)z * plane + hcol);
      Pl[hslot] = hv;
    }
    return v;
  };

  int zcls_cur = -1;
  T c[kCoefStride];
#pragma unroll
  for (int k = 0; k < kCoefStride; k++) c[k] = T(0);
  T xm = (z0 > 0 && cl.own) ? load((int64_t)(z0 - 1) * plane + cl.col) : T(0);
  T xc = stage(z0, sm + (z0 % 3) * PS);
  for (int z = z0; z < z1; ++z) {
    T xp = stage(z + 1, sm + ((z + 1) % 3) * PS);
    __syncthreads();
    const T* Pl = sm + (z % 3) * PS;
    const int zcl = g.cz[z];
    if (zcl != zcls_cur) {
      zcls_cur = zcl;
      const T* row = coef_b + ((int64_t)zcl * g.ncy * g.ncx + cl.xy) * kCoefStride;
#pragma unroll
      for (int k = 0; k < kCoefStride; k++) c[k] = row[k];
    }
    if (cl.own) {
      const int64_t idx = (int64_t)z * plane + cl.col;
      T y;
      if (kResid) {
        y = (T)base(idx);
        y = fma(-c[6], xc, y);
        y = fma(-c[0], Pl[oslot - 1], y);
        y = fma(-c[1], Pl[oslot + 1], y);
        y = fma(-c[2], Pl[oslot - PW], y);
        y = fma(-c[3], Pl[oslot + PW], y);
        y = fma(-c[4], xm, y);
        y = fma(-c[5], xp, y);
      } else {
        y = c[6] * xc;
        y = fma(c[0], Pl[oslot - 1], y);
        y = fma(c[1], Pl[oslot + 1], y);
        y = fma(c[2], Pl[oslot - PW], y);
        y = fma(c[3], Pl[oslot + PW], y);
        y = fma(c[4], xm, y);
        y = fma(c[5], xp, y);
      }
      consume(idx, xc, y, c[7]);
    }
    xm = xc;
    xc = xp;
  }
}

struct TilePos {
  int x0, y0, z0, z1, part;
};

// The block a kernel body works on: blockIdx and gridDim.x of an ordinary launch, or a
// work item of the persistent iteration kernel.
struct VBlk {
  int x, y, z, gx;
  __device__ __forceinline__ static VBlk here() { return VBlk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x}; }
};

__device__ __forceinline__ TilePos tile_pos_v(const Geo& g, int tiles_x, int zc, const VBlk& v) {
  TilePos t;
  t.x0 = (v.x % tiles_x) * blockDim.x;
  t.y0 = (v.x / tiles_x) * blockDim.y;
  t.z0 = v.y * zc;
  t.z1 = min(g.nz, t.z0 + zc);
  t.part = v.y * v.gx + v.x;
  return t;
}

__device__ __forceinline__ TilePos tile_pos(const Geo& g, int tiles_x, int zc) {
  TilePos t;
  const int tile = blockIdx.x;
  t.x0 = (tile % tiles_x) * blockDim.x;
  t.y0 = (tile / tiles_x) * blockDim.y;
  t.z0 = blockIdx.y * zc;
  t.z1 = min(g.nz, t.z0 + zc);
  t.part = blockIdx.y * gridDim.x + blockIdx.x;
  return t;
}

// ---------------------------------------------------------------------------
// Coefficient tables
// ---------------------------------------------------------------------------
__global__ void k_coef_tables(Geo g, const int8_t* __restrict__ kx, const int8_t* __restrict__ ky,
                              const int8_t* __restrict__ kz, int bx, int by,
                              const uint8_t* __restrict__ segq, double sx, double sy, double sz, int Q,
                              const double* __restrict__ mu, int B, double* __restrict__ coef64,
                              float* __restrict__ coef32) {
  const int ncls = g.ncls();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ncls * B) return;
  const int b = (int)(t / ncls), e = (int)(t % ncls);
  const int cxi = e % g.ncx, cyi = (e / g.ncx) % g.ncy, czi = e / (g.ncx * g.ncy);
  const int ox = kx[3 * cxi], lx = kx[3 * cxi + 1], hx = kx[3 * cxi + 2];
  const int oy = ky[3 * cyi], ly = ky[3 * cyi + 1], hy = ky[3 * cyi + 2];
  const int oz = kz[3 * czi], lz = kz[3 * czi + 1], hz = kz[3 * czi + 2];
  const double* m = mu + (int64_t)b * Q;
  auto kap = [&](int ax, int ay, int az) {
    const int box = (az * by + ay) * bx + ax;
    return m[segq ? segq[box] : box];
  };
  const double kc = kap(ox, oy, oz);
  // face coefficient: arithmetic mean of the two kappas; Dirichlet boundary face (key -1):
  // own kappa; no face past a Neumann face (key -2)
  auto face = [&](int nb, double knb, double s) { return nb >= 0 ? 0.5 * (kc + knb) * s : (nb == -1 ? kc * s : 0.0); };
  // a node on a Neumann face has half a control volume: its faces across the other axes
  // have half the area
  const double wx = hx == -2 ? 0.5 : 1.0, wy = hy == -2 ? 0.5 : 1.0, wz = hz == -2 ? 0.5 : 1.0;
  const double kW = face(lx, lx >= 0 ? kap(lx, oy, oz) : 0.0, sx) * (wy * wz);
  const double kE = face(hx, hx >= 0 ? kap(hx, oy, oz) : 0.0, sx) * (wy * wz);
  const double kS = face(ly, ly >= 0 ? kap(ox, ly, oz) : 0.0, sy) * (wx * wz);
  const double kN = face(hy, hy >= 0 ? kap(ox, hy, oz) : 0.0, sy) * (wx * wz);
  const double kD = face(lz, lz >= 0 ? kap(ox, oy, lz) : 0.0, sz) * (wx * wy);
  const double kU = face(hz, hz >= 0 ? kap(ox, oy, hz) : 0.0, sz) * (wx * wy);
  const double D = kW + kE + kS + kN + kD + kU;
  const double v[kCoefStride] = {-kW, -kE, -kS, -kN, -kD, -kU, D, 1.0 / D};
  double* o64 = coef64 + ((int64_t)b * ncls + e) * kCoefStride;
  for (int k = 0; k < kCoefStride; k++) o64[k] = v[k];
  if (coef32) {
    float* o32 = coef32 + ((int64_t)b * ncls + e) * kCoefStride;
    for (int k = 0; k < kCoefStride; k++) o32[k] = (float)v[k];
    o32[7] = 1.0f / (float)D;
  }
}

// ---------------------------------------------------------------------------
// y = A(mu) x
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_apply(Geo g, int tiles_x, int zc, const T* __restrict__ coef, const T* __restrict__ x,
                        int64_t x_stride, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.z;
  const TilePos tp = tile_pos(g, tiles_x, zc);
  const T* xb = x + (int64_t)b * x_stride;
  T* yb = y + (int64_t)b * g.n;
  const T* cb = coef + (int64_t)b * g.ncls() * kCoefStride;
  zmarch<T>(
      g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm, [&](int64_t idx) { return xb[idx]; },
      [&](int64_t idx, T, T v, T) { yb[idx] = v; });
}

// r = f - A u in FP64 with partial sums of r.r per CTA.
__global__ void k_residual64(Geo g, int tiles_x, int zc, const double* __restrict__ coef,
                             const double* __restrict__ f, int64_t f_stride, const double* __restrict__ u,
                             double* __restrict__ r, double* __restrict__ rr_part, int P,
                             const int* __restrict__ mask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int b = blockIdx.z;
  if (mask && !mask[b]) return;
  const TilePos tp = tile_pos(g, tiles_x, zc);
  const double* ub = u + (int64_t)b * g.n;
  const double* fb = f ? f + (int64_t)b * f_stride : nullptr;
  double* rb = r ? r + (int64_t)b * g.n : nullptr;
  const double* cb = coef + (int64_t)b * g.ncls() * kCoefStride;
  double acc = 0.0;
  zmarch<double, true>(
      g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm, [&](int64_t idx) { return ub[idx]; },
      [&](int64_t idx, double, double rv, double) {  // rv = f - A u
        if (rb) rb[idx] = rv;
        acc = fma(rv, rv, acc);
      },
      [&](int64_t idx) { return fb ? fb[idx] : 1.0; });
  double dummy = 0.0;
  block_sum2(acc, dummy, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) rr_part[(int64_t)b * P + tp.part] = acc;
}

// The same residual from the float-float solution of the mixed-precision iteration: each
// staged value is hi + lo converted to FP64 (ff_to_f64), and each node's value is written
// to u (the FP64 solution that the check decides on), so no separate conversion pass reads
// and writes the solution first.
__global__ void k_residual64_ff(Geo g, int tiles_x, int zc, const double* __restrict__ coef,
                                const double* __restrict__ f, int64_t f_stride, const float* __restrict__ uh,
                                const float* __restrict__ ul, double* __restrict__ u, double* __restrict__ r,
                                double* __restrict__ rr_part, int P, const int* __restrict__ mask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int b = blockIdx.z;
  if (mask && !mask[b]) return;
  const TilePos tp = tile_pos(g, tiles_x, zc);
  const int64_t off = (int64_t)b * g.n;
  const float* hb = uh + off;
  const float* lb = ul + off;
  double* ub = u + off;
  const double* fb = f ? f + (int64_t)b * f_stride : nullptr;
  double* rb = r ? r + off : nullptr;
  const double* cb = coef + (int64_t)b * g.ncls() * kCoefStride;
  double acc = 0.0;
  zmarch<double, true>(
      g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm, [&](int64_t idx) { return ff_to_f64(hb[idx], lb[idx]); },
      [&](int64_t idx, double uc, double rv, double) {  // uc = u at the node, rv = f - A u
        ub[idx] = uc;
        if (rb) rb[idx] = rv;
        acc = fma(rv, rv, acc);
      },
      [&](int64_t idx) { return fb ? fb[idx] : 1.0; });
  double dummy = 0.0;
  block_sum2(acc, dummy, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) rr_part[(int64_t)b * P + tp.part] = acc;
}

// ---------------------------------------------------------------------------
// PCG phase kernels.  Per iteration k (parity = k % 2):
//   A: beta = rho_k / rho_{k-1};  p_new = s + beta p_old (staged, halo too);
//      q = A p_new;  gamma partials = p_new . q.       Stops converged ones.
//   B: alpha = rho_k / gamma;  u += alpha p;  r -= alpha q;  s = D^{-1} r;
//      partials of rho_{k+1} = r.s and r.r.
// Search directions ping-pong: A(parity) reads pbuf[parity], writes
// pbuf[parity^1]; rho/rr partials ping-pong the same way.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cg_init_body(const CGArgs<T>& a, int parity, const VBlk& v) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int b = v.z;
  const TilePos tp = tile_pos_v(a.g, a.tiles_x, a.zc, v);
  const int64_t off = (int64_t)b * a.g.n;
  const T* cb = a.coef + (int64_t)b * a.g.ncls() * kCoefStride;
  T* pold = (parity ? a.p1 : a.p0) + off;
  T* ub = a.u + off;
  T* rb = a.r + off;
  T* sb = a.s + off;
  const bool jac = a.precond != RBWS_PREC_NONE;  // Jacobi, or D^{-1} r as MSRB's first sweep
  // MSRB and MG compute s and rho = r.s in their own passes
  const bool msrb = a.precond == RBWS_PREC_MSRB || a.precond == RBWS_PREC_MG;
  T rho = T(0), rr = T(0);
  if (a.rhs64 == nullptr) {
    zmarch<T>(
        a.g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm, [&](int64_t idx) { return ub[idx]; },
        [&](int64_t idx, T, T v, T dinv) {
          const T rv = (a.f ? a.f[(int64_t)b * a.f_stride + idx] : T(1)) - v;
          const T sv = jac ? dinv * rv : rv;
          rb[idx] = rv;
          if (jac) sb[idx] = sv;
          pold[idx] = T(0);
          rho = fma(rv, sv, rho);
          rr = fma(rv, rv, rr);
        });
  } else {
    // FP32_IR inner system: right-hand side = FP64 outer residual / ||residual||
    const Column cl = make_column(a.g, tp.x0, tp.y0);
    const double scale = 1.0 / a.rhs_scale[b];
    const double* hb = a.rhs64 + off;
    const int64_t plane = (int64_t)a.g.nx * a.g.ny;
    if (cl.own) {
      int zcls_cur = -1;
      T dinv = T(1);
      for (int z = tp.z0; z < tp.z1; ++z) {
        const int zcl = a.g.cz[z];
        if (zcl != zcls_cur) {
          zcls_cur = zcl;
          dinv = cb[((int64_t)zcl * a.g.ncy * a.g.ncx + cl.xy) * kCoefStride + 7];
        }
        const int64_t idx = (int64_t)z * plane + cl.col;
        const T rv = (T)(hb[idx] * scale);
        const T sv = jac ? dinv * rv : rv;
        ub[idx] = T(0);
        rb[idx] = rv;
        if (jac) sb[idx] = sv;
        pold[idx] = T(0);
        rho = fma(rv, sv, rho);
        rr = fma(rv, rv, rr);
      }
    }
  }
  double drho = msrb ? 0.0 : (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    a.rho_rr[((int64_t)parity * a.B + b) * a.P + tp.part] = make_double2(drho, drr);
    // rho_{k-1} := 1 (p_old = 0, so beta only has to be finite)
    a.rho_rr[((int64_t)(parity ^ 1) * a.B + b) * a.P + tp.part] =
        make_double2(tp.part == 0 ? 1.0 : 0.0, 0.0);
  }
}

template <typename T>
__global__ void k_cg_init(CGArgs<T> a, int parity) {
  cg_init_body<T>(a, parity, VBlk::here());
}

// Called by a full warp (lane 0..31) for instance b.
template <typename T>
__device__ __forceinline__ void cg_finalize_body(const CGArgs<T>& a, int parity, int mode, int max_restarts, int b,
                                                 int lane) {
  if (b >= a.B) return;
  const double2 v = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, lane);
  if (lane != 0) return;
  InstState& s = a.st[b];
  const double rel = sqrt(v.y) / a.fnorm[b];
  if (a.hist) {
    const int k = mode == 0 ? 0 : s.iters;
    if (k < a.hist_len) a.hist[(int64_t)b * a.hist_len + k] = rel;
  }
  if (mode == 0) {
    s.relres0 = rel;
    s.relres = rel;
    s.iters = 0;
    s.restarts = 0;
    s.t_done = global_ns();
    if (rel < a.tol) {
      s.status = ST_CONVERGED;
    } else if (!(rel == rel) || a.max_iters <= 0) {
      s.status = (rel == rel) ? ST_MAX_ITERS : ST_BREAKDOWN;
    } else {
      s.status = ST_ACTIVE;
      atomicAdd(a.active, 1);
    }
  } else {
    s.relres = rel;
    if (s.status == ST_CONVERGED && !(rel < a.tol)) {
      if (s.restarts < max_restarts && s.iters < a.max_iters && rel == rel) {
        s.restarts += 1;
        s.status = ST_ACTIVE;
        atomicAdd(a.active, 1);
      } else {
        s.status = ST_MAX_ITERS;
      }
    }
  }
}

template <typename T>
__global__ void k_cg_finalize(CGArgs<T> a, int parity, int mode, int max_restarts) {
  cg_finalize_body<T>(a, parity, mode, max_restarts, (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)),
                      (int)(threadIdx.x & 31));
}

template <typename T>
__device__ __forceinline__ void cg_a_body(const CGArgs<T>& a, int parity, const VBlk& v) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ double s_beta;
  __shared__ int s_run;
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int b = v.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const TilePos tp = tile_pos_v(a.g, a.tiles_x, a.zc, v);
  const bool leader = tp.part == 0;
  if (tid < 32) {
    InstState* st = a.st + b;
    const int status = st->status;
    double2 cur = make_double2(0.0, 0.0);
    double prev = 0.0;
    if (status == ST_ACTIVE) {
      cur = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, tid);
      const double2 pv = sum_partials2(a.rho_rr + ((int64_t)(parity ^ 1) * a.B + b) * a.P, a.P, tid);
      prev = pv.x;
    }
    if (tid == 0) {
      int run = 0;
      if (status == ST_ACTIVE) {
        const double rel = sqrt(cur.y) / a.fnorm[b];
        if (leader && a.hist && st->iters < a.hist_len) a.hist[(int64_t)b * a.hist_len + st->iters] = rel;
        if (rel < a.tol) {
          if (leader) {
            st->status = a.ru ? ST_PAUSED : ST_CONVERGED;
            st->relres = rel;
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else if (st->iters >= a.max_iters || !(rel == rel)) {
          if (leader) {
            st->status = (rel == rel) ? ST_MAX_ITERS : ST_BREAKDOWN;
            st->relres = rel;
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else {
          run = 1;
          s_beta = cur.x / prev;
        }
      }
      s_run = run;
    }
  }
  __syncthreads();
  if (!s_run) return;
  const T beta = (T)s_beta;
  const int64_t off = (int64_t)b * a.g.n;
  const T* cb = a.coef + (int64_t)b * a.g.ncls() * kCoefStride;
  const T* sb = (a.precond != RBWS_PREC_NONE ? a.s : a.r) + off;
  const T* pold = (parity ? a.p1 : a.p0) + off;
  T* pnew = (parity ? a.p0 : a.p1) + off;
  T* qb = a.q + off;
  T gam = T(0);
  zmarch<T>(
      a.g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm,
      [&](int64_t idx) { return fma(beta, pold[idx], sb[idx]); },
      [&](int64_t idx, T pc, T v, T) {
        pnew[idx] = pc;
        qb[idx] = v;
        gam = fma(pc, v, gam);
      });
  double dg = (double)gam, dummy = 0.0;
  block_sum2(dg, dummy, red);
  if (tid == 0) a.gam[(int64_t)b * a.P + tp.part] = dg;
}

template <typename T>
__global__ void k_cg_a(CGArgs<T> a, int parity) {
  cg_a_body<T>(a, parity, VBlk::here());
}

template <typename T>
__device__ __forceinline__ void cg_b_body(const CGArgs<T>& a, int parity, const VBlk& v) {
  __shared__ double red[64];
  __shared__ double s_alpha;
  __shared__ int s_run;
  const int b = v.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const TilePos tp = tile_pos_v(a.g, a.tiles_x, a.zc, v);
  const bool leader = tp.part == 0;
  if (tid < 32) {
    InstState* st = a.st + b;
    const int status = st->status;
    double rho = 0.0, gam = 0.0, rr = 0.0;
    if (status == ST_ACTIVE) {
      const double2 cur = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, tid);
      rho = cur.x;
      rr = cur.y;
      gam = sum_partials(a.gam + (int64_t)b * a.P, a.P, tid);
    }
    if (tid == 0) {
      int run = 0;
      if (status == ST_ACTIVE) {
        const double alpha = rho / gam;
        if (!(gam > 0.0) || !(alpha == alpha) || alpha == INFINITY) {
          if (leader) {
            st->status = ST_BREAKDOWN;
            st->relres = sqrt(rr) / a.fnorm[b];
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else {
          run = 1;
          s_alpha = alpha;
          if (leader) st->iters += 1;
        }
      }
      s_run = run;
    }
  }
  __syncthreads();
  if (!s_run) return;
  const T alpha = (T)s_alpha;
  const int64_t off = (int64_t)b * a.g.n;
  const T* cb = a.coef + (int64_t)b * a.g.ncls() * kCoefStride;
  const T* pn = (parity ? a.p0 : a.p1) + off;
  const T* qb = a.q + off;
  T* ub = a.u + off;
  T* rb = a.r + off;
  T* sb = a.s + off;
  const bool jac = a.precond != RBWS_PREC_NONE;
  const bool msrb = a.precond == RBWS_PREC_MSRB || a.precond == RBWS_PREC_MG;
  const Column cl = make_column(a.g, tp.x0, tp.y0);
  const int64_t plane = (int64_t)a.g.nx * a.g.ny;
  T rho = T(0), rr = T(0);
  if (cl.own) {
    int zcls_cur = -1;
    T dinv = T(1);
    for (int z = tp.z0; z < tp.z1; ++z) {
      const int zcl = a.g.cz[z];
      if (zcl != zcls_cur) {
        zcls_cur = zcl;
        dinv = cb[((int64_t)zcl * a.g.ncy * a.g.ncx + cl.xy) * kCoefStride + 7];
      }
      const int64_t idx = (int64_t)z * plane + cl.col;
      const T pv = pn[idx];
      const T qv = qb[idx];
      ub[idx] = fma(alpha, pv, ub[idx]);
      const T rv = fma(-alpha, qv, rb[idx]);
      rb[idx] = rv;
      T sv = rv;
      if (jac) {
        sv = dinv * rv;
        sb[idx] = sv;
      }
      rho = fma(rv, sv, rho);
      rr = fma(rv, rv, rr);
    }
  }
  double drho = msrb ? 0.0 : (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (tid == 0)
    a.rho_rr[((int64_t)(parity ^ 1) * a.B + b) * a.P + tp.part] = make_double2(drho, drr);
}

template <typename T>
__global__ void k_cg_b(CGArgs<T> a, int parity) {
  cg_b_body<T>(a, parity, VBlk::here());
}

// ---------------------------------------------------------------------------
// MSRB preconditioner (Algorithm 3) for the active instances.  On entry s
// holds u~ = D^{-1} r (one undamped Jacobi sweep from zero).
//   1. q = r - A u~                                  (stencil; q is free here)
//   2. g = W^T q                                     (two-stage projections)
//   3. c = A_N(mu)^{-1} g                            (cached Cholesky factor)
//   4. s = u~ + W c,  partial rho = r.s              (into parity slot `slot`)
// ---------------------------------------------------------------------------
__global__ void k_msrb_residual(CGArgs<double> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE) return;
  const TilePos tp = tile_pos(a.g, a.tiles_x, a.zc);
  const int64_t off = (int64_t)b * a.g.n;
  const double* cb = a.coef + (int64_t)b * a.g.ncls() * kCoefStride;
  const double* ut = a.s + off;
  const double* rb = a.r + off;
  double* qb = a.q + off;
  zmarch<double>(
      a.g, cb, tp.x0, tp.y0, tp.z0, tp.z1, sm, [&](int64_t idx) { return ut[idx]; },
      [&](int64_t idx, double, double v, double) { qb[idx] = rb[idx] - v; });
}

constexpr int kProjJ = 8;  // basis vectors per pass of the projection kernel

// part[b][chunk][j] = sum over the chunk's nodes of W[j][i] q[b][i]
__global__ void k_msrb_project(CGArgs<double> a) {
  __shared__ double red[kProjJ][32];
  const int b = blockIdx.y;
  if (a.st[b].status != ST_ACTIVE) return;
  const int chunk = blockIdx.x, chunks = gridDim.x;
  const int64_t n = a.g.n;
  const double* qb = a.q + (int64_t)b * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j0 = 0; j0 < a.N; j0 += kProjJ) {
    double acc[kProjJ];
#pragma unroll
    for (int k = 0; k < kProjJ; k++) acc[k] = 0.0;
    for (int64_t i = (int64_t)chunk * blockDim.x + threadIdx.x; i < n; i += (int64_t)chunks * blockDim.x) {
      const double qv = qb[i];
#pragma unroll
      for (int k = 0; k < kProjJ; k++)
        if (j0 + k < a.N) acc[k] = fma(a.W[(int64_t)(j0 + k) * n + i], qv, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kProjJ; k++) {
      double v = warp_sum_down(acc[k]);
      if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int k = 0; k < kProjJ; k++) {
        double v = lane < nw ? red[k][lane] : 0.0;
        v = warp_sum_down(v);
        if (lane == 0 && j0 + k < a.N)
          a.proj_part[((int64_t)b * chunks + chunk) * a.N + j0 + k] = v;
      }
    }
    __syncthreads();
  }
}

// One warp per instance: g = sum of the chunk partials, then c = L^{-T} L^{-1} g.
__global__ void k_msrb_reduce_solve(CGArgs<double> a) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= a.B || a.st[b].status != ST_ACTIVE) return;
  const int N = a.N, chunks = a.proj_chunks;
  double* g = a.G + (int64_t)b * N;
  for (int j = 0; j < N; j++) {
    double v = 0.0;
    for (int c = lane; c < chunks; c += 32) v += a.proj_part[((int64_t)b * chunks + c) * N + j];
    v = warp_sum_down(v);
    if (lane == 0) g[j] = v;
  }
  __syncwarp();
  if (lane == 0) {
    const double* L = a.L + (int64_t)b * N * N;
    double* c = a.C + (int64_t)b * N;
    for (int i = 0; i < N; i++) {
      double v = g[i];
      for (int k = 0; k < i; k++) v = fma(-L[i * N + k], c[k], v);
      c[i] = v / L[i * N + i];
    }
    for (int i = N - 1; i >= 0; i--) {
      double v = c[i];
      for (int k = i + 1; k < N; k++) v = fma(-L[k * N + i], c[k], v);
      c[i] = v / L[i * N + i];
    }
  }
}

// s = u~ + W c and the partials of rho = r.s (same tiling as the update phase).
__global__ void k_msrb_lift(CGArgs<double> a, int slot) {
  __shared__ double red[64];
  __shared__ double cs[256];
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int j = tid; j < a.N; j += blockDim.x * blockDim.y) cs[j] = a.C[(int64_t)b * a.N + j];
  __syncthreads();
  const TilePos tp = tile_pos(a.g, a.tiles_x, a.zc);
  const int64_t off = (int64_t)b * a.g.n;
  const Column cl = make_column(a.g, tp.x0, tp.y0);
  const int64_t plane = (int64_t)a.g.nx * a.g.ny;
  double rho = 0.0;
  if (cl.own) {
    for (int z = tp.z0; z < tp.z1; ++z) {
      const int64_t idx = (int64_t)z * plane + cl.col;
      double sv = a.s[off + idx];
      for (int j = 0; j < a.N; j++) sv = fma(cs[j], a.W[(int64_t)j * a.g.n + idx], sv);
      a.s[off + idx] = sv;
      rho = fma(a.r[off + idx], sv, rho);
    }
  }
  double dummy = 0.0;
  block_sum2(rho, dummy, red);
  if (tid == 0) a.rho_rr[((int64_t)slot * a.B + b) * a.P + tp.part].x = rho;
}

// Partials of rho = r.s after an external preconditioner (the MG V-cycle) has
// written s; same tiling and slot layout as the update phase.
template <typename T>
__global__ void k_precond_rho(CGArgs<T> a, int slot, const int* mask) {
  __shared__ double red[64];
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (mask && !mask[b])) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const TilePos tp = tile_pos(a.g, a.tiles_x, a.zc);
  const int64_t off = (int64_t)b * a.g.n;
  const Column cl = make_column(a.g, tp.x0, tp.y0);
  const int64_t plane = (int64_t)a.g.nx * a.g.ny;
  double rho = 0.0;
  if (cl.own)
    for (int z = tp.z0; z < tp.z1; ++z) {
      const int64_t idx = off + (int64_t)z * plane + cl.col;
      rho = fma((double)a.r[idx], (double)a.s[idx], rho);
    }
  double dummy = 0.0;
  block_sum2(rho, dummy, red);
  if (tid == 0) a.rho_rr[((int64_t)slot * a.B + b) * a.P + tp.part].x = rho;
}

// ---------------------------------------------------------------------------
// FP32 PCG with FP64 reliable updates.  At the end of every block of
// iterations (parity 0 again), k_ru_decide flags the instances that need an
// FP64 update: ACTIVE ones whose FP32 residual fell below sqrt(ru_delta2)
// times the residual at their last update (the search direction is kept),
// and PAUSED ones (FP32 residual met tol; the direction restarts if the FP64
// check fails).  An update folds the FP32 correction d into u64, forms the
// FP64 residual, and resets the FP32 residual from it.
// ---------------------------------------------------------------------------
__global__ void k_ru_decide(CGArgs<float> a) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= a.B) return;
  InstState& s = a.st[b];
  const int status = s.status;
  double rr = 0.0;
  if (status == ST_ACTIVE) rr = sum_partials2(a.rho_rr + (int64_t)b * a.P, a.P, lane).y;  // slot 0
  if (lane != 0) return;
  int u = 0;
  if (status == ST_ACTIVE && rr < a.ru_delta2 * a.rr_ref[b]) {
    u = 1;
    s.status = ST_UPDATE;
    atomicSub(a.active, 1);
  } else if (status == ST_PAUSED) {
    u = 2;
  }
  a.upd[b] = u;
  if (u) atomicAdd(a.pending, 1);
}

// u64 += d; d = 0 for flagged instances.  With the 32-byte schedule the
// update alpha p of the last iteration is still pending: it is added here
// (parity 0 for updates at a block boundary, the recorded parity otherwise).
__global__ void k_ru_fold(CGArgs<float> a) {
  const int b = blockIdx.y;
  const int mode = a.upd[b];
  if (!mode) return;
  const int par = mode == 1 ? 0 : a.st[b].pad;
  const double al = a.alpha ? a.alpha[(int64_t)par * a.B + b] : 0.0;
  const float* pp = (par ? a.p1 : a.p0) + (int64_t)b * a.g.n;
  const int64_t off = (int64_t)b * a.g.n, n = a.g.n;
  double* u64 = a.u64 + off;
  float* d = a.u + off;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const bool vec = (n & 3) == 0 && ((reinterpret_cast<uintptr_t>(u64) | reinterpret_cast<uintptr_t>(d) |
                                     reinterpret_cast<uintptr_t>(pp)) & 15) == 0;
  if (vec) {  // 4 nodes per thread: 16-byte accesses
    for (int64_t k = t0; k < (n >> 2); k += stride) {
      const float4 dv = reinterpret_cast<const float4*>(d)[k];
      double2 lo = reinterpret_cast<const double2*>(u64)[2 * k], hi = reinterpret_cast<const double2*>(u64)[2 * k + 1];
      lo.x += (double)dv.x;
      lo.y += (double)dv.y;
      hi.x += (double)dv.z;
      hi.y += (double)dv.w;
      if (al != 0.0) {
        const float4 pv = reinterpret_cast<const float4*>(pp)[k];
        lo.x = fma(al, (double)pv.x, lo.x);
        lo.y = fma(al, (double)pv.y, lo.y);
        hi.x = fma(al, (double)pv.z, hi.x);
        hi.y = fma(al, (double)pv.w, hi.y);
      }
      reinterpret_cast<double2*>(u64)[2 * k] = lo;
      reinterpret_cast<double2*>(u64)[2 * k + 1] = hi;
      reinterpret_cast<float4*>(d)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  for (int64_t i = t0; i < n; i += stride) {
    double v = u64[i] + (double)d[i];
    if (al != 0.0) v = fma(al, (double)pp[i], v);
    u64[i] = v;
    d[i] = 0.f;
  }
}

// After the FP64 residual of the flagged instances: new status from rel64,
// r = (float) r64, s = D^{-1} r, partials of rho and ||r||^2 into slot 0.  With
// upd == 2 (or at the start) the search direction restarts: p_old = 0 and a
// dummy rho in slot 1.
__global__ void k_ru_reset(CGArgs<float> a, int start) {
  __shared__ double red[64];
  const int b = blockIdx.z;
  const int mode = a.upd[b];
  if (!mode) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const TilePos tp = tile_pos(a.g, a.tiles_x, a.zc);
  const bool leader = tp.part == 0;
  InstState* st = a.st + b;
  const double rel = a.rel64[b];
  const int iters = start ? 0 : st->iters;
  int ns;
  if (rel < a.tol) ns = ST_CONVERGED;
  else if (!(rel == rel)) ns = ST_BREAKDOWN;
  else if (iters >= a.max_iters) ns = ST_MAX_ITERS;
  else ns = ST_ACTIVE;
  __syncthreads();  // every thread has read the old state before the leader writes
  if (leader && tid == 0) {
    if (start) {
      st->iters = 0;
      st->restarts = 0;
      st->relres0 = rel;
    }
    st->status = ns;
    st->relres = rel;
    if (ns != ST_ACTIVE) st->t_done = global_ns();
    if (a.alpha) a.alpha[b] = 0.0;  // the fold applied any pending update
    a.rr_ref[b] = (rel * a.fnorm[b]) * (rel * a.fnorm[b]);
    if (ns == ST_ACTIVE) atomicAdd(a.active, 1);
    if (ns == ST_ACTIVE && mode == 2 && !start) st->restarts += 1;
  }
  if (ns != ST_ACTIVE) return;
  const bool restart = start || mode == 2;
  const int64_t off = (int64_t)b * a.g.n;
  const float* cb = a.coef + (int64_t)b * a.g.ncls() * kCoefStride;
  const bool jac = a.precond != RBWS_PREC_NONE;
  const Column cl = make_column(a.g, tp.x0, tp.y0);
  const int64_t plane = (int64_t)a.g.nx * a.g.ny;
  float rho = 0.f, rr = 0.f;
  if (cl.own) {
    int zcls_cur = -1;
    float dinv = 1.f;
    for (int z = tp.z0; z < tp.z1; ++z) {
      const int zcl = a.g.cz[z];
      if (zcl != zcls_cur) {
        zcls_cur = zcl;
        dinv = cb[((int64_t)zcl * a.g.ncy * a.g.ncx + cl.xy) * kCoefStride + 7];
      }
      const int64_t idx = off + (int64_t)z * plane + cl.col;
      const float rv = (float)a.r64[idx];
      const float sv = jac ? dinv * rv : rv;
      a.r[idx] = rv;
      if (jac) a.s[idx] = sv;
      if (restart) a.p0[idx] = 0.f;
      rho = fmaf(rv, sv, rho);
      rr = fmaf(rv, rv, rr);
    }
  }
  // with MG, s and rho follow from a V-cycle after the reset
  double drho = a.precond == RBWS_PREC_MG ? 0.0 : (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (tid == 0) {
    a.rho_rr[(int64_t)b * a.P + tp.part] = make_double2(drho, drr);
    if (restart)
      a.rho_rr[((int64_t)a.B + b) * a.P + tp.part] = make_double2(tp.part == 0 ? 1.0 : 0.0, 0.0);
  }
}

// ---------------------------------------------------------------------------
// Persistent FP64 PCG: Algorithm 1 (preconditioner none or Jacobi) with the
// true-residual check and restarts of Algorithm 4, for one or several problems
// (grids of different sizes) in one cooperative launch.  Each CTA takes work items
// (tile, z-chunk, instance) of every task with a grid stride; the phases are the
// bodies of k_cg_init / k_cg_finalize / k_cg_a / k_cg_b, separated by grid
// barriers; the loop ends on the device when no instance of any task is active.
// Every barrier wait is bounded: when it runs out the CTA sets *err and every CTA
// leaves at its next barrier.
// ---------------------------------------------------------------------------
struct PTask {
  CGArgs<double> a;
  int ntiles;  // tiles_x * tiles_y
  int items;   // ntiles * nzc * B: work items of a stencil or update phase
};

struct PCtl {
  int* bar;               // [2]: arrivals, generation
  int* err;               // a barrier wait ran out
  long long wait_cycles;  // bound of each barrier wait (clock64 cycles)
  int max_restarts;
  int max_rounds;         // cap on iterations plus checks (a safety net)
};

__device__ bool grid_sync(const PCtl& c) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile int* vgen = c.bar + 1;
    const int gen = *vgen;  // read before arriving: the last arrival bumps it
    __threadfence();
    const int nb = (int)(gridDim.x * gridDim.y * gridDim.z);
    int ok = 1;
    if (atomicAdd(c.bar, 1) == nb - 1) {
      atomicExch(c.bar, 0);
      __threadfence();
      atomicAdd(c.bar + 1, 1);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > c.wait_cycles) {
          ok = 0;
          atomicExch(c.err, 1);
          break;
        }
      }
    }
    __threadfence();  // the other CTAs' writes of the phase are visible from here on
    s_ok = ok && *reinterpret_cast<volatile int*>(c.err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kPMaxTasks = 16;

// Loop-invariant state lives in shared memory, not registers: the phase bodies are
// inlined into the loop, and every register the loop keeps live costs resident CTAs.
struct PShared {
  PCtl c;
  int ntasks, total, total_fin, cur;
  int items[kPMaxTasks], ntiles[kPMaxTasks], nzc[kPMaxTasks], fin[kPMaxTasks];
  const PTask* tasks;
};

// Four CTAs per SM (64 registers, a few spilled): the bodies inlined into one loop need 80
// registers otherwise, and three resident CTAs left the FP64 pipe underfed (measured: 746
// against 667 ms for 256 solves at 64^3).
__global__ void __launch_bounds__(256, 4) k_pcg_persistent(const PTask* __restrict__ tasks, int ntasks, PCtl c) {
  // the arguments of the task being worked on, in shared memory: the phase bodies read
  // them at every plane, and global loads would miss L1 after each grid barrier
  __shared__ __align__(16) unsigned s_args[(sizeof(CGArgs<double>) + 3) / 4];
  __shared__ PShared S;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) {
    const int warps = (blockDim.x * blockDim.y) >> 5;
    S.c = c;
    S.tasks = tasks;
    S.ntasks = ntasks;
    S.total = S.total_fin = 0;
    S.cur = -1;
    for (int t = 0; t < ntasks; t++) {
      S.items[t] = tasks[t].items;
      S.ntiles[t] = tasks[t].ntiles;
      S.nzc[t] = tasks[t].a.nzc;
      S.fin[t] = (tasks[t].a.B + warps - 1) / warps;
      S.total += S.items[t];
      S.total_fin += S.fin[t];
    }
  }
  __syncthreads();
  auto args = [&](int t) -> const CGArgs<double>& {
    if (t != S.cur) {  // S.cur changes only between the two barriers below: uniform
      __syncthreads();
      const unsigned* src = reinterpret_cast<const unsigned*>(&S.tasks[t].a);
      for (int w = tid; w < (int)(sizeof(CGArgs<double>) / 4); w += blockDim.x * blockDim.y) s_args[w] = src[w];
      __syncthreads();
      if (tid == 0) S.cur = t;
      __syncthreads();
    }
    return *reinterpret_cast<const CGArgs<double>*>(s_args);
  };
  // item -> (task, virtual block)
  auto locate = [&](int item, int& t) -> VBlk {
    t = 0;
    while (item >= S.items[t]) item -= S.items[t++];
    const int nt = S.ntiles[t];
    return VBlk{item % nt, (item / nt) % S.nzc[t], item / (nt * S.nzc[t]), nt};
  };
  auto active = [&]() {
    int n = 0;
    for (int t = 0; t < S.ntasks; t++) n += *reinterpret_cast<volatile int*>(S.tasks[t].a.active);
    return n;
  };
  auto init = [&]() {
    for (int item = blockIdx.x; item < S.total; item += gridDim.x) {
      int t;
      const VBlk v = locate(item, t);
      const CGArgs<double>& a = args(t);
      __syncthreads();
      cg_init_body<double>(a, 0, v);
    }
  };
  auto finalize = [&](int mode) {
    for (int item = blockIdx.x; item < S.total_fin; item += gridDim.x) {
      int t = 0, rest = item;
      while (rest >= S.fin[t]) rest -= S.fin[t++];
      const CGArgs<double>& a = args(t);
      cg_finalize_body<double>(a, 0, mode, S.c.max_restarts, rest * ((blockDim.x * blockDim.y) >> 5) + (tid >> 5),
                               tid & 31);
    }
  };
  init();
  if (!grid_sync(S.c)) return;
  finalize(0);
  if (!grid_sync(S.c)) return;
  int parity = 0;
  for (int round = 0; round < S.c.max_rounds; round++) {
    if (active() == 0) {
      // every instance stopped: check the true residual f - A u, restart the failures
      init();
      if (!grid_sync(S.c)) return;
      finalize(1);
      if (!grid_sync(S.c)) return;
      if (active() == 0) return;
      parity = 0;
    }
    for (int item = blockIdx.x; item < S.total; item += gridDim.x) {
      int t;
      const VBlk v = locate(item, t);
      const CGArgs<double>& a = args(t);
      __syncthreads();
      cg_a_body<double>(a, parity, v);
    }
    if (!grid_sync(S.c)) return;
    for (int item = blockIdx.x; item < S.total; item += gridDim.x) {
      int t;
      const VBlk v = locate(item, t);
      const CGArgs<double>& a = args(t);
      __syncthreads();
      cg_b_body<double>(a, parity, v);
    }
    if (!grid_sync(S.c)) return;
    parity ^= 1;
  }
}

// ---------------------------------------------------------------------------
// y = A x in the mu-interleaved layout [nz][ny][nx][B] (instance fastest): a warp
// takes 32 consecutive instances of one node, so every load and store of x, y and of
// the coefficients is one 32-element run; the 6 neighbours come through L1/L2.  The
// coefficient table is interleaved too: cI[cls][8][B].  An alternative layout for the
// autotuner to time against the planar z-march (rbws_autotune_layout).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_coef_interleave(const T* __restrict__ c, int ncls, int B, T* __restrict__ cI) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ncls * kCoefStride * B) return;
  const int b = (int)(t % B), k = (int)((t / B) % kCoefStride), cls = (int)(t / ((int64_t)B * kCoefStride));
  cI[t] = c[((int64_t)b * ncls + cls) * kCoefStride + k];
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply_il(Geo g, int B, const T* __restrict__ cI, const T* __restrict__ x,
                                                 T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int groups = (B + 31) >> 5;
  const int64_t node = warp / groups;
  if (node >= g.n) return;
  const int b = (int)(warp % groups) * 32 + lane;
  if (b >= B) return;
  const int i = (int)(node % g.nx), j = (int)((node / g.nx) % g.ny), k = (int)(node / ((int64_t)g.nx * g.ny));
  const int cls = ((int)g.cz[k] * g.ncy + (int)g.cy[j]) * g.ncx + (int)g.cx[i];
  const T* cr = cI + (int64_t)cls * kCoefStride * B + b;
  const int64_t sx = B, sy = (int64_t)g.nx * B, sz = (int64_t)g.nx * g.ny * B;
  const T* xp = x + node * B + b;
  T v = cr[6 * B] * xp[0];
  if (i > 0) v = fma(cr[0], xp[-sx], v);
  if (i < g.nx - 1) v = fma(cr[1 * B], xp[sx], v);
  if (j > 0) v = fma(cr[2 * B], xp[-sy], v);
  if (j < g.ny - 1) v = fma(cr[3 * B], xp[sy], v);
  if (k > 0) v = fma(cr[4 * B], xp[-sz], v);
  if (k < g.nz - 1) v = fma(cr[5 * B], xp[sz], v);
  y[node * B + b] = v;
}

inline size_t plane_smem(Tile t, size_t elem) { return 3 * (size_t)(t.tx + 2) * (t.ty + 2) * elem; }

template <typename T>
dim3 cg_grid(const CGArgs<T>& a) {
  return dim3(a.tiles_x * a.tiles_y, a.nzc, a.B);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void launch_coef_tables(const Geo& g, const int8_t* kx, const int8_t* ky, const int8_t* kz, int bx,
                        int by, const uint8_t* segq, double sx, double sy, double sz, int Q,
                        const double* mu, int B, double* coef64, float* coef32, cudaStream_t s) {
  const int64_t total = (int64_t)g.ncls() * B;
  const int threads = 128;
  const int blocks = (int)((total + threads - 1) / threads);
  k_coef_tables<<<blocks, threads, 0, s>>>(g, kx, ky, kz, bx, by, segq, sx, sy, sz, Q, mu, B, coef64,
                                           coef32);
}

template <typename T>
void launch_apply(const Geo& g, Tile t, const T* coef, int B, const T* x, int64_t x_stride, T* y,
                  cudaStream_t s) {
  const int tiles_x = (g.nx + t.tx - 1) / t.tx, tiles_y = (g.ny + t.ty - 1) / t.ty;
  // z-chunks: enough CTAs to fill the GPU a few times over
  int nzc = 1;
  const int64_t per_chunk = (int64_t)tiles_x * tiles_y * B;
  while (per_chunk * nzc < 4 * 152 && nzc * 2 <= g.nz / 4) nzc *= 2;
  const int zc = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + zc - 1) / zc;
  dim3 grid(tiles_x * tiles_y, nzc, B), block(t.tx, t.ty);
  k_apply<T><<<grid, block, plane_smem(t, sizeof(T)), s>>>(g, tiles_x, zc, coef, x, x_stride, y);
}

void launch_residual64(const Geo& g, Tile t, int zc, const double* coef, int B, const double* f,
                       const double* u, double* r, double* rr_part, int P, const int* mask,
                       cudaStream_t s, int64_t f_stride) {
  const int tiles_x = (g.nx + t.tx - 1) / t.tx, tiles_y = (g.ny + t.ty - 1) / t.ty;
  const int nzc = (g.nz + zc - 1) / zc;
  (void)P;
  dim3 grid(tiles_x * tiles_y, nzc, B), block(t.tx, t.ty);
  k_residual64<<<grid, block, plane_smem(t, sizeof(double)), s>>>(g, tiles_x, zc, coef, f, f_stride, u, r,
                                                                  rr_part, tiles_x * tiles_y * nzc, mask);
}

void launch_residual64_ff(const Geo& g, Tile t, int zc, const double* coef, int B, const double* f,
                          const float* uh, const float* ul, double* u_out, double* r, double* rr_part, int P,
                          const int* mask, cudaStream_t s, int64_t f_stride) {
  const int tiles_x = (g.nx + t.tx - 1) / t.tx, tiles_y = (g.ny + t.ty - 1) / t.ty;
  const int nzc = (g.nz + zc - 1) / zc;
  (void)P;
  dim3 grid(tiles_x * tiles_y, nzc, B), block(t.tx, t.ty);
  k_residual64_ff<<<grid, block, plane_smem(t, sizeof(double)), s>>>(g, tiles_x, zc, coef, f, f_stride, uh, ul,
                                                                     u_out, r, rr_part, tiles_x * tiles_y * nzc,
                                                                     mask);
}

template <typename T>
void launch_cg_init(const CGArgs<T>& a, Tile t, int parity, int only_status, cudaStream_t s) {
  (void)only_status;
  k_cg_init<T><<<cg_grid(a), dim3(t.tx, t.ty), plane_smem(t, sizeof(T)), s>>>(a, parity);
}
template <typename T>
void launch_cg_a(const CGArgs<T>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_a<T><<<cg_grid(a), dim3(t.tx, t.ty), plane_smem(t, sizeof(T)), s>>>(a, parity);
}
template <typename T>
void launch_cg_b(const CGArgs<T>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_b<T><<<cg_grid(a), dim3(t.tx, t.ty), 0, s>>>(a, parity);
}
template <typename T>
void launch_cg_finalize(const CGArgs<T>& a, int parity, int mode, int max_restarts, cudaStream_t s) {
  const int warps = 4;
  k_cg_finalize<T><<<(a.B + warps - 1) / warps, 32 * warps, 0, s>>>(a, parity, mode, max_restarts);
}

int launch_pcg_persistent(const std::vector<CGArgs<double>>& args, Tile t, int* bar, int* err,
                          long long wait_cycles, int max_restarts, int max_rounds, void* d_tasks, cudaStream_t s) {
  const int ntasks = (int)args.size();
  if (ntasks < 1 || ntasks > kPMaxTasks) return -1;
  std::vector<PTask> h(ntasks);
  int total = 0;
  for (int i = 0; i < ntasks; i++) {
    h[i].a = args[i];
    h[i].ntiles = args[i].tiles_x * args[i].tiles_y;
    h[i].items = h[i].ntiles * args[i].nzc * args[i].B;
    total += h[i].items;
  }
  if (cudaMemcpyAsync(d_tasks, h.data(), sizeof(PTask) * ntasks, cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(int), s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return -1;
  const size_t smem = plane_smem(t, sizeof(double));
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent, t.tx * t.ty, smem) != cudaSuccess ||
      per_sm < 1)
    return -1;
  // every CTA must be resident at once (the grid barriers): at most the occupancy limit
  const int grid = std::max(1, std::min(total, sms * per_sm));
  PTask* tp = static_cast<PTask*>(d_tasks);
  PCtl c{bar, err, wait_cycles > 0 ? wait_cycles : 4000000000LL, max_restarts, max_rounds};
  void* params[] = {&tp, (void*)&ntasks, &c};
  if (cudaLaunchCooperativeKernel((const void*)k_pcg_persistent, dim3(grid), dim3(t.tx, t.ty), params, smem, s) !=
      cudaSuccess)
    return -1;
  return grid;
}

size_t pcg_persistent_task_bytes() { return sizeof(PTask); }

template <typename T>
void launch_apply_interleaved(const Geo& g, const T* coef, int B, T* coefI, const T* x, T* y, cudaStream_t s) {
  const int64_t nc = (int64_t)g.ncls() * kCoefStride * B;
  k_coef_interleave<T><<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(coef, g.ncls(), B, coefI);
  const int64_t warps = g.n * ((B + 31) / 32);
  k_apply_il<T><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(g, B, coefI, x, y);
}
template void launch_apply_interleaved<double>(const Geo&, const double*, int, double*, const double*, double*,
                                               cudaStream_t);
template void launch_apply_interleaved<float>(const Geo&, const float*, int, float*, const float*, float*,
                                              cudaStream_t);

void launch_ru_decide(const CGArgs<float>& a, cudaStream_t s) {
  k_ru_decide<<<(a.B + 3) / 4, 128, 0, s>>>(a);
}
namespace {
__global__ void k_loop_condition(cudaGraphConditionalHandle h, const int* __restrict__ counts, int* ctr, int cap) {
  const int blocks = ++*ctr;
  cudaGraphSetConditional(h, (counts[0] > 0 && counts[2] == 0 && blocks < cap) ? 1u : 0u);
}
}  // namespace

namespace {
__global__ void k_copy_words(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, size_t words) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < words; k += (size_t)gridDim.x * blockDim.x)
    dst[k] = src[k];
}
}  // namespace

void launch_copy_words(const uint32_t* src, uint32_t* dst, size_t words, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, 64);
  k_copy_words<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(src, dst, words);
}

void launch_loop_condition(cudaGraphConditionalHandle h, const int* counts, int* ctr, int cap, cudaStream_t s) {
  k_loop_condition<<<1, 1, 0, s>>>(h, counts, ctr, cap);
}

void launch_ru_fold(const CGArgs<float>& a, cudaStream_t s) {
  const int threads = 256;
  const int64_t work = (a.g.n & 3) == 0 ? a.g.n / 4 : a.g.n;  // the kernel falls back to one node per
                                                                  // thread (a grid-stride loop) if unaligned
  const int64_t blocks = std::min<int64_t>((work + threads - 1) / threads, 152 * 4);
  k_ru_fold<<<dim3((unsigned)blocks, a.B), threads, 0, s>>>(a);
}
void launch_ru_reset(const CGArgs<float>& a, Tile t, int start, cudaStream_t s) {
  k_ru_reset<<<cg_grid(a), dim3(t.tx, t.ty), 0, s>>>(a, start);
}

template <typename T>
void launch_precond_rho(const CGArgs<T>& a, Tile t, int slot, const int* mask, cudaStream_t s) {
  k_precond_rho<T><<<cg_grid(a), dim3(t.tx, t.ty), 0, s>>>(a, slot, mask);
}
template void launch_precond_rho<double>(const CGArgs<double>&, Tile, int, const int*, cudaStream_t);
template void launch_precond_rho<float>(const CGArgs<float>&, Tile, int, const int*, cudaStream_t);

void launch_msrb_apply(const CGArgs<double>& a, Tile t, int slot, cudaStream_t s) {
  k_msrb_residual<<<cg_grid(a), dim3(t.tx, t.ty), plane_smem(t, sizeof(double)), s>>>(a);
  k_msrb_project<<<dim3(a.proj_chunks, a.B), 256, 0, s>>>(a);
  k_msrb_reduce_solve<<<(a.B + 3) / 4, 128, 0, s>>>(a);
  k_msrb_lift<<<cg_grid(a), dim3(t.tx, t.ty), 0, s>>>(a, slot);
}

template void launch_apply<double>(const Geo&, Tile, const double*, int, const double*, int64_t,
                                   double*, cudaStream_t);
template void launch_apply<float>(const Geo&, Tile, const float*, int, const float*, int64_t, float*,
                                  cudaStream_t);
#define RBWS_INST(T)                                                                       \
  template void launch_cg_init<T>(const CGArgs<T>&, Tile, int, int, cudaStream_t);        \
  template void launch_cg_a<T>(const CGArgs<T>&, Tile, int, cudaStream_t);                \
  template void launch_cg_b<T>(const CGArgs<T>&, Tile, int, cudaStream_t);                \
  template void launch_cg_finalize<T>(const CGArgs<T>&, int, int, int, cudaStream_t);
RBWS_INST(double)
RBWS_INST(float)
#undef RBWS_INST

}  // namespace rbws
