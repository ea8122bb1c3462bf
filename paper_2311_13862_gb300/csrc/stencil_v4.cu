// stencil_v4.cu -- FP32 PCG phase kernels with 4 nodes per thread.
//
// The FP32 inner iterations are HBM-bound, and the one-node-per-thread
// kernels of stencil.cu leave too few bytes in flight on GB300 (a load is
// issued right before each plane's barrier and waited on at once).  Here a
// thread owns 4 consecutive x nodes (16-byte loads and stores; requires
// nx % 4 == 0), and the stencil phase prefetches the next plane's loads into
// registers before the barrier of the current plane, so a plane's memory
// latency overlaps the previous plane's arithmetic.
//
// Tiles: TXT threads x 4 nodes in x (TXT in {4, 8, 16, 32}), TY rows, 256
// threads or fewer; each CTA marches a chunk of zc planes.  The partial-sum
// decomposition (one partial per CTA) is shared by all kernels of a solve
// that use these tiles: k_cg_a_v4, k_cg_b_v4, k_ru_reset_v4.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rbws {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_down(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  a = warp_sum_down(a);
  b = warp_sum_down(b);
  __syncthreads();
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

__device__ __forceinline__ double2 sum_partials2(const double2* part, int P, int lane) {
  double x = 0.0, y = 0.0;
  for (int c = lane; c < P; c += 32) {
    double2 v = part[c];
    x += v.x;
    y += v.y;
  }
  return make_double2(warp_sum_down(x), warp_sum_down(y));
}
__device__ __forceinline__ double sum_partials(const double* part, int P, int lane) {
  double s = 0.0;
  for (int c = lane; c < P; c += 32) s += part[c];
  return warp_sum_down(s);
}

struct Pos4 {
  int x0, y0, z0, z1, part;  // tile origin (nodes), z range, partial index
  int i, j;                  // first node of this thread
  bool own;
};

__device__ __forceinline__ Pos4 pos4(const Geo& g, int tiles_x, int zc) {
  Pos4 p;
  const int tile = blockIdx.x;
  p.x0 = (tile % tiles_x) * (blockDim.x * 4);
  p.y0 = (tile / tiles_x) * blockDim.y;
  p.z0 = blockIdx.y * zc;
  p.z1 = min(g.nz, p.z0 + zc);
  p.part = blockIdx.y * gridDim.x + blockIdx.x;
  p.i = p.x0 + 4 * (int)threadIdx.x;
  p.j = p.y0 + (int)threadIdx.y;
  p.own = p.i < g.nx && p.j < g.ny;  // nx % 4 == 0: all 4 nodes in range together
  return p;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float f4(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Stencil coefficients (-kW, -kE, -kS, -kN, -kD, -kU, D) of the thread's 4
// nodes for z class zcl (1/D is not needed by the stencil phase).
__device__ __forceinline__ void load_coef4(const Geo& g, const float* cb, int zcl, int i, int j, float c[4][7]) {
  const int yc = (int)g.cy[j];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
    const float4 a = ld4(row);
    const float2 b = *reinterpret_cast<const float2*>(row + 4);
    c[e][0] = a.x; c[e][1] = a.y; c[e][2] = a.z; c[e][3] = a.w;
    c[e][4] = b.x; c[e][5] = b.y; c[e][6] = row[6];
  }
}

// Shared-memory plane: rows -1..TY, row pitch PW floats; node x (tile-local,
// -1..TXN) lives at column 4 + x, so the 4-node groups are 16-byte aligned.
struct Plane {
  int PW, PS;
  __device__ __forceinline__ int at(int x, int y) const { return (y + 1) * PW + 4 + x; }
};

// Halo duty of a thread in the v4 tiles: y-halo rows by 4-node groups
// (2*blockDim.x threads), then x-halo columns by single nodes (2*TY threads).
struct Halo4 {
  int kind;      // 0 none, 1 y-row group (4 nodes), 2 x-column node
  int hx, hy;    // tile-local position
  bool in;       // inside the domain
  int64_t col;   // gj*nx + gi
  int slot;      // shared-memory offset
};

__device__ __forceinline__ Halo4 halo4(const Geo& g, const Pos4& ps, const Plane& pl, int tid) {
  Halo4 h{0, 0, 0, false, 0, 0};
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  const int nyh = 2 * blockDim.x;
  if (tid < nyh) {
    h.kind = 1;
    h.hx = 4 * (tid % blockDim.x);
    h.hy = tid < (int)blockDim.x ? -1 : TY;
  } else if (tid < nyh + 2 * TY) {
    h.kind = 2;
    const int t = tid - nyh;
    h.hx = t < TY ? -1 : TXN;
    h.hy = t < TY ? t : t - TY;
  }
  const int gi = ps.x0 + h.hx, gj = ps.y0 + h.hy;
  h.in = h.kind != 0 && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
  h.col = (int64_t)gj * g.nx + gi;
  h.slot = pl.at(h.hx, h.hy);
  return h;
}

// y = A x for the thread's 4 nodes from the staged plane P (x, y neighbours)
// and the column registers xm (z-1), xc (z), xp (z+1).
__device__ __forceinline__ void stencil4(const float* P, const Plane& pl, int oslot, const float c[4][7],
                                         float4 xm, float4 xc, float4 xp, float y[4]) {
  const float left = P[oslot - 1], right = P[oslot + 4];
  const float4 sth = ld4(P + oslot - pl.PW), nth = ld4(P + oslot + pl.PW);
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const float xce = f4(xc, e);
    const float xw = e == 0 ? left : f4(xc, e - 1);
    const float xe = e == 3 ? right : f4(xc, e + 1);
    float v = c[e][6] * xce;
    v = fmaf(c[e][0], xw, v);
    v = fmaf(c[e][1], xe, v);
    v = fmaf(c[e][2], f4(sth, e), v);
    v = fmaf(c[e][3], f4(nth, e), v);
    v = fmaf(c[e][4], f4(xm, e), v);
    v = fmaf(c[e][5], f4(xp, e), v);
    y[e] = v;
  }
}

// 1/D of node (i, j) in z class zcl (from the coefficient table).
__device__ __forceinline__ float dinv_at(const Geo& g, const float* cb, int zcl, int i, int j) {
  return cb[(((int64_t)zcl * g.ncy + g.cy[j]) * g.ncx + g.cx[i]) * kCoefStride + 7];
}

}  // namespace

// ---------------------------------------------------------------------------
// Phase A: beta = rho_k / rho_{k-1}; p = s + beta p_old (halo recomputed);
// q = A p; partial p.q.  Same scalars and stopping logic as k_cg_a.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_cg_a_v4(CGArgs<float> a, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ double s_beta;
  __shared__ int s_run;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
  if (tid < 32) {
    InstState* st = a.st + b;
    const int status = st->status;
    double2 cur = make_double2(0.0, 0.0);
    double prev = 0.0;
    if (status == ST_ACTIVE) {
      cur = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, tid);
      prev = sum_partials2(a.rho_rr + ((int64_t)(parity ^ 1) * a.B + b) * a.P, a.P, tid).x;
    }
    if (tid == 0) {
      int run = 0;
      if (status == ST_ACTIVE) {
        const double rel = sqrt(cur.y) / a.fnorm[b];
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
  const float beta = (float)s_beta;
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const float* sb = (a.precond != RBWS_PREC_NONE ? a.s : a.r) + off;
  const float* pold = (parity ? a.p1 : a.p0) + off;
  float* pnew = (parity ? a.p0 : a.p1) + off;
  float* qb = a.q + off;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  Plane pl{TXN + 8, 0};
  pl.PS = pl.PW * (TY + 2);
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  // Halo assignment: y-halo rows by 4-node groups (2*blockDim.x threads),
  // then x-halo columns by single nodes (2*TY threads).
  const int nyh = 2 * blockDim.x;
  int hx = 0, hy = 0, hkind = 0;  // 0 none, 1 y-row group (4 nodes), 2 x-column node
  if (tid < nyh) {
    hkind = 1;
    hx = 4 * (tid % blockDim.x);
    hy = tid < (int)blockDim.x ? -1 : TY;
  } else if (tid < nyh + 2 * TY) {
    hkind = 2;
    const int t = tid - nyh;
    hx = t < TY ? -1 : TXN;
    hy = t < TY ? t : t - TY;
  }
  const int gi = ps.x0 + hx, gj = ps.y0 + hy;
  const bool hin = hkind != 0 && gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
  const int64_t hcol = (int64_t)gj * g.nx + gi;
  const int hslot = pl.at(hx, hy), oslot = pl.at(lx, ly);

  // register prefetch of (s, p_old) for the own group and the halo element(s)
  float4 s_own, p_own, s_h, p_h;
  auto fetch = [&](int z) {
    const bool zin = z >= 0 && z < g.nz;
    s_own = p_own = make_float4(0.f, 0.f, 0.f, 0.f);
    s_h = p_h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zin && ps.own) {
      s_own = ld4(sb + z * plane + col);
      p_own = ld4(pold + z * plane + col);
    }
    if (zin && hin) {
      if (hkind == 1) {
        s_h = ld4(sb + z * plane + hcol);
        p_h = ld4(pold + z * plane + hcol);
      } else {
        s_h.x = sb[z * plane + hcol];
        p_h.x = pold[z * plane + hcol];
      }
    }
  };
  // p_new of the fetched plane into a smem slot; returns the own group
  auto commit = [&](float* P) -> float4 {
    const float4 v = fma4(beta, p_own, s_own);
    st4(P + oslot, v);
    if (hkind == 1) st4(P + hslot, fma4(beta, p_h, s_h));
    else if (hkind == 2) P[hslot] = fmaf(beta, p_h.x, s_h.x);
    return v;
  };

  float c[4][7];
  int zcls_cur = -1;
  const int z0 = ps.z0, z1 = ps.z1;
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
  if (z0 > 0 && ps.own) xm = fma4(beta, ld4(pold + (z0 - 1) * plane + col), ld4(sb + (z0 - 1) * plane + col));
  fetch(z0);
  float4 xc = commit(sm + (z0 % 3) * pl.PS);
  fetch(z0 + 1);
  float gam = 0.f;
  for (int z = z0; z < z1; ++z) {
    const float4 xp = commit(sm + ((z + 1) % 3) * pl.PS);  // plane z+1 (zeros past nz)
    fetch(z + 2);                                          // in flight during plane z
    __syncthreads();
    const float* P = sm + (z % 3) * pl.PS;
    const int zcl = g.cz[z];
    if (zcl != zcls_cur && ps.own) {
      zcls_cur = zcl;
      load_coef4(g, cb, zcl, ps.i, ps.j, c);
    }
    if (ps.own) {
      const float left = P[oslot - 1], right = P[oslot + 4];
      const float4 sth = ld4(P + oslot - pl.PW), nth = ld4(P + oslot + pl.PW);
      float y[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const float xce = f4(xc, e);
        const float xw = e == 0 ? left : f4(xc, e - 1);
        const float xe = e == 3 ? right : f4(xc, e + 1);
        float v = c[e][6] * xce;
        v = fmaf(c[e][0], xw, v);
        v = fmaf(c[e][1], xe, v);
        v = fmaf(c[e][2], f4(sth, e), v);
        v = fmaf(c[e][3], f4(nth, e), v);
        v = fmaf(c[e][4], f4(xm, e), v);
        v = fmaf(c[e][5], f4(xp, e), v);
        y[e] = v;
        gam = fmaf(xce, v, gam);
      }
      st4(pnew + z * plane + col, xc);
      st4(qb + z * plane + col, make_float4(y[0], y[1], y[2], y[3]));
    }
    xm = xc;
    xc = xp;
  }
  double dg = (double)gam, dummy = 0.0;
  block_sum2(dg, dummy, red);
  if (tid == 0) a.gam[(int64_t)b * a.P + ps.part] = dg;
}

// ---------------------------------------------------------------------------
// Phase B: alpha = rho / gamma; u += alpha p; r -= alpha q; s = D^{-1} r;
// partials of rho = r.s and r.r.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_cg_b_v4(CGArgs<float> a, int parity) {
  __shared__ double red[64];
  __shared__ double s_alpha;
  __shared__ int s_run;
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
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
  const float alpha = (float)s_alpha;
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const float* pn = (parity ? a.p0 : a.p1) + off;
  const float* qb = a.q + off;
  float* ub = a.u + off;
  float* rb = a.r + off;
  float* sb = a.s + off;
  const bool mg = a.precond == RBWS_PREC_MG;  // the V-cycle writes s and rho after this phase
  const bool jac = a.precond != RBWS_PREC_NONE && !mg;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  float rho = 0.f, rr = 0.f;
  if (ps.own) {
    int zcls_cur = -1;
    float dinv[4] = {1.f, 1.f, 1.f, 1.f};
    const int yc = (int)g.cy[ps.j];
    // two planes per step: all eight loads are issued before any use
    for (int z = ps.z0; z < ps.z1; z += 2) {
      const bool two = z + 1 < ps.z1;
      const int64_t i0 = z * plane + col, i1 = i0 + plane;
      const float4 p0v = ld4(pn + i0), q0v = ld4(qb + i0), u0v = ld4(ub + i0), r0v = ld4(rb + i0);
      float4 p1v = p0v, q1v = q0v, u1v = u0v, r1v = r0v;
      if (two) {
        p1v = ld4(pn + i1);
        q1v = ld4(qb + i1);
        u1v = ld4(ub + i1);
        r1v = ld4(rb + i1);
      }
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (h == 1 && !two) break;
        const int zz = z + h;
        const int zcl = g.cz[zz];
        if (zcl != zcls_cur) {
          zcls_cur = zcl;
#pragma unroll
          for (int e = 0; e < 4; e++)
            dinv[e] = cb[(((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[ps.i + e]) * kCoefStride + 7];
        }
        const float4 pv = h ? p1v : p0v, qv = h ? q1v : q0v, uv = h ? u1v : u0v, rv0 = h ? r1v : r0v;
        const float4 uo = fma4(alpha, pv, uv);
        const float4 ro = fma4(-alpha, qv, rv0);
        float4 so = ro;
        if (jac) so = make_float4(dinv[0] * ro.x, dinv[1] * ro.y, dinv[2] * ro.z, dinv[3] * ro.w);
        const int64_t ii = h ? i1 : i0;
        st4(ub + ii, uo);
        st4(rb + ii, ro);
        if (jac) st4(sb + ii, so);
        rho = fmaf(ro.x, so.x, rho);
        rho = fmaf(ro.y, so.y, rho);
        rho = fmaf(ro.z, so.z, rho);
        rho = fmaf(ro.w, so.w, rho);
        rr = fmaf(ro.x, ro.x, rr);
        rr = fmaf(ro.y, ro.y, rr);
        rr = fmaf(ro.z, ro.z, rr);
        rr = fmaf(ro.w, ro.w, rr);
      }
    }
  }
  double drho = mg ? 0.0 : (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (tid == 0) a.rho_rr[((int64_t)(parity ^ 1) * a.B + b) * a.P + ps.part] = make_double2(drho, drr);
}

// Reliable-update reset with the v4 tiles (see k_ru_reset in stencil.cu).
__global__ void __launch_bounds__(256) k_ru_reset_v4(CGArgs<float> a, int start) {
  __shared__ double red[64];
  const int b = blockIdx.z;
  const int mode = a.upd[b];
  if (!mode) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
  InstState* st = a.st + b;
  const double rel = a.rel64[b];
  const int iters = start ? 0 : st->iters;
  int ns;
  if (rel < a.tol) ns = ST_CONVERGED;
  else if (!(rel == rel)) ns = ST_BREAKDOWN;
  else if (iters >= a.max_iters) ns = ST_MAX_ITERS;
  else ns = ST_ACTIVE;
  __syncthreads();
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
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const bool mg = a.precond == RBWS_PREC_MG;  // s and rho follow from a V-cycle after the reset
  const bool jac = a.precond != RBWS_PREC_NONE;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  float rho = 0.f, rr = 0.f;
  if (ps.own) {
    int zcls_cur = -1;
    float dinv[4] = {1.f, 1.f, 1.f, 1.f};
    const int yc = (int)g.cy[ps.j];
    for (int z = ps.z0; z < ps.z1; ++z) {
      const int zcl = g.cz[z];
      if (zcl != zcls_cur) {
        zcls_cur = zcl;
#pragma unroll
        for (int e = 0; e < 4; e++)
          dinv[e] = cb[(((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[ps.i + e]) * kCoefStride + 7];
      }
      const int64_t idx = off + z * plane + col;
      const double2 ra = *reinterpret_cast<const double2*>(a.r64 + idx);
      const double2 rb2 = *reinterpret_cast<const double2*>(a.r64 + idx + 2);
      const float4 rv = make_float4((float)ra.x, (float)ra.y, (float)rb2.x, (float)rb2.y);
      float4 sv = rv;
      if (jac) sv = make_float4(dinv[0] * rv.x, dinv[1] * rv.y, dinv[2] * rv.z, dinv[3] * rv.w);
      st4(a.r + idx, rv);
      if (!mg) st4(a.s + idx, sv);  // s = r without a preconditioner (the s-form schedule reads s)
      if (restart) st4(a.p0 + idx, make_float4(0.f, 0.f, 0.f, 0.f));
      rho = fmaf(rv.x, sv.x, fmaf(rv.y, sv.y, fmaf(rv.z, sv.z, fmaf(rv.w, sv.w, rho))));
      rr = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, rr))));
    }
  }
  double drho = mg ? 0.0 : (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (tid == 0) {
    a.rho_rr[(int64_t)b * a.P + ps.part] = make_double2(drho, drr);
    if (restart)
      a.rho_rr[((int64_t)a.B + b) * a.P + ps.part] = make_double2(ps.part == 0 ? 1.0 : 0.0, 0.0);
  }
}

// Partials of rho = r.s after the FP32 V-cycle wrote s, with the v4 tiling of
// the update phase (slot `slot`); instances with mask[b] == 0 are skipped.
__global__ void __launch_bounds__(256) k_precond_rho_v4(CGArgs<float> a, int slot, const int* mask) {
  __shared__ double red[64];
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (mask && !mask[b])) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const int64_t off = (int64_t)b * a.g.n;
  const int64_t plane = (int64_t)a.g.nx * a.g.ny;
  const int64_t col = (int64_t)ps.j * a.g.nx + ps.i;
  float rho = 0.f;
  if (ps.own)
    for (int z = ps.z0; z < ps.z1; ++z) {
      const int64_t idx = off + z * plane + col;
      const float4 rv = ld4(a.r + idx), sv = ld4(a.s + idx);
      rho = fmaf(rv.x, sv.x, fmaf(rv.y, sv.y, fmaf(rv.z, sv.z, fmaf(rv.w, sv.w, rho))));
    }
  double drho = (double)rho, dummy = 0.0;
  block_sum2(drho, dummy, red);
  if (tid == 0) a.rho_rr[((int64_t)slot * a.B + b) * a.P + ps.part].x = drho;
}

__global__ void k_tune_prep(CGArgs<float> a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nP = (int64_t)a.B * a.P;
  if (i < a.B) {
    a.st[i].status = ST_ACTIVE;
    a.st[i].iters = 0;
    if (a.alpha) a.alpha[i] = a.alpha[a.B + i] = 0.0;
  }
  if (i < nP) {
    a.rho_rr[i] = make_double2(1.0, 1e300);
    a.rho_rr[nP + i] = make_double2(1.0, 1e300);
    a.gam[i] = 1.0;
  }
}

void launch_tune_prep(const CGArgs<float>& a, cudaStream_t s) {
  const int64_t n = std::max<int64_t>(a.B, (int64_t)a.B * a.P);
  k_tune_prep<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
}

size_t v4_plane_smem(Tile t) { return sizeof(float) * 3 * (size_t)(4 * t.tx + 8) * (t.ty + 2); }

// ---------------------------------------------------------------------------
// 32-byte schedule.  Phase A of iteration k (parity = k % 2):
//   u += alpha_{k-1} p_{k-1}            (the update phase B deferred)
//   p_k = D^{-1} r_k + beta_k p_{k-1}   (D^{-1} r formed on the fly, halo too)
//   partial gamma_k = p_k . A p_k       (A p_k not stored)
// reads r, p_old (+halo), u; writes p, u: 20 B per DoF.
// Phase B: alpha_k = rho_k / gamma_k; r -= alpha_k A p_k (A p_k recomputed from
// the staged p_k); partials rho_{k+1} = r.D^{-1}r, ||r||^2; reads r, p (+halo),
// writes r: 12 B per DoF.  alpha_k goes to a.alpha[parity ^ 1][b]; an instance
// that stops in phase A keeps its pending update, and records its parity in
// InstState::pad for the reliable-update fold.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3) k_cg_a32_v4(CGArgs<float> a, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ double s_beta, s_alpha;
  __shared__ int s_run;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
  if (tid < 32) {
    InstState* st = a.st + b;
    const int status = st->status;
    double2 cur = make_double2(0.0, 0.0);
    double prev = 0.0;
    if (status == ST_ACTIVE) {
      cur = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, tid);
      prev = sum_partials2(a.rho_rr + ((int64_t)(parity ^ 1) * a.B + b) * a.P, a.P, tid).x;
    }
    if (tid == 0) {
      int run = 0;
      if (status == ST_ACTIVE) {
        const double rel = sqrt(cur.y) / a.fnorm[b];
        if (rel < a.tol || st->iters >= a.max_iters || !(rel == rel)) {
          if (leader) {
            st->status = rel < a.tol ? (a.ru ? ST_PAUSED : ST_CONVERGED)
                                     : ((rel == rel) ? ST_MAX_ITERS : ST_BREAKDOWN);
            st->relres = rel;
            st->pad = parity;  // the update alpha[parity] * p_old is still pending
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else {
          run = 1;
          s_beta = cur.x / prev;
          s_alpha = a.alpha[(int64_t)parity * a.B + b];
        }
      }
      s_run = run;
    }
  }
  __syncthreads();
  if (!s_run) return;
  const float beta = (float)s_beta, alpha = (float)s_alpha;
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const bool jac = a.precond != RBWS_PREC_NONE;
  const float* rb = a.r + off;
  const float* pold = (parity ? a.p1 : a.p0) + off;
  float* pnew = (parity ? a.p0 : a.p1) + off;
  float* ub = a.u + off;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  Plane pl{TXN + 8, 0};
  pl.PS = pl.PW * (TY + 2);
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  const int oslot = pl.at(4 * (int)threadIdx.x, (int)threadIdx.y);
  const Halo4 h = halo4(g, ps, pl, tid);
  const int hi = ps.x0 + h.hx, hj = ps.y0 + h.hy;

  float c[4][7];
  int zcls_cur = -1;
  auto coefs = [&](int z) {
    const int zcl = g.cz[z];
    if (zcl != zcls_cur && ps.own) {
      zcls_cur = zcl;
      load_coef4(g, cb, zcl, ps.i, ps.j, c);
    }
  };
  float4 r_own, p_own, r_h, p_h;
  auto fetch = [&](int z) {
    const bool zin = z >= 0 && z < g.nz;
    r_own = p_own = r_h = p_h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zin && ps.own) {
      r_own = ld4(rb + z * plane + col);
      p_own = ld4(pold + z * plane + col);
    }
    if (zin && h.in) {
      if (h.kind == 1) {
        r_h = ld4(rb + z * plane + h.col);
        p_h = ld4(pold + z * plane + h.col);
      } else {
        r_h.x = rb[z * plane + h.col];
        p_h.x = pold[z * plane + h.col];
      }
    }
  };
  // p of plane z into a smem slot (needs the own 1/D of plane z); returns the own group
  auto commit = [&](float* P, int z) -> float4 {
    float4 sv = r_own;
    if (jac && z < g.nz && ps.own) {
      // own nodes: 1/D of plane z (the cached rows may belong to another z class)
      const int zcl = g.cz[z];
      sv = make_float4(r_own.x * dinv_at(g, cb, zcl, ps.i, ps.j), r_own.y * dinv_at(g, cb, zcl, ps.i + 1, ps.j),
                       r_own.z * dinv_at(g, cb, zcl, ps.i + 2, ps.j), r_own.w * dinv_at(g, cb, zcl, ps.i + 3, ps.j));
    }
    const float4 v = fma4(beta, p_own, sv);
    st4(P + oslot, v);
    if (h.kind != 0) {
      float4 sh = r_h;
      if (jac && h.in && z < g.nz) {
        const int zcl = g.cz[z];
        if (h.kind == 1)
          sh = make_float4(r_h.x * dinv_at(g, cb, zcl, hi, hj), r_h.y * dinv_at(g, cb, zcl, hi + 1, hj),
                           r_h.z * dinv_at(g, cb, zcl, hi + 2, hj), r_h.w * dinv_at(g, cb, zcl, hi + 3, hj));
        else
          sh.x = r_h.x * dinv_at(g, cb, zcl, hi, hj);
      }
      if (h.kind == 1) st4(P + h.slot, fma4(beta, p_h, sh));
      else P[h.slot] = fmaf(beta, p_h.x, sh.x);
    }
    return v;
  };

  const int z0 = ps.z0, z1 = ps.z1;
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
  if (z0 > 0 && ps.own) {
    fetch(z0 - 1);
    float4 sv = r_own;
    if (jac) {
      const int zcl = g.cz[z0 - 1];
      sv = make_float4(r_own.x * dinv_at(g, cb, zcl, ps.i, ps.j), r_own.y * dinv_at(g, cb, zcl, ps.i + 1, ps.j),
                       r_own.z * dinv_at(g, cb, zcl, ps.i + 2, ps.j), r_own.w * dinv_at(g, cb, zcl, ps.i + 3, ps.j));
    }
    xm = fma4(beta, p_own, sv);
  }
  fetch(z0);
  float4 xc = commit(sm + (z0 % 3) * pl.PS, z0);
  fetch(z0 + 1);
  float gam = 0.f;
  for (int z = z0; z < z1; ++z) {
    // own u and p_old of plane z for the deferred update (in flight over the barrier)
    float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f), po4 = u4;
    if (ps.own) {
      u4 = ld4(ub + z * plane + col);
      po4 = ld4(pold + z * plane + col);
    }
    const float4 xp = commit(sm + ((z + 1) % 3) * pl.PS, z + 1);
    fetch(z + 2);
    __syncthreads();
    coefs(z);
    if (ps.own) {
      float y[4];
      stencil4(sm + (z % 3) * pl.PS, pl, oslot, c, xm, xc, xp, y);
      gam = fmaf(xc.x, y[0], fmaf(xc.y, y[1], fmaf(xc.z, y[2], fmaf(xc.w, y[3], gam))));
      st4(pnew + z * plane + col, xc);
      st4(ub + z * plane + col, fma4(alpha, po4, u4));
    }
    xm = xc;
    xc = xp;
  }
  double dg = (double)gam, dummy = 0.0;
  block_sum2(dg, dummy, red);
  if (tid == 0) a.gam[(int64_t)b * a.P + ps.part] = dg;
}

__global__ void __launch_bounds__(256, 3) k_cg_b32_v4(CGArgs<float> a, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ double s_alpha;
  __shared__ int s_run;
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
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
            st->pad = parity ^ 1;  // no valid alpha_k: nothing pending
            a.alpha[(int64_t)(parity ^ 1) * a.B + b] = 0.0;
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else {
          run = 1;
          s_alpha = alpha;
          if (leader) {
            st->iters += 1;
            a.alpha[(int64_t)(parity ^ 1) * a.B + b] = alpha;
          }
        }
      }
      s_run = run;
    }
  }
  __syncthreads();
  if (!s_run) return;
  const float alpha = (float)s_alpha;
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const bool jac = a.precond != RBWS_PREC_NONE;
  const float* pb = (parity ? a.p0 : a.p1) + off;
  float* rb = a.r + off;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  Plane pl{TXN + 8, 0};
  pl.PS = pl.PW * (TY + 2);
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  const int oslot = pl.at(4 * (int)threadIdx.x, (int)threadIdx.y);
  const Halo4 h = halo4(g, ps, pl, tid);

  float c[4][7];
  float dinv[4] = {1.f, 1.f, 1.f, 1.f};
  int zcls_cur = -1;
  float4 p_own, p_h;
  auto fetch = [&](int z) {
    const bool zin = z >= 0 && z < g.nz;
    p_own = p_h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zin && ps.own) p_own = ld4(pb + z * plane + col);
    if (zin && h.in) {
      if (h.kind == 1) p_h = ld4(pb + z * plane + h.col);
      else p_h.x = pb[z * plane + h.col];
    }
  };
  auto commit = [&](float* P) -> float4 {
    st4(P + oslot, p_own);
    if (h.kind == 1) st4(P + h.slot, p_h);
    else if (h.kind == 2) P[h.slot] = p_h.x;
    return p_own;
  };
  const int z0 = ps.z0, z1 = ps.z1;
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
  if (z0 > 0 && ps.own) xm = ld4(pb + (z0 - 1) * plane + col);
  fetch(z0);
  float4 xc = commit(sm + (z0 % 3) * pl.PS);
  fetch(z0 + 1);
  float rho = 0.f, rr = 0.f;
  for (int z = z0; z < z1; ++z) {
    float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ps.own) r4 = ld4(rb + z * plane + col);  // in flight over the barrier
    const float4 xp = commit(sm + ((z + 1) % 3) * pl.PS);
    fetch(z + 2);
    __syncthreads();
    const int zcl = g.cz[z];
    if (zcl != zcls_cur && ps.own) {
      zcls_cur = zcl;
      load_coef4(g, cb, zcl, ps.i, ps.j, c);
#pragma unroll
      for (int e = 0; e < 4; e++) dinv[e] = dinv_at(g, cb, zcl, ps.i + e, ps.j);
    }
    if (ps.own) {
      float y[4];
      stencil4(sm + (z % 3) * pl.PS, pl, oslot, c, xm, xc, xp, y);
      const float4 rn = make_float4(fmaf(-alpha, y[0], r4.x), fmaf(-alpha, y[1], r4.y),
                                    fmaf(-alpha, y[2], r4.z), fmaf(-alpha, y[3], r4.w));
      st4(rb + z * plane + col, rn);
      const float4 sv = jac ? make_float4(dinv[0] * rn.x, dinv[1] * rn.y, dinv[2] * rn.z, dinv[3] * rn.w) : rn;
      rho = fmaf(rn.x, sv.x, fmaf(rn.y, sv.y, fmaf(rn.z, sv.z, fmaf(rn.w, sv.w, rho))));
      rr = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, fmaf(rn.z, rn.z, fmaf(rn.w, rn.w, rr))));
    }
    xm = xc;
    xc = xp;
  }
  double drho = (double)rho, drr = (double)rr;
  block_sum2(drho, drr, red);
  if (tid == 0) a.rho_rr[((int64_t)(parity ^ 1) * a.B + b) * a.P + ps.part] = make_double2(drho, drr);
}

void launch_cg_a32_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_a32_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), v4_plane_smem(t), s>>>(a, parity);
}
void launch_cg_b32_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_b32_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), v4_plane_smem(t), s>>>(a, parity);
}

// ---------------------------------------------------------------------------
// Fine-level multigrid steps (Algorithm 2 on the finest grid) with the v4
// tiles and the iteration's tiling, FP32.  The staged field x is
//   kStage 0: xin;   kStage 1: omega D^-1 rhs (the first smoothing step from
//   zero, formed where it is staged);
// and the output is
//   kOut 0: out = x + omega D^-1 (rhs - A x)      (a damped Jacobi step)
//   kOut 1: out = rhs - A x                        (the residual)
//   kOut 2: as 0, plus the partials of rho = rhs . out into slot `slot` of
//           the iteration's partials (out is the preconditioned residual s).
// ---------------------------------------------------------------------------
template <int kStage, int kOut>
__global__ void __launch_bounds__(256, 3) k_mg_fine_v4(CGArgs<float> a, MGFineArgs m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (m.mask && !m.mask[b])) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Pos4 ps = pos4(a.g, a.tiles_x, a.zc);
  const Geo& g = a.g;
  const int64_t off = (int64_t)b * g.n;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const float* rhs = m.rhs + off;
  const float* xin = kStage == 1 ? nullptr : m.xin + off;
  float* out = m.out + off;
  const float omega = m.omega;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  Plane pl{TXN + 8, 0};
  pl.PS = pl.PW * (TY + 2);
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  const Halo4 h = halo4(g, ps, pl, tid);
  const int oslot = pl.at(4 * (int)threadIdx.x, (int)threadIdx.y);
  const int gi = ps.x0 + h.hx, gj = ps.y0 + h.hy;

  // raw loads of plane z (register prefetch): the array the staged field is
  // formed from, for the own group and the halo element(s)
  const float* src = kStage == 1 ? rhs : xin;
  float4 v_own, v_h;
  auto fetch = [&](int z) {
    v_own = v_h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (z < 0 || z >= g.nz) return;
    if (ps.own) v_own = ld4(src + z * plane + col);
    if (h.in) {
      if (h.kind == 1) v_h = ld4(src + z * plane + h.col);
      else v_h.x = src[z * plane + h.col];
    }
  };
  // staged values from raw ones: omega D^-1 raw (kStage 1; 1/D cached per z
  // class for the own group and the halo element)
  int own_zc = -1, h_zc = -1;
  float own_di[4] = {0.f, 0.f, 0.f, 0.f}, h_di[4] = {0.f, 0.f, 0.f, 0.f};
  auto commit = [&](float* P, int z) -> float4 {
    const bool zin = z >= 0 && z < g.nz;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zin && ps.own) {
      if (kStage == 1) {
        const int zc = g.cz[z];
        if (zc != own_zc) {
          own_zc = zc;
#pragma unroll
          for (int e = 0; e < 4; e++) own_di[e] = omega * dinv_at(g, cb, zc, ps.i + e, ps.j);
        }
        v = make_float4(own_di[0] * v_own.x, own_di[1] * v_own.y, own_di[2] * v_own.z, own_di[3] * v_own.w);
      } else {
        v = v_own;
      }
    }
    st4(P + oslot, v);
    if (h.kind != 0) {
      float4 hv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (zin && h.in) {
        const int nh = h.kind == 1 ? 4 : 1;
        if (kStage == 1) {
          const int zc = g.cz[z];
          if (zc != h_zc) {
            h_zc = zc;
#pragma unroll
            for (int e = 0; e < 4; e++)
              if (e < nh) h_di[e] = omega * dinv_at(g, cb, zc, gi + e, gj);
          }
          hv = make_float4(h_di[0] * v_h.x, h_di[1] * v_h.y, h_di[2] * v_h.z, h_di[3] * v_h.w);
        } else {
          hv = v_h;
        }
      }
      if (h.kind == 1) st4(P + h.slot, hv);
      else P[h.slot] = hv.x;
    }
    return v;
  };

  float c[4][7];
  float dinv[4] = {0.f, 0.f, 0.f, 0.f};
  int zcls_cur = -1;
  const int z0 = ps.z0, z1 = ps.z1;
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
  if (z0 > 0 && ps.own) {  // plane z0 - 1 of the own column, staged like the others
    const float4 raw = ld4(src + (z0 - 1) * plane + col);
    if (kStage == 1) {
      const int zc = g.cz[z0 - 1];
      xm = make_float4(omega * dinv_at(g, cb, zc, ps.i, ps.j) * raw.x, omega * dinv_at(g, cb, zc, ps.i + 1, ps.j) * raw.y,
                       omega * dinv_at(g, cb, zc, ps.i + 2, ps.j) * raw.z,
                       omega * dinv_at(g, cb, zc, ps.i + 3, ps.j) * raw.w);
    } else {
      xm = raw;
    }
  }
  fetch(z0);
  float4 xc = commit(sm + (z0 % 3) * pl.PS, z0);
  fetch(z0 + 1);
  float rho = 0.f;
  for (int z = z0; z < z1; ++z) {
    const float4 xp = commit(sm + ((z + 1) % 3) * pl.PS, z + 1);  // plane z+1 (zeros past nz)
    fetch(z + 2);                                                  // in flight during plane z
    __syncthreads();
    const float* P = sm + (z % 3) * pl.PS;
    const int zcl = g.cz[z];
    if (zcl != zcls_cur && ps.own) {
      zcls_cur = zcl;
      load_coef4(g, cb, zcl, ps.i, ps.j, c);
#pragma unroll
      for (int e = 0; e < 4; e++) dinv[e] = dinv_at(g, cb, zcl, ps.i + e, ps.j);
    }
    if (ps.own) {
      float y[4];
      stencil4(P, pl, oslot, c, xm, xc, xp, y);
      const float4 bv = ld4(rhs + z * plane + col);
      float4 o;
      if (kOut == 1) {
        o = make_float4(bv.x - y[0], bv.y - y[1], bv.z - y[2], bv.w - y[3]);
      } else {
        o = make_float4(fmaf(omega * dinv[0], bv.x - y[0], xc.x), fmaf(omega * dinv[1], bv.y - y[1], xc.y),
                        fmaf(omega * dinv[2], bv.z - y[2], xc.z), fmaf(omega * dinv[3], bv.w - y[3], xc.w));
        if (kOut == 2) rho = fmaf(bv.x, o.x, fmaf(bv.y, o.y, fmaf(bv.z, o.z, fmaf(bv.w, o.w, rho))));
      }
      st4(out + z * plane + col, o);
    }
    xm = xc;
    xc = xp;
  }
  if (kOut == 2) {
    double drho = (double)rho, dummy = 0.0;
    block_sum2(drho, dummy, red);
    if (tid == 0) a.rho_rr[((int64_t)m.slot * a.B + b) * a.P + ps.part].x = drho;
  }
}

int launch_mg_fine_v4(const CGArgs<float>& a, Tile t, int stage, int outk, const MGFineArgs& m, cudaStream_t s) {
  const dim3 grid(a.tiles_x * a.tiles_y, a.nzc, a.B), block(t.tx, t.ty);
  const size_t smem = v4_plane_smem(t);
  if (stage == 1 && outk == 0) {
    if (launch_mg_smooth_tma(a, t, 1, m, false, s)) k_mg_fine_v4<1, 0><<<grid, block, smem, s>>>(a, m);
  }
  else if (stage == 0 && outk == 1) k_mg_fine_v4<0, 1><<<grid, block, smem, s>>>(a, m);
  else if (stage == 0 && outk == 2) {
    if (launch_mg_smooth_tma(a, t, 0, m, true, s)) k_mg_fine_v4<0, 2><<<grid, block, smem, s>>>(a, m);
  } else if (stage == 0 && outk == 0) {
    if (launch_mg_smooth_tma(a, t, 0, m, false, s)) k_mg_fine_v4<0, 0><<<grid, block, smem, s>>>(a, m);
  }
  else if (stage == 0 && outk == 3) return launch_mg_fine_rr_tma(a, t, m, s);
  else return -1;
  return 0;
}

void launch_cg_a_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_a_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), v4_plane_smem(t), s>>>(a, parity);
}
void launch_cg_b_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s) {
  k_cg_b_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), 0, s>>>(a, parity);
}
void launch_precond_rho_v4(const CGArgs<float>& a, Tile t, int slot, const int* mask, cudaStream_t s) {
  k_precond_rho_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), 0, s>>>(a, slot, mask);
}

void launch_ru_reset_v4(const CGArgs<float>& a, Tile t, int start, cudaStream_t s) {
  k_ru_reset_v4<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), 0, s>>>(a, start);
}

}  // namespace rbws
