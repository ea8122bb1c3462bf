// ru_ff.cu -- reliable updates of the mixed-precision iteration in float-float
// arithmetic, on the FP32 pipe.
//
// The FP32 iteration (Algorithm 1 with FP32 vectors) accumulates a correction d
// since its last reliable update.  An update folds d into the solution and
// replaces the FP32 recursive residual by the true residual.  GB300 runs FP64 at
// about 1/60 of its FP32 rate, so an FP64 update (u += d, r = f - A u) is bound
// by the FP64 pipe.  Here the solution and the true residual are carried as
// unevaluated sums of two floats (hi + lo, about 48 significant bits) and an
// update is
//     r <- r - A d,    u <- u + d,
// with A d formed from float-float coefficients and the FP32 d.  Because the
// residual is updated rather than recomputed from u, its rounding error is
// relative to the size of the correction, not to |A| |u|.
//
// Arithmetic (all in round-to-nearest FP32, no reassociation):
//   two_sum(a, b) = (s, e) with s + e = a + b exactly (Knuth's TwoSum, The Art
//     of Computer Programming vol. 2, 1969; 6 operations, no ordering condition);
//   the product of a float-float coefficient (ch, cl) and a float x is
//     p = ch*x, e = fma(ch, x, -p) (the exact error of p, as in Dekker's
//     splitting, "A floating-point technique for extending the available
//     precision", 1971, with the fused multiply-add standing in for the split),
//     t = fma(cl, x, e), so c*x = p + t up to about 2^-48 |c x|;
//   sums of such products keep (hi, lo) with two_sum on the high parts and plain
//   addition of the low parts, then renormalise with two_sum.
//
// Convergence is decided in true FP64: an instance whose float-float residual
// meets tol has u = hi + lo written in FP64 and its FP64 residual f - A u formed
// (k_residual64); only that decides.  If it fails, the tracked residual is reset
// from the FP64 one.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rbws {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += (ch + cl) * x
__device__ __forceinline__ void acc_prod(float ch, float cl, float x, float& sh, float& sl) {
  const float p = __fmul_rn(ch, x);
  const float e = __fmaf_rn(ch, x, -p);
  const float t = __fmaf_rn(cl, x, e);
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, t));
}

// (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& h, float& l) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  two_sum(s, e, h, l);
}

// A double that holds a float value, as that float (exact then; otherwise the
// double truncated to 24 significant bits).  Integer operations only: zero and
// values below the float range give 0, above it the float conversion.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(bits >> 32), lw = (unsigned)bits;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return 0.f;
  if (e >= 255) return __double2float_rn(x);
  const unsigned m = ((hw & 0xfffffu) << 3) | (lw >> 29);
  return __uint_as_float((hw & 0x80000000u) | ((unsigned)e << 23) | m);
}

__device__ __forceinline__ void split_f64(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

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

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float f4(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 trunc4(const double* p) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  return make_float4(f64_to_f32_trunc(a.x), f64_to_f32_trunc(a.y), f64_to_f32_trunc(b.x), f64_to_f32_trunc(b.y));
}

// The v4 tiling of the FP32 phase kernels (stencil_v4.cu): 4 consecutive x nodes
// per thread, one CTA per (tile, z-chunk, instance), one partial per CTA.
struct Pos4 {
  int x0, y0, z0, z1, part;
  int i, j;
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
  p.own = p.i < g.nx && p.j < g.ny;
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Float-float coefficient tables: [B][ncls][16], the hi parts of the 8 values of
// the FP64 table, then their lo parts (value - hi, rounded).
// ---------------------------------------------------------------------------
__global__ void k_coef_ff(const double* __restrict__ c64, int64_t entries, float* __restrict__ cff) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= entries) return;
  const double* s = c64 + t * kCoefStride;
  float* o = cff + t * 2 * kCoefStride;
  for (int k = 0; k < kCoefStride; k++) split_f64(s[k], o[k], o[kCoefStride + k]);
}

// ---------------------------------------------------------------------------
// The update of the instances with upd[b] != 0 (1: at a block boundary, the
// deferred alpha p of the 32-byte schedules at parity 0; 2: a paused instance,
// at the parity recorded when it stopped):
//   d' = d + alpha p;  r <- r - A d';  u <- u + d';  r32 = hi(r);  ||r32||^2 partials.
// kStart: the first update of a solve, from u0 (FP64, holding FP32 values: the
// mixed-precision starts are FP32 lifts) with u = 0 and r = f before it.
// d is read (with its halo) but not written: neighbouring CTAs still read it;
// k_ru_reset_ff clears it afterwards.
// ---------------------------------------------------------------------------
template <bool kStart>
__global__ void __launch_bounds__(256, 2) k_ru_ff(CGArgs<float> a, FFState ff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z;
  const int mode = a.upd[b];
  if (!mode) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Geo& g = a.g;
  const Pos4 ps = pos4(g, a.tiles_x, a.zc);
  const int64_t off = (int64_t)b * g.n;
  const int par = mode == 1 ? 0 : a.st[b].pad;
  const float al = (!kStart && a.alpha) ? (float)a.alpha[(int64_t)par * a.B + b] : 0.f;
  const float* db = a.u + off;
  const float* pb = (par ? a.p1 : a.p0) + off;
  const double* u0 = a.u64 + off;
  const float* cb = ff.coef + (int64_t)b * g.ncls() * 2 * kCoefStride;
  const double* fb = ff.f ? ff.f + (int64_t)b * ff.f_stride : nullptr;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  const int PW = TXN + 8, PS = PW * (TY + 2);
  auto at = [&](int x, int y) { return (y + 1) * PW + 4 + x; };
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  // halo duty: y-halo rows by 4-node groups (2*blockDim.x threads), then x-halo
  // columns by single nodes (2*TY threads)
  const int nyh = 2 * blockDim.x;
  int hx = 0, hy = 0, hkind = 0;
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
  const int hslot = at(hx, hy), oslot = at(lx, ly);

  // the correction d' at a group of 4 nodes / one node
  auto val4 = [&](int64_t idx) -> float4 {
    if (kStart) return trunc4(u0 + idx);
    float4 v = ld4(db + idx);
    if (al != 0.f) v = fma4(al, ld4(pb + idx), v);
    return v;
  };
  auto val1 = [&](int64_t idx) -> float {
    if (kStart) return f64_to_f32_trunc(u0[idx]);
    float v = db[idx];
    if (al != 0.f) v = fmaf(al, pb[idx], v);
    return v;
  };
  float4 v_own, v_h;
  auto fetch = [&](int z) {
    const bool zin = z >= 0 && z < g.nz;
    v_own = v_h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zin && ps.own) v_own = val4(z * plane + col);
    if (zin && hin) {
      if (hkind == 1) v_h = val4(z * plane + hcol);
      else v_h.x = val1(z * plane + hcol);
    }
  };
  auto commit = [&](float* P) -> float4 {
    st4(P + oslot, v_own);
    if (hkind == 1) st4(P + hslot, v_h);
    else if (hkind == 2) P[hslot] = v_h.x;
    return v_own;
  };

  float ch[4][7], cl[4][7];
  int zcls_cur = -1;
  const int z0 = ps.z0, z1 = ps.z1;
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
  if (z0 > 0 && ps.own) xm = val4((z0 - 1) * plane + col);
  fetch(z0);
  float4 xc = commit(sm + (z0 % 3) * PS);
  fetch(z0 + 1);
  float rr = 0.f;
  for (int z = z0; z < z1; ++z) {
    const float4 xp = commit(sm + ((z + 1) % 3) * PS);
    fetch(z + 2);
    // own-node streams of plane z (issued before the barrier)
    const int64_t idx = off + z * plane + col;
    float4 rh4 = make_float4(1.f, 1.f, 1.f, 1.f), rl4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 uh4 = make_float4(0.f, 0.f, 0.f, 0.f), ul4 = uh4;
    if (ps.own) {
      if (!kStart) {
        rh4 = ld4(ff.rh + idx);
        rl4 = ld4(ff.rl + idx);
        uh4 = ld4(ff.uh + idx);
        ul4 = ld4(ff.ul + idx);
      } else if (fb) {
        const double* fz = fb + z * plane + col;
        float h, l;
        split_f64(fz[0], h, l); rh4.x = h; rl4.x = l;
        split_f64(fz[1], h, l); rh4.y = h; rl4.y = l;
        split_f64(fz[2], h, l); rh4.z = h; rl4.z = l;
        split_f64(fz[3], h, l); rh4.w = h; rl4.w = l;
      }
    }
    __syncthreads();
    const float* P = sm + (z % 3) * PS;
    const int zcl = g.cz[z];
    if (zcl != zcls_cur && ps.own) {
      zcls_cur = zcl;
      const int yc = (int)g.cy[ps.j];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[ps.i + e]) * 2 * kCoefStride;
#pragma unroll
        for (int m = 0; m < 7; m++) {
          ch[e][m] = row[m];
          cl[e][m] = row[kCoefStride + m];
        }
      }
    }
    if (ps.own) {
      const float left = P[oslot - 1], right = P[oslot + 4];
      const float4 sth = ld4(P + oslot - PW), nth = ld4(P + oslot + PW);
      float ro[4], rlo[4], uo[4], ulo[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const float xce = f4(xc, e);
        const float xw = e == 0 ? left : f4(xc, e - 1);
        const float xe = e == 3 ? right : f4(xc, e + 1);
        // (sh, sl) = (A d')(node) in float-float; table order -kW -kE -kS -kN -kD -kU D
        float sh = 0.f, sl = 0.f;
        acc_prod(ch[e][6], cl[e][6], xce, sh, sl);
        acc_prod(ch[e][0], cl[e][0], xw, sh, sl);
        acc_prod(ch[e][1], cl[e][1], xe, sh, sl);
        acc_prod(ch[e][2], cl[e][2], f4(sth, e), sh, sl);
        acc_prod(ch[e][3], cl[e][3], f4(nth, e), sh, sl);
        acc_prod(ch[e][4], cl[e][4], f4(xm, e), sh, sl);
        acc_prod(ch[e][5], cl[e][5], f4(xp, e), sh, sl);
        ff_add(f4(rh4, e), f4(rl4, e), -sh, -sl, ro[e], rlo[e]);
        float s, err;
        two_sum(f4(uh4, e), xce, s, err);
        two_sum(s, __fadd_rn(err, f4(ul4, e)), uo[e], ulo[e]);
        rr = fmaf(ro[e], ro[e], rr);
      }
      const float4 r4 = make_float4(ro[0], ro[1], ro[2], ro[3]);
      st4(ff.rh + idx, r4);
      st4(ff.rl + idx, make_float4(rlo[0], rlo[1], rlo[2], rlo[3]));
      st4(ff.uh + idx, make_float4(uo[0], uo[1], uo[2], uo[3]));
      st4(ff.ul + idx, make_float4(ulo[0], ulo[1], ulo[2], ulo[3]));
      st4(a.r + idx, r4);
    }
    xm = xc;
    xc = xp;
  }
  double drr = (double)rr, dummy = 0.0;
  block_sum2(drr, dummy, red);
  if (tid == 0) ff.part[(int64_t)b * a.P + ps.part] = drr;
}

// chk[b] = 1 for the updated instances whose float-float residual meets tol:
// they take the FP64 check.
__global__ void k_ru_mark(CGArgs<float> a, FFState ff) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  ff.chk[b] = (a.upd[b] != 0 && ff.rel[b] < a.tol) ? 1 : 0;
}

// u64 = hi + lo for the instances with mask[b] != 0.  Usually few instances are masked in:
// each CTA compacts the mask (1024 instances at a time) into a shared list in ascending
// order (a block-wide prefix sum, so every CTA holds the same list) and the grid sweeps the
// flattened (listed instance, node) range, so every element is independent work instead of
// one instance after another.
__global__ void __launch_bounds__(256) k_ff_to64(int64_t n, int B, const float* __restrict__ uh,
                                                 const float* __restrict__ ul, const int* __restrict__ mask,
                                                 double* __restrict__ u64) {
  __shared__ int s_list[1024];
  __shared__ int s_warp[8];
  __shared__ int s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;  // 256 threads
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c0 = 0; c0 < B; c0 += 1024) {
    // thread tid takes the chunk's entries 4 tid .. 4 tid + 3
    int flags[4], cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int b = c0 + 4 * tid + q;
      flags[q] = b < B && mask[b] != 0;
      cnt += flags[q];
    }
    int incl = cnt;  // inclusive scan over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; w++) base += s_warp[w];
    int pos = base + incl - cnt;
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (flags[q]) s_list[pos++] = c0 + 4 * tid + q;
    if (tid == 255) s_cnt = pos;
    __syncthreads();
    const int64_t total = (int64_t)s_cnt * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + tid; t < total; t += stride) {
      const int64_t e = (int64_t)s_list[t / n] * n + t % n;
      u64[e] = ff_to_f64(uh[e], ul[e]);
    }
    __syncthreads();  // the list and the warp sums are rebuilt for the next chunk
  }
}

// u <- u + d + alpha p (float-float) and d = 0 for the instances with upd[b] != 0
// (the fold of instances that stopped between updates; parity as in k_ru_ff).
__global__ void k_ff_fold(CGArgs<float> a, FFState ff) {
  const int b = blockIdx.y;
  const int mode = a.upd[b];
  if (!mode) return;
  const int par = mode == 1 ? 0 : a.st[b].pad;
  const float al = a.alpha ? (float)a.alpha[(int64_t)par * a.B + b] : 0.f;
  const int64_t off = (int64_t)b * a.g.n;
  const float* pp = (par ? a.p1 : a.p0) + off;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.g.n; i += (int64_t)gridDim.x * blockDim.x) {
    float dv = a.u[off + i];
    if (al != 0.f) dv = fmaf(al, pp[i], dv);
    float s, err;
    two_sum(ff.uh[off + i], dv, s, err);
    two_sum(s, __fadd_rn(err, ff.ul[off + i]), ff.uh[off + i], ff.ul[off + i]);
    a.u[off + i] = 0.f;
  }
}

// After an update: the new status of each updated instance, from the FP64
// residual where it took the check (chk), else from the float-float one.
//  - chk and rel64 < tol: converged (u64 was written for the check);
//  - chk and rel64 >= tol: the tracked residual is reset from the FP64 one and
//    the search direction restarts;
//  - otherwise active (mode 2 or the start restarts the direction), or
//    max_iters / breakdown.
// Every updated instance gets d = 0; an active one r = hi(r) (already written by
// k_ru_ff, or from the FP64 residual), s = D^{-1} r (Jacobi), p_old = 0 on a
// restart, and the partials of rho = r.s and ||r||^2 in slot 0.
__global__ void __launch_bounds__(256) k_ru_reset_ff(CGArgs<float> a, FFState ff, int start) {
  __shared__ double red[64];
  const int b = blockIdx.z;
  const int mode = a.upd[b];
  if (!mode) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const Geo& g = a.g;
  const Pos4 ps = pos4(g, a.tiles_x, a.zc);
  const bool leader = ps.part == 0;
  InstState* st = a.st + b;
  const bool chk = ff.chk[b] != 0;
  const double rel = chk ? a.rel64[b] : ff.rel[b];
  const int iters = start ? 0 : st->iters;
  int ns;
  if (chk && rel < a.tol) ns = ST_CONVERGED;
  else if (!(rel == rel)) ns = ST_BREAKDOWN;
  else if (iters >= a.max_iters) ns = ST_MAX_ITERS;
  else ns = ST_ACTIVE;
  const bool resync = chk && ns == ST_ACTIVE;
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
    if (a.alpha) a.alpha[b] = 0.0;  // the update applied any pending alpha p
    a.rr_ref[b] = (rel * a.fnorm[b]) * (rel * a.fnorm[b]);
    if (ns == ST_ACTIVE) atomicAdd(a.active, 1);
    if (ns == ST_ACTIVE && (mode == 2 || resync) && !start) st->restarts += 1;
  }
  const bool active = ns == ST_ACTIVE;
  const bool restart = start || mode == 2 || resync;
  const bool mg = a.precond == RBWS_PREC_MG;
  const bool jac = a.precond != RBWS_PREC_NONE;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const int64_t off = (int64_t)b * g.n;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)ps.j * g.nx + ps.i;
  // With MG and no resync the residual is the one k_ru_ff just wrote, and its r.r partials
  // are that kernel's (same tiling, in ff.part): r need not be read again.
  const bool reuse_rr = mg && !resync;
  float rho = 0.f, rr = 0.f;
  if (ps.own) {
    int zcls_cur = -1;
    float dinv[4] = {1.f, 1.f, 1.f, 1.f};
    const int yc = (int)g.cy[ps.j];
    for (int z = ps.z0; z < ps.z1; ++z) {
      const int64_t idx = off + z * plane + col;
      st4(a.u + idx, make_float4(0.f, 0.f, 0.f, 0.f));
      if (!active) continue;
      if (reuse_rr) {
        if (restart) st4(a.p0 + idx, make_float4(0.f, 0.f, 0.f, 0.f));
        continue;
      }
      const int zcl = g.cz[z];
      if (zcl != zcls_cur) {
        zcls_cur = zcl;
#pragma unroll
        for (int e = 0; e < 4; e++)
          dinv[e] = cb[(((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[ps.i + e]) * kCoefStride + 7];
      }
      float4 rv;
      if (resync) {
        const double2 ra = *reinterpret_cast<const double2*>(a.r64 + idx);
        const double2 rb2 = *reinterpret_cast<const double2*>(a.r64 + idx + 2);
        float h[4], l[4];
        split_f64(ra.x, h[0], l[0]);
        split_f64(ra.y, h[1], l[1]);
        split_f64(rb2.x, h[2], l[2]);
        split_f64(rb2.y, h[3], l[3]);
        rv = make_float4(h[0], h[1], h[2], h[3]);
        st4(ff.rh + idx, rv);
        st4(ff.rl + idx, make_float4(l[0], l[1], l[2], l[3]));
        st4(a.r + idx, rv);
      } else {
        rv = ld4(a.r + idx);
      }
      float4 sv = rv;
      if (jac) sv = make_float4(dinv[0] * rv.x, dinv[1] * rv.y, dinv[2] * rv.z, dinv[3] * rv.w);
      if (!mg) st4(a.s + idx, sv);
      if (restart) st4(a.p0 + idx, make_float4(0.f, 0.f, 0.f, 0.f));
      rho = fmaf(rv.x, sv.x, fmaf(rv.y, sv.y, fmaf(rv.z, sv.z, fmaf(rv.w, sv.w, rho))));
      rr = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, rr))));
    }
  }
  if (!active) return;  // uniform over the CTA
  // with MG, s and rho follow from a V-cycle after the reset
  double drho = mg ? 0.0 : (double)rho, drr = (double)rr;
  if (!reuse_rr) block_sum2(drho, drr, red);
  else drr = ff.part[(int64_t)b * a.P + ps.part];
  if (tid == 0) {
    a.rho_rr[(int64_t)b * a.P + ps.part] = make_double2(drho, drr);
    if (restart) a.rho_rr[((int64_t)a.B + b) * a.P + ps.part] = make_double2(ps.part == 0 ? 1.0 : 0.0, 0.0);
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void launch_coef_ff(const double* coef64, int64_t entries, float* coefff, cudaStream_t s) {
  k_coef_ff<<<(unsigned)((entries + 127) / 128), 128, 0, s>>>(coef64, entries, coefff);
}

void launch_ru_ff(const CGArgs<float>& a, Tile t, const FFState& ff, bool start, cudaStream_t s) {
  const dim3 grid(a.tiles_x * a.tiles_y, a.nzc, a.B), block(t.tx, t.ty);
  const size_t smem = sizeof(float) * 3 * (size_t)(4 * t.tx + 8) * (t.ty + 2);
  if (start) k_ru_ff<true><<<grid, block, smem, s>>>(a, ff);
  else k_ru_ff<false><<<grid, block, smem, s>>>(a, ff);
}

void launch_ru_mark(const CGArgs<float>& a, const FFState& ff, cudaStream_t s) {
  k_ru_mark<<<(a.B + 127) / 128, 128, 0, s>>>(a, ff);
}

void launch_ff_to64(const CGArgs<float>& a, const FFState& ff, const int* mask, cudaStream_t s) {
  k_ff_to64<<<152 * 8, 256, 0, s>>>(a.g.n, a.B, ff.uh, ff.ul, mask, a.u64);
}

void launch_ff_fold(const CGArgs<float>& a, const FFState& ff, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((a.g.n + 255) / 256, 152 * 2);
  k_ff_fold<<<dim3((unsigned)blocks, a.B), 256, 0, s>>>(a, ff);
}

void launch_ru_reset_ff(const CGArgs<float>& a, Tile t, const FFState& ff, int start, cudaStream_t s) {
  k_ru_reset_ff<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), 0, s>>>(a, ff, start);
}

}  // namespace rbws
