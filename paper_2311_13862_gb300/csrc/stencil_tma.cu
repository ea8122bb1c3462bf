// stencil_tma.cu -- FP32 PCG stencil phase fed by the Tensor Memory Accelerator.
//
// Same arithmetic as k_cg_a_v4 (p = s + beta p_old, q = A p, partial p.q), but
// the (s, p_old) tiles of each z plane -- a (4*tx + 8) x (ty + 2) box that
// includes the x/y halo -- are copied into a ring of kStages shared-memory
// stages by cp.async.bulk.tensor, issued by one thread and completed on one
// mbarrier per stage.  Up to kStages planes are in flight per CTA without
// holding registers, and the tensor map's zero fill supplies the Dirichlet
// halo at the domain faces (boxes may start at x = -4, y = -1, z = -1; x
// starts stay 16-byte aligned because tiles start at multiples of 4 nodes).
// p at the neighbours is formed from the staged s and p_old when it is read.
//
// The same ring feeds the other TMA kernels of this file: phase B of the
// 32-byte schedule (k_cg_b_s_tma), and the finest-level multigrid steps --
// the damped Jacobi steps (k_mg_smooth_tma, k_mg_smooth_od_tma with omega/D
// staged beside r) and the residual + restriction pass (k_mg_fine_rr_tma).
//
// Every mbarrier wait is bounded (about 2 s of clock64 time).  A CTA whose
// wait runs out sets *err, lets its outstanding copies land (again bounded)
// and returns; the host reports RBWS_ERR_DEVICE_TIMEOUT.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rbws {

namespace {

constexpr int kStages = 4;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for phase `parity` of the barrier; false if it ran out.  budget:
// clock64 cycles (<= 0: kWaitCycles).  The waits of the normal pipeline take the
// call's budget (rbws_options.wait_cycles); the drain after a timeout always takes
// kWaitCycles, so that a CTA returns only once its copies in flight have landed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long budget = kWaitCycles) {
  if (budget <= 0) budget = kWaitCycles;
  // try_wait may suspend the thread for a while before it returns false, so a
  // short budget (a test of the timeout path) polls with the non-blocking test_wait
  const bool poll = budget < 1000000;
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    if (poll)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ double warp_sum_down(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
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

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float f4(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

}  // namespace

// kMode 0: 44-byte schedule (writes p and q = A p).
// kMode 1: 32-byte s-form schedule (writes p; q is not stored; also applies
//          the update u += alpha_{k-1} p_{k-1} deferred by phase B, own nodes).
template <int kMode>
__global__ void __launch_bounds__(256, 3)
    k_cg_a_tma(const __grid_constant__ CUtensorMap tm_s, const __grid_constant__ CUtensorMap tm_p0,
               const __grid_constant__ CUtensorMap tm_p1, const __grid_constant__ CUtensorMap tm_u,
               CGArgs<float> a, int parity, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ double red[64];
  __shared__ double s_beta, s_alpha;
  __shared__ int s_run;
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tiles_x = a.tiles_x;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  const int x0 = (blockIdx.x % tiles_x) * TXN, y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = blockIdx.y * a.zc, z1 = min(a.g.nz, z0 + a.zc);
  const int part = blockIdx.y * gridDim.x + blockIdx.x;
  const bool leader = part == 0;
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
      // an earlier CTA's wait ran out: do not wait again (decided by one thread, shared below)
      if (status == ST_ACTIVE && !*reinterpret_cast<volatile int*>(err)) {
        const double rel = sqrt(cur.y) / a.fnorm[b];
        if (rel < a.tol) {
          if (leader) {
            st->status = a.ru ? ST_PAUSED : ST_CONVERGED;
            st->relres = rel;
            st->pad = parity;  // kMode 1: the update alpha[parity] * p_old is still pending
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else if (st->iters >= a.max_iters || !(rel == rel)) {
          if (leader) {
            st->status = (rel == rel) ? ST_MAX_ITERS : ST_BREAKDOWN;
            st->relres = rel;
            st->pad = parity;
            st->t_done = global_ns();
            atomicSub(a.active, 1);
          }
        } else {
          run = 1;
          s_beta = cur.x / prev;
          s_alpha = kMode == 1 ? a.alpha[(int64_t)parity * a.B + b] : 0.0;
        }
      }
      s_run = run;
    }
  }
  __syncthreads();
  if (!s_run) return;
  const float beta = (float)s_beta;
  const float alpha_prev = (float)s_alpha;
  const Geo& g = a.g;
  const int BX = TXN + 8, BY = TY + 2;
  const unsigned box_bytes = (unsigned)(BX * BY * sizeof(float));
  const int arr_floats = ((BX * BY * 4 + 127) / 128) * 32;  // 128-byte aligned arrays
  // kMode 1 also stages the own (halo-free) TXN x TY tile of u for planes z0 .. z1-1
  const unsigned own_bytes = (unsigned)(TXN * TY * sizeof(float));
  const int own_floats = kMode == 1 ? ((TXN * TY * 4 + 127) / 128) * 32 : 0;
  const int stage_floats = 2 * arr_floats + own_floats;
  float* stage_base = reinterpret_cast<float*>(smem_raw);
  auto s_tile = [&](int st) { return stage_base + st * stage_floats; };
  auto p_tile = [&](int st) { return stage_base + st * stage_floats + arr_floats; };
  auto u_tile = [&](int st) { return stage_base + st * stage_floats + 2 * arr_floats; };
  const CUtensorMap* mp = parity ? &tm_p1 : &tm_p0;
  const int nq = z1 - z0 + 2;  // planes z0-1 .. z1
  auto issue = [&](int j) {    // plane z0-1+j into stage j % kStages (thread 0 only)
    const int st = j % kStages;
    const bool with_u = kMode == 1 && j >= 1 && j <= nq - 2;
    mbar_expect_tx(&bars[st], 2 * box_bytes + (with_u ? own_bytes : 0u));
    tma_load_4d(s_tile(st), &tm_s, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    tma_load_4d(p_tile(st), mp, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    if (with_u) tma_load_4d(u_tile(st), &tm_u, x0, y0, z0 - 1 + j, b, &bars[st]);
  };
  if (tid == 0) {
    for (int st = 0; st < kStages; st++) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int n_issued = 0;  // meaningful in thread 0 only
  int next_wait = 0; // first plane index not yet waited for (uniform)
  if (tid == 0)
    for (int j = 0; j < kStages && j < nq; j++) {
      issue(j);
      n_issued = j + 1;
    }

  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  const int i = x0 + lx, jn = y0 + ly;
  const bool own = i < g.nx && jn < g.ny;
  const int cofs = (ly + 1) * BX + lx + 4;  // own group in a box
  const int lofs = ly * TXN + lx;           // own group in an own-tile array
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)jn * g.nx + i;
  float* pnew = (parity ? a.p0 : a.p1) + (int64_t)b * g.n;
  float* qb = a.q + (int64_t)b * g.n;
  float* ub = a.u + (int64_t)b * g.n;
  auto own_p = [&](int st) { return fma4(beta, ld4s(p_tile(st) + cofs), ld4s(s_tile(st) + cofs)); };

  // prologue: planes z0-1 (own column only) and z0
  bool timed_out = !mbar_wait(&bars[0], 0, a.wait_cycles);
  float4 xm = own_p(0);
  if (!timed_out) timed_out = !mbar_wait(&bars[1 % kStages], (1 / kStages) & 1, a.wait_cycles);
  float4 xc = own_p(1 % kStages);
  if (__syncthreads_or(timed_out)) goto abort;
  next_wait = 2;
  if (tid == 0 && kStages < nq) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(kStages);  // stage 0 is free again
    n_issued = kStages + 1;
  }
  {
    float c[4][7];
    int zcls_cur = -1;
    float gam = 0.f;
    for (int z = z0; z < z1; ++z) {
      const int k = z - z0 + 1;  // index of plane z; plane z+1 is k+1
      const int sk = k % kStages, sn = (k + 1) % kStages;
      bool to = !mbar_wait(&bars[sn], ((k + 1) / kStages) & 1, a.wait_cycles);
      if (!to && own) {
        const float4 xp = own_p(sn);
        const int zcl = g.cz[z];
        if (zcl != zcls_cur) {
          zcls_cur = zcl;
          const int yc = (int)g.cy[jn];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
#pragma unroll
            for (int m = 0; m < 7; m++) c[e][m] = row[m];
          }
        }
        const float* S = s_tile(sk);
        const float* Pp = p_tile(sk);
        const float left = fmaf(beta, Pp[cofs - 1], S[cofs - 1]);
        const float right = fmaf(beta, Pp[cofs + 4], S[cofs + 4]);
        const float4 sth = fma4(beta, ld4s(Pp + cofs - BX), ld4s(S + cofs - BX));
        const float4 nth = fma4(beta, ld4s(Pp + cofs + BX), ld4s(S + cofs + BX));
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
        *reinterpret_cast<float4*>(pnew + z * plane + col) = xc;
        if (kMode == 0) {
          *reinterpret_cast<float4*>(qb + z * plane + col) = make_float4(y[0], y[1], y[2], y[3]);
        } else {
          const float4 po4 = ld4s(Pp + cofs);  // own p_old and u of plane z, from the stage
          *reinterpret_cast<float4*>(ub + z * plane + col) = fma4(alpha_prev, po4, ld4s(u_tile(sk) + lofs));
        }
        xm = xc;
        xc = xp;
      } else if (!to) {
        xm = xc;
        xc = own_p(sn);
      }
      if (__syncthreads_or(to)) goto abort;
      next_wait = k + 2;
      // plane z's stage is free: refill it with plane index k + kStages
      if (tid == 0 && k + kStages < nq) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + kStages);
        n_issued = k + kStages + 1;
      }
    }
    double dg = (double)gam, dummy = 0.0;
    // deterministic block sum (same tree as the other kernels)
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    dg = warp_sum_down(dg);
    if (lane == 0) red[warp] = dg;
    __syncthreads();
    if (warp == 0) {
      double x = lane < nw ? red[lane] : 0.0;
      x = warp_sum_down(x);
      if (lane == 0) a.gam[(int64_t)b * a.P + part] = x;
    }
    (void)dummy;
  }
  return;
abort:
  // a wait ran out: flag it and let the copies already issued land before returning
  if (tid == 0) {
    atomicExch(err, 1);
    // copies issued for planes next_wait .. n_issued-1 may still be landing
    for (int j = next_wait; j < n_issued; j++) mbar_wait(&bars[j % kStages], (j / kStages) & 1);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Phase B of the 32-byte s-form schedule.  The stored residual is
// s = D^{-1} r (s = r without a preconditioner).  alpha_k = rho_k / gamma_k;
// s -= alpha_k D^{-1} A p_k with A p_k recomputed from TMA-staged planes of
// p_k; r = D s; partials rho_{k+1} = r.s and ||r||^2.  Reads s (own tile,
// staged in the same ring) and p (halo from L2), writes s: 12 bytes per DoF.
// alpha_k goes to a.alpha[parity ^ 1][b] for the next phase A.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3)
    k_cg_b_s_tma(const __grid_constant__ CUtensorMap tm_p0, const __grid_constant__ CUtensorMap tm_p1,
                 const __grid_constant__ CUtensorMap tm_s, CGArgs<float> a, int parity, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ double red[64];
  __shared__ double s_alpha;
  __shared__ int s_run;
  const int b = blockIdx.z;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int tiles_x = a.tiles_x;
  const int TXN = blockDim.x * 4, TY = blockDim.y;
  const int x0 = (blockIdx.x % tiles_x) * TXN, y0 = (blockIdx.x / tiles_x) * TY;
  const int z0 = blockIdx.y * a.zc, z1 = min(a.g.nz, z0 + a.zc);
  const int part = blockIdx.y * gridDim.x + blockIdx.x;
  const bool leader = part == 0;
  if (tid < 32) {
    InstState* st = a.st + b;
    const int status = st->status;
    double rho = 0.0, gam = 0.0, rr = 0.0;
    if (status == ST_ACTIVE) {
      const double2 cur = sum_partials2(a.rho_rr + ((int64_t)parity * a.B + b) * a.P, a.P, tid);
      rho = cur.x;
      rr = cur.y;
      double gs = 0.0;
      for (int c = tid; c < a.P; c += 32) gs += a.gam[(int64_t)b * a.P + c];
      gam = warp_sum_down(gs);
    }
    if (tid == 0) {
      int run = 0;
      if (status == ST_ACTIVE && !*reinterpret_cast<volatile int*>(err)) {
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
  const bool jac = a.precond != RBWS_PREC_NONE;
  const int BX = TXN + 8, BY = TY + 2;
  const unsigned box_bytes = (unsigned)(BX * BY * sizeof(float));
  const int arr_floats = ((BX * BY * 4 + 127) / 128) * 32;
  const unsigned own_bytes = (unsigned)(TXN * TY * sizeof(float));
  const int stage_floats = arr_floats + ((TXN * TY * 4 + 127) / 128) * 32;
  float* stage_base = reinterpret_cast<float*>(smem_raw);
  auto p_tile = [&](int st) { return stage_base + st * stage_floats; };
  auto s_tile = [&](int st) { return stage_base + st * stage_floats + arr_floats; };
  const CUtensorMap* mp = parity ? &tm_p0 : &tm_p1;  // p_k = pbuf[parity ^ 1]
  const int nq = z1 - z0 + 2;
  auto issue = [&](int j) {  // p of plane z0-1+j with its halo; s of it for planes z0 .. z1-1
    const int st = j % kStages;
    const bool with_s = j >= 1 && j <= nq - 2;
    mbar_expect_tx(&bars[st], box_bytes + (with_s ? own_bytes : 0u));
    tma_load_4d(p_tile(st), mp, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    if (with_s) tma_load_4d(s_tile(st), &tm_s, x0, y0, z0 - 1 + j, b, &bars[st]);
  };
  if (tid == 0) {
    for (int st = 0; st < kStages; st++) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int n_issued = 0, next_wait = 0;
  if (tid == 0)
    for (int j = 0; j < kStages && j < nq; j++) {
      issue(j);
      n_issued = j + 1;
    }
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  const int i = x0 + lx, jn = y0 + ly;
  const bool own = i < g.nx && jn < g.ny;
  const int cofs = (ly + 1) * BX + lx + 4;
  const int lofs = ly * TXN + lx;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)jn * g.nx + i;
  float* sb = a.s + (int64_t)b * g.n;
  float rho = 0.f, rr = 0.f;
  bool timed_out = !mbar_wait(&bars[0], 0, a.wait_cycles);
  float4 xm = ld4s(p_tile(0) + cofs);
  if (!timed_out) timed_out = !mbar_wait(&bars[1 % kStages], (1 / kStages) & 1, a.wait_cycles);
  float4 xc = ld4s(p_tile(1 % kStages) + cofs);
  if (__syncthreads_or(timed_out)) goto abort;
  next_wait = 2;
  if (tid == 0 && kStages < nq) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(kStages);
    n_issued = kStages + 1;
  }
  {
    float c[4][8];
    int zcls_cur = -1;
    // the planes in groups of kStages, so that a plane's ring stages and its wait
    // parity's offset within the group are compile-time constants
    for (int kb = 0; z0 + kb < z1; kb += kStages)
#pragma unroll
    for (int q = 0; q < kStages; q++) {
      const int z = z0 + kb + q;
      if (z >= z1) break;
      const int k = kb + q + 1;
      const int sk = (q + 1) % kStages, sn = (q + 2) % kStages;
      bool to = !mbar_wait(&bars[sn], ((kb / kStages) + (q + 2) / kStages) & 1, a.wait_cycles);
      if (!to && own) {
        const float4 xp = ld4s(p_tile(sn) + cofs);
        const float4 s4 = ld4s(s_tile(sk) + lofs);
        const int zcl = g.cz[z];
        if (zcl != zcls_cur) {
          zcls_cur = zcl;
          const int yc = (int)g.cy[jn];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
#pragma unroll
            for (int m = 0; m < 8; m++) c[e][m] = row[m];
          }
        }
        const float* Pp = p_tile(sk);
        const float left = Pp[cofs - 1], right = Pp[cofs + 4];
        const float4 sth = ld4s(Pp + cofs - BX), nth = ld4s(Pp + cofs + BX);
        float sn4[4];
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
          const float dinv = jac ? c[e][7] : 1.f;
          const float snew = fmaf(-alpha * dinv, v, f4(s4, e));
          const float rnew = jac ? c[e][6] * snew : snew;
          rho = fmaf(rnew, snew, rho);
          rr = fmaf(rnew, rnew, rr);
          sn4[e] = snew;
        }
        *reinterpret_cast<float4*>(sb + z * plane + col) = make_float4(sn4[0], sn4[1], sn4[2], sn4[3]);
        xm = xc;
        xc = xp;
      } else if (!to) {
        xm = xc;
        xc = ld4s(p_tile(sn) + cofs);
      }
      if (__syncthreads_or(to)) goto abort;
      next_wait = k + 2;
      if (tid == 0 && k + kStages < nq) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + kStages);
        n_issued = k + kStages + 1;
      }
    }
    double drho = (double)rho, drr = (double)rr;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    drho = warp_sum_down(drho);
    drr = warp_sum_down(drr);
    if (lane == 0) {
      red[warp] = drho;
      red[32 + warp] = drr;
    }
    __syncthreads();
    if (warp == 0) {
      double x = lane < nw ? red[lane] : 0.0, y = lane < nw ? red[32 + lane] : 0.0;
      x = warp_sum_down(x);
      y = warp_sum_down(y);
      if (lane == 0) a.rho_rr[((int64_t)(parity ^ 1) * a.B + b) * a.P + part] = make_double2(x, y);
    }
  }
  return;
abort:
  if (tid == 0) {
    atomicExch(err, 1);
    for (int j = next_wait; j < n_issued; j++) mbar_wait(&bars[j % kStages], (j / kStages) & 1);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Finest multigrid level: the residual r = rhs - A x and its restriction
// rc = P^T r in one pass (the residual and restriction steps of Algorithm 2),
// without storing r.  A CTA owns the coarse nodes whose centre (fine node
// 2I+1, 0-based) lies in its tile and z-chunk; their support reaches one fine
// node past the tile on the high side of each axis, so the residual is also
// formed on the extra column x0+TXN, the extra row y0+TY and the extra plane
// z1.  Each plane of x (a (TXN+8) x (TY+3) box from x0-4, y0-1) and of rhs (a
// (TXN+4) x (TY+1) box from x0, y0) arrives by TMA in a ring of kStages
// stages.  The residuals of a plane go to one of two shared-memory planes;
// after one barrier each thread sums the x/y weights (1/2, 1, 1/2) of its
// coarse column, and the z weights are applied as the march passes the
// coarse planes.  Requires an even TY and zc (tile origins on even nodes).
// ---------------------------------------------------------------------------
// Two CTAs per SM: the ring keeps about three planes per CTA in flight without
// registers, so occupancy is not what feeds HBM here.
__global__ void __launch_bounds__(256, 3)
    k_mg_fine_rr_tma(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_r,
                     CGArgs<float> a, MGFineArgs m, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ int s_go;
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (m.mask && !m.mask[b])) return;
  const Geo& g = a.g;
  const int TXT = blockDim.x, TY = blockDim.y, TXN = 4 * TXT;
  const int tid = (int)threadIdx.y * TXT + (int)threadIdx.x;
  // an earlier CTA's wait ran out: do not wait again (read by one thread, shared)
  if (tid == 0) s_go = !*reinterpret_cast<volatile int*>(err);
  __syncthreads();
  if (!s_go) return;
  const int x0 = (blockIdx.x % a.tiles_x) * TXN, y0 = (blockIdx.x / a.tiles_x) * TY;
  const int z0 = blockIdx.y * a.zc, z1 = min(g.nz, z0 + a.zc), zlast = min(z1, g.nz - 1);
  const int PW = TXN + 8, RP = TXN + 4;  // row pitch of the x box and of the rhs box (and R)
  const int xfl = ((PW * (TY + 3) * 4 + 127) / 128) * 32, rfl = ((RP * (TY + 1) * 4 + 127) / 128) * 32;
  float* base = reinterpret_cast<float*>(smem_raw);
  auto xs = [&](int st) { return base + st * (xfl + rfl); };
  auto rs = [&](int st) { return base + st * (xfl + rfl) + xfl; };
  const int rpl = RP * (TY + 1);
  float* R = base + kStages * (xfl + rfl);  // two residual planes [TY+1][RP]
  float* exc_all = R + 2 * rpl;             // 8 floats per extra node: its cached coefficients
  const unsigned xbytes = (unsigned)(PW * (TY + 3) * 4), rbytes = (unsigned)(RP * (TY + 1) * 4);
  const int nq = zlast - z0 + 3;  // planes z0-1 .. zlast+1
  auto issue = [&](int j) {       // plane z0-1+j into stage j % kStages (thread 0 only)
    const int st = j % kStages;
    const bool with_r = j >= 1 && j <= nq - 2;
    mbar_expect_tx(&bars[st], xbytes + (with_r ? rbytes : 0u));
    tma_load_4d(xs(st), &tm_x, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    if (with_r) tma_load_4d(rs(st), &tm_r, x0, y0, z0 - 1 + j, b, &bars[st]);
  };
  if (tid == 0) {
    for (int st = 0; st < kStages; st++) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int n_issued = 0;   // thread 0 only
  int next_wait = 0;  // first plane index not yet waited for (uniform)
  if (tid == 0)
    for (int j = 0; j < kStages && j < nq; j++) {
      issue(j);
      n_issued = j + 1;
    }
  // duties: own group; at most one extra node (the TXN nodes of the extra row, then
  // the TY + 1 of the extra column), extra node d going to lane d / warps of warp
  // d % warps, so that every warp takes about the same share and runs the one-node
  // path once per plane; coarse column (every thread: 2 TXT x TY/2 of them)
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  const int i = x0 + lx, j = y0 + ly;
  const bool own = i < g.nx && j < g.ny;
  const int xo = (ly + 1) * PW + 4 + lx, ro = ly * RP + lx;
  const int nthr = TXT * TY;
  const int dix = (nthr & 31) == 0 ? (tid & 31) * (nthr >> 5) + (tid >> 5) : tid;
  const bool ex_duty = dix < TXN + TY + 1;
  const int exl = dix < TXN ? dix : TXN, eyl = dix < TXN ? TY : dix - TXN;
  const int exi = x0 + exl, exj = y0 + eyl;
  const bool ex_in = ex_duty && exi < g.nx && exj < g.ny;
  float* exc = exc_all + (dix < TXN ? dix : TXN + eyl) * 8;
  const int Il = tid % (2 * TXT), Jl = tid / (2 * TXT);
  const int I = x0 / 2 + Il, J = y0 / 2 + Jl;
  const bool cown = I < m.cnx && J < m.cny;
  float* rc = m.out + (int64_t)b * m.cnx * m.cny * m.cnz + (int64_t)J * m.cnx + I;
  const int64_t cplane = (int64_t)m.cnx * m.cny;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;

  bool to = !mbar_wait(&bars[0], 0, a.wait_cycles);
  if (!to) to = !mbar_wait(&bars[1 % kStages], (1 / kStages) & 1, a.wait_cycles);
  if (__syncthreads_or(to)) goto abort;
  next_wait = 2;
  {
    float c[4][7];
    int zcls_cur = -1, ex_zcls = -1;
    float acc = 0.f;
    // the planes in groups of kStages: z0 is even and each group starts kStages planes
    // after the last, so a plane's ring stages, its wait parity's offset within the group
    // and its parity along z (the restriction's branch) are compile-time constants
    for (int kb = 0; z0 + kb <= zlast; kb += kStages)
#pragma unroll
    for (int q = 0; q < kStages; q++) {
      const int z = z0 + kb + q;
      if (z > zlast) break;
      const int k = kb + q + 1;  // plane index of z
      const int sm_ = q, sk = (q + 1) % kStages, sn = (q + 2) % kStages;
      to = !mbar_wait(&bars[sn], ((kb / kStages) + (q + 2) / kStages) & 1, a.wait_cycles);
      float* Rz = R + (q & 1) * rpl;
      if (!to) {
        const float* Pm = xs(sm_);
        const float* Pc = xs(sk);
        const float* Pp = xs(sn);
        const float* Rh = rs(sk);
        const int zcl = g.cz[z];
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (own) {
          if (zcl != zcls_cur) {
            zcls_cur = zcl;
            const int yc = (int)g.cy[j];
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
#pragma unroll
              for (int q = 0; q < 7; q++) c[e][q] = row[q];
            }
          }
          const float left = Pc[xo - 1], right = Pc[xo + 4];
          const float4 xc = ld4s(Pc + xo), sth = ld4s(Pc + xo - PW), nth = ld4s(Pc + xo + PW);
          const float4 xm = ld4s(Pm + xo), xp = ld4s(Pp + xo), bv = ld4s(Rh + ro);
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
            y[e] = f4(bv, e) - v;
          }
          r = make_float4(y[0], y[1], y[2], y[3]);
        }
        *reinterpret_cast<float4*>(Rz + ro) = r;
        if (ex_duty) {
          if (ex_in && zcl != ex_zcls) {  // refresh the cached coefficients at a z class change
            ex_zcls = zcl;
            const float* row = cb + (((int64_t)zcl * g.ncy + g.cy[exj]) * g.ncx + g.cx[exi]) * kCoefStride;
#pragma unroll
            for (int q = 0; q < 7; q++) exc[q] = row[q];
          }
          const int o = (eyl + 1) * PW + 4 + exl;
          float rv = 0.f;
          if (ex_in) {
            float v = exc[6] * Pc[o];
            v = fmaf(exc[0], Pc[o - 1], v);
            v = fmaf(exc[1], Pc[o + 1], v);
            v = fmaf(exc[2], Pc[o - PW], v);
            v = fmaf(exc[3], Pc[o + PW], v);
            v = fmaf(exc[4], Pm[o], v);
            v = fmaf(exc[5], Pp[o], v);
            rv = Rh[eyl * RP + exl] - v;
          }
          Rz[eyl * RP + exl] = rv;
        }
      }
      if (__syncthreads_or(to)) goto abort;
      next_wait = k + 2;
      // plane k-1's stage is free: refill it with plane index k-1 + kStages
      if (tid == 0 && k - 1 + kStages < nq) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k - 1 + kStages);
        n_issued = k + kStages;
      }
      // x/y weights (1/2, 1, 1/2) of the coarse column over this plane
      const float* r0 = Rz + 2 * Jl * RP + 2 * Il;
      const float* r1 = r0 + RP;
      const float* r2 = r1 + RP;
      const float qv = 0.5f * fmaf(0.5f, r0[0] + r0[2], r0[1]) + fmaf(0.5f, r1[0] + r1[2], r1[1]) +
                       0.5f * fmaf(0.5f, r2[0] + r2[2], r2[1]);
      if (q & 1) {
        acc += qv;  // the centre plane of coarse K = (z - 1) / 2
      } else {
        if (kb + q > 0) {  // plane z closes coarse K = z/2 - 1
          acc = fmaf(0.5f, qv, acc);
          const int K = z / 2 - 1;
          if (cown && K < m.cnz) rc[K * cplane] = acc;
        }
        acc = 0.5f * qv;  // and opens K = z/2 (not owned when z = z1)
      }
    }
    if (zlast == z1 - 1 && (zlast & 1)) {  // the last chunk of an even axis: plane nz is outside
      const int K = (zlast - 1) / 2;
      if (cown && K < m.cnz) rc[K * cplane] = acc;
    }
  }
  return;
abort:
  if (tid == 0) {
    atomicExch(err, 1);
    for (int jq = next_wait; jq < n_issued; jq++) mbar_wait(&bars[jq % kStages], (jq / kStages) & 1);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Finest multigrid level: one damped Jacobi step out = x + omega D^-1 (rhs - A x)
// (Algorithm 2's smoother), kRho: also the partials of rho = rhs . out into
// slot m.slot of the iteration's partials (the launch then uses the iteration's
// tiling).  The box of each plane ((4 tx + 8) x (ty + 2), halo included) and
// the own rhs tile arrive by TMA in the kStages ring, as in phase B.  The
// staged field x is
//   kStage 0: xin;
//   kStage 1: omega D^-1 rhs (the box is rhs; the first step from zero).
// For kStage 1 each thread scales its own group of each plane in place when the
// copy lands, one plane ahead of the stencil, so one barrier per plane stays
// enough; the halo keeps the staged rhs and the tile's edge threads scale the
// outside neighbours they read.
// ---------------------------------------------------------------------------
template <int kStage, bool kRho>
__global__ void __launch_bounds__(256, 3)
    k_mg_smooth_tma(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_r,
                    CGArgs<float> a, MGFineArgs m, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ double red[32];
  __shared__ int s_go;
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (m.mask && !m.mask[b])) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) s_go = !*reinterpret_cast<volatile int*>(err);  // an earlier wait ran out: do not wait again
  __syncthreads();
  if (!s_go) return;
  const Geo& g = a.g;
  const int TXT = blockDim.x, TXN = TXT * 4, TY = blockDim.y;
  const int x0 = (blockIdx.x % a.tiles_x) * TXN, y0 = (blockIdx.x / a.tiles_x) * TY;
  const int z0 = blockIdx.y * a.zc, z1 = min(g.nz, z0 + a.zc);
  const int BX = TXN + 8, BY = TY + 2;
  const unsigned box_bytes = (unsigned)(BX * BY * sizeof(float)), own_bytes = (unsigned)(TXN * TY * sizeof(float));
  const int arr_floats = ((BX * BY * 4 + 127) / 128) * 32;
  const int stage_floats = arr_floats + ((TXN * TY * 4 + 127) / 128) * 32;
  float* stage_base = reinterpret_cast<float*>(smem_raw);
  auto x_tile = [&](int st) { return stage_base + st * stage_floats; };
  auto r_tile = [&](int st) { return stage_base + st * stage_floats + arr_floats; };
  const int nq = z1 - z0 + 2;
  auto issue = [&](int j) {  // the box of plane z0-1+j; the own rhs of it for planes z0 .. z1-1
    const int st = j % kStages;
    const bool with_r = j >= 1 && j <= nq - 2;
    mbar_expect_tx(&bars[st], box_bytes + (with_r ? own_bytes : 0u));
    tma_load_4d(x_tile(st), &tm_x, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    if (with_r) tma_load_4d(r_tile(st), &tm_r, x0, y0, z0 - 1 + j, b, &bars[st]);
  };
  if (tid == 0) {
    for (int st = 0; st < kStages; st++) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int n_issued = 0, next_wait = 0;
  if (tid == 0)
    for (int j = 0; j < kStages && j < nq; j++) {
      issue(j);
      n_issued = j + 1;
    }
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  const int i = x0 + lx, jn = y0 + ly;
  const bool own = i < g.nx && jn < g.ny;
  const int cofs = (ly + 1) * BX + lx + 4;
  const int lofs = ly * TXN + lx;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)jn * g.nx + i;
  float* ob = m.out + (int64_t)b * g.n;
  const float omega = m.omega;
  // kStage 1: each thread scales its own group of every staged plane in place by omega / D,
  // one plane ahead of the stencil.  The halo of the box keeps the staged rhs: a thread on
  // the tile's edge scales the outside neighbours it reads (the column x0-1 or x0+TXN, the
  // row y0-1 or y0+TY) by their omega / D as it reads them (no thread works for the halo,
  // so no warp carries extra work to the plane barrier).  Tiles are at least 2 x 2 threads.
  int own_tz = -1;  // z class of the cached omega / D of the own group
  float own_od[4] = {0.f, 0.f, 0.f, 0.f};
  const bool eW = kStage != 0 && lx == 0, eE = kStage != 0 && lx == TXN - 4;
  const bool eS = kStage != 0 && ly == 0, eN = kStage != 0 && ly == TY - 1;
  const int nbx = eW ? i - 1 : i + 4, nby = eS ? jn - 1 : jn + 1;
  const bool nbx_in = (eW || eE) && own && nbx >= 0 && nbx < g.nx;
  const bool nby_in = (eS || eN) && own && nby >= 0 && nby < g.ny;
  float odx = 0.f, ody[4] = {0.f, 0.f, 0.f, 0.f};  // omega / D of the outside neighbours (z class zcls_cur)
  // scale the own group at box offset cofs of plane z by omega / D
  auto xform = [&](float* X, int z) {
    float4 v = ld4s(X + cofs);
    const int zcl = g.cz[z];
    if (zcl != own_tz) {
      own_tz = zcl;
#pragma unroll
      for (int e = 0; e < 4; e++)
        own_od[e] = omega * cb[(((int64_t)zcl * g.ncy + g.cy[jn]) * g.ncx + g.cx[i + e]) * kCoefStride + 7];
    }
    v = make_float4(own_od[0] * v.x, own_od[1] * v.y, own_od[2] * v.z, own_od[3] * v.w);
    *reinterpret_cast<float4*>(X + cofs) = v;
    return v;
  };
  // transform plane index j's stage (own group); returns the own group
  auto xform_plane = [&](int j) -> float4 {
    const int z = z0 - 1 + j;
    float* X = x_tile(j % kStages);
    const bool zin = z >= 0 && z < g.nz;
    float4 v = ld4s(X + cofs);
    if (kStage != 0 && zin && own) v = xform(X, z);
    return v;
  };
  float rho = 0.f;
  bool timed_out = !mbar_wait(&bars[0], 0, a.wait_cycles);
  float4 xm = timed_out ? make_float4(0.f, 0.f, 0.f, 0.f) : xform_plane(0);
  if (!timed_out) timed_out = !mbar_wait(&bars[1 % kStages], (1 / kStages) & 1, a.wait_cycles);
  float4 xc = timed_out ? make_float4(0.f, 0.f, 0.f, 0.f) : xform_plane(1);
  if (__syncthreads_or(timed_out)) goto abort;
  next_wait = 2;
  if (tid == 0 && kStages < nq) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(kStages);
    n_issued = kStages + 1;
  }
  {
    float c[4][8];
    int zcls_cur = -1;
    // one plane per iteration (U = 1): groups of kStages planes, as in the residual +
    // restriction pass, measured slower here (the kStage 1 body spills when unrolled, the
    // kStage 0 steps gained nothing)
    constexpr int U = 1;
    for (int kb = 0; z0 + kb < z1; kb += U)
#pragma unroll
    for (int q = 0; q < U; q++) {
      const int z = z0 + kb + q;
      if (U > 1 && z >= z1) break;
      const int k = kb + q + 1;
      const int sk = U > 1 ? (q + 1) % kStages : k % kStages, sn = U > 1 ? (q + 2) % kStages : (k + 1) % kStages;
      const unsigned par = U > 1 ? ((kb / kStages) + (q + 2) / kStages) & 1 : ((k + 1) / kStages) & 1;
      bool to = !mbar_wait(&bars[sn], par, a.wait_cycles);
      if (!to) {
        const float4 xp = xform_plane(k + 1);  // plane z+1, own group transformed
        if (own) {
          const float4 bv = ld4s(r_tile(sk) + lofs);
          const int zcl = g.cz[z];
          if (zcl != zcls_cur) {
            zcls_cur = zcl;
            const int yc = (int)g.cy[jn];
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
#pragma unroll
              for (int q = 0; q < 8; q++) c[e][q] = row[q];
            }
            if (nbx_in) odx = omega * cb[(((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[nbx]) * kCoefStride + 7];
            if (nby_in)
#pragma unroll
              for (int e = 0; e < 4; e++)
                ody[e] = i + e < g.nx
                             ? omega * cb[(((int64_t)zcl * g.ncy + g.cy[nby]) * g.ncx + g.cx[i + e]) * kCoefStride + 7]
                             : 0.f;
          }
          const float* X = x_tile(sk);
          float left = X[cofs - 1], right = X[cofs + 4];
          float4 sth = ld4s(X + cofs - BX), nth = ld4s(X + cofs + BX);
          if (kStage != 0) {  // outside neighbours still hold the rhs: scale them now
            if (eW) left *= odx;
            if (eE) right *= odx;
            if (eS) sth = make_float4(ody[0] * sth.x, ody[1] * sth.y, ody[2] * sth.z, ody[3] * sth.w);
            if (eN) nth = make_float4(ody[0] * nth.x, ody[1] * nth.y, ody[2] * nth.z, ody[3] * nth.w);
          }
          float o4[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float xce = f4(xc, e);
            float v = c[e][6] * xce;
            v = fmaf(c[e][0], e == 0 ? left : f4(xc, e - 1), v);
            v = fmaf(c[e][1], e == 3 ? right : f4(xc, e + 1), v);
            v = fmaf(c[e][2], f4(sth, e), v);
            v = fmaf(c[e][3], f4(nth, e), v);
            v = fmaf(c[e][4], f4(xm, e), v);
            v = fmaf(c[e][5], f4(xp, e), v);
            o4[e] = fmaf(omega * c[e][7], f4(bv, e) - v, xce);
            if (kRho) rho = fmaf(f4(bv, e), o4[e], rho);
          }
          *reinterpret_cast<float4*>(ob + z * plane + col) = make_float4(o4[0], o4[1], o4[2], o4[3]);
        }
        xm = xc;
        xc = xp;
      }
      if (__syncthreads_or(to)) goto abort;
      next_wait = k + 2;
      if (tid == 0 && k + kStages < nq) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + kStages);
        n_issued = k + kStages + 1;
      }
    }
    if (kRho) {  // deterministic block sum of the rho partial
      double v = (double)rho;
      const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
      v = warp_sum_down(v);
      if (lane == 0) red[warp] = v;
      __syncthreads();
      if (warp == 0) {
        double x = lane < nw ? red[lane] : 0.0;
        x = warp_sum_down(x);
        if (lane == 0) a.rho_rr[((int64_t)m.slot * a.B + b) * a.P + blockIdx.y * gridDim.x + blockIdx.x].x = x;
      }
    }
  }
  return;
abort:
  if (tid == 0) {
    atomicExch(err, 1);
    for (int jq = next_wait; jq < n_issued; jq++) mbar_wait(&bars[jq % kStages], (jq / kStages) & 1);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The first pre-smoothing step from the staged rhs and a staged omega / D: two
// damped Jacobi steps from zero, Y = X1 + omega D^-1 (r - A X1) with X1 =
// omega D^-1 r, where omega / D per node of the finest level (od, [B][n], formed
// once per solve by k_omega_dinv) arrives by TMA beside r, so every X1 the
// stencil needs, halo included, is one product of two staged values: no pass
// scales a plane in place and no thread treats the tile's edge apart.  Reads r
// and od, writes Y: 12 B/DoF.  The products and their order are those of
// k_mg_smooth_tma<1, ...>, so its results are the same.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 3)
    k_mg_smooth_od_tma(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_d,
                       CGArgs<float> a, MGFineArgs m, int* err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ int s_go;
  const int b = blockIdx.z;
  if (a.st[b].status != ST_ACTIVE || (m.mask && !m.mask[b])) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) s_go = !*reinterpret_cast<volatile int*>(err);  // an earlier wait ran out: do not wait again
  __syncthreads();
  if (!s_go) return;
  const Geo& g = a.g;
  const int TXT = blockDim.x, TXN = TXT * 4, TY = blockDim.y;
  const int x0 = (blockIdx.x % a.tiles_x) * TXN, y0 = (blockIdx.x / a.tiles_x) * TY;
  const int z0 = blockIdx.y * a.zc, z1 = min(g.nz, z0 + a.zc);
  const int BX = TXN + 8, BY = TY + 2;
  const unsigned box_bytes = (unsigned)(BX * BY * sizeof(float));
  const int arr_floats = ((BX * BY * 4 + 127) / 128) * 32;
  float* stage_base = reinterpret_cast<float*>(smem_raw);
  auto r_box = [&](int st) { return stage_base + st * 2 * arr_floats; };
  auto d_box = [&](int st) { return stage_base + st * 2 * arr_floats + arr_floats; };
  const int nq = z1 - z0 + 2;
  auto issue = [&](int j) {  // the r and od boxes of plane z0-1+j
    const int st = j % kStages;
    mbar_expect_tx(&bars[st], 2 * box_bytes);
    tma_load_4d(r_box(st), &tm_r, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
    tma_load_4d(d_box(st), &tm_d, x0 - 4, y0 - 1, z0 - 1 + j, b, &bars[st]);
  };
  if (tid == 0) {
    for (int st = 0; st < kStages; st++) mbar_init(&bars[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int n_issued = 0, next_wait = 0;
  if (tid == 0)
    for (int j = 0; j < kStages && j < nq; j++) {
      issue(j);
      n_issued = j + 1;
    }
  const int lx = 4 * (int)threadIdx.x, ly = (int)threadIdx.y;
  const int i = x0 + lx, jn = y0 + ly;
  const bool own = i < g.nx && jn < g.ny;
  const int cofs = (ly + 1) * BX + lx + 4;
  const float* cb = a.coef + (int64_t)b * g.ncls() * kCoefStride;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const int64_t col = (int64_t)jn * g.nx + i;
  float* ob = m.out + (int64_t)b * g.n;
  auto mul4 = [](float4 u, float4 v) { return make_float4(u.x * v.x, u.y * v.y, u.z * v.z, u.w * v.w); };
  // own group of plane index j: X1 = od r, and the raw r and od
  float4 rc, dc, rp, dp;
  auto own_plane = [&](int j, float4& r4, float4& d4) -> float4 {
    const int st = j % kStages;
    r4 = ld4s(r_box(st) + cofs);
    d4 = ld4s(d_box(st) + cofs);
    return mul4(d4, r4);
  };
  bool timed_out = !mbar_wait(&bars[0], 0, a.wait_cycles);
  float4 xm = make_float4(0.f, 0.f, 0.f, 0.f), xc = xm;
  rc = dc = rp = dp = xm;
  if (!timed_out) xm = own_plane(0, rp, dp);
  if (!timed_out) timed_out = !mbar_wait(&bars[1 % kStages], (1 / kStages) & 1, a.wait_cycles);
  if (!timed_out) xc = own_plane(1, rc, dc);
  if (__syncthreads_or(timed_out)) goto abort;
  next_wait = 2;
  if (tid == 0 && kStages < nq) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(kStages);
    n_issued = kStages + 1;
  }
  {
    float c[4][7];
    int zcls_cur = -1;
    for (int z = z0; z < z1; ++z) {
      const int k = z - z0 + 1;
      const int sk = k % kStages, sn = (k + 1) % kStages;
      bool to = !mbar_wait(&bars[sn], ((k + 1) / kStages) & 1, a.wait_cycles);
      if (!to) {
        const float4 xp = own_plane(k + 1, rp, dp);  // plane z+1
        if (own) {
          const int zcl = g.cz[z];
          if (zcl != zcls_cur) {
            zcls_cur = zcl;
            const int yc = (int)g.cy[jn];
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float* row = cb + (((int64_t)zcl * g.ncy + yc) * g.ncx + g.cx[i + e]) * kCoefStride;
#pragma unroll
              for (int q = 0; q < 7; q++) c[e][q] = row[q];
            }
          }
          const float* R = r_box(sk);
          const float* D = d_box(sk);
          const float left = D[cofs - 1] * R[cofs - 1], right = D[cofs + 4] * R[cofs + 4];
          const float4 sth = mul4(ld4s(D + cofs - BX), ld4s(R + cofs - BX));
          const float4 nth = mul4(ld4s(D + cofs + BX), ld4s(R + cofs + BX));
          float o4[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float xce = f4(xc, e);
            float v = c[e][6] * xce;
            v = fmaf(c[e][0], e == 0 ? left : f4(xc, e - 1), v);
            v = fmaf(c[e][1], e == 3 ? right : f4(xc, e + 1), v);
            v = fmaf(c[e][2], f4(sth, e), v);
            v = fmaf(c[e][3], f4(nth, e), v);
            v = fmaf(c[e][4], f4(xm, e), v);
            v = fmaf(c[e][5], f4(xp, e), v);
            o4[e] = fmaf(f4(dc, e), f4(rc, e) - v, xce);
          }
          *reinterpret_cast<float4*>(ob + z * plane + col) = make_float4(o4[0], o4[1], o4[2], o4[3]);
        }
        xm = xc;
        xc = xp;
        rc = rp;
        dc = dp;
      }
      if (__syncthreads_or(to)) goto abort;
      next_wait = k + 2;
      if (tid == 0 && k + kStages < nq) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + kStages);
        n_issued = k + kStages + 1;
      }
    }
  }
  return;
abort:
  if (tid == 0) {
    atomicExch(err, 1);
    for (int jq = next_wait; jq < n_issued; jq++) mbar_wait(&bars[jq % kStages], (jq / kStages) & 1);
  }
  __syncthreads();
}

// od[b][node] = omega / D of the node (the FP32 table's reciprocal diagonal, times omega).
// Four x-consecutive nodes per thread (nx % 4 == 0, as every TMA-fed step requires), one
// 16-byte store; grid (chunks, B) with a grid-stride loop over the instance's groups.
__global__ void k_omega_dinv(Geo g, const float* __restrict__ coef32, float omega, float* __restrict__ od) {
  const int b = blockIdx.y;
  const int gx = g.nx >> 2, groups = (int)(g.n >> 2);
  const float* cb = coef32 + (int64_t)b * g.ncls() * kCoefStride;
  float4* o = reinterpret_cast<float4*>(od + (int64_t)b * g.n);
  for (int e4 = blockIdx.x * blockDim.x + threadIdx.x; e4 < groups; e4 += gridDim.x * blockDim.x) {
    const int i = (e4 % gx) * 4, row = e4 / gx;
    const int j = row % g.ny, k = row / g.ny;
    const int cyz = ((int)g.cz[k] * g.ncy + (int)g.cy[j]) * g.ncx;
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = omega * cb[(int64_t)(cyz + (int)g.cx[i + q]) * kCoefStride + 7];
    o[e4] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// Host side: tensor maps over [B][nz][ny][nx] float arrays with a box of
// (4*tx + 8) x (ty + 2) x 1 x 1 and zero fill outside the tensor.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver entry point is the same for every device: looked up once per process (the
// initialisation of a function-local static is thread-safe).
static EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

// halo = true: the (4*tx + 8) x (ty + 2) box of a stencil operand; false: the
// 4*tx x ty own tile of a streamed operand.
static int make_map_box(CUtensorMap* m, const float* base, const Geo& g, int B, int bx, int by) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || bx > 256 || by > 256 || (bx * 4) % 16) return -1;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4, (cuuint64_t)g.n * 4};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

static int make_map(CUtensorMap* m, const float* base, const Geo& g, int B, Tile t, bool halo = true) {
  return make_map_box(m, base, g, B, 4 * t.tx + (halo ? 8 : 0), t.ty + (halo ? 2 : 0));
}

// Dynamic shared memory of the ring: halo boxes per stage (2 for phase A, 1
// for phase B) and own tiles per stage (1 for the s-form phases, else 0).
static size_t ring_bytes(Tile t, int halo_boxes, int own_tiles) {
  const int BX = 4 * t.tx + 8, BY = t.ty + 2;
  const size_t arr = (size_t)((BX * BY * 4 + 127) / 128) * 128;
  const size_t own = (size_t)((4 * t.tx * t.ty * 4 + 127) / 128) * 128;
  return kStages * (halo_boxes * arr + own_tiles * own) + 128;
}

size_t tma_smem_bytes(Tile t) { return ring_bytes(t, 2, 1); }

bool tma_supported(const Geo& g, Tile t) {
  return encode_fn() != nullptr && g.nx % 4 == 0 && 4 * t.tx + 8 <= 256 && t.ty + 2 <= 256 &&
         tma_smem_bytes(t) <= 200 * 1024;
}

// Raises the TMA kernels' shared-memory limit on the current device; called before their
// launches, outside any stream capture (cheap to repeat).
void tma_prepare() {
  cudaFuncSetAttribute(k_cg_a_tma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_cg_a_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_cg_b_s_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mg_fine_rr_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mg_smooth_od_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mg_smooth_tma<0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mg_smooth_tma<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mg_smooth_tma<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int launch_mg_smooth_tma(const CGArgs<float>& a, Tile t, int stage, const MGFineArgs& m, bool rho, cudaStream_t s) {
  if (!tma_supported(a.g, t) || (rho && m.slot < 0) || (rho && stage != 0) || stage < 0 || stage > 1) return -1;
  CUtensorMap mx, mr;
  const float* boxed = stage == 1 ? m.rhs : m.xin;
  if (make_map(&mx, boxed, a.g, a.B, t) || make_map(&mr, m.rhs, a.g, a.B, t, false)) return -1;
  if (stage == 1 && m.od) {  // X1 formed from the staged omega / D (k_mg_smooth_od_tma)
    CUtensorMap md;
    if (make_map(&md, m.od, a.g, a.B, t)) return -1;
    int* err = a.active + 2;
    k_mg_smooth_od_tma<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), ring_bytes(t, 2, 0), s>>>(
        mx, md, a, m, err);
    if (cudaPeekAtLastError() != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    return 0;
  }
  if (stage == 1 && (t.tx < 2 || t.ty < 2)) return -1;  // an edge thread would face two outside neighbours
  const size_t smem = ring_bytes(t, 1, 1);
  const dim3 grid(a.tiles_x * a.tiles_y, a.nzc, a.B), block(t.tx, t.ty);
  int* err = a.active + 2;
  if (rho) k_mg_smooth_tma<0, true><<<grid, block, smem, s>>>(mx, mr, a, m, err);
  else if (stage == 0) k_mg_smooth_tma<0, false><<<grid, block, smem, s>>>(mx, mr, a, m, err);
  else k_mg_smooth_tma<1, false><<<grid, block, smem, s>>>(mx, mr, a, m, err);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

// Ring stages (x box + rhs box), two residual planes, the extra nodes' coefficients.
static size_t rr_smem_bytes(Tile t) {
  const int TXN = 4 * t.tx, PW = TXN + 8, RP = TXN + 4;
  const size_t xfl = (size_t)((PW * (t.ty + 3) * 4 + 127) / 128) * 32;
  const size_t rfl = (size_t)((RP * (t.ty + 1) * 4 + 127) / 128) * 32;
  return sizeof(float) * (kStages * (xfl + rfl) + 2 * (size_t)RP * (t.ty + 1) + (size_t)(TXN + t.ty + 1) * 8);
}

int launch_mg_fine_rr_tma(const CGArgs<float>& a, Tile t, const MGFineArgs& m, cudaStream_t s) {
  // one extra node per thread at most: the CTA needs TXN + TY + 1 threads
  if ((t.ty & 1) || (a.zc & 1) || a.g.nx % 4 || rr_smem_bytes(t) > 200 * 1024 || t.tx * t.ty < 4 * t.tx + t.ty + 1)
    return -1;
  CUtensorMap mx, mr;
  if (make_map_box(&mx, m.xin, a.g, a.B, 4 * t.tx + 8, t.ty + 3) ||
      make_map_box(&mr, m.rhs, a.g, a.B, 4 * t.tx + 4, t.ty + 1))
    return -1;
  // the error flag is the third counter of the solve (active, pending, TMA error)
  k_mg_fine_rr_tma<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), rr_smem_bytes(t), s>>>(
      mx, mr, a, m, a.active + 2);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

int launch_cg_a_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s) {
  CUtensorMap ms, m0, m1;
  const float* sarr = a.precond != RBWS_PREC_NONE ? a.s : a.r;
  if (make_map(&ms, sarr, a.g, a.B, t) || make_map(&m0, a.p0, a.g, a.B, t) || make_map(&m1, a.p1, a.g, a.B, t))
    return -1;
  // the own-tile map is unused in this mode: any valid map fills the slot
  k_cg_a_tma<0><<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), ring_bytes(t, 2, 0), s>>>(
      ms, m0, m1, ms, a, parity, err);
  return 0;
}

int launch_cg_a_s_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s) {
  CUtensorMap ms, m0, m1, mu;
  if (make_map(&ms, a.s, a.g, a.B, t) || make_map(&m0, a.p0, a.g, a.B, t) || make_map(&m1, a.p1, a.g, a.B, t) ||
      make_map(&mu, a.u, a.g, a.B, t, false))
    return -1;
  k_cg_a_tma<1><<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), ring_bytes(t, 2, 1), s>>>(
      ms, m0, m1, mu, a, parity, err);
  return 0;
}

int launch_cg_b_s_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s) {
  CUtensorMap m0, m1, ms;
  if (make_map(&m0, a.p0, a.g, a.B, t) || make_map(&m1, a.p1, a.g, a.B, t) || make_map(&ms, a.s, a.g, a.B, t, false))
    return -1;
  k_cg_b_s_tma<<<dim3(a.tiles_x * a.tiles_y, a.nzc, a.B), dim3(t.tx, t.ty), ring_bytes(t, 1, 1), s>>>(
      m0, m1, ms, a, parity, err);
  return 0;
}

}  // namespace rbws

namespace rbws {
void launch_omega_dinv(const Geo& g, const float* coef32, int B, float omega, float* od, cudaStream_t s) {
  const int64_t groups = g.n / 4;
  const unsigned chunks = (unsigned)std::min<int64_t>((groups + 255) / 256, std::max<int64_t>(1, 152 * 8 / B));
  k_omega_dinv<<<dim3(chunks, (unsigned)B), 256, 0, s>>>(g, coef32, omega, od);
}
}  // namespace rbws
