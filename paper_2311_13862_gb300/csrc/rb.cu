// rb.cu -- reduced basis kernels: batched reduced Galerkin solve (Sec. 2.3),
// lift u0 = W c (Algorithm 4, line 2), and the dense helpers of the offline
// greedy (projections W^T y, Gram-Schmidt updates), in FP64; for the
// mixed-precision starts the FP32 lift (k_lift32) and the projections W^T f_b of
// per-instance sources (k_project_tc on the tensor cores with split TF32
// operands, k_project32 on the CUDA cores above N = 48), FP64 sums across runs;
// the Gaussian sources of the per-instance-source workload and the L1 indicator.
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

// One CTA per parameter: A = sum_q mu_q ANq[q] in shared memory, right-looking
// Cholesky, then the two triangular solves for c = A^{-1} fN.
__global__ void k_reduced_solve(int N, int Q, const double* __restrict__ ANq,
                                const double* __restrict__ fN, int64_t f_sb, int64_t f_sj,
                                const double* __restrict__ mu, double* __restrict__ c, int* __restrict__ info,
                                double* __restrict__ L_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // N*N
  double* x = A + N * N;                             // N
  __shared__ int bad;
  const int b = blockIdx.x;
  const double* m = mu + (int64_t)b * Q;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < Q; q++) s = fma(m[q], ANq[(int64_t)q * N * N + e], s);
    A[e] = s;
  }
  for (int e = threadIdx.x; e < N; e += blockDim.x) x[e] = fN[(int64_t)b * f_sb + (int64_t)e * f_sj];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < N; j++) {
    if (threadIdx.x == 0) {
      const double d = A[j * N + j];
      if (!(d > 0.0)) bad = 1;
      A[j * N + j] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double ljj = A[j * N + j];
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) A[i * N + j] /= ljj;
    __syncthreads();
    const int m2 = N - j - 1;
    for (int e = threadIdx.x; e < m2 * m2; e += blockDim.x) {
      const int i = j + 1 + e / m2, k = j + 1 + e % m2;
      if (k <= i) A[i * N + k] = fma(-A[i * N + j], A[k * N + j], A[i * N + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < N; i++) {  // L y = f
      double s = x[i];
      for (int k = 0; k < i; k++) s = fma(-A[i * N + k], x[k], s);
      x[i] = s / A[i * N + i];
    }
    for (int i = N - 1; i >= 0; i--) {  // L^T c = y
      double s = x[i];
      for (int k = i + 1; k < N; k++) s = fma(-A[k * N + i], x[k], s);
      x[i] = s / A[i * N + i];
    }
    info[b] = bad ? -1 : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N; e += blockDim.x) c[(int64_t)b * N + e] = x[e];
  if (L_out)
    for (int e = threadIdx.x; e < N * N; e += blockDim.x)
      L_out[(int64_t)b * N * N + e] = (e % N) <= (e / N) ? A[e] : 0.0;
}

// u[b][i] = sum_j c[b][j] W[j][i]; each thread one node for kLiftB instances.
constexpr int kLiftB = 8;
__global__ void k_lift(int64_t n, int N, const double* __restrict__ W, const double* __restrict__ c,
                       int B, double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* cs = reinterpret_cast<double*>(smem_raw);  // [kLiftB][N]
  const int b0 = blockIdx.y * kLiftB;
  const int nb = min(kLiftB, B - b0);
  for (int e = threadIdx.x; e < nb * N; e += blockDim.x) cs[e] = c[(int64_t)b0 * N + e];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc[kLiftB];
#pragma unroll
    for (int k = 0; k < kLiftB; k++) acc[k] = 0.0;
    for (int j = 0; j < N; j++) {
      const double w = W[(int64_t)j * n + i];
#pragma unroll
      for (int k = 0; k < kLiftB; k++) acc[k] = fma(cs[k * N + j], w, acc[k]);
    }
    for (int k = 0; k < nb; k++) u[(int64_t)(b0 + k) * n + i] = acc[k];
  }
}

// The same with an FP32 copy of W and FP32 accumulation (u to about 1e-7
// relative: the start of the mixed-precision solver, whose FP64 residual is
// formed from the u actually written).
__global__ void k_lift32(int64_t n, int N, const float* __restrict__ W, const double* __restrict__ c, int B,
                         double* __restrict__ u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* cs = reinterpret_cast<float*>(smem_raw);  // [kLiftB][N]
  const int b0 = blockIdx.y * kLiftB;
  const int nb = min(kLiftB, B - b0);
  for (int e = threadIdx.x; e < nb * N; e += blockDim.x) cs[e] = (float)c[(int64_t)b0 * N + e];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc[kLiftB];
#pragma unroll
    for (int k = 0; k < kLiftB; k++) acc[k] = 0.f;
    for (int j = 0; j < N; j++) {
      const float w = W[(int64_t)j * n + i];
#pragma unroll
      for (int k = 0; k < kLiftB; k++) acc[k] = fmaf(cs[k * N + j], w, acc[k]);
    }
    for (int k = 0; k < nb; k++) u[(int64_t)(b0 + k) * n + i] = (double)acc[k];
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// Stage 1 of out[k] = X[k].y: partial sums over fixed chunks.
__global__ void k_dot_stage1(int64_t n, const double* __restrict__ X, int64_t ldx,
                             const double* __restrict__ y, double* __restrict__ part, int chunks) {
  __shared__ double red[32];
  const int k = blockIdx.y;
  const double* xk = X + (int64_t)k * ldx;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)chunks * blockDim.x)
    s = fma(xk[i], y[i], s);
  s = warp_sum_down(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum_down(v);
    if (lane == 0) part[(int64_t)k * chunks + blockIdx.x] = v;
  }
}

__global__ void k_dot_stage2(const double* __restrict__ part, int chunks, int K,
                             double* __restrict__ out) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  double s = 0.0;
  for (int c = lane; c < chunks; c += 32) s += part[(int64_t)k * chunks + c];
  s = warp_sum_down(s);
  if (lane == 0) out[k] = s;
}

__global__ void k_sub_combination(int64_t n, int K, const double* __restrict__ W,
                                  const double* __restrict__ coef, double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = w[i];
    for (int j = 0; j < K; j++) v = fma(-coef[j], W[(int64_t)j * n + i], v);
    w[i] = v;
  }
}

__global__ void k_scale_inv(int64_t n, const double* __restrict__ alpha, double* __restrict__ w) {
  const double s = 1.0 / alpha[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] *= s;
}

__global__ void k_norms_from_partials(const double* __restrict__ part, int B, int P, double fnorm,
                                      const double* __restrict__ fnorms, double* __restrict__ out) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  double s = 0.0;
  for (int c = lane; c < P; c += 32) s += part[(int64_t)b * P + c];
  s = warp_sum_down(s);
  if (lane == 0) out[b] = sqrt(s) / (fnorms ? fnorms[b] : fnorm);
}

// out[b] = ||X[b]||_2 for rows of length n, stride ldx (one CTA per row, FP64).
__global__ void k_row_norms(int64_t n, const double* __restrict__ X, int64_t ldx, double* __restrict__ out) {
  __shared__ double red[32];
  const double* x = X + (int64_t)blockIdx.x * ldx;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  s = warp_sum_down(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    s = warp_sum_down(s);
    if (lane == 0) out[blockIdx.x] = sqrt(s);
  }
}

// f[b][node] = exp(-|x(node) - c_b|^2 / (2 s_b^2)) at the interior nodes x = ((i+1) hx,
// (j+1) hy, (k+1) hz); prm[b] = (c_x, c_y, c_z, s_b).
// f[b] = (offset + amplitude exp(-|x - c|^2 / width)) times the node's relative control
// volume; prm [B][6] = (c_x, c_y, c_z, width, amplitude, offset).  Node coordinates along an
// axis: (i+1)/(n+1), or (i+1)/n on an axis with a Neumann face (nm = 1), where the last
// node has half a control volume.
__global__ void k_gaussian_source(int nx, int ny, int nz, int nmx, int nmy, int nmz, const double* __restrict__ prm,
                                  double* __restrict__ f) {
  const int b = blockIdx.y;
  const int64_t n = (int64_t)nx * ny * nz;
  const double* pr = prm + 6 * b;
  const double cx = pr[0], cy = pr[1], cz = pr[2], amp = pr[4], off = pr[5];
  const double hx = 1.0 / (nmx ? nx : nx + 1), hy = 1.0 / (nmy ? ny : ny + 1), hz = 1.0 / (nmz ? nz : nz + 1);
  const double inv = 1.0 / pr[3];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((int64_t)nx * ny));
    const double dx = (i + 1) * hx - cx, dy = (j + 1) * hy - cy, dz = (k + 1) * hz - cz;
    const double w = (nmx && i == nx - 1 ? 0.5 : 1.0) * (nmy && j == ny - 1 ? 0.5 : 1.0) *
                     (nmz && k == nz - 1 ? 0.5 : 1.0);
    f[(int64_t)b * n + t] = (off + amp * exp(-(dx * dx + dy * dy + dz * dz) * inv)) * w;
  }
}

// eta[b] = || R^{-1} c[b] ||_1 (R upper triangular [Nmax][Nmax]): the L1 norm of
// the RB coefficients with respect to the unorthogonalised snapshots.  An
// instance whose reduced solve failed (info[b] != 0) gets +inf.
__global__ void k_l1_indicator(int N, int Nmax, const double* __restrict__ R, const double* __restrict__ c,
                               const int* __restrict__ info, int B, double* __restrict__ eta) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (info[b] != 0) {
    eta[b] = INFINITY;
    return;
  }
  double x[160];
  const double* cb = c + (int64_t)b * N;
  double l1 = 0.0;
  for (int i = N - 1; i >= 0; i--) {
    double s = cb[i];
    for (int k = i + 1; k < N; k++) s = fma(-R[i * Nmax + k], x[k], s);
    x[i] = s / R[i * Nmax + i];
    l1 += fabs(x[i]);
  }
  eta[b] = l1;
}

// The reduced right-hand sides of per-instance sources for the mixed-precision start,
// FN[j][b] = (W^T f_b)_j, from the FP32 copy of W: products of FP32 values, summed in FP32
// over runs of kProjRun nodes and in FP64 across runs.  A CTA takes kProjInst instances
// (one per lane) and one split of the nodes; warp w accumulates the basis vectors
// j = w, w + 8, ... (JPT of them).  The run's sources are staged node-major (row pitch
// kProjInst + 1: no bank conflicts), W row-major; part[s][j][b] receives the split's sum.
constexpr int kProjRun = 128;
constexpr int kProjInst = 32;
template <int JPT>
__global__ void __launch_bounds__(256) k_project32(int64_t n, int N, int B, const float* __restrict__ W,
                                                  const double* __restrict__ F, int64_t ldf, int64_t per_split,
                                                  double* __restrict__ part) {
  __shared__ float Fs[kProjRun][kProjInst + 1];
  extern __shared__ __align__(16) float Ws[];  // [N][kProjRun]
  const int sp = blockIdx.x, b0 = blockIdx.y * kProjInst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t lo = (int64_t)sp * per_split, hi = min(n, lo + per_split);
  double acc[JPT];
#pragma unroll
  for (int q = 0; q < JPT; q++) acc[q] = 0.0;
  for (int64_t i0 = lo; i0 < hi; i0 += kProjRun) {
    const int len = (int)min((int64_t)kProjRun, hi - i0);
#pragma unroll 4
    for (int e = tid; e < kProjInst * kProjRun; e += 256) {
      const int r = e / kProjRun, c = e % kProjRun, bb = b0 + r;
      Fs[c][r] = (bb < B && c < len) ? (float)F[(int64_t)bb * ldf + i0 + c] : 0.f;
    }
    for (int e = tid; e < N * kProjRun; e += 256) {
      const int j = e / kProjRun, c = e % kProjRun;
      Ws[e] = c < len ? W[(int64_t)j * n + i0 + c] : 0.f;
    }
    __syncthreads();
    float a32[JPT];
#pragma unroll
    for (int q = 0; q < JPT; q++) a32[q] = 0.f;
    for (int c = 0; c < kProjRun; c += 4) {
      const float f0 = Fs[c][lane], f1 = Fs[c + 1][lane], f2 = Fs[c + 2][lane], f3 = Fs[c + 3][lane];
#pragma unroll
      for (int q = 0; q < JPT; q++) {
        const int j = warp + 8 * q;
        if (j < N) {
          const float4 w4 = *reinterpret_cast<const float4*>(Ws + j * kProjRun + c);
          a32[q] = fmaf(w4.x, f0, a32[q]);
          a32[q] = fmaf(w4.y, f1, a32[q]);
          a32[q] = fmaf(w4.z, f2, a32[q]);
          a32[q] = fmaf(w4.w, f3, a32[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < JPT; q++) acc[q] += (double)a32[q];
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < JPT; q++) {
    const int j = warp + 8 * q;
    if (j < N && b0 + lane < B) part[((int64_t)sp * N + j) * B + b0 + lane] = acc[q];
  }
}

// ---------------------------------------------------------------------------
// The same projection on the tensor cores (mma.sync m16n8k8, TF32 operands, FP32
// accumulation), for N <= 48 (its staging ring is static shared memory, 48 KB at most).  part[s][j][b] = sum over split s of W[j][i] F[b][i]:
// an M x Nb x K product with M = N (padded to 16 MT rows), Nb = 64 instances per CTA
// (8 per warp) and K = the split's nodes.  Each operand is split into a TF32 high part
// and the TF32 rounding of the rest, and the product keeps hi*hi + hi*lo + lo*hi (three
// MMAs), which carries about 21 significant bits: the accuracy of FP32 products.  The
// sources arrive in FP64 and are rounded to FP32 with integer operations (the FP64 pipe
// is slow on this part).  FP32 sums over runs of 128 nodes, FP64 across runs, as in
// k_project32.  Tiles of 32 nodes are staged by cp.async into a two-stage ring.
// ---------------------------------------------------------------------------
constexpr int kPtcK = 32;      // nodes per staged tile
constexpr int kPtcInst = 64;   // instances per CTA
constexpr int kPtcFp = kPtcK + 2;   // pitch (doubles) of a staged source row
constexpr int kPtcWp = kPtcK + 4;   // pitch (floats) of a staged W row

__device__ __forceinline__ float f64_to_f32_int(double x) {
  // round toward zero to FP32 with integer operations; zero below the normal range
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(bits >> 32), lw = (unsigned)bits;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return 0.f;
  if (e >= 255) return __uint_as_float((hw & 0x80000000u) | 0x7f800000u);
  return __uint_as_float((hw & 0x80000000u) | ((unsigned)e << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
}

__device__ __forceinline__ void tf32_split(float a, unsigned& hi, unsigned& lo) {
  const unsigned h = __float_as_uint(a) & 0xffffe000u;  // the 10 mantissa bits the MMA reads
  hi = h;
  lo = __float_as_uint(a - __uint_as_float(h)) & 0xffffe000u;
}

__device__ __forceinline__ void mma_tf32(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}

template <int MT>
__global__ void __launch_bounds__(256) k_project_tc(int64_t n, int N, int B, const float* __restrict__ W,
                                                   const double* __restrict__ F, int64_t ldf, int64_t per_split,
                                                   double* __restrict__ part) {
  __shared__ __align__(16) double Fs[2][kPtcInst][kPtcFp];
  __shared__ __align__(16) float Ws[2][MT * 16][kPtcWp];
  const int sp = blockIdx.x, b0 = blockIdx.y * kPtcInst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const int64_t lo = (int64_t)sp * per_split, hi = min(n, lo + per_split);
  const int ntile = (int)((hi - lo + kPtcK - 1) / kPtcK);
  // stage tile t (nodes lo + t*32 ..): sources of 64 instances (16-byte chunks of two
  // doubles) and W rows (chunks of four floats); past the end of the split, or of B / N,
  // the chunk is zero-filled
  auto stage = [&](int t, int buf) {
    const int64_t i0 = lo + (int64_t)t * kPtcK;
    for (int c = tid; c < kPtcInst * (kPtcK / 2); c += 256) {
      const int r = c / (kPtcK / 2), col = 2 * (c % (kPtcK / 2));
      const int bb = b0 + r;
      const int64_t i = i0 + col;
      int bytes = 0;
      if (bb < B && i < hi) bytes = i + 1 < hi ? 16 : 8;
      const double* src = bytes ? F + (int64_t)bb * ldf + i : F;
      cp_async16(&Fs[buf][r][col], src, bytes);
    }
    for (int c = tid; c < MT * 16 * (kPtcK / 4); c += 256) {
      const int j = c / (kPtcK / 4), col = 4 * (c % (kPtcK / 4));
      const int64_t i = i0 + col;
      int bytes = 0;
      if (j < N && i < hi) bytes = (int)min((int64_t)16, (hi - i) * 4);
      const float* src = bytes ? W + (int64_t)j * n + i : W;
      cp_async16(&Ws[buf][j][col], src, bytes);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float c[MT][4];
  double acc[MT][4];
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int q = 0; q < 4; q++) c[m][q] = 0.f, acc[m][q] = 0.0;
  if (ntile > 0) stage(0, 0);
  for (int t = 0; t < ntile; t++) {
    const int buf = t & 1;
    if (t + 1 < ntile) {
      stage(t + 1, buf ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kPtcK / 8; ks++) {
      const int k0 = ks * 8;
      // B fragment (8 x 8, column major): B[k][nn] = F[b0 + 8 warp + nn][k0 + k]
      unsigned bh[2], bl[2];
      tf32_split(f64_to_f32_int(Fs[buf][8 * warp + g][k0 + tig]), bh[0], bl[0]);
      tf32_split(f64_to_f32_int(Fs[buf][8 * warp + g][k0 + tig + 4]), bh[1], bl[1]);
#pragma unroll
      for (int m = 0; m < MT; m++) {
        // A fragment (16 x 8, row major): A[r][k] = W[16 m + r][k0 + k]
        unsigned ah[4], al[4];
        tf32_split(Ws[buf][16 * m + g][k0 + tig], ah[0], al[0]);
        tf32_split(Ws[buf][16 * m + g + 8][k0 + tig], ah[1], al[1]);
        tf32_split(Ws[buf][16 * m + g][k0 + tig + 4], ah[2], al[2]);
        tf32_split(Ws[buf][16 * m + g + 8][k0 + tig + 4], ah[3], al[3]);
        mma_tf32(c[m], al, bh);
        mma_tf32(c[m], ah, bl);
        mma_tf32(c[m], ah, bh);
      }
    }
    // FP32 runs of 128 nodes (4 tiles), FP64 across runs
    if ((t & 3) == 3 || t + 1 == ntile) {
#pragma unroll
      for (int m = 0; m < MT; m++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[m][q] += (double)c[m][q], c[m][q] = 0.f;
    }
    __syncthreads();  // the buffer is refilled by the next iteration's stage
  }
  // D fragment: (row g, cols 2 tig, 2 tig + 1) and (row g + 8, same cols)
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int j = 16 * m + g + (q >= 2 ? 8 : 0);
      const int bb = b0 + 8 * warp + 2 * tig + (q & 1);
      if (j < N && bb < B) part[((int64_t)sp * N + j) * B + bb] = acc[m][q];
    }
}

// FN[j * B + b] = sum over the S splits, in split order.
__global__ void k_project_reduce(int S, int N, int B, const double* __restrict__ part, double* __restrict__ FN) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * B) return;
  double v = 0.0;
  for (int sp = 0; sp < S; sp++) v += part[(int64_t)sp * N * B + t];
  FN[t] = v;
}

inline int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

void launch_reduced_solve(int N, int Q, const double* ANq, const double* fN, const double* mu, int B,
                          double* c, int* info, double* L_out, cudaStream_t s, int64_t f_sb, int64_t f_sj) {
  const size_t smem = sizeof(double) * ((size_t)N * N + N);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_reduced_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_reduced_solve<<<B, 128, smem, s>>>(N, Q, ANq, fN, f_sb, f_sj, mu, c, info, L_out);
}

void launch_l1_indicator(int N, int Nmax, const double* R, const double* c, const int* info, int B,
                         double* eta, cudaStream_t s) {
  k_l1_indicator<<<(B + 127) / 128, 128, 0, s>>>(N, Nmax, R, c, info, B, eta);
}

void launch_lift(int64_t n, int N, const double* W, const double* c, int B, double* u,
                 cudaStream_t s) {
  const int threads = 256;
  dim3 grid(grid_for(n, threads, 152 * 4), (B + kLiftB - 1) / kLiftB);
  k_lift<<<grid, threads, sizeof(double) * kLiftB * N, s>>>(n, N, W, c, B, u);
}

void launch_lift32(int64_t n, int N, const float* W, const double* c, int B, double* u, cudaStream_t s) {
  const int threads = 256;
  dim3 grid(grid_for(n, threads, 152 * 4), (B + kLiftB - 1) / kLiftB);
  k_lift32<<<grid, threads, sizeof(float) * kLiftB * N, s>>>(n, N, W, c, B, u);
}

void launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  k_to_f32<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(n, x, y);
}

void launch_multi_dot(int64_t n, int K, const double* X, int64_t ldx, const double* y, double* out,
                      double* scratch, int scratch_len, cudaStream_t s) {
  int chunks = 256;
  while ((int64_t)chunks * K > scratch_len && chunks > 1) chunks /= 2;
  k_dot_stage1<<<dim3(chunks, K), 256, 0, s>>>(n, X, ldx, y, scratch, chunks);
  k_dot_stage2<<<(K + 3) / 4, 128, 0, s>>>(scratch, chunks, K, out);
}

void launch_sub_combination(int64_t n, int K, const double* W, const double* coef, double* w,
                            cudaStream_t s) {
  k_sub_combination<<<grid_for(n, 256), 256, 0, s>>>(n, K, W, coef, w);
}

void launch_scale_inv(int64_t n, const double* alpha, double* w, cudaStream_t s) {
  k_scale_inv<<<grid_for(n, 256), 256, 0, s>>>(n, alpha, w);
}

void launch_norms_from_partials(const double* part, int B, int P, double fnorm, double* out,
                                cudaStream_t s, const double* fnorms) {
  k_norms_from_partials<<<(B + 3) / 4, 128, 0, s>>>(part, B, P, fnorm, fnorms, out);
}

void launch_row_norms(int64_t n, int B, const double* X, int64_t ldx, double* out, cudaStream_t s) {
  if (B > 0) k_row_norms<<<B, 256, 0, s>>>(n, X, ldx, out);
}

// Splits of the nodes: the CUDA-core kernel's (32-instance groups) and the tensor-core
// kernel's (64-instance groups), each about four CTAs per SM.
int splits_cc(int64_t n, int B) {
  const int groups = (B + kProjInst - 1) / kProjInst;
  int64_t S = std::max<int64_t>(1, (4 * 152 + groups - 1) / groups);
  S = std::min<int64_t>(S, (n + kProjRun - 1) / kProjRun);
  return (int)std::max<int64_t>(S, 1);
}
int splits_tc(int64_t n, int B) {
  const int groups = (B + kPtcInst - 1) / kPtcInst;
  return (int)std::max<int64_t>(1, std::min<int64_t>((4 * 152 + groups - 1) / groups, n / (4 * kPtcK)));
}

// The partial sums' scratch is sized for either kernel.
int project32_splits(int64_t n, int B) { return std::max(splits_cc(n, B), splits_tc(n, B)); }

int launch_project32(int64_t n, int N, int B, const float* W, const double* F, int64_t ldf, double* part,
                     double* FN, cudaStream_t s) {
  if (N < 1 || N > 160 || B < 1) return -1;
  // the tensor-core kernel needs 16-byte aligned rows for its cp.async chunks
  const bool tc = N <= 48 && n % 4 == 0 && ldf % 2 == 0 && (reinterpret_cast<uintptr_t>(F) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  if (tc) {
    const int S = splits_tc(n, B);
    int64_t per = (n + S - 1) / S;
    per = (per + kPtcK - 1) / kPtcK * kPtcK;
    const int Sused = (int)((n + per - 1) / per);
    const dim3 grid((unsigned)Sused, (unsigned)((B + kPtcInst - 1) / kPtcInst));
    const int MT = (N + 15) / 16;
    if (MT == 1) k_project_tc<1><<<grid, 256, 0, s>>>(n, N, B, W, F, ldf, per, part);
    else if (MT == 2) k_project_tc<2><<<grid, 256, 0, s>>>(n, N, B, W, F, ldf, per, part);
    else k_project_tc<3><<<grid, 256, 0, s>>>(n, N, B, W, F, ldf, per, part);
    k_project_reduce<<<(N * B + 255) / 256, 256, 0, s>>>(Sused, N, B, part, FN);
    return 0;
  }
  const int S = splits_cc(n, B);
  int64_t per = (n + S - 1) / S;
  per = (per + kProjRun - 1) / kProjRun * kProjRun;
  const int Sused = (int)((n + per - 1) / per);
  const dim3 grid((unsigned)Sused, (unsigned)((B + kProjInst - 1) / kProjInst));
  const size_t smem = sizeof(float) * (size_t)N * kProjRun;
  // The shared-memory limit is a per-device attribute of each kernel: set it on every call
  // (cheap), so a problem on any device, and concurrent callers, launch with it raised.
  auto raise = [](const void* k) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024); };
  if (smem > 48 * 1024) {
    if (N <= 16) raise((const void*)k_project32<2>);
    else if (N <= 40) raise((const void*)k_project32<5>);
    else if (N <= 80) raise((const void*)k_project32<10>);
    else raise((const void*)k_project32<20>);
  }
  if (N <= 16) k_project32<2><<<grid, 256, smem, s>>>(n, N, B, W, F, ldf, per, part);
  else if (N <= 40) k_project32<5><<<grid, 256, smem, s>>>(n, N, B, W, F, ldf, per, part);
  else if (N <= 80) k_project32<10><<<grid, 256, smem, s>>>(n, N, B, W, F, ldf, per, part);
  else k_project32<20><<<grid, 256, smem, s>>>(n, N, B, W, F, ldf, per, part);
  k_project_reduce<<<(N * B + 255) / 256, 256, 0, s>>>(Sused, N, B, part, FN);
  return 0;
}

void launch_gaussian_source(int nx, int ny, int nz, const int* neumann, const double* prm, int B, double* f,
                            cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (B > 0)
    k_gaussian_source<<<dim3(blocks, B), 256, 0, s>>>(nx, ny, nz, neumann[0], neumann[1], neumann[2], prm, f);
}

}  // namespace rbws
