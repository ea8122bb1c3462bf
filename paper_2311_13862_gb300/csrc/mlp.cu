// mlp.cu -- the learned warm start: a fully connected network mu -> c
// (p -> H -> H -> H -> N, GELU with erf) trained on reduced Galerkin
// coefficients.  BF16 weights and activations as tensor-core operands, FP32
// accumulation and FP32 master weights for Adam.
//
// The GEMMs are tiny (batch x 256 x 256), so they are latency-bound: one
// generic kernel covers the forward (X W^T), data-gradient (dZ W) and
// weight-gradient (dZ^T X) products through strided operand addressing, with
// mma.sync m16n8k16 BF16 tensor-core instructions and a bias / GELU epilogue.
// Weight gradients are computed by one accumulator per output element in a
// fixed k order, so training is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <cuda_runtime.h>

#include "internal.h"

namespace rbws {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, BKP = BK + 8;

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float ld_any(const void* p, int is_bf16, int64_t i) {
  return is_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i])
                 : reinterpret_cast<const float*>(p)[i];
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kGemmThreads = 128;
constexpr int kStageElems = BM * BK / kGemmThreads;  // elements of a k-tile per thread and operand
static_assert(BM == BN && BM * BK % kGemmThreads == 0, "k-tile staging");

// One k-tile of both operands into registers, every load issued before any is used:
// A(m0 + r, k0 + c) and B(k0 + c, n0 + r) for the elements e = tid + 128 u (r = e / BK,
// c = e % BK), zero outside the operands.
__device__ __forceinline__ void gemm_load_tile(const MlpGemm& g, int m0, int n0, int k0, float (&va)[kStageElems],
                                               float (&vb)[kStageElems]) {
#pragma unroll
  for (int u = 0; u < kStageElems; u++) {
    const int e = threadIdx.x + kGemmThreads * u, r = e / BK, c = e % BK, m = m0 + r, k = k0 + c;
    va[u] = (m < g.M && k < g.K) ? ld_any(g.A, g.a_bf16, (int64_t)m * g.sam + (int64_t)k * g.sak) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kStageElems; u++) {
    const int e = threadIdx.x + kGemmThreads * u, r = e / BK, c = e % BK, n = n0 + r, k = k0 + c;
    vb[u] = (n < g.N && k < g.K) ? ld_any(g.B, g.b_bf16, (int64_t)k * g.sbk + (int64_t)n * g.sbn) : 0.f;
  }
}

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]); Z = C, Aout = GELU(C).
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]; operands are rounded to
// BF16 when staged in shared memory.  4 warps, 64x64 CTA tile, 32x32 per warp.  The
// next k-tile's loads are in flight while the MMAs of the current one run.
__global__ void __launch_bounds__(kGemmThreads) k_gemm_bf16(MlpGemm g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BKP];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BKP];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int k = 0; k < 4; k++) acc[i][j][k] = 0.f;
  float va[kStageElems], vb[kStageElems];
  if (g.K > 0) gemm_load_tile(g, m0, n0, 0, va, vb);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int u = 0; u < kStageElems; u++) {
      const int e = threadIdx.x + kGemmThreads * u;
      As[e / BK][e % BK] = __float2bfloat16(va[u]);
      Bs[e / BK][e % BK] = __float2bfloat16(vb[u]);
    }
    __syncthreads();
    if (k0 + BK < g.K) gemm_load_tile(g, m0, n0, k0 + BK, va, vb);
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      const int rb = wm + mt * 16;
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(&As[rb + gid][tig * 2]);
      a[1] = *reinterpret_cast<const uint32_t*>(&As[rb + gid + 8][tig * 2]);
      a[2] = *reinterpret_cast<const uint32_t*>(&As[rb + gid][tig * 2 + 8]);
      a[3] = *reinterpret_cast<const uint32_t*>(&As[rb + gid + 8][tig * 2 + 8]);
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int cb = wn + nt * 8;
        uint32_t b[2];
        b[0] = *reinterpret_cast<const uint32_t*>(&Bs[cb + gid][tig * 2]);
        b[1] = *reinterpret_cast<const uint32_t*>(&Bs[cb + gid][tig * 2 + 8]);
        mma_bf16(acc[mt][nt], a, b);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int m = m0 + wm + mt * 16 + gid + h * 8;
        if (m >= g.M) continue;
#pragma unroll
        for (int e = 0; e < 2; e++) {
          const int n = n0 + wn + nt * 8 + tig * 2 + e;
          if (n >= g.N) continue;
          float v = acc[mt][nt][h * 2 + e];
          if (g.bias) v += g.bias[n];
          g.Z[(int64_t)m * g.ldz + n] = v;
          if (g.Aout) g.Aout[(int64_t)m * g.ldz + n] = gelu_f(v);
        }
      }
}

// x[b][q] = 2 (log mu - log lo) / (log hi - log lo) - 1
__global__ void k_mlp_inputs(const double* __restrict__ mu, int B, int p, double lo, double hi,
                             float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * p) return;
  const double l0 = log(lo), l1 = log(hi);
  x[i] = (float)(2.0 * (log(mu[i]) - l0) / (l1 - l0) - 1.0);
}

// dY = 2 (Y - T) / (B N); loss partial sums per block (deterministic two-level).
__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ t, int total,
                           float scale, float* __restrict__ dy, float* __restrict__ loss_out) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const float e = y[i] - t[i];
    dy[i] = 2.f * e * scale;
    s = fmaf(e, e, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *loss_out = v * scale;
  }
}

// dZ = dA * GELU'(Z)
__global__ void k_gelu_back(const float* __restrict__ da, const float* __restrict__ z, int total,
                            float* __restrict__ dz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) dz[i] = da[i] * gelu_grad_f(z[i]);
}

// db[n] = sum_m dZ[m][n], rows in order.
__global__ void k_bias_grad(const float* __restrict__ dz, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; m++) s += dz[(int64_t)m * N + n];
  db[n] = s;
}

// Adam on the FP32 master weights; refreshes the BF16 copy.  step[0] counts.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ w16, const float* __restrict__ g,
                       float* __restrict__ m1, float* __restrict__ m2, int64_t P, float lr,
                       int* __restrict__ step) {
  const int t = *step + 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = m1[i] = b1 * m1[i] + (1.f - b1) * gi;
    const float v = m2[i] = b2 * m2[i] + (1.f - b2) * gi * gi;
    const float wi = w[i] - lr * (a * c1) / (sqrtf(v * c2) + eps);
    w[i] = wi;
    w16[i] = __float2bfloat16(wi);
  }
}

__global__ void k_adam_step(int* step) { *step += 1; }

// U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from splitmix64(seed + index) (Steele,
// Lea & Flood, 2014), 53-bit mantissa -> [0, 1).
__global__ void k_init_params(float* __restrict__ w, __nv_bfloat16* __restrict__ w16, int64_t P,
                              const int64_t* __restrict__ seg_end, const float* __restrict__ seg_bound,
                              int nseg, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    int s = 0;
    while (s < nseg - 1 && i >= seg_end[s]) s++;
    const float v = (float)((2.0 * u - 1.0) * seg_bound[s]);
    w[i] = v;
    w16[i] = __float2bfloat16(v);
  }
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16, int64_t P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16(w[i]);
}

// t[b][j] = c[b][j] / scale[j]  (float); also c (double) -> scaled targets
__global__ void k_scale_targets(const double* __restrict__ c, const float* __restrict__ scale, int B, int N,
                                float* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * N) t[i] = (float)(c[i] / (double)scale[i % N]);
}

// scale[j] = sqrt(mean_b c[b][j]^2) (1 if zero), rows in order.
__global__ void k_rms_scale(const double* __restrict__ c, int B, int N, float* __restrict__ scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int b = 0; b < B; b++) s += c[(int64_t)b * N + j] * c[(int64_t)b * N + j];
  const double r = sqrt(s / B);
  scale[j] = r > 0.0 ? (float)r : 1.f;
}

// c[b][j] = y[b][j] * scale[j] (double)
__global__ void k_unscale(const float* __restrict__ y, const float* __restrict__ scale, int B, int N,
                          double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * N) c[i] = (double)y[i] * (double)scale[i % N];
}

// One reduced CG step on A_N(mu) c = f_N from c: r = f_N - A c;
// c += (r.r / r.A r) r.  One warp per instance; A_N(mu) formed on the fly.
__global__ void k_reduced_cg_step(int N, int Q, const double* __restrict__ ANq, const double* __restrict__ fN,
                                  const double* __restrict__ mu, int B, double* __restrict__ c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wpb = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * wpb + w;
  double* r = reinterpret_cast<double*>(smem_raw) + (size_t)w * 2 * N;
  double* Ar = r + N;
  if (b >= B) return;
  const double* m = mu + (int64_t)b * Q;
  double* cb = c + (int64_t)b * N;
  auto Aentry = [&](int i, int j) {
    double s = 0.0;
    for (int q = 0; q < Q; q++) s = fma(m[q], ANq[((int64_t)q * N + i) * N + j], s);
    return s;
  };
  for (int i = lane; i < N; i += 32) {
    double s = fN[i];
    for (int j = 0; j < N; j++) s = fma(-Aentry(i, j), cb[j], s);
    r[i] = s;
  }
  __syncwarp();
  for (int i = lane; i < N; i += 32) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s = fma(Aentry(i, j), r[j], s);
    Ar[i] = s;
  }
  __syncwarp();
  if (lane == 0) {
    double rr = 0.0, rAr = 0.0;
    for (int i = 0; i < N; i++) {
      rr = fma(r[i], r[i], rr);
      rAr = fma(r[i], Ar[i], rAr);
    }
    const double alpha = rAr > 0.0 ? rr / rAr : 0.0;
    for (int i = 0; i < N; i++) cb[i] = fma(alpha, r[i], cb[i]);
  }
}

inline int blocks_for(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 152 * 8); }

}  // namespace

void launch_mlp_gemm(const MlpGemm& g, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  k_gemm_bf16<<<grid, kGemmThreads, 0, s>>>(g);
}

void launch_mlp_inputs(const double* mu, int B, int p, double lo, double hi, float* x, cudaStream_t s) {
  k_mlp_inputs<<<(B * p + 255) / 256, 256, 0, s>>>(mu, B, p, lo, hi, x);
}

void launch_mlp_loss(const float* y, const float* t, int total, float scale, float* dy, float* loss,
                     cudaStream_t s) {
  k_mlp_loss<<<1, 1024, 0, s>>>(y, t, total, scale, dy, loss);
}

void launch_gelu_back(const float* da, const float* z, int total, float* dz, cudaStream_t s) {
  k_gelu_back<<<(total + 255) / 256, 256, 0, s>>>(da, z, total, dz);
}

void launch_bias_grad(const float* dz, int M, int N, float* db, cudaStream_t s) {
  k_bias_grad<<<(N + 127) / 128, 128, 0, s>>>(dz, M, N, db);
}

void launch_adam(float* w, void* w16, const float* g, float* m1, float* m2, int64_t P, float lr, int* step,
                 cudaStream_t s) {
  k_adam<<<blocks_for(P, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16*>(w16), g, m1, m2, P, lr, step);
  k_adam_step<<<1, 1, 0, s>>>(step);
}

void launch_init_params(float* w, void* w16, int64_t P, const int64_t* seg_end, const float* seg_bound, int nseg,
                        uint64_t seed, cudaStream_t s) {
  k_init_params<<<blocks_for(P, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16*>(w16), P, seg_end,
                                                   seg_bound, nseg, seed);
}

void launch_to_bf16(const float* w, void* w16, int64_t P, cudaStream_t s) {
  k_to_bf16<<<blocks_for(P, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16*>(w16), P);
}

void launch_rms_scale(const double* c, int B, int N, float* scale, cudaStream_t s) {
  k_rms_scale<<<(N + 127) / 128, 128, 0, s>>>(c, B, N, scale);
}

void launch_scale_targets(const double* c, const float* scale, int B, int N, float* t, cudaStream_t s) {
  k_scale_targets<<<(B * N + 255) / 256, 256, 0, s>>>(c, scale, B, N, t);
}

void launch_unscale(const float* y, const float* scale, int B, int N, double* c, cudaStream_t s) {
  k_unscale<<<(B * N + 255) / 256, 256, 0, s>>>(y, scale, B, N, c);
}

void launch_reduced_cg_step(int N, int Q, const double* ANq, const double* fN, const double* mu, int B,
                            double* c, cudaStream_t s) {
  const int wpb = 4;
  k_reduced_cg_step<<<(B + wpb - 1) / wpb, 32 * wpb, sizeof(double) * 2 * N * wpb, s>>>(N, Q, ANq, fN, mu, B, c);
}

}  // namespace rbws
