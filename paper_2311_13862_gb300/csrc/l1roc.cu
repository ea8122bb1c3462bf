// l1roc.cu -- device kernels of the L1-based reduced over-collocation method
// (L1ROC, Sec. 3.1): the DEIM point search (largest |entry|), gathers of
// vector entries at collocation nodes, and the batched over-collocation
// least-squares solve min_c ||P (f - A(mu) W c)||_2 by Householder QR.
#include <cmath>

#include "internal.h"

namespace rbws {
namespace {

// (value, index) of the largest |v[i]| over a chunk; ties keep the smaller index.
__device__ __forceinline__ void amax_merge(double& v, int64_t& i, double v2, int64_t i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__device__ __forceinline__ void amax_block(double& v, int64_t& i) {
  __shared__ double sv[32];
  __shared__ int64_t si[32];
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int64_t i2 = __shfl_down_sync(0xffffffffu, i, o);
    amax_merge(v, i, v2, i2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    sv[warp] = v;
    si[warp] = i;
  }
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sv[lane] : -1.0;
    i = lane < nw ? si[lane] : INT64_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_down_sync(0xffffffffu, v, o);
      const int64_t i2 = __shfl_down_sync(0xffffffffu, i, o);
      amax_merge(v, i, v2, i2);
    }
  }
}

__global__ void k_amax_stage1(int64_t n, const double* __restrict__ x, int chunks, double* pv, int64_t* pi) {
  const int64_t per = (n + chunks - 1) / chunks;
  const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
  double v = -1.0;
  int64_t i = INT64_MAX;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) amax_merge(v, i, fabs(x[t]), t);
  amax_block(v, i);
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = v;
    pi[blockIdx.x] = i;
  }
}

__global__ void k_amax_stage2(int chunks, const double* __restrict__ pv, const int64_t* __restrict__ pi,
                              const double* __restrict__ x, int64_t* out_idx, double* out_val) {
  double v = -1.0;
  int64_t i = INT64_MAX;
  for (int t = threadIdx.x; t < chunks; t += blockDim.x) amax_merge(v, i, pv[t], pi[t]);
  amax_block(v, i);
  if (threadIdx.x == 0) {
    *out_idx = i;
    *out_val = v;  // max |x| (the first pass)
  }
}

// Second pass: the smallest index with |x| >= (1 - 1e-8) max |x| (near-ties
// resolve to the smaller index whatever the rounding).
__global__ void k_amax_first(int64_t n, const double* __restrict__ x, const double* __restrict__ vmax, int chunks,
                             int64_t* pi) {
  const double thr = (1.0 - 1e-8) * *vmax;
  const int64_t per = (n + chunks - 1) / chunks;
  const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
  int64_t i = INT64_MAX;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x)
    if (fabs(x[t]) >= thr) i = min(i, t);
  for (int o = 16; o > 0; o >>= 1) i = min(i, __shfl_down_sync(0xffffffffu, i, o));
  __shared__ int64_t si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) si[warp] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t m = INT64_MAX;
    for (int w = 0; w < nw; w++) m = min(m, si[w]);
    pi[blockIdx.x] = m;
  }
}

__global__ void k_amax_first_final(int chunks, const int64_t* __restrict__ pi, const double* __restrict__ x,
                                   int64_t* out_idx, double* out_val) {
  if (threadIdx.x != 0) return;
  int64_t m = INT64_MAX;
  for (int t = 0; t < chunks; t++) m = min(m, pi[t]);
  *out_idx = m;
  *out_val = x[m];  // signed entry at the point
}

// out[t] = X[col[t] * ld + idx[t]] (0 where idx[t] < 0).
__global__ void k_gather(const double* __restrict__ X, int64_t ld, const int* __restrict__ col,
                         const int64_t* __restrict__ idx, int L, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L) return;
  out[t] = idx[t] >= 0 ? X[(int64_t)col[t] * ld + idx[t]] : 0.0;
}

// One instance per CTA: G = sum_q mu_q PAWq[q] (M x N), g = Pf; Householder QR of
// [G | g] column by column (one warp per column update), then R c = Q^T g.
// info[b] = 1 if a diagonal entry of R vanishes (rank deficiency).
__global__ void k_colloc_ls(int M, int N, int Q, const double* __restrict__ PAWq, const double* __restrict__ Pf,
                            const double* __restrict__ mu, double* __restrict__ c, int* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* G = reinterpret_cast<double*>(smem_raw);  // column-major [N + 1][M]; column N = g
  __shared__ double s_alpha, s_vn2;
  __shared__ int s_bad;
  const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < M * N; e += nt) {
    const int i = e / N, j = e % N;
    double v = 0.0;
    for (int q = 0; q < Q; q++) v = fma(mu[(int64_t)b * Q + q], PAWq[((int64_t)q * M + i) * N + j], v);
    G[(int64_t)j * M + i] = v;
  }
  for (int i = tid; i < M; i += nt) G[(int64_t)N * M + i] = Pf[i];
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < N; k++) {
    double* ck = G + (int64_t)k * M;
    if (warp == 0) {
      double sg = 0.0;
      for (int i = k + 1 + lane; i < M; i += 32) sg = fma(ck[i], ck[i], sg);
      for (int o = 16; o > 0; o >>= 1) sg += __shfl_down_sync(0xffffffffu, sg, o);
      if (lane == 0) {
        const double x0 = ck[k];
        const double nrm = sqrt(sg + x0 * x0);
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        s_alpha = alpha;
        s_vn2 = sg + v0 * v0;
        ck[k] = v0;  // the reflector's first entry (its others are the column below)
        if (!(nrm > 0.0)) s_bad = 1;
      }
    }
    __syncthreads();
    const double vn2 = s_vn2;
    if (vn2 > 0.0)
      for (int j = k + 1 + warp; j <= N; j += nw) {  // columns right of k and the right-hand side
        double* cj = G + (int64_t)j * M;
        double t = 0.0;
        for (int i = k + lane; i < M; i += 32) t = fma(ck[i], cj[i], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const double f = 2.0 * t / vn2;
        for (int i = k + lane; i < M; i += 32) cj[i] = fma(-f, ck[i], cj[i]);
      }
    __syncthreads();
    if (tid == 0) ck[k] = s_alpha;  // R[k][k]
    __syncthreads();
  }
  if (tid == 0) {
    double* cb = c + (int64_t)b * N;
    for (int k = N - 1; k >= 0; k--) {
      double v = G[(int64_t)N * M + k];
      for (int j = k + 1; j < N; j++) v = fma(-G[(int64_t)j * M + k], cb[j], v);
      cb[k] = v / G[(int64_t)k * M + k];
    }
    info[b] = s_bad;
  }
}

}  // namespace

void launch_argmax_abs(int64_t n, const double* x, double* scratch_v, int64_t* scratch_i, int chunks,
                       int64_t* out_idx, double* out_val, cudaStream_t s) {
  k_amax_stage1<<<chunks, 256, 0, s>>>(n, x, chunks, scratch_v, scratch_i);
  k_amax_stage2<<<1, 256, 0, s>>>(chunks, scratch_v, scratch_i, x, out_idx, out_val);  // out_val = max |x|
  k_amax_first<<<chunks, 256, 0, s>>>(n, x, out_val, chunks, scratch_i);
  k_amax_first_final<<<1, 32, 0, s>>>(chunks, scratch_i, x, out_idx, out_val);
}

void launch_gather(const double* X, int64_t ld, const int* col, const int64_t* idx, int L, double* out,
                   cudaStream_t s) {
  if (L > 0) k_gather<<<(L + 255) / 256, 256, 0, s>>>(X, ld, col, idx, L, out);
}

size_t colloc_ls_smem(int M, int N) { return sizeof(double) * (size_t)(N + 1) * M; }

void colloc_ls_prepare() {
  cudaFuncSetAttribute(k_colloc_ls, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_colloc_ls(int M, int N, int Q, const double* PAWq, const double* Pf, const double* mu, int B, double* c,
                      int* info, cudaStream_t s) {
  k_colloc_ls<<<B, 128, colloc_ls_smem(M, N), s>>>(M, N, Q, PAWq, Pf, mu, c, info);
}

}  // namespace rbws
