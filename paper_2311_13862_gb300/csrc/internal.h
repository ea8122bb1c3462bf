// internal.h -- shared declarations of librbws (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rbws.h"

namespace rbws {

// ---------------------------------------------------------------------------
// Geometry and coefficient classes.
//
// With block-constant kappa, the seven coefficients of a node's stencil row
// depend only on which block the node and each of its neighbours lie in (or
// whether a neighbour is on the boundary).  Along one axis a node's "class"
// is the triple (own block, lower neighbour's block or -1, upper neighbour's
// block or -1); a node's full class is (z class, y class, x class).  There
// are at most 3b+2 classes per axis, so each instance's coefficients fit in a
// small table [ncz][ncy][ncx] of 8 values:
//   -kW, -kE, -kS, -kN, -kD, -kU  (negated face coefficients, 1/h^2 included),
//   D = kW+kE+kS+kN+kD+kU,  Dinv = 1/D.
// The stencil is then y = D x_c + sum_f (-k_f) x_f: 1 multiply + 6 FMAs.
// ---------------------------------------------------------------------------
constexpr int kCoefStride = 8;  // values per class entry
constexpr int kMaxQ = 64;
constexpr int kMaxAxis = 1024;
constexpr int kL1RocMaxN = 64;  // L1ROC basis size limit (collocation solve in shared memory)
constexpr int kMaxClassPerAxis = 3 * 16 + 2;

struct AxisClasses {
  int n = 0, b = 0;           // nodes, segments (blocks) along the axis
  std::vector<uint8_t> cls;   // [n] class id of each node
  std::vector<int8_t> key;    // [ncls][3] (own, lo, hi) segments, -1 = boundary
  int ncls() const { return (int)key.size() / 3; }
};

// Device-side view of the grid shared by the kernels.
struct Geo {
  int nx, ny, nz;
  int ncx, ncy, ncz;          // classes per axis
  int64_t n;                  // nx*ny*nz
  const uint8_t* cx;          // [nx] class ids (device)
  const uint8_t* cy;          // [ny]
  const uint8_t* cz;          // [nz]
  __host__ __device__ int ncls() const { return ncx * ncy * ncz; }
};

// Per-instance solver state kept on the device.
enum : int {
  ST_ACTIVE = -1,
  ST_CONVERGED = 0,
  ST_MAX_ITERS = 1,
  ST_BREAKDOWN = 2,
  ST_IDLE = 3,
  ST_PAUSED = 4,  // FP32 recursive residual met tol: awaiting the FP64 check
  ST_UPDATE = 5   // FP32 residual dropped by the update factor: awaiting an FP64 update
};

struct InstState {
  int status;    // ST_*
  int iters;     // applications of A to a search direction
  int restarts;  // true-residual restarts used
  int pad;
  double relres; // last relative residual (true residual after finalisation)
  double relres0;
  unsigned long long t_done;  // %globaltimer (ns) when the status last became final
};

#ifdef __CUDACC__
// Interpolation weights of the prolongation along one axis: fine node j
// (0-based) of an axis whose coarse grid has m nodes takes coarse k0 (weight
// w0) and, if k1 >= 0, coarse k1 (weight w1).  An even 1-based index takes its
// coarse node whole, an odd one half of each neighbour that exists (the
// boundary contributes zero).
struct PRows {
  int k0, k1;
  float w0, w1;
};
__device__ __forceinline__ PRows prows(int j, int m) {
  const int t = j + 1;
  PRows r{-1, -1, 0.f, 0.f};
  if (t % 2 == 0) {
    r.k0 = t / 2 - 1;
    r.w0 = 1.f;
  } else {
    if ((t - 1) / 2 >= 1) r.k0 = (t - 1) / 2 - 1, r.w0 = 0.5f;
    if ((t + 1) / 2 <= m) r.k1 = (t + 1) / 2 - 1, r.w1 = 0.5f;
  }
  return r;
}
#endif

#ifdef __CUDACC__
// hi + lo as a double, with integer operations only (the FP64 pipe runs at a small
// fraction of the FP32 rate on this part).  For a float-float pair |lo| <= ulp(hi): the
// 24-bit significand of hi goes to the top of a 53-bit one and lo, shifted to the same
// scale (its bits below the double's last place dropped), is added or subtracted.  The
// result is hi + lo to within one unit in the last place of the double.  A zero or
// subnormal hi gives lo converted alone (subnormal floats count as zero).
__device__ __forceinline__ double ff_to_f64(float hi, float lo) {
  unsigned H = __float_as_uint(hi), L = __float_as_uint(lo);
  int eh = (int)((H >> 23) & 0xffu);
  if (eh == 0) {  // hi is zero (or subnormal): the result is lo
    H = L;
    L = 0u;
    eh = (int)((H >> 23) & 0xffu);
    if (eh == 0) return 0.0;
  }
  const int el = (int)((L >> 23) & 0xffu);
  long long M = (long long)((H & 0x7fffffu) | 0x800000u) << 29;  // hi's significand in 53 bits
  if (el != 0) {
    const long long ml = (long long)((L & 0x7fffffu) | 0x800000u);
    const int sh = el - eh + 29;  // lo's significand scaled to M's last place
    long long t = 0;
    if (sh >= 0) t = ml << sh;
    else if (sh > -25) t = ml >> (-sh);
    M += ((H ^ L) & 0x80000000u) ? -t : t;
  }
  int e = eh + 896;  // double's biased exponent for M in [2^52, 2^53)
  if (M >= (1ll << 53)) {
    M >>= 1;
    e += 1;
  } else if (M < (1ll << 52)) {
    M <<= 1;
    e -= 1;
  }
  const unsigned long long bits = ((unsigned long long)(H & 0x80000000u) << 32) |
                                  ((unsigned long long)e << 52) | ((unsigned long long)M & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif

// Arguments of the CG phase kernels (one struct so launches stay short).
template <typename T>
struct CGArgs {
  Geo g;
  int B;                // instances in the launch
  int tiles_x, tiles_y; // tiles per plane
  int zc;               // planes per z-chunk
  int nzc;              // z-chunks
  int P;                // CTAs (partials) per instance = tiles_x*tiles_y*nzc
  const T* coef;        // [B][ncls][8]
  const T* f;           // right-hand side [n] (shared) or nullptr -> 1 (init kernel only)
  int64_t f_stride;     // 0: one f for every instance; n: f is [B][n]
  const double* rhs64;  // FP32_IR init: FP64 residual [B][n] to be scaled, else nullptr
  const double* rhs_scale; // FP32_IR init: per-instance norm of rhs64 (the inner rhs is rhs64/norm)
  T* u;                 // [B][n]
  T* r;
  T* s;
  T* p0;                // ping-pong search directions
  T* p1;
  T* q;                 // A p
  double2* rho_rr;      // [2][B][P] partials (rho = r.s, rr = r.r)
  double* gam;          // [B][P] partials of p.Ap
  InstState* st;        // [B]
  const double* fnorm;  // [B] norm of the right-hand side of each instance
  double tol;
  int max_iters;
  int* active;          // number of active instances
  int precond;          // RBWS_PREC_NONE / JACOBI / MSRB
  // MSRB preconditioner (Algorithm 3), FP64 only
  const double* W;      // [N][n] reduced basis
  int N;
  const double* L;      // [B][N][N] Cholesky factors of A_N(mu_b)
  double* G;            // [B][N] projections W^T (r - A D^{-1} r)
  double* C;            // [B][N] reduced corrections
  double* proj_part;    // [B][proj_chunks][N] partial projections
  int proj_chunks;
  // FP32 iterations with FP64 reliable updates (T = float)
  int ru;               // 1: converged instances pause for an FP64 check
  double ru_delta2;     // update when ||r||^2 < ru_delta2 * ||r at last update||^2
  double* rr_ref;       // [B] FP64 ||r||^2 at the last update
  int* pending;         // instances flagged for an update
  int* upd;             // [B] 0 none, 1 update keeping p, 2 update restarting p
  double* u64;          // [B][n] FP64 solution
  double* r64;          // [B][n] FP64 residual f - A u64
  double* rel64;        // [B] ||r64|| / ||f||
  // 32-byte FP32 schedule (k_cg_a32_v4 / k_cg_b32_v4): s is never stored and
  // the u update of iteration k is applied by phase A of iteration k+1.
  double* alpha;        // [2][B] alpha_k by parity; 0 = no pending update
  // residual history (FP64 iteration): hist[b][k] = ||r_k|| / ||f||
  double* hist;         // [B][hist_len] or nullptr
  int hist_len;
  // multigrid preconditioner (host pointer, read by the launchers only)
  const struct MGBatch* mg;
  // bound of each device-side wait in the pipelined kernels, clock64 cycles (0: the
  // built-in default of about 2 s)
  long long wait_cycles;
};

// ---------------------------------------------------------------------------
// Launchers (stencil.cu)
// ---------------------------------------------------------------------------
struct Tile {
  int tx, ty;  // threads per CTA in x and y (one node per thread per plane)
};

// Builds per-instance coefficient tables: coef64 [B][ncls][8] (and coef32 if
// non-null) from mu [B][Q] on the device.  The subdomain of segment box
// (sx, sy, sz) is segq[(sz*by + sy)*bx + sx], or that index itself when segq
// is null (the block rule).
void launch_coef_tables(const Geo& g, const int8_t* keys_x, const int8_t* keys_y,
                        const int8_t* keys_z, int bx, int by, const uint8_t* segq, double sx,
                        double sy, double sz, int Q, const double* mu, int B, double* coef64,
                        float* coef32, cudaStream_t s);
// Tables of a face-field problem (one class per node): coef[b][node] = sum_q mu[b][q]
// rows[q][node] for the 7 stencil values, entry 7 = 1 / D (FP64 and, if coef32, FP32).
void launch_field_tables(int Q, int64_t n, const double* rows, const double* mu, int B, double* coef64,
                         float* coef32, cudaStream_t s);
// lift[q][node] = sum over the node's boundary faces of -rows[q][node][face] * g there;
// gb: the six boundary planes (device), see rbws_dirichlet_lift.
void launch_dirichlet_lift(const Geo& g, int Q, const double* rows, const double* gb, double* lift,
                           cudaStream_t s);
// out[b] = sum_k theta[b][k] F[k], F [K][n], theta [B][K] (device).
void launch_affine_sources(int64_t n, int K, const double* F, const double* theta, int B, double* out,
                           cudaStream_t s);

// y = A x in the mu-interleaved layout [n][B] (instance fastest); coef: the planar
// tables [B][ncls][8], coefI: device scratch of ncls * 8 * B elements for their
// interleaved copy.  Two launches.
template <typename T>
void launch_apply_interleaved(const Geo& g, const T* coef, int B, T* coefI, const T* x, T* y, cudaStream_t s);

// y[b] = A(mu_b) x[b]; x_stride = 0 broadcasts one x to every instance.
template <typename T>
void launch_apply(const Geo& g, Tile t, const T* coef, int B, const T* x, int64_t x_stride, T* y,
                  cudaStream_t s);

// r = f - A u (FP64) per instance; rr partials [B][P] and the residual
// written to r (if non-null); instances with mask[b] == 0 are skipped.
// f: the right-hand side ([n], or [B][n] with f_stride = n; nullptr: f = 1).
void launch_residual64(const Geo& g, Tile t, int zc, const double* coef, int B, const double* f,
                       const double* u, double* r, double* rr_part, int P, const int* mask,
                       cudaStream_t s, int64_t f_stride = 0);
// FP32 phase kernels with 4 nodes per thread (stencil_v4.cu; nx % 4 == 0).
// Tile: t.tx threads x 4 nodes in x, t.ty rows.
void launch_cg_a_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s);
void launch_cg_b_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s);
void launch_ru_reset_v4(const CGArgs<float>& a, Tile t, int start, cudaStream_t s);
// 32-byte schedule: phase A reads r, p_old, u and writes p, u; phase B reads
// r, p (halo) and writes r (A p recomputed); 32 B per DoF and iteration.
void launch_cg_a32_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s);
void launch_cg_b32_v4(const CGArgs<float>& a, Tile t, int parity, cudaStream_t s);
// TMA-fed FP32 stencil phase (stencil_tma.cu): same result as
// launch_cg_a_v4.  Returns -1 if the tensor maps cannot be built.
bool tma_supported(const Geo& g, Tile t);
size_t tma_smem_bytes(Tile t);
int launch_cg_a_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s);
void tma_prepare();  // kernel attributes; call outside stream capture
// 32-byte s-form schedule with both phases TMA-fed (schedule 3): the stored
// residual is s = D^{-1} r; phase A: p = s + beta p_old, u += alpha_{k-1} p_old,
// partial p.A p (20 B/DoF); phase B: s -= alpha D^{-1} A p (A p recomputed),
// partials r.s and r.r with r = D s (12 B/DoF).
int launch_cg_a_s_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s);
int launch_cg_b_s_tma(const CGArgs<float>& a, Tile t, int parity, int* err, cudaStream_t s);
// Autotuning: puts every instance in a runnable state with benign scalars
// (status ACTIVE, rho = 1, ||r||^2 huge, gamma = 1) so one phase kernel can be timed.
void launch_tune_prep(const CGArgs<float>& a, cudaStream_t s);
// Float-float reliable updates (ru_ff.cu): the solution and the tracked true
// residual as hi + lo float pairs, updated on the FP32 pipe; FP64 only for the
// convergence check.
struct FFState {
  float* uh;           // [B][n] solution, hi parts
  float* ul;           //        lo parts
  float* rh;           // [B][n] tracked residual f - A u, hi parts
  float* rl;           //        lo parts
  const float* coef;   // [B][ncls][16]: hi parts of the FP64 table values, then lo parts
  double* part;        // [B][P] partials of ||r||^2 (v4 tiling)
  double* rel;         // [B] ||r|| / ||f|| from part
  int* chk;            // [B] 1: the instance takes the FP64 check
  const double* f;     // right-hand side (nullptr: f = 1); row b at f + b * f_stride
  int64_t f_stride;
};
void launch_coef_ff(const double* coef64, int64_t entries, float* coefff, cudaStream_t s);
// r -= A d', u += d' for instances with upd[b] != 0 (start: from u0 = a.u64, u = 0, r = f)
void launch_ru_ff(const CGArgs<float>& a, Tile t, const FFState& ff, bool start, cudaStream_t s);
void launch_ru_mark(const CGArgs<float>& a, const FFState& ff, cudaStream_t s);
void launch_ff_to64(const CGArgs<float>& a, const FFState& ff, const int* mask, cudaStream_t s);
void launch_ff_fold(const CGArgs<float>& a, const FFState& ff, cudaStream_t s);
void launch_ru_reset_ff(const CGArgs<float>& a, Tile t, const FFState& ff, int start, cudaStream_t s);

// Reliable-update kernels of the FP32 path (see stencil.cu).
void launch_ru_decide(const CGArgs<float>& a, cudaStream_t s);
// dst[k] = src[k] for k < words (dst may be pinned, mapped host memory).
void launch_copy_words(const uint32_t* src, uint32_t* dst, size_t words, cudaStream_t s);
// launch_residual64 from the float-float solution: u = hi + lo (ff_to_f64) formed as the
// planes are staged, written to u_out for the masked instances, and r = f - A u.
void launch_residual64_ff(const Geo& g, Tile t, int zc, const double* coef, int B, const double* f,
                          const float* uh, const float* ul, double* u_out, double* r, double* rr_part, int P,
                          const int* mask, cudaStream_t s, int64_t f_stride);
// The end of one block of a graph-resident solve loop: counts the block in *ctr and sets the
// while node's condition to (counts[0] > 0, the active instances) && (counts[2] == 0, no
// TMA wait ran out) && (*ctr < cap).
void launch_loop_condition(cudaGraphConditionalHandle h, const int* counts, int* ctr, int cap, cudaStream_t s);
void launch_ru_fold(const CGArgs<float>& a, cudaStream_t s);
void launch_ru_reset(const CGArgs<float>& a, Tile t, int start, cudaStream_t s);

// Persistent FP64 PCG (preconditioner none or Jacobi) of one or several problems in one
// cooperative launch: start, iterations and true-residual checks with restarts, until no
// instance is active.  bar (device int[2]) and err (device int) are the grid barrier and its
// timeout flag; d_tasks: device scratch of args.size() * pcg_persistent_task_bytes().
// Returns the grid size, or -1 if the launch could not be made.
int launch_pcg_persistent(const std::vector<CGArgs<double>>& args, Tile t, int* bar, int* err,
                          long long wait_cycles, int max_restarts, int max_rounds, void* d_tasks, cudaStream_t s);
size_t pcg_persistent_task_bytes();

template <typename T>
void launch_cg_init(const CGArgs<T>& a, Tile t, int parity, int only_status, cudaStream_t s);
template <typename T>
void launch_cg_a(const CGArgs<T>& a, Tile t, int parity, cudaStream_t s);
template <typename T>
void launch_cg_b(const CGArgs<T>& a, Tile t, int parity, cudaStream_t s);
// MSRB preconditioner s = D^{-1} r + W A_N^{-1} W^T (r - A D^{-1} r) for the
// active instances; on entry s holds D^{-1} r; the rho partials r.s are
// written into parity slot `slot` (Algorithm 3 applied as P in Algorithm 1).
void launch_msrb_apply(const CGArgs<double>& a, Tile t, int slot, cudaStream_t s);
// Per-instance finalisation after an init pass: mode 0 = start (record
// relres0, set ACTIVE/CONVERGED, count active); mode 1 = true-residual check
// (record relres, restart CONVERGED instances that fail tol).
template <typename T>
void launch_cg_finalize(const CGArgs<T>& a, int parity, int mode, int max_restarts,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// Reduced basis kernels (rb.cu)
// ---------------------------------------------------------------------------
// c[b] = (sum_q mu[b][q] ANq[q])^{-1} fN; info[b] = 0 or -1 (not SPD).  If
// L_out is non-null the Cholesky factor of each A_N(mu_b) is stored there
// ([B][N][N], lower triangle, upper part zero).
// fN element (b, j) at fN[b * f_sb + j * f_sj]: (0, 1) = one reduced right-hand side for all.
void launch_reduced_solve(int N, int Q, const double* ANq, const double* fN, const double* mu,
                          int B, double* c, int* info, double* L_out, cudaStream_t s, int64_t f_sb = 0,
                          int64_t f_sj = 1);
// eta[b] = ||R^{-1} c[b]||_1 with R upper triangular [Nmax][Nmax] (L1 indicator);
// +inf where info[b] != 0.
void launch_l1_indicator(int N, int Nmax, const double* R, const double* c, const int* info, int B,
                         double* eta, cudaStream_t s);
// u = W c with an FP32 copy of W and FP32 accumulation (u written in FP64).
void launch_lift32(int64_t n, int N, const float* W, const double* c, int B, double* u, cudaStream_t s);
// y = (float) x.
void launch_to_f32(int64_t n, const double* x, float* y, cudaStream_t s);
// u[b] = sum_j c[b][j] W[j]  (W: [N][n]).
void launch_lift(int64_t n, int N, const double* W, const double* c, int B, double* u,
                 cudaStream_t s);
// out[k] = X[k] . y for k < K (X rows of length n, row stride ldx), two-stage deterministic.
void launch_multi_dot(int64_t n, int K, const double* X, int64_t ldx, const double* y,
                      double* out, double* scratch, int scratch_len, cudaStream_t s);
// w -= sum_j coef[j] W[j]   (coef device [K])
void launch_sub_combination(int64_t n, int K, const double* W, const double* coef, double* w,
                            cudaStream_t s);
// w *= 1/alpha (alpha device scalar)
void launch_scale_inv(int64_t n, const double* alpha, double* w, cudaStream_t s);
// per-instance eta[b] = sqrt(sum partials)/fnorm
// out[b] = sqrt(sum of the P partials of b) / (fnorms ? fnorms[b] : fnorm).
void launch_norms_from_partials(const double* part, int B, int P, double fnorm, double* out,
                                cudaStream_t s, const double* fnorms = nullptr);
// out[b] = ||X[b]||_2, rows of length n with stride ldx.
void launch_row_norms(int64_t n, int B, const double* X, int64_t ldx, double* out, cudaStream_t s);
// FN[j * B + b] = (W^T f_b)_j from the FP32 copy of W (device [N][n]) and the FP64 sources
// F (row b at F + b * ldf): FP32 products, summed in FP32 over runs of 128 nodes and in
// FP64 across runs and splits (fixed order).  part: device scratch of
// project32_splits(n, B) * N * B doubles.  N in 1..160; returns -1 otherwise.  Two launches.
int project32_splits(int64_t n, int B);
int launch_project32(int64_t n, int N, int B, const float* W, const double* F, int64_t ldf, double* part,
                     double* FN, cudaStream_t s);
// f[b] = (offset + amplitude exp(-|x - c_b|^2 / width)) times each node's relative control
// volume, prm device [B][6] = (c_x, c_y, c_z, width, amplitude, offset); neumann (host [3]):
// the axes with a Neumann face at coordinate 1 (node coordinates i/n there).
void launch_gaussian_source(int nx, int ny, int nz, const int* neumann, const double* prm, int B, double* f,
                            cudaStream_t s);

// ---------------------------------------------------------------------------
// Learned warm start (mlp.cu)
// ---------------------------------------------------------------------------
// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]) with BF16 operands, FP32 accumulation;
// Z = C and, if Aout is non-null, Aout = GELU(C) (both [M][ldz] row-major).
struct MlpGemm {
  int M, N, K;
  const void* A;
  int64_t sam, sak;
  int a_bf16;
  const void* B;
  int64_t sbk, sbn;
  int b_bf16;
  const float* bias;
  float* Z;
  float* Aout;
  int64_t ldz;
};
void launch_mlp_gemm(const MlpGemm& g, cudaStream_t s);
void launch_mlp_inputs(const double* mu, int B, int p, double lo, double hi, float* x, cudaStream_t s);
void launch_mlp_loss(const float* y, const float* t, int total, float scale, float* dy, float* loss,
                     cudaStream_t s);
void launch_gelu_back(const float* da, const float* z, int total, float* dz, cudaStream_t s);
void launch_bias_grad(const float* dz, int M, int N, float* db, cudaStream_t s);
void launch_adam(float* w, void* w16, const float* g, float* m1, float* m2, int64_t P, float lr, int* step,
                 cudaStream_t s);
void launch_init_params(float* w, void* w16, int64_t P, const int64_t* seg_end, const float* seg_bound,
                        int nseg, uint64_t seed, cudaStream_t s);
void launch_to_bf16(const float* w, void* w16, int64_t P, cudaStream_t s);
void launch_rms_scale(const double* c, int B, int N, float* scale, cudaStream_t s);
void launch_scale_targets(const double* c, const float* scale, int B, int N, float* t, cudaStream_t s);
void launch_unscale(const float* y, const float* scale, int B, int N, double* c, cudaStream_t s);
void launch_reduced_cg_step(int N, int Q, const double* ANq, const double* fN, const double* mu, int B,
                            double* c, cudaStream_t s);

// rho = r.s partials after an external preconditioner wrote s, in slot `slot`
// of the phase kernels' partials (one-node tiling: stencil.cu; v4 tiling:
// stencil_v4.cu); instances with mask[b] == 0 are skipped (mask may be null).
template <typename T>
void launch_precond_rho(const CGArgs<T>& a, Tile t, int slot, const int* mask, cudaStream_t s);
void launch_precond_rho_v4(const CGArgs<float>& a, Tile t, int slot, const int* mask, cudaStream_t s);

// ---------------------------------------------------------------------------
// Multigrid V-cycle preconditioner, Algorithm 2 (mg.cu)
//
// Every level's operator is stored the way the finest one is: by per-axis
// node classes and a per-instance table of rows by class.  The finest level
// uses the 7-point tables of k_coef_tables; a coarse node's class along an
// axis is the tuple of fine classes at fine nodes 2J-2 .. 2J+2 (or "outside"),
// which fixes its Galerkin row (P^T A P), a 27-point stencil.  The rows of
// each affine term are formed once on the host; per instance a table is the
// mu-combination of them.  The coarsest level is solved with an explicit
// inverse per instance.
// ---------------------------------------------------------------------------
constexpr int kMGMaxLevels = 12;
constexpr int kMGCoarsest = 64;     // coarsen while a level has more unknowns than this
constexpr int kMGMaxDense = 1024;   // largest coarsest level accepted
constexpr int kMGTailMax = 4096;    // levels up to this size run in one kernel per V-cycle
constexpr int kMGNu = 2;            // pre- and post-smoothing steps
constexpr double kMGOmega = 2.0 / 3.0;

struct MGPlan {
  struct Level {
    int nx = 0, ny = 0, nz = 0;
    int64_t n = 0;
    int ncx = 0, ncy = 0, ncz = 0;
    std::vector<uint8_t> cx, cy, cz;  // class of each node along each axis
    std::vector<double> tq;           // [Q][ncls][27] rows by class (offset (dz+1)*9+(dy+1)*3+dx+1)
    int ncls() const { return ncx * ncy * ncz; }
  };
  int J = -1;  // finest level; levels 0 (coarsest) .. J
  int Q = 0;
  int n0 = 0;  // unknowns on level 0
  std::vector<Level> lv;
  std::vector<double> a0q;  // [Q][n0][n0] level-0 matrices of the affine terms
  // device copies
  uint8_t* d_cls[kMGMaxLevels] = {};
  double* d_tq[kMGMaxLevels] = {};
  double* d_a0q = nullptr;
  ~MGPlan();
};

// Builds the hierarchy from the finest grid's axis classes and the 27-wide rows of
// each affine term on it by class ([Q][ncls][27], fine_rows_q or a face-field
// problem's node rows); "" or the reason multigrid is not available for this grid.
// Device copies are made here.
std::string mg_build_plan(const AxisClasses& ax, const AxisClasses& ay, const AxisClasses& az,
                          std::vector<double> fine_tq, int Q, MGPlan* plan);

// Device view of one level for the V-cycle kernels (element type: the batch's).
struct MGLevel {
  int nx, ny, nz;
  int64_t n;
  int ncx, ncy, ncz;
  const uint8_t* cx;
  const uint8_t* cy;
  const uint8_t* cz;
  const void* coef;  // [B][ncls][stride]
  int stride;        // 8: the finest 7-point table; 28: 27 entries + 1/diagonal
};

// Per-batch state of the V-cycle: level views, work vectors, level-0 inverses.
// fp32: every vector, table and inverse is float (the inner iteration of the
// mixed-precision solver), else double.
struct MGBatch {
  const MGPlan* plan = nullptr;
  int B = 0;
  int fp32 = 0;
  const InstState* st = nullptr;  // instances whose status is not ACTIVE are skipped
  const int* mask = nullptr;      // and, if set, those with mask[b] == 0
  // FP32 iteration with the v4 tiles: the finest level runs fused steps with
  // the iteration's tiling and writes the rho partials itself
  const CGArgs<float>* fine_cg = nullptr;
  Tile fine_tile{0, 0};
  // tiling of the fused steps that write no partials (wider tiles: less halo)
  Tile mg_tile{0, 0};
  int mg_tiles_x = 0, mg_tiles_y = 0, mg_zc = 0, mg_nzc = 0;
  cudaEvent_t* ev = nullptr;  // if set: 8 events bracketing the four fused finest-level steps, and a
                              // ninth (ev[8]) between the prolongation pass and step 2's smoothing
  MGLevel lv[kMGMaxLevels];
  void* rhs[kMGMaxLevels] = {};
  void* sol[kMGMaxLevels] = {};
  void* w1[kMGMaxLevels] = {};
  void* w2[kMGMaxLevels] = {};
  const void* ainv = nullptr;  // [B][n0][n0]
  const float* od = nullptr;    // FP32 finest level: omega / D per node [B][n] (see MGFineArgs)
};

// Per-instance coarse tables (element type per fp32) and level-0 inverses
// for B parameters (device mu [B][Q]).  The inverses are formed in FP64
// (dense_a, dense_l, ainv64) and, with fp32, rounded into ainv32.  info[b] != 0
// where a level-0 matrix is not positive definite.
void launch_mg_setup(const MGPlan& plan, const double* mu, int B, int fp32, void* const* tables, double* dense_a,
                     double* dense_l, double* ainv64, float* ainv32, int* info, cudaStream_t s);
// out = MG(rhs) on the finest level (Algorithm 2 at level J); returns launches.
// With m.fine_cg set the partials of rho = rhs . out go to slot `slot` too.
int launch_mg_vcycle(const MGBatch& m, const void* rhs, void* out, int slot, cudaStream_t s);
// Fine-level FP32 multigrid steps with the v4 tiles (stencil_v4.cu).
struct MGFineArgs {
  const float* rhs;  // [B][n] right-hand side of the level (the iteration's r)
  const float* xin;  // staged input (stage 0)
  float* out;
  int cnx, cny, cnz;  // the coarse grid of output kind 3
  const int* mask;   // skip instances with mask[b] == 0 (may be null)
  float omega;
  int slot;          // partial slot of rho (output kind 2)
  const float* od = nullptr;  // [B][n] omega / D of the level's nodes (stage 1 from staged od), or null
};
// od[b][node] = omega / D from the FP32 coefficient tables (the first pre-smoothing step's
// scaling, staged beside the rhs).
void launch_omega_dinv(const Geo& g, const float* coef32, int B, float omega, float* od, cudaStream_t s);
// stage 0: x = xin, 1: x = omega D^-1 rhs;  outk 0: Jacobi
// step, 1: residual, 2: Jacobi step and rho partials, 3 (stage 0): the
// restricted residual P^T (rhs - A x) into out (the coarse grid cnx x cny x
// cnz).  Returns -1 for a combination that is not built, or (outk 3) a tiling
// it does not take.
int launch_mg_fine_v4(const CGArgs<float>& a, Tile t, int stage, int outk, const MGFineArgs& m, cudaStream_t s);
// outk 3 of the above: the TMA-fed residual + restriction kernel (stencil_tma.cu).
// Needs an even ty and zc, tensor-map support and tma_prepare(); -1 otherwise.
// A stage wait that runs out sets the error flag a.active[2].
int launch_mg_fine_rr_tma(const CGArgs<float>& a, Tile t, const MGFineArgs& m, cudaStream_t s);
// Stages 0 and 1 with outk 0, and stage 0 with outk 2, of launch_mg_fine_v4 with the
// planes fed by TMA (stencil_tma.cu): -1 where tensor maps or the tiling do not allow
// it (the register-prefetch kernel runs then).
int launch_mg_smooth_tma(const CGArgs<float>& a, Tile t, int stage, const MGFineArgs& m, bool rho,
                         cudaStream_t s);
// y = D^-1 x on the FP64 level view L (instances all active).
void launch_diag_inverse(const MGLevel& L, int B, const double* x, double* y, cudaStream_t s);

// ---------------------------------------------------------------------------
// L1ROC (l1roc.cu): DEIM point search, gathers, over-collocation least squares
// ---------------------------------------------------------------------------
// (index, signed value) of the first entry of x whose magnitude is within a
// factor 1 - 1e-8 of the largest (near-ties: the smaller index); scratch of
// `chunks` entries each.
void launch_argmax_abs(int64_t n, const double* x, double* scratch_v, int64_t* scratch_i, int chunks,
                       int64_t* out_idx, double* out_val, cudaStream_t s);
// out[t] = X[col[t] * ld + idx[t]] (0 where idx[t] < 0), t < L.
void launch_gather(const double* X, int64_t ld, const int* col, const int64_t* idx, int L, double* out,
                   cudaStream_t s);
// c[b] = argmin ||sum_q mu[b][q] PAWq[q] c - Pf||_2 (PAWq [Q][M][N] row-major) by
// Householder QR, one CTA per instance; info[b] = 1 on rank deficiency.  Needs
// colloc_ls_smem(M, N) bytes of shared memory (colloc_ls_prepare raises the limit).
size_t colloc_ls_smem(int M, int N);
void colloc_ls_prepare();
void launch_colloc_ls(int M, int N, int Q, const double* PAWq, const double* Pf, const double* mu, int B, double* c,
                      int* info, cudaStream_t s);

// Rows of each affine term on the finest grid by class: [Q][ncls][27] (offset
// (dz+1)*9 + (dy+1)*3 + dx+1; kappa = e_q), as the coefficient tables form them.
std::vector<double> fine_rows_q(const AxisClasses& ax, const AxisClasses& ay, const AxisClasses& az, int bx, int by,
                                const uint8_t* segq, int Q, double sx, double sy, double sz);

// ---------------------------------------------------------------------------
// Operator apply with static scratch (static_scratch.cu)
// ---------------------------------------------------------------------------
size_t static_scratch_need(int Q, int ncls, int B, bool fp32);
size_t static_scratch_capacity();
int apply_operator_static(int device, const Geo& g, const int8_t* kx, const int8_t* ky, const int8_t* kz,
                          int bx, int by, const uint8_t* segq, double sx, double sy, double sz, int Q,
                          const double* mu_host, int B, const void* x, void* y, int precision,
                          cudaStream_t s, Tile t);

// ---------------------------------------------------------------------------
// Error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);  // sets message, returns RBWS_ERR_CUDA

}  // namespace rbws
