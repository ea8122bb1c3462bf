// api.cu -- the C ABI of librbws and the host-side orchestration: problem
// set-up (block rule, explicit maps, anisotropic / Neumann axes, face-field
// problems), the batched PCG driver (CUDA-graph captured iterations with device
// convergence masks), FP32-inner / FP64-outer refinement (its blocks looped on
// the device by a conditional graph node), the warm starts (Galerkin, L1ROC,
// learned), the offline greedy, uneven request batches, the autotuner and
// checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

using namespace rbws;

namespace rbws {

static thread_local std::string g_last_error = "";

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return RBWS_ERR_CUDA;
}

}  // namespace rbws

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return (rbws_status)cuda_fail(e_, #call); \
  } while (0)

#define CKI(call)                                       \
  do {                                                  \
    int r_ = (call);                                    \
    if (r_ != 0) return (rbws_status)r_;                \
  } while (0)

namespace {

// Grow-only device buffer.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Classes of one axis from the segment of every node (seg: [n], values < b).
// Keys (own, lo, hi): lo / hi the neighbour's segment, -1 past a Dirichlet boundary, -2
// past the last node of an axis whose face at coordinate 1 is a Neumann face.
AxisClasses make_axis_segments(const std::vector<int>& seg, int b, bool neumann = false) {
  const int n = (int)seg.size();
  AxisClasses a;
  a.n = n;
  a.b = b;
  a.cls.resize(n);
  auto blk = [&](int i) { return seg[i - 1]; };  // i: 1..n
  std::map<std::tuple<int, int, int>, int> ids;
  for (int i = 1; i <= n; i++) {
    const int own = blk(i), lo = i > 1 ? blk(i - 1) : -1, hi = i < n ? blk(i + 1) : (neumann ? -2 : -1);
    auto key = std::make_tuple(own, lo, hi);
    auto it = ids.find(key);
    int id;
    if (it == ids.end()) {
      id = (int)ids.size();
      ids[key] = id;
      a.key.push_back((int8_t)own);
      a.key.push_back((int8_t)lo);
      a.key.push_back((int8_t)hi);
    } else {
      id = it->second;
    }
    a.cls[i - 1] = (uint8_t)id;
  }
  return a;
}

// Block rule: along an axis with n nodes and b blocks, node i (1..n) lies in
// block min(floor(b*i/(n+1)), b-1); on an axis with a Neumann face (nodes at i/n)
// in block min(floor(b*i/n), b-1): blocks by coordinate either way.
AxisClasses make_axis(int n, int b, bool neumann = false) {
  std::vector<int> seg(n);
  const int64_t cells = neumann ? n : n + 1;
  for (int i = 1; i <= n; i++) {
    const int k = (int)(((int64_t)b * i) / cells);
    seg[i - 1] = k < b - 1 ? k : b - 1;
  }
  return make_axis_segments(seg, b, neumann);
}

// An explicit map [nz][ny][nx] is cut by every grid plane across which it
// changes somewhere; between consecutive cuts the map does not change along
// any axis, so it is constant on each box of that tensor-product partition
// and the per-axis class machinery of the block rule applies unchanged.
// Fills the per-axis segments and the box -> subdomain table; returns "" or
// the reason the map is rejected.
constexpr int kMaxSegments = 64;       // per axis (class ids stay below 256)
constexpr int kMaxClasses = 1 << 16;   // coefficient rows per instance

std::string map_segments(int nx, int ny, int nz, const uint8_t* map, int Q, std::vector<int>& sx,
                         std::vector<int>& sy, std::vector<int>& sz, std::vector<uint8_t>& segq) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t t = 0; t < n; t++)
    if (map[t] >= Q) return "map value " + std::to_string(map[t]) + " >= Q";
  auto at = [&](int i, int j, int k) { return map[((int64_t)k * ny + j) * nx + i]; };
  std::vector<char> cx(nx, 0), cy(ny, 0), cz(nz, 0);  // cut before node index
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        const uint8_t v = at(i, j, k);
        if (i > 0 && at(i - 1, j, k) != v) cx[i] = 1;
        if (j > 0 && at(i, j - 1, k) != v) cy[j] = 1;
        if (k > 0 && at(i, j, k - 1) != v) cz[k] = 1;
      }
  auto segs = [](const std::vector<char>& c, std::vector<int>& s) {
    s.assign(c.size(), 0);
    for (size_t i = 1; i < c.size(); i++) s[i] = s[i - 1] + c[i];
    return s.back() + 1;
  };
  const int bx = segs(cx, sx), by = segs(cy, sy), bz = segs(cz, sz);
  if (bx > kMaxSegments || by > kMaxSegments || bz > kMaxSegments)
    return "the map needs more than " + std::to_string(kMaxSegments) + " segments along an axis";
  segq.assign((size_t)bx * by * bz, 0);
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) segq[((size_t)sz[k] * by + sy[j]) * bx + sx[i]] = at(i, j, k);
  return "";
}

}  // namespace

struct rbws_problem_s {
  int device = 0;
  int nx = 0, ny = 0, nz = 0, bx = 1, by = 1, bz = 1, Q = 1;
  double kscale[3] = {1.0, 1.0, 1.0};  // diagonal of the diffusion tensor
  int neumann[3] = {0, 0, 0};          // Neumann face at coordinate 1 of each axis
  bool default_f = false;              // f = the node weights (no f given, a Neumann face)
  int64_t n = 0;
  double sx = 0, sy = 0, sz = 0;
  AxisClasses ax, ay, az;
  uint8_t* d_cls = nullptr;  // cx | cy | cz
  int8_t* d_keys = nullptr;  // kx | ky | kz
  std::vector<uint8_t> h_map;  // explicit subdomain map [n] (empty: block rule)
  std::vector<uint8_t> h_segq; // explicit map: box (bx*by*bz segments) -> subdomain
  uint8_t* d_segq = nullptr;
  // Face-field problems (rbws_problem_create_field): every node is its own class and the
  // coefficient rows of each term, [Q][n][7] (-kW -kE -kS -kN -kD -kU D, already scaled by
  // 1/h^2), are combined per instance by k_field_tables; the face arrays are kept for
  // checkpoints (kfx | kfy | kfz, each [Q][...]).
  bool field = false;
  std::vector<double> h_frows;
  double* d_frows = nullptr;
  std::vector<double> h_faces;
  // L1ROC online data (Sec. 3.1): collocation nodes, P A_q W and P f, and T
  // with U = W T (snapshots U); empty unless the basis came from rbws_offline_l1roc
  struct L1Roc {
    int N = 0, M = 0;
    std::vector<int64_t> pts;
    std::vector<double> T;        // [N][N], row-major, upper triangular
    double* d_PAWq = nullptr;     // [Q][M][N]
    double* d_Pf = nullptr;       // [M]
  } l1;
  std::unique_ptr<MGPlan> mg;  // multigrid hierarchy, built on first use
  std::string mg_err;
  bool mg_tried = false;
  Geo geo{};
  double* d_f = nullptr;     // nullptr: f == 1
  double* d_ones = nullptr;  // ones vector (for W^T f when f == 1)
  double fnorm = 0.0;
  // Per-instance right-hand sides of the current call (f == nullptr: the problem's f above):
  // f_b = f + b * stride, ||f_b|| = norms[b]; the reduced right-hand sides W^T f_b at
  // fN[b * fN_sb + j * fN_sj] when precomputed (else formed where needed).
  struct RhsView {
    const double* f = nullptr;
    int64_t stride = 0;
    const double* norms = nullptr;
    const double* fN = nullptr;
    int64_t fN_sb = 0, fN_sj = 1;
  } rhs;
  cudaStream_t stream = nullptr;  // internal stream (used when the caller passes none)
  cudaStream_t cur = nullptr;     // work stream of the current call
  cudaEvent_t ev = nullptr;
  cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};  // profiling events
  cudaEvent_t mgev[10] = {};                                 // ... of the fused MG steps
  int64_t launches = 0;           // kernels launched by the current call
  // pinned, mapped host memory for the mixed-precision solve's own small reads (read_small)
  void* h_small = nullptr;
  void* d_small = nullptr;
  size_t small_bytes = 0;
  // reduced basis
  int N = 0;
  double* d_W = nullptr;    // [N][n]
  float* d_W32 = nullptr;   // FP32 copy of W for the mixed-precision start (built on first use)
  double* d_ANq = nullptr;  // [Q][N][N]
  double* d_fN = nullptr;   // [N]
  std::vector<double> h_ANq, h_fN;  // packed [Q][N][N], [N]
  // surrogate network mu -> c (learned warm start)
  int net_H = 0, net_N = 0;
  int64_t net_P = 0;
  float* d_w32 = nullptr;     // FP32 master parameters [P]
  void* d_w16 = nullptr;      // BF16 copy [P]
  float* d_cscale = nullptr;  // [N] coefficient scales
  double net_lo = 0.0, net_hi = 0.0;
  std::map<std::string, DevBuf> bufs;
  struct Tuned {
    int tx, ty, zc;
    double ms;
    int sched;  // 0: 44 B, 1: 32 B, 2: 44 B with TMA stencil phase, 3: 32 B s-form, both phases TMA
  };
  std::map<int, Tuned> tuned32;  // batch size -> tuned FP32 tile

  void* buf(const std::string& name, size_t bytes, int* err) {
    DevBuf& d = bufs[name];
    if (d.bytes < bytes) {
      if (d.ptr) cudaFree(d.ptr);
      d.ptr = nullptr;
      d.bytes = 0;
      cudaError_t e = cudaMalloc(&d.ptr, bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("out of device memory allocating " + name + " (" + std::to_string(bytes) + " B)");
        *err = RBWS_ERR_OOM;
        return nullptr;
      }
      d.bytes = bytes;
    }
    return d.ptr;
  }
};

namespace {

Tile choose_tile(int nx) {
  Tile t;
  t.tx = nx >= 64 ? 64 : (nx > 16 ? 32 : 16);
  t.ty = 256 / t.tx;
  return t;
}

// Tile of the 4-node-per-thread FP32 kernels: widest row segment (4*tx nodes,
// tx in {32,16,8,4}) dividing nx (else the widest that fits), up to 256
// threads.  tx = 0 when nx % 4 != 0 (the one-node kernels are used then).
Tile choose_tile_v4(int nx, int ny) {
  Tile t{0, 0};
  if (nx % 4) return t;
  for (int tx : {32, 16, 8, 4})
    if (4 * tx <= nx && nx % (4 * tx) == 0) {
      t.tx = tx;
      break;
    }
  if (!t.tx)  // no exact fit: widest segment that fits, last tile ragged
    for (int tx : {32, 16, 8, 4})
      if (4 * tx <= nx) {
        t.tx = tx;
        break;
      }
  if (!t.tx) return t;
  t.ty = std::min(256 / t.tx, ny);
  return t;
}

// z-chunking of the v4 kernels: a few waves of 4 resident CTAs per SM.
int choose_zc_v4(int nz, int64_t ctas_per_chunk) {
  int nzc = 1;
  while (ctas_per_chunk * nzc < 4 * 608 && (nz / (nzc * 2)) >= 8) nzc *= 2;
  return (nz + nzc - 1) / nzc;
}

// z-chunking: enough CTAs for several waves, chunks of at least 8 planes.
int choose_zc(int nz, int64_t ctas_per_chunk) {
  int nzc = 1;
  while (ctas_per_chunk * nzc < 8 * 1216 && (nz / (nzc * 2)) >= 8) nzc *= 2;
  return (nz + nzc - 1) / nzc;
}

struct StreamGuard {
  rbws_problem p;
  bool ok = true;
  StreamGuard(rbws_problem p_, void* user) : p(p_) {
    cudaSetDevice(p->device);
    p->launches = 0;
    if (user) {
      p->cur = (cudaStream_t)user;
    } else {
      // order after earlier work on the legacy default stream
      cudaEventRecord(p->ev, 0);
      cudaStreamWaitEvent(p->stream, p->ev, 0);
      p->cur = p->stream;
    }
  }
  ~StreamGuard() { p->cur = p->stream; }
};

// Reads `bytes` (a multiple of 4) of device memory into host memory: a kernel writes them to
// pinned, mapped host memory, then the host waits for stream s.  A plain device-to-host copy
// would take a copy engine and queue behind any large copy the caller has in flight (the
// previous batch's solutions going back to the host while this batch solves), and the solve
// would stall until that copy ended.
rbws_status read_small(rbws_problem p, const void* dev, size_t bytes, void* host, cudaStream_t s) {
  if (bytes > p->small_bytes) {
    CK(cudaStreamSynchronize(s));  // nothing still writes the old buffer
    if (p->h_small) cudaFreeHost(p->h_small);
    p->h_small = p->d_small = nullptr;
    p->small_bytes = 0;
    const size_t nb = std::max<size_t>(bytes, 4096);
    CK(cudaHostAlloc(&p->h_small, nb, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(&p->d_small, p->h_small, 0));
    p->small_bytes = nb;
  }
  launch_copy_words(static_cast<const uint32_t*>(dev), static_cast<uint32_t*>(p->d_small), bytes / 4, s);
  p->launches += 1;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  std::memcpy(host, p->h_small, bytes);
  return RBWS_OK;
}

// Coefficient tables for B parameters already on the device.
rbws_status coef_tables(rbws_problem p, const double* d_mu, int B, double** c64, float** c32) {
  int err = 0;
  const size_t ncls = (size_t)p->geo.ncls();
  *c64 = (double*)p->buf("coef64", sizeof(double) * ncls * kCoefStride * B, &err);
  if (err) return (rbws_status)err;
  if (c32) {
    *c32 = (float*)p->buf("coef32", sizeof(float) * ncls * kCoefStride * B, &err);
    if (err) return (rbws_status)err;
  }
  if (p->field) {
    launch_field_tables(p->Q, p->n, p->d_frows, d_mu, B, *c64, c32 ? *c32 : nullptr, p->cur);
  } else {
    const int8_t* kx = p->d_keys;
    const int8_t* ky = kx + p->ax.key.size();
    const int8_t* kz = ky + p->ay.key.size();
    launch_coef_tables(p->geo, kx, ky, kz, p->bx, p->by, p->d_segq, p->sx, p->sy, p->sz, p->Q, d_mu, B, *c64,
                       c32 ? *c32 : nullptr, p->cur);
  }
  p->launches += 1;
  CK(cudaGetLastError());
  return RBWS_OK;
}

rbws_status upload_mu(rbws_problem p, const double* mu, int B, double** d_mu, const char* name) {
  int err = 0;
  *d_mu = (double*)p->buf(name, sizeof(double) * (size_t)B * p->Q, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(*d_mu, mu, sizeof(double) * (size_t)B * p->Q, cudaMemcpyHostToDevice,
                     p->cur));
  return RBWS_OK;
}

// Sets the inner states of finished instances to CONVERGED before an inner solve.
__global__ void k_mask_done(InstState* st, const int* done, int B, int* active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (done[b] && st[b].status == ST_ACTIVE) {
    st[b].status = ST_CONVERGED;
    atomicSub(active, 1);
  }
}

// One PCG iteration of the given parity: phase A, phase B and, for MSRB, the
// preconditioner application (Algorithm 3) that completes s = P(r).
template <typename T>
int launch_iteration(const CGArgs<T>& a, Tile t, int parity, cudaStream_t s) {
  launch_cg_a<T>(a, t, parity, s);
  launch_cg_b<T>(a, t, parity, s);
  if constexpr (sizeof(T) == 8) {
    if (a.precond == RBWS_PREC_MSRB) {
      launch_msrb_apply(a, t, parity ^ 1, s);
      return 6;
    }
    if (a.precond == RBWS_PREC_MG) {
      const int l = launch_mg_vcycle(*a.mg, a.r, a.s, -1, s);
      launch_precond_rho<double>(a, t, parity ^ 1, nullptr, s);
      return 3 + l;
    }
  }
  return 2;
}

// Completes the initial s = P(r0) for MSRB after an init pass.
template <typename T>
int launch_precond_start(const CGArgs<T>& a, Tile t, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (a.precond == RBWS_PREC_MSRB) {
      launch_msrb_apply(a, t, 0, s);
      return 4;
    }
    if (a.precond == RBWS_PREC_MG) {
      const int l = launch_mg_vcycle(*a.mg, a.r, a.s, -1, s);
      launch_precond_rho<double>(a, t, 0, nullptr, s);
      return 1 + l;
    }
  }
  return 0;
}

// The batched PCG driver.  On entry a.u holds the initial values.  Runs
// Algorithm 1 with the true-residual restarts of Algorithm 4.
// `done` (device [B] or nullptr) marks instances that must not run; with
// check_true = false the true-residual check is skipped (inner solves of
// FP32_IR, whose outer loop checks the FP64 residual itself).
// Iterations run in blocks of M = check_every (even): a captured CUDA graph
// of M (A, B) phase pairs is relaunched until the device-side active count
// reaches zero.  With a profile record the blocks are launched directly and
// the first pair of each block is timed with CUDA events.
template <typename T>
rbws_status run_pcg(rbws_problem p, CGArgs<T>& a, Tile t, int max_restarts, int check_every,
                    const int* done, bool check_true, rbws_profile* prof) {
  cudaStream_t s = p->cur;
  CK(cudaMemsetAsync(a.active, 0, sizeof(int), s));
  launch_cg_init<T>(a, t, 0, 0, s);
  launch_cg_finalize<T>(a, 0, 0, max_restarts, s);
  p->launches += 2;
  if (done) {
    k_mask_done<<<(a.B + 127) / 128, 128, 0, s>>>(a.st, done, a.B, a.active);
    p->launches += 1;
  }
  p->launches += launch_precond_start<T>(a, t, s);
  CK(cudaGetLastError());
  int M = check_every > 0 ? check_every : 8;
  if (M % 2) M++;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t ce;
  int per_iter = 2;
  if (!prof) {
    // Capture M iterations (parities 0,1,0,1,...) once; relaunch until done.
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < M; k++) per_iter = launch_iteration<T>(a, t, k & 1, s);
    ce = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) return (rbws_status)cuda_fail(ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      return (rbws_status)cuda_fail(ce, "cudaGraphInstantiate");
    }
  } else {
    prof->elem_bytes = (int32_t)sizeof(T);
    prof->schedule = -1;
  }
  rbws_status rc = RBWS_OK;
  for (;;) {
    int active = 0;  // read off the copy engines (read_small)
    if ((rc = read_small(p, a.active, sizeof(int), &active, s)) != RBWS_OK) break;
    if (active > 0) {
      if (!prof) {
        if ((ce = cudaGraphLaunch(exec, s)) != cudaSuccess) {
          rc = (rbws_status)cuda_fail(ce, "cudaGraphLaunch");
          break;
        }
      } else {
        cudaEventRecord(p->tev[0], s);
        launch_cg_a<T>(a, t, 0, s);
        cudaEventRecord(p->tev[1], s);
        launch_cg_b<T>(a, t, 0, s);
        cudaEventRecord(p->tev[2], s);
        if constexpr (sizeof(T) == 8) {
          if (a.precond == RBWS_PREC_MSRB) {
            launch_msrb_apply(a, t, 1, s);
            per_iter = 6;
          }
          if (a.precond == RBWS_PREC_MG) {
            per_iter = 3 + launch_mg_vcycle(*a.mg, a.r, a.s, -1, s);
            launch_precond_rho<double>(a, t, 1, nullptr, s);
          }
        }
        for (int k = 1; k < M; k++) launch_iteration<T>(a, t, k & 1, s);
        if ((ce = cudaEventSynchronize(p->tev[2])) != cudaSuccess) {
          rc = (rbws_status)cuda_fail(ce, "profile events");
          break;
        }
        float ta = 0.f, tb = 0.f;
        cudaEventElapsedTime(&ta, p->tev[0], p->tev[1]);
        cudaEventElapsedTime(&tb, p->tev[1], p->tev[2]);
        prof->stencil_ms += ta;
        prof->update_ms += tb;
        prof->active_dofs += (double)active * (double)p->n;
        prof->samples += 1;
      }
      p->launches += (int64_t)per_iter * M;
      continue;
    }
    if (!check_true) break;
    // all stopped: check the true residual f - A u, restart the failures
    launch_cg_init<T>(a, t, 0, 0, s);
    launch_cg_finalize<T>(a, 0, 1, max_restarts, s);
    p->launches += 2;
    p->launches += launch_precond_start<T>(a, t, s);
    int restarted = 0;
    if ((rc = read_small(p, a.active, sizeof(int), &restarted, s)) != RBWS_OK) break;
    if (restarted == 0) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  return rc;
}

template <typename T>
rbws_status make_cg_args(rbws_problem p, int B, Tile t, const T* coef, T* u, CGArgs<T>* out,
                         const std::string& tag, int vec = 1, int zc_force = 0) {
  int err = 0;
  CGArgs<T> a{};
  a.g = p->geo;
  a.B = B;
  a.tiles_x = (p->nx + vec * t.tx - 1) / (vec * t.tx);
  a.tiles_y = (p->ny + t.ty - 1) / t.ty;
  a.zc = zc_force > 0 ? std::min(zc_force, p->nz)
         : vec == 4 ? choose_zc_v4(p->nz, (int64_t)a.tiles_x * a.tiles_y * B)
                    : choose_zc(p->nz, (int64_t)a.tiles_x * a.tiles_y * B);
  a.nzc = (p->nz + a.zc - 1) / a.zc;
  a.P = a.tiles_x * a.tiles_y * a.nzc;
  a.coef = coef;
  a.u = u;
  const size_t vb = sizeof(T) * (size_t)B * p->n;
  a.r = (T*)p->buf(tag + "r", vb, &err);
  if (!err) a.s = (T*)p->buf(tag + "s", vb, &err);
  if (!err) a.p0 = (T*)p->buf(tag + "p0", vb, &err);
  if (!err) a.p1 = (T*)p->buf(tag + "p1", vb, &err);
  if (!err) a.q = (T*)p->buf(tag + "q", vb, &err);
  if (!err) a.rho_rr = (double2*)p->buf(tag + "rho_rr", sizeof(double2) * 2 * (size_t)B * a.P, &err);
  if (!err) a.gam = (double*)p->buf(tag + "gam", sizeof(double) * (size_t)B * a.P, &err);
  if (!err) a.st = (InstState*)p->buf(tag + "st", sizeof(InstState) * (size_t)B, &err);
  if (!err) a.active = (int*)p->buf(tag + "active", sizeof(int) * 4, &err);
  if (!err) a.fnorm = (const double*)p->buf(tag + "fnorm", sizeof(double) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  *out = a;
  return RBWS_OK;
}

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

void fill(double* x, int64_t n, double v, cudaStream_t s) {
  k_fill<<<152 * 4, 256, 0, s>>>(x, n, v);
}

__global__ void k_fill_f(float* x, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

void fill_f(float* x, int64_t n, float v, cudaStream_t s) { k_fill_f<<<152 * 4, 256, 0, s>>>(x, n, v); }

// Per-instance FP64 true residual norms ||f - A u|| / ||f||  (B values, device).
rbws_status residual_norms(rbws_problem p, const double* coef64, int B, const double* u,
                           double* r_out, double* rel_dev, const int* mask = nullptr, const float* uh = nullptr,
                           const float* ul = nullptr) {
  Tile t = choose_tile(p->nx);
  const int tiles = ((p->nx + t.tx - 1) / t.tx) * ((p->ny + t.ty - 1) / t.ty);
  const int zc = choose_zc(p->nz, (int64_t)tiles * B);
  const int P = tiles * ((p->nz + zc - 1) / zc);
  int err = 0;
  double* part = (double*)p->buf("res_part", sizeof(double) * (size_t)B * P, &err);
  if (err) return (rbws_status)err;
  const bool own_f = p->rhs.f != nullptr;
  if (uh)  // u = hi + lo formed on the way, and written to u
    launch_residual64_ff(p->geo, t, zc, coef64, B, own_f ? p->rhs.f : p->d_f, uh, ul, const_cast<double*>(u), r_out,
                         part, P, mask, p->cur, own_f ? p->rhs.stride : 0);
  else
    launch_residual64(p->geo, t, zc, coef64, B, own_f ? p->rhs.f : p->d_f, u, r_out, part, P, mask, p->cur,
                      own_f ? p->rhs.stride : 0);
  launch_norms_from_partials(part, B, P, p->fnorm, rel_dev, p->cur, own_f ? p->rhs.norms : nullptr);
  p->launches += 2;
  CK(cudaGetLastError());
  return RBWS_OK;
}

// Galerkin warm start u[b] = W A_N(mu_b)^{-1} fN.
// u = W c; fp32: with the FP32 copy of W (the mixed-precision solver's start).
// The FP32 copy of W used by the mixed-precision start (built on first use).
rbws_status ensure_w32(rbws_problem p) {
  if (!p->d_W32) {
    CK(cudaMalloc(&p->d_W32, sizeof(float) * (size_t)p->N * p->n));
    launch_to_f32((int64_t)p->N * p->n, p->d_W, p->d_W32, p->cur);
    p->launches += 1;
  }
  return RBWS_OK;
}

rbws_status lift(rbws_problem p, const double* C, int B, double* u, bool fp32) {
  if (fp32) {
    CKI(ensure_w32(p));
    launch_lift32(p->n, p->N, p->d_W32, C, B, u, p->cur);
  } else {
    launch_lift(p->n, p->N, p->d_W, C, B, u, p->cur);
  }
  p->launches += 1;
  return RBWS_OK;
}

rbws_status galerkin_start(rbws_problem p, const double* d_mu, int B, double* u, bool fp32 = false) {
  if (p->N <= 0) {
    set_error("no reduced basis: run rbws_offline_greedy or rbws_set_basis first");
    return RBWS_ERR_NO_BASIS;
  }
  int err = 0;
  double* C = (double*)p->buf("C", sizeof(double) * (size_t)B * p->N, &err);
  int* info = err ? nullptr : (int*)p->buf("info", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  if (p->rhs.f) {  // per-instance right-hand sides: W^T f_b (given, or formed over the batch)
    const double* fN = p->rhs.fN;
    int64_t sb = p->rhs.fN_sb, sj = p->rhs.fN_sj;
    if (!fN) {
      double* FN = (double*)p->buf("rhs_FN", sizeof(double) * (size_t)p->N * B, &err);
      if (err) return (rbws_status)err;
      if (fp32) {
        // the mixed-precision start: one pass over the sources with the FP32 copy of W (as
        // its lift uses), FP32 products and FP64 sums.  The start is a starting guess; the
        // FP64 residual of u0 is what the iteration corrects, so its accuracy is not at stake.
        CKI(ensure_w32(p));
        double* part = (double*)p->buf("rhs_proj",
                                       sizeof(double) * (size_t)project32_splits(p->n, B) * p->N * B, &err);
        if (err) return (rbws_status)err;
        if (launch_project32(p->n, p->N, B, p->d_W32, p->rhs.f, p->rhs.stride, part, FN, p->cur)) {
          set_error("reduced basis too large for the projection (N > 160)");
          return RBWS_ERR_INVALID_ARG;
        }
        p->launches += 2;
      } else {  // FP64: N dot launches over the batch
        const int scratch_len = 256 * (B + 2);
        double* scr = (double*)p->buf("rhs_scr", sizeof(double) * scratch_len, &err);
        if (err) return (rbws_status)err;
        for (int j = 0; j < p->N; j++)
          launch_multi_dot(p->n, B, p->rhs.f, p->rhs.stride, p->d_W + (int64_t)j * p->n, FN + (int64_t)j * B,
                           scr, scratch_len, p->cur);
        p->launches += p->N;
      }
      fN = FN;
      sb = 1;
      sj = B;
    }
    launch_reduced_solve(p->N, p->Q, p->d_ANq, fN, d_mu, B, C, info, nullptr, p->cur, sb, sj);
  } else {
    launch_reduced_solve(p->N, p->Q, p->d_ANq, p->d_fN, d_mu, B, C, info, nullptr, p->cur);
  }
  p->launches += 1;
  CKI(lift(p, C, B, u, fp32));
  CK(cudaGetLastError());
  std::vector<int> h(B);
  CKI(read_small(p, info, sizeof(int) * B, h.data(), p->cur));
  for (int b = 0; b < B; b++)
    if (h[b] != 0) {
      set_error("reduced matrix A_N(mu) is not positive definite for instance " + std::to_string(b));
      return RBWS_ERR_NOT_SPD;
    }
  return RBWS_OK;
}

// The 27-wide rows of each affine term on the finest level, by class ([Q][ncls][27]):
// from the block description, or, for a face-field problem, each node's 7-point row.
std::vector<double> fine_rows(rbws_problem p) {
  if (!p->field)
    return fine_rows_q(p->ax, p->ay, p->az, p->bx, p->by, p->h_segq.empty() ? nullptr : p->h_segq.data(), p->Q,
                       p->sx, p->sy, p->sz);
  std::vector<double> tq((size_t)p->Q * p->n * 27, 0.0);
  // table order -kW -kE -kS -kN -kD -kU D; 27-wide offsets (dz+1)*9 + (dy+1)*3 + (dx+1)
  static const int o27[7] = {12, 14, 10, 16, 4, 22, 13};
  for (size_t r = 0; r < (size_t)p->Q * p->n; r++)
    for (int m = 0; m < 7; m++) tq[r * 27 + o27[m]] = p->h_frows[r * 7 + m];
  return tq;
}

// The multigrid hierarchy of the problem (built on first use).
rbws_status mg_plan(rbws_problem p, const MGPlan** out) {
  if (!p->mg_tried) {
    p->mg_tried = true;
    auto plan = std::make_unique<MGPlan>();
    p->mg_err = mg_build_plan(p->ax, p->ay, p->az, fine_rows(p), p->Q, plan.get());
    if (p->mg_err.empty()) p->mg = std::move(plan);
  }
  if (!p->mg) {
    set_error(p->mg_err);
    return RBWS_ERR_UNSUPPORTED;
  }
  *out = p->mg.get();
  return RBWS_OK;
}

// Per-batch V-cycle state: level views, work vectors, coarse tables and the
// level-0 inverses for B parameters (device mu); coef = the finest level's
// tables, FP32 (fp32 = 1, the mixed-precision inner iteration) or FP64.
rbws_status mg_batch(rbws_problem p, const double* d_mu, int B, const void* coef, int fp32, const InstState* st,
                     MGBatch* m) {
  const MGPlan* plan = nullptr;
  CKI(mg_plan(p, &plan));
  m->plan = plan;
  m->B = B;
  m->fp32 = fp32;
  m->st = st;
  const size_t el = fp32 ? sizeof(float) : sizeof(double);
  const std::string tag = fp32 ? "mg32_" : "mg64_";
  int err = 0;
  void* tables[kMGMaxLevels] = {};
  for (int i = 0; i <= plan->J && !err; i++) {
    const MGPlan::Level& L = plan->lv[i];
    MGLevel& v = m->lv[i];
    v.nx = L.nx, v.ny = L.ny, v.nz = L.nz, v.n = L.n;
    v.ncx = L.ncx, v.ncy = L.ncy, v.ncz = L.ncz;
    const std::string k = std::to_string(i);
    const size_t vec = el * (size_t)B * L.n;
    if (i == plan->J) {
      v.cx = p->geo.cx, v.cy = p->geo.cy, v.cz = p->geo.cz;
      v.coef = coef;
      v.stride = kCoefStride;
    } else {
      v.cx = plan->d_cls[i], v.cy = v.cx + L.nx, v.cz = v.cy + L.ny;
      v.stride = 28;
      m->rhs[i] = p->buf(tag + "rhs" + k, vec, &err);
      if (!err) m->sol[i] = p->buf(tag + "sol" + k, vec, &err);
      if (i >= 1 && !err) {
        tables[i] = p->buf(tag + "tab" + k, el * (size_t)B * L.ncls() * 28, &err);
        v.coef = tables[i];
      }
    }
    if (i >= 1 && !err) {
      m->w1[i] = p->buf(tag + "w1_" + k, vec, &err);
      if (!err) m->w2[i] = p->buf(tag + "w2_" + k, vec, &err);
    }
  }
  const size_t dense = (size_t)B * plan->n0 * plan->n0;
  double* da = err ? nullptr : (double*)p->buf("mg_dense_a", sizeof(double) * dense, &err);
  double* dl = err ? nullptr : (double*)p->buf("mg_dense_l", sizeof(double) * dense, &err);
  double* ai = err ? nullptr : (double*)p->buf("mg_dense_inv", sizeof(double) * dense, &err);
  float* ai32 = (err || !fp32) ? nullptr : (float*)p->buf("mg_dense_inv32", sizeof(float) * dense, &err);
  int* info = err ? nullptr : (int*)p->buf("mg_info", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  m->ainv = fp32 ? (const void*)ai32 : (const void*)ai;
  launch_mg_setup(*plan, d_mu, B, fp32, tables, da, dl, ai, ai32, info, p->cur);
  p->launches += plan->J + 1;
  CK(cudaGetLastError());
  std::vector<int> h(B);
  CKI(read_small(p, info, sizeof(int) * B, h.data(), p->cur));
  for (int b = 0; b < B; b++)
    if (h[b]) {
      set_error("multigrid: coarsest-level matrix not positive definite");
      return RBWS_ERR_NOT_SPD;
    }
  return RBWS_OK;
}

// The FP64 iteration state of one problem's batch, ready for the PCG loop.
struct Fp64Batch {
  CGArgs<double> a{};
  Tile t{0, 0};
  MGBatch mgb;  // outlives the loop: the launchers read it while capturing
};

bool persistent_ok(const rbws_options& o) {
  return o.persistent != 0 && o.precision == RBWS_FP64 && !o.profile &&
         (o.precond == RBWS_PREC_NONE || o.precond == RBWS_PREC_JACOBI);
}

rbws_status prepare_fp64(rbws_problem p, const double* d_mu, int B, double tol, const rbws_options& o, double* u,
                         Fp64Batch* fb, Tile t) {
  double* coef64 = nullptr;
  CKI(coef_tables(p, d_mu, B, &coef64, nullptr));
  fb->t = t;
  CGArgs<double>& a = fb->a;
  CKI(make_cg_args<double>(p, B, t, coef64, u, &a, "d_"));
  a.f = p->rhs.f ? p->rhs.f : p->d_f;
  a.f_stride = p->rhs.f ? p->rhs.stride : 0;
  a.tol = tol;
  a.max_iters = o.max_iters;
  a.precond = o.precond;
  a.wait_cycles = o.wait_cycles;
  if (o.precond == RBWS_PREC_MSRB) {
    if (p->N <= 0) {
      set_error("MSRB preconditioner needs a reduced basis");
      return RBWS_ERR_NO_BASIS;
    }
    int err = 0;
    const int N = p->N;
    a.W = p->d_W;
    a.N = N;
    a.proj_chunks = (int)std::max<int64_t>(8, std::min<int64_t>(256, (4 * 1216 + B - 1) / B));
    double* L = (double*)p->buf("msrb_L", sizeof(double) * (size_t)B * N * N, &err);
    if (!err) a.G = (double*)p->buf("msrb_G", sizeof(double) * (size_t)B * N, &err);
    if (!err) a.C = (double*)p->buf("msrb_C", sizeof(double) * (size_t)B * N, &err);
    if (!err) a.proj_part = (double*)p->buf("msrb_part", sizeof(double) * (size_t)B * a.proj_chunks * N, &err);
    int* info = err ? nullptr : (int*)p->buf("msrb_info", sizeof(int) * (size_t)B, &err);
    if (err) return (rbws_status)err;
    a.L = L;
    launch_reduced_solve(N, p->Q, p->d_ANq, p->d_fN, d_mu, B, a.C, info, L, p->cur);
    p->launches += 1;
    std::vector<int> h(B);
    CK(cudaMemcpyAsync(h.data(), info, sizeof(int) * B, cudaMemcpyDeviceToHost, p->cur));
    CK(cudaStreamSynchronize(p->cur));
    for (int b = 0; b < B; b++)
      if (h[b]) {
        set_error("MSRB: A_N(mu) not positive definite");
        return RBWS_ERR_NOT_SPD;
      }
  }
  if (o.precond == RBWS_PREC_MG) {
    CKI(mg_batch(p, d_mu, B, coef64, 0, a.st, &fb->mgb));
    a.mg = &fb->mgb;
  }
  if (p->rhs.f) CK(cudaMemcpyAsync((double*)a.fnorm, p->rhs.norms, sizeof(double) * B, cudaMemcpyDeviceToDevice, p->cur));
  else fill((double*)a.fnorm, B, p->fnorm, p->cur);
  p->launches += 1;
  if (o.relres_hist) {
    int err = 0;
    a.hist_len = o.hist_len;
    a.hist = (double*)p->buf("hist", sizeof(double) * (size_t)B * o.hist_len, &err);
    if (err) return (rbws_status)err;
    fill(a.hist, (int64_t)B * o.hist_len, std::nan(""), p->cur);
    p->launches += 1;
  }
  return RBWS_OK;
}

// One cooperative launch of the persistent FP64 PCG over the prepared batches (one per
// problem), on the stream s; returns after it completed.
rbws_status run_persistent(rbws_problem p, const std::vector<CGArgs<double>>& args, Tile t, const rbws_options& o,
                           cudaStream_t s) {
  int err = 0;
  int* ctl = (int*)p->buf("pcg_ctl", sizeof(int) * 4, &err);
  void* tasks = err ? nullptr : p->buf("pcg_tasks", pcg_persistent_task_bytes() * args.size(), &err);
  if (err) return (rbws_status)err;
  int max_it = 0;
  for (const auto& a : args) max_it = std::max(max_it, a.max_iters);
  // each round is one iteration or one true-residual check
  const int rounds = (int)std::min<int64_t>((int64_t)(max_it + 2) * (o.max_restarts + 2), 1 << 30);
  if (launch_pcg_persistent(args, t, ctl, ctl + 2, o.wait_cycles, o.max_restarts, rounds, tasks, s) < 0) {
    cudaGetLastError();
    set_error("persistent PCG: the cooperative launch failed");
    return RBWS_ERR_CUDA;
  }
  p->launches += 1;
  int terr = 0;
  CK(cudaMemcpyAsync(&terr, ctl + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (terr) {
    set_error("persistent PCG: a grid barrier wait ran out of time");
    return RBWS_ERR_DEVICE_TIMEOUT;
  }
  return RBWS_OK;
}

rbws_status solve_fp64(rbws_problem p, const double* d_mu, int B, double tol, const rbws_options& o,
                       double* u, std::vector<InstState>& st) {
  Fp64Batch fb;
  CKI(prepare_fp64(p, d_mu, B, tol, o, u, &fb, choose_tile(p->nx)));
  CGArgs<double>& a = fb.a;
  if (persistent_ok(o)) {
    CKI(run_persistent(p, {a}, fb.t, o, p->cur));
  } else {
    CKI(run_pcg<double>(p, a, fb.t, o.max_restarts, o.check_every, nullptr, true, o.profile));
  }
  st.resize(B);
  CK(cudaMemcpyAsync(st.data(), a.st, sizeof(InstState) * B, cudaMemcpyDeviceToHost, p->cur));
  if (o.relres_hist)
    CK(cudaMemcpyAsync(o.relres_hist, a.hist, sizeof(double) * (size_t)B * o.hist_len, cudaMemcpyDeviceToHost,
                       p->cur));
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

// The FP32 V-cycle state for a batch: the level tables and vectors, and with the
// 4-node kernels (v4) the finest level fused on the iteration's arguments a (tile t)
// and the wider MG tiles of the steps that write no partials.
rbws_status mg_fp32_batch(rbws_problem p, const double* d_mu, int B, const float* coef32, bool v4, Tile t,
                          CGArgs<float>* a, MGBatch* mgb) {
  CKI(mg_batch(p, d_mu, B, coef32, 1, a->st, mgb));
  if (v4) {
    tma_prepare();  // the TMA-fed finest-level steps
    mgb->fine_cg = a;
    mgb->fine_tile = t;
    const Tile tm = choose_tile_v4(p->nx, p->ny);
    mgb->mg_tile = tm;
    mgb->mg_tiles_x = (p->nx + 4 * tm.tx - 1) / (4 * tm.tx);
    mgb->mg_tiles_y = (p->ny + tm.ty - 1) / tm.ty;
    mgb->mg_zc = choose_zc_v4(p->nz, (int64_t)mgb->mg_tiles_x * mgb->mg_tiles_y * B);
    mgb->mg_nzc = (p->nz + mgb->mg_zc - 1) / mgb->mg_zc;
    // omega / D per node, staged beside the rhs by the first pre-smoothing step (nx % 4 == 0)
    if (p->nx % 4 == 0) {
      int err = 0;
      float* od = (float*)p->buf("mg_od", sizeof(float) * (size_t)B * p->n, &err);
      if (err) return (rbws_status)err;
      launch_omega_dinv(p->geo, coef32, B, (float)kMGOmega, od, p->cur);
      p->launches += 1;
      CK(cudaGetLastError());
      mgb->od = od;
    }
  }
  return RBWS_OK;
}

// FP32 Jacobi-PCG inside FP64 iterative refinement, with reliable updates:
// the FP32 iteration accumulates its correction d; whenever an instance's
// FP32 residual has dropped by the factor inner_tol since its last update (or
// meets tol), the correction is folded into the FP64 solution u, the FP64
// residual f - A u is formed, and the FP32 residual is reset from it.  The
// search direction is kept across updates (restarted only when an FP64 check
// after apparent convergence fails), so the Krylov space is not thrown away
// at every refinement step.  Convergence is decided on the FP64 residual.
rbws_status solve_fp32_ir(rbws_problem p, const double* d_mu, int B, double tol,
                          const rbws_options& o, double* u, std::vector<InstState>& st) {
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &coef64, &coef32));
  Tile t4 = choose_tile_v4(p->nx, p->ny);
  // Schedules: 0 = 44 bytes per DoF-iteration (s and A p stored), stencil
  // phase with register prefetch; 2 = the same with the stencil phase fed by
  // TMA (default where the tensor maps can be built); 1 = 32 bytes (s formed
  // on the fly, A p recomputed); 3 = 32 bytes with s = D^{-1} r as the stored
  // residual and both phases fed by TMA.  The 44-byte update phase is a pure stream
  // (97% of HBM on the 64^3 workload) while both 32-byte phases are stencil
  // kernels; the autotuner picks whichever is fastest.
  int zc_force = 0, sched = 2;
  auto tu = p->tuned32.find(B);
  if (t4.tx > 0 && tu != p->tuned32.end()) {
    t4 = Tile{tu->second.tx, tu->second.ty};
    zc_force = tu->second.zc;
    sched = tu->second.sched;
  }
  const bool v4 = t4.tx > 0;
  if (!v4) sched = 0;
  const bool mg = o.precond == RBWS_PREC_MG;
  if (mg && sched == 1) sched = 0;  // the 32-byte schedules store no separate s: Jacobi only
  if (mg && sched == 3) sched = 2;
  const Tile t = v4 ? t4 : choose_tile(p->nx);
  if ((sched == 2 || sched == 3) && !tma_supported(p->geo, t)) sched = 0;
  if (sched == 2 || sched == 3) tma_prepare();
  const int sched32 = sched == 1 || sched == 3;
  int* tma_err = nullptr;  // set by make_cg_args below: the third int of the counter block
  auto phase_a = [&](const CGArgs<float>& aa, int par, cudaStream_t ss) {
    if (sched == 1) launch_cg_a32_v4(aa, t, par, ss);
    else if (sched == 2) {
      if (launch_cg_a_tma(aa, t, par, tma_err, ss)) launch_cg_a_v4(aa, t, par, ss);
    } else if (sched == 3) launch_cg_a_s_tma(aa, t, par, tma_err, ss);
    else if (v4) launch_cg_a_v4(aa, t, par, ss);
    else launch_cg_a<float>(aa, t, par, ss);
  };
  MGBatch mgb;  // FP32 V-cycle state; outlives the captured graph's launches
  int mg_launches = 0;
  // s = MG(r) and the partials of rho = r.s into `slot`, for the instances in
  // mgb.mask (all when null)
  auto mg_apply = [&](const CGArgs<float>& aa, int slot, cudaStream_t ss) {
    const bool fused = mgb.fine_cg && mgb.plan->J > 0;  // the fused finest level writes rho itself
    int l = launch_mg_vcycle(mgb, aa.r, aa.s, fused ? slot : -1, ss);
    if (fused) return l;
    if (v4) launch_precond_rho_v4(aa, t, slot, mgb.mask, ss);
    else launch_precond_rho<float>(aa, t, slot, mgb.mask, ss);
    return l + 1;
  };
  auto phase_b_core = [&](const CGArgs<float>& aa, int par, cudaStream_t ss) {
    if (sched == 1) launch_cg_b32_v4(aa, t, par, ss);
    else if (sched == 3) launch_cg_b_s_tma(aa, t, par, tma_err, ss);
    else if (v4) launch_cg_b_v4(aa, t, par, ss);
    else launch_cg_b<float>(aa, t, par, ss);
  };
  auto phase_b = [&](const CGArgs<float>& aa, int par, cudaStream_t ss) {
    phase_b_core(aa, par, ss);
    if (mg) mg_launches = mg_apply(aa, par ^ 1, ss);
  };
  // With MG the V-cycle of a block's last iteration is deferred to the start of
  // the next block (slot 0), after any reliable update: an instance whose FP32
  // residual is replaced then takes one V-cycle, on its new residual, not two.
  auto reset = [&](const CGArgs<float>& aa, int start, cudaStream_t ss) {
    if (v4) launch_ru_reset_v4(aa, t, start, ss);
    else launch_ru_reset(aa, t, start, ss);
  };
  cudaStream_t s = p->cur;
  int err = 0;
  float* d = (float*)p->buf("ir_d", sizeof(float) * (size_t)B * p->n, &err);
  double* r64 = err ? nullptr : (double*)p->buf("ir_r64", sizeof(double) * (size_t)B * p->n, &err);
  double* rel = err ? nullptr : (double*)p->buf("ir_rel", sizeof(double) * (size_t)B, &err);
  double* rr_ref = err ? nullptr : (double*)p->buf("ir_rr_ref", sizeof(double) * (size_t)B, &err);
  int* upd = err ? nullptr : (int*)p->buf("ir_upd", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  CGArgs<float> a{};
  CKI(make_cg_args<float>(p, B, t, coef32, d, &a, "f_", v4 ? 4 : 1, zc_force));
  tma_err = a.active + 2;  // counters: active, pending, TMA error flag
  a.f = nullptr;
  a.tol = tol;
  a.max_iters = o.max_iters;
  a.precond = o.precond;
  a.wait_cycles = o.wait_cycles;
  a.ru = 1;
  // auto: 1e-2.  With MG (about a decade per iteration) and blocks of 2 iterations
  // that keeps the FP32 recursion within about four decades of its last update.
  // Smaller factors save FP64 updates but were not robust: 1e-3 left zero-start
  // instances of the 64^3 workload at twice the FP64 iteration count, and 1e-4
  // let a contrast-1e4 test instance take 142 iterations instead of 17.
  const double delta = (o.inner_tol > 0.0 && o.inner_tol < 1.0) ? o.inner_tol : 1e-2;
  a.ru_delta2 = delta * delta;
  a.rr_ref = rr_ref;
  a.pending = a.active + 1;
  a.upd = upd;
  a.u64 = u;
  a.r64 = r64;
  a.rel64 = rel;
  if (mg) CKI(mg_fp32_batch(p, d_mu, B, coef32, v4, t, &a, &mgb));
  if (sched32) {
    a.alpha = (double*)p->buf("ir_alpha", sizeof(double) * 2 * (size_t)B, &err);
    if (err) return (rbws_status)err;
    CK(cudaMemsetAsync(a.alpha, 0, sizeof(double) * 2 * (size_t)B, s));
  }
  if (p->rhs.f) CK(cudaMemcpyAsync((double*)a.fnorm, p->rhs.norms, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
  else fill((double*)a.fnorm, B, p->fnorm, s);
  // Reliable updates in float-float on the FP32 pipe (ru_ff.cu) with the 4-node tiles; FP64
  // updates otherwise or when asked for.  Either way convergence is decided in FP64.
  const bool ffu = v4 && o.ru_mode != 1;
  FFState ff{};
  if (ffu) {
    const size_t vb = sizeof(float) * (size_t)B * p->n;
    ff.uh = (float*)p->buf("ff_uh", vb, &err);
    if (!err) ff.ul = (float*)p->buf("ff_ul", vb, &err);
    if (!err) ff.rh = (float*)p->buf("ff_rh", vb, &err);
    if (!err) ff.rl = (float*)p->buf("ff_rl", vb, &err);
    float* cff = err ? nullptr
                     : (float*)p->buf("ff_coef", sizeof(float) * 2 * kCoefStride * (size_t)B * p->geo.ncls(), &err);
    if (!err) ff.part = (double*)p->buf("ff_part", sizeof(double) * (size_t)B * a.P, &err);
    if (!err) ff.rel = (double*)p->buf("ff_rel", sizeof(double) * (size_t)B, &err);
    if (!err) ff.chk = (int*)p->buf("ff_chk", sizeof(int) * (size_t)B, &err);
    if (err) return (rbws_status)err;
    ff.coef = cff;
    ff.f = p->rhs.f ? p->rhs.f : p->d_f;
    ff.f_stride = p->rhs.f ? p->rhs.stride : 0;
    launch_coef_ff(coef64, (int64_t)B * p->geo.ncls(), cff, s);
    p->launches += 1;
  }
  // one reliable update of the flagged instances (upd), inside or outside a capture:
  // float-float r -= A d, u += d; the FP64 check of those meeting tol; the reset
  auto update_ff = [&](bool start, cudaStream_t ss) -> rbws_status {
    launch_ru_ff(a, t, ff, start, ss);
    launch_norms_from_partials(ff.part, B, a.P, p->fnorm, ff.rel, ss, a.fnorm);
    launch_ru_mark(a, ff, ss);
    // the FP64 check of the marked: u = hi + lo written as the residual kernel stages it
    const rbws_status rr = residual_norms(p, coef64, B, u, r64, rel, ff.chk, ff.uh, ff.ul);
    launch_ru_reset_ff(a, t, ff, start ? 1 : 0, ss);
    return rr;
  };
  CK(cudaMemsetAsync(d, 0, sizeof(float) * (size_t)B * p->n, s));
  // start: every instance takes an update from u (restarting its direction)
  std::vector<int> two(B, 2);
  CK(cudaMemcpyAsync(upd, two.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(a.active, 0, 3 * sizeof(int), s));
  if (ffu) {
    CKI(update_ff(true, s));
    p->launches += 6;
  } else {
    CKI(residual_norms(p, coef64, B, u, r64, rel, upd));
    reset(a, 1, s);
    p->launches += 2;
  }
  CK(cudaGetLastError());
  // The reliable-update test runs at block boundaries.  A multigrid-preconditioned
  // iteration gains about a decade per step, so blocks of 8 would carry the FP32
  // recursion far below its own accuracy floor (it then stagnates or breaks down);
  // with MG the blocks are 2 iterations long.
  int M = o.check_every > 0 ? o.check_every : (mg ? 2 : 8);
  if (M % 2) M++;
  rbws_profile* prof = o.profile;
  if (prof) {
    prof->elem_bytes = 4;
    prof->schedule = v4 ? sched : -1;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t ce;
  // One block: the previous block's last preconditioning, M iterations, the decision and the
  // reliable update of the instances it flagged (the others leave those kernels at once).
  auto record_block = [&](cudaStream_t ss) -> rbws_status {
    if (mg) mg_launches = mg_apply(a, 0, ss);
    for (int k = 0; k < M; k++) {
      phase_a(a, k & 1, ss);
      if (mg && k == M - 1) phase_b_core(a, k & 1, ss);
      else phase_b(a, k & 1, ss);
    }
    cudaMemsetAsync(a.pending, 0, sizeof(int), ss);
    launch_ru_decide(a, ss);
    if (ffu) return update_ff(false, ss);
    launch_ru_fold(a, ss);
    const rbws_status rr = residual_norms(p, coef64, B, u, r64, rel, upd);
    reset(a, 0, ss);
    return rr;
  };
  // The blocks run inside one graph launch: a conditional while node repeats the block while
  // a one-thread kernel at its end finds instances still active (and no TMA wait ran out,
  // and fewer than loop_cap blocks ran).  The host then reads nothing between blocks: such a
  // read (a device-to-host copy of the counts and a wait) queues behind any large copy the
  // caller has on the same copy engine, e.g. the previous batch's solutions going back to
  // the host, and the GPU would idle until that copy ends.  If the driver cannot build the
  // conditional graph, the host loop below launches one block at a time.
  int* loop_ctr = nullptr;
  bool in_graph_loop = false;
  const int loop_cap = 2 * std::max(o.max_iters, 1) / M + 64;
  if (!prof) {
    const int64_t launches0 = p->launches;
    int err = 0;
    loop_ctr = (int*)p->buf("loop_ctr", sizeof(int), &err);
    if (err) return (rbws_status)err;
    cudaGraphConditionalHandle handle;
    cudaGraph_t body = nullptr;
    ce = cudaGraphCreate(&graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (ce == cudaSuccess) {
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node;
      ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
      if (ce == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (ce == cudaSuccess) ce = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      const rbws_status rr = record_block(s);
      launch_loop_condition(handle, a.active, loop_ctr, loop_cap, s);
      cudaGraph_t captured = nullptr;
      ce = cudaStreamEndCapture(s, &captured);
      if (rr != RBWS_OK) {
        cudaGraphDestroy(graph);
        return rr;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    }
    if (ce == cudaSuccess) {
      in_graph_loop = true;
    } else {  // the one-block graph of the host loop
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const rbws_status rr = record_block(s);
      ce = cudaStreamEndCapture(s, &graph);
      if (rr != RBWS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rr;
      }
      if (ce != cudaSuccess) return (rbws_status)cuda_fail(ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&exec, graph, 0);
      if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return (rbws_status)cuda_fail(ce, "cudaGraphInstantiate");
      }
    }
    p->launches = launches0;
  }
  rbws_status rc = RBWS_OK;
  int counts[3];
  if (in_graph_loop) {
    // the counts before the first block come from the start (no block has run yet)
    rc = read_small(p, a.active, 3 * sizeof(int), counts, s);
    if (rc == RBWS_OK && counts[0] > 0 && !counts[2]) {
      int blocks = 0;
      cudaMemsetAsync(loop_ctr, 0, sizeof(int), s);
      if ((ce = cudaGraphLaunch(exec, s)) != cudaSuccess) rc = (rbws_status)cuda_fail(ce, "cudaGraphLaunch");
      if (rc == RBWS_OK) rc = read_small(p, loop_ctr, sizeof(int), &blocks, s);
      p->launches += (int64_t)blocks * ((2 + mg_launches) * M + 2 + (ffu ? 7 : 4));
    }
  }
  for (; !in_graph_loop;) {
    if ((rc = read_small(p, a.active, 3 * sizeof(int), counts, s)) != RBWS_OK) break;
    if (counts[2]) break;  // a TMA stage wait ran out; reported below
    const int active = counts[0];
    if (active == 0) break;
    if (!prof) {
      if ((ce = cudaGraphLaunch(exec, s)) != cudaSuccess) {
        rc = (rbws_status)cuda_fail(ce, "cudaGraphLaunch");
        break;
      }
    } else {
      if (mg) mg_launches = mg_apply(a, 0, s);
      cudaEventRecord(p->tev[0], s);
      phase_a(a, 0, s);
      cudaEventRecord(p->tev[1], s);
      phase_b_core(a, 0, s);
      cudaEventRecord(p->tev[2], s);
      if (mg) {
        if (mgb.fine_cg && mgb.plan->J > 0) mgb.ev = p->mgev;
        mg_launches = mg_apply(a, 1, s);
        mgb.ev = nullptr;
      }
      cudaEventRecord(p->tev[3], s);
      for (int k = 1; k < M; k++) {
        phase_a(a, k & 1, s);
        if (mg && k == M - 1) phase_b_core(a, k & 1, s);
        else phase_b(a, k & 1, s);
      }
      cudaMemsetAsync(a.pending, 0, sizeof(int), s);
      launch_ru_decide(a, s);
      if (ffu) {
        if ((rc = update_ff(false, s)) != RBWS_OK) break;
      } else {
        launch_ru_fold(a, s);
        if ((rc = residual_norms(p, coef64, B, u, r64, rel, upd)) != RBWS_OK) break;
        reset(a, 0, s);
      }
      if ((ce = cudaEventSynchronize(p->tev[3])) != cudaSuccess) {
        rc = (rbws_status)cuda_fail(ce, "profile events");
        break;
      }
      float ta = 0.f, tb = 0.f, tp = 0.f;
      cudaEventElapsedTime(&ta, p->tev[0], p->tev[1]);
      cudaEventElapsedTime(&tb, p->tev[1], p->tev[2]);
      cudaEventElapsedTime(&tp, p->tev[2], p->tev[3]);
      prof->stencil_ms += ta;
      prof->update_ms += tb;
      if (mg) {
        prof->precond_ms += tp;
        if (mgb.fine_cg && mgb.plan->J > 0)
          for (int k = 0; k < 4; k++) {
            float tk = 0.f;
            cudaEventElapsedTime(&tk, p->mgev[2 * k], p->mgev[2 * k + 1]);
            prof->mg_fine_ms[k] += tk;
            if (k == 2) {  // the prolongation pass alone (the first part of step 2)
              cudaEventElapsedTime(&tk, p->mgev[4], p->mgev[8]);
              prof->mg_prolong_ms += tk;
            }
          }
      }
      prof->active_dofs += (double)active * (double)p->n;
      prof->samples += 1;
    }
    // + decide and the update: fold, residual, norms, reset (FP64); or the float-float
    // update, norms, mark, conversion, FP64 residual and norms (masked), reset
    p->launches += (2 + mg_launches) * M + 1 + (ffu ? 7 : 4);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc != RBWS_OK) return rc;
  {
    int terr = 0;
    CKI(read_small(p, tma_err, sizeof(int), &terr, s));
    if (terr) {
      set_error("a TMA stage wait ran out of time in the FP32 stencil phase");
      return RBWS_ERR_DEVICE_TIMEOUT;
    }
  }
  // instances stopped by max_iters or breakdown still hold a correction in d
  std::vector<InstState> h(B);
  static_assert(sizeof(InstState) % 4 == 0, "read_small copies 4-byte words");
  CKI(read_small(p, a.st, sizeof(InstState) * B, h.data(), s));
  std::vector<int> fin(B);
  int nfin = 0;
  // mode 2: the fold adds the update still pending at the parity recorded when the instance stopped
  for (int b = 0; b < B; b++) nfin += (fin[b] = (h[b].status == ST_MAX_ITERS || h[b].status == ST_BREAKDOWN) ? 2 : 0) != 0;
  if (nfin) {
    CK(cudaMemcpyAsync(upd, fin.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
    if (ffu) {
      launch_ff_fold(a, ff, s);
      launch_ff_to64(a, ff, upd, s);
      p->launches += 1;
    } else {
      launch_ru_fold(a, s);
    }
    CKI(residual_norms(p, coef64, B, u, r64, rel, upd));
    std::vector<double> hr(B);
    CKI(read_small(p, rel, sizeof(double) * B, hr.data(), s));
    for (int b = 0; b < B; b++)
      if (fin[b]) h[b].relres = hr[b];
    p->launches += 3;
  }
  st = h;
  return RBWS_OK;
}


// ---------------------------------------------------------------------------
// Surrogate network p -> H -> H -> H -> N (GELU), parameters laid out as
// W1[H][p] b1[H] W2[H][H] b2[H] W3[H][H] b3[H] W4[N][H] b4[N].
// ---------------------------------------------------------------------------
struct NetLayout {
  int p, H, N;
  int64_t W[4], b[4], P;
  int in[4], out[4];
};

NetLayout net_layout(int p, int H, int N) {
  NetLayout L;
  L.p = p;
  L.H = H;
  L.N = N;
  const int in[4] = {p, H, H, H}, out[4] = {H, H, H, N};
  int64_t o = 0;
  for (int l = 0; l < 4; l++) {
    L.in[l] = in[l];
    L.out[l] = out[l];
    L.W[l] = o;
    o += (int64_t)in[l] * out[l];
    L.b[l] = o;
    o += out[l];
  }
  L.P = o;
  return L;
}

// Activations of one batch (device buffers owned by the problem).
struct NetBufs {
  float *x, *Z[3], *A[3], *Y, *dY, *dA, *dZ, *loss;
};

rbws_status net_bufs(rbws_problem p, const NetLayout& L, int B, NetBufs* nb) {
  int err = 0;
  const size_t bh = sizeof(float) * (size_t)B * L.H;
  nb->x = (float*)p->buf("net_x", sizeof(float) * (size_t)B * L.p, &err);
  for (int l = 0; l < 3 && !err; l++) {
    nb->Z[l] = (float*)p->buf("net_Z" + std::to_string(l), bh, &err);
    if (!err) nb->A[l] = (float*)p->buf("net_A" + std::to_string(l), bh, &err);
  }
  if (!err) nb->Y = (float*)p->buf("net_Y", sizeof(float) * (size_t)B * L.N, &err);
  if (!err) nb->dY = (float*)p->buf("net_dY", sizeof(float) * (size_t)B * L.N, &err);
  if (!err) nb->dA = (float*)p->buf("net_dA", bh, &err);
  if (!err) nb->dZ = (float*)p->buf("net_dZ", bh, &err);
  if (!err) nb->loss = (float*)p->buf("net_loss1", sizeof(float) * 4, &err);
  return (rbws_status)err;
}

// Forward pass on inputs x [B][p] (float); output nb.Y [B][N].
void net_forward(rbws_problem p, const NetLayout& L, int B, const float* x, const NetBufs& nb, cudaStream_t s) {
  const char* w16 = static_cast<const char*>(p->d_w16);
  const void* in = x;
  int in_dim = L.p;
  for (int l = 0; l < 4; l++) {
    MlpGemm g{};
    g.M = B;
    g.N = L.out[l];
    g.K = L.in[l];
    g.A = in;
    g.sam = in_dim;
    g.sak = 1;
    g.a_bf16 = 0;
    g.B = w16 + 2 * L.W[l];
    g.sbk = 1;
    g.sbn = L.in[l];
    g.b_bf16 = 1;
    g.bias = p->d_w32 + L.b[l];
    g.Z = l < 3 ? nb.Z[l] : nb.Y;
    g.Aout = l < 3 ? nb.A[l] : nullptr;
    g.ldz = L.out[l];
    launch_mlp_gemm(g, s);
    in = nb.A[l < 3 ? l : 2];
    in_dim = L.H;
  }
  p->launches += 4;
}

// Backward pass from dY (nb.dY) into grad [P] (float).
void net_backward(rbws_problem p, const NetLayout& L, int B, const float* x, const NetBufs& nb, float* grad,
                  cudaStream_t s) {
  const char* w16 = static_cast<const char*>(p->d_w16);
  const float* dout = nb.dY;  // gradient w.r.t. the output of layer l
  for (int l = 3; l >= 0; l--) {
    const int no = L.out[l], ni = L.in[l];
    const float* ain = l == 0 ? x : nb.A[l - 1];
    // dW_l = dout^T a_in  ([no][ni], k over the batch)
    MlpGemm gw{};
    gw.M = no;
    gw.N = ni;
    gw.K = B;
    gw.A = dout;
    gw.sam = 1;
    gw.sak = no;
    gw.B = ain;
    gw.sbk = ni;
    gw.sbn = 1;
    gw.Z = grad + L.W[l];
    gw.ldz = ni;
    launch_mlp_gemm(gw, s);
    launch_bias_grad(dout, B, no, grad + L.b[l], s);
    p->launches += 2;
    if (l == 0) break;
    // d a_in = dout W_l  ([B][ni]), then through GELU of layer l-1
    MlpGemm gd{};
    gd.M = B;
    gd.N = ni;
    gd.K = no;
    gd.A = dout;
    gd.sam = no;
    gd.sak = 1;
    gd.B = w16 + 2 * L.W[l];
    gd.sbk = ni;
    gd.sbn = 1;
    gd.b_bf16 = 1;
    gd.Z = nb.dA;
    gd.ldz = ni;
    launch_mlp_gemm(gd, s);
    launch_gelu_back(nb.dA, nb.Z[l - 1], B * ni, nb.dZ, s);
    p->launches += 2;
    // every read of the previous dout (dW, db, dA) is ordered before this
    // overwrite of dZ on the stream, so one buffer serves all layers
    dout = nb.dZ;
  }
}

// c[b] = W^T-coefficients predicted by the network for mu[b] (device mu).
rbws_status net_predict(rbws_problem p, const double* d_mu, int B, double* c, bool corrected) {
  if (!p->d_w32 || p->net_N != p->N || p->N <= 0) {
    set_error("learned warm start needs a reduced basis and a surrogate trained for it");
    return RBWS_ERR_NO_BASIS;
  }
  const NetLayout L = net_layout(p->Q, p->net_H, p->net_N);
  NetBufs nb{};
  CKI(net_bufs(p, L, B, &nb));
  launch_mlp_inputs(d_mu, B, p->Q, p->net_lo, p->net_hi, nb.x, p->cur);
  net_forward(p, L, B, nb.x, nb, p->cur);
  launch_unscale(nb.Y, p->d_cscale, B, L.N, c, p->cur);
  p->launches += 2;
  if (corrected) {
    launch_reduced_cg_step(p->N, p->Q, p->d_ANq, p->d_fN, d_mu, B, c, p->cur);
    p->launches += 1;
  }
  CK(cudaGetLastError());
  return RBWS_OK;
}

rbws_status learned_start(rbws_problem p, const double* d_mu, int B, double* u, bool corrected, bool fp32) {
  int err = 0;
  double* C = (double*)p->buf("C", sizeof(double) * (size_t)B * (p->N > 0 ? p->N : 1), &err);
  if (err) return (rbws_status)err;
  CKI(net_predict(p, d_mu, B, C, corrected));
  CKI(lift(p, C, B, u, fp32));
  CK(cudaGetLastError());
  return RBWS_OK;
}

rbws_status net_alloc(rbws_problem p, int H, int N) {
  const NetLayout L = net_layout(p->Q, H, N);
  cudaFree(p->d_w32);
  cudaFree(p->d_w16);
  cudaFree(p->d_cscale);
  p->d_w32 = nullptr;
  p->d_w16 = nullptr;
  p->d_cscale = nullptr;
  p->net_H = p->net_N = 0;
  CK(cudaMalloc(&p->d_w32, sizeof(float) * L.P));
  CK(cudaMalloc(&p->d_w16, 2 * L.P));
  CK(cudaMalloc(&p->d_cscale, sizeof(float) * N));
  p->net_H = H;
  p->net_N = N;
  p->net_P = L.P;
  return RBWS_OK;
}


rbws_status check_solve_options(const rbws_options& o, double tol, int warm) {
  if (!(tol > 0.0) || o.max_iters < 0 || o.max_restarts < 0) {
    set_error("solve: invalid tolerance or limits");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.precond != RBWS_PREC_NONE && o.precond != RBWS_PREC_JACOBI && o.precond != RBWS_PREC_MSRB &&
      o.precond != RBWS_PREC_MG) {
    set_error("solve: unknown preconditioner");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.precond == RBWS_PREC_MSRB && o.precision != RBWS_FP64) {
    set_error("solve: the MSRB preconditioner runs in FP64 only");
    return RBWS_ERR_UNSUPPORTED;
  }
  if (warm < RBWS_WARM_ZERO || warm > RBWS_WARM_L1ROC) {
    set_error("solve: unknown warm-start mode");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.precision != RBWS_FP64 && o.precision != RBWS_FP32_IR) {
    set_error("solve: unknown precision");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.persistent != 0 && o.persistent != 1) {
    set_error("solve: persistent must be 0 or 1");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.ru_mode < 0 || o.ru_mode > 2) {
    set_error("solve: ru_mode must be 0, 1 or 2");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.wait_cycles < 0) {
    set_error("solve: wait_cycles must be >= 0");
    return RBWS_ERR_INVALID_ARG;
  }
  if (o.relres_hist && (o.precision != RBWS_FP64 || o.hist_len < 1)) {
    set_error("solve: the residual history needs FP64 precision and hist_len >= 1");
    return RBWS_ERR_INVALID_ARG;
  }
  return RBWS_OK;
}

// Warm start + PCG for B parameters (host mu) on the problem's current work
// stream; u: device [B][n].
// L1ROC online solve (Sec. 3.1): c[b] = argmin ||P (f - A(mu_b) W c)||_2.
rbws_status l1roc_coefficients(rbws_problem p, const double* d_mu, int B, double** C_out) {
  if (p->l1.N <= 0 || p->l1.N != p->N) {
    set_error("no L1ROC basis: run rbws_offline_l1roc first");
    return RBWS_ERR_NO_BASIS;
  }
  int err = 0;
  double* C = (double*)p->buf("C", sizeof(double) * (size_t)B * p->N, &err);
  int* info = err ? nullptr : (int*)p->buf("info", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  colloc_ls_prepare();
  launch_colloc_ls(p->l1.M, p->l1.N, p->Q, p->l1.d_PAWq, p->l1.d_Pf, d_mu, B, C, info, p->cur);
  p->launches += 1;
  CK(cudaGetLastError());
  std::vector<int> h(B);
  CK(cudaMemcpyAsync(h.data(), info, sizeof(int) * B, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  for (int b = 0; b < B; b++)
    if (h[b]) {
      set_error("L1ROC: the collocation matrix is rank deficient for instance " + std::to_string(b));
      return RBWS_ERR_STATE;
    }
  *C_out = C;
  return RBWS_OK;
}

rbws_status l1roc_start(rbws_problem p, const double* d_mu, int B, double* u, bool fp32) {
  double* C = nullptr;
  CKI(l1roc_coefficients(p, d_mu, B, &C));
  return lift(p, C, B, u, fp32);
}

// The parameters on the device and the initial value u0 (Algorithm 4, line 2).
rbws_status warm_start(rbws_problem p, const double* mu, int B, int warm, const rbws_options& o, double* u,
                       double** d_mu_out) {
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_solve"));
  if (warm == RBWS_WARM_ZERO) {
    CK(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)B * p->n, p->cur));
  } else if (warm == RBWS_WARM_GALERKIN) {
    CKI(galerkin_start(p, d_mu, B, u, o.precision == RBWS_FP32_IR));
  } else if (warm == RBWS_WARM_L1ROC) {
    CKI(l1roc_start(p, d_mu, B, u, o.precision == RBWS_FP32_IR));
  } else {
    CKI(learned_start(p, d_mu, B, u, warm == RBWS_WARM_LEARNED_CORRECTED, o.precision == RBWS_FP32_IR));
  }
  *d_mu_out = d_mu;
  return RBWS_OK;
}

rbws_status solve_batch_impl(rbws_problem p, const double* mu, int B, double tol, int warm,
                             const rbws_options& o, double* u, std::vector<InstState>& st) {
  if (o.profile) std::memset(o.profile, 0, sizeof(rbws_profile));
  double* d_mu = nullptr;
  CKI(warm_start(p, mu, B, warm, o, u, &d_mu));
  if (o.precision == RBWS_FP64) {
    CKI(solve_fp64(p, d_mu, B, tol, o, u, st));
  } else {
    CKI(solve_fp32_ir(p, d_mu, B, tol, o, u, st));
  }
  return RBWS_OK;
}

__global__ void k_stamp(unsigned long long* t) { *t = global_ns(); }
void launch_stamp(unsigned long long* t, cudaStream_t s) { k_stamp<<<1, 1, 0, s>>>(t); }

}  // namespace

// ===========================================================================
// L1ROC offline (Algorithm 5): DEIM on snapshots and on RB residuals, the
// over-collocation RB system (Sec. 3.1), and the L1 indicator.
// ===========================================================================
namespace {

// Solves the k x k system A x = b (row-major, partial pivoting); false if singular.
bool small_solve(int k, std::vector<double> A, std::vector<double>& b) {
  for (int c = 0; c < k; c++) {
    int piv = c;
    for (int r = c + 1; r < k; r++)
      if (std::fabs(A[(size_t)r * k + c]) > std::fabs(A[(size_t)piv * k + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * k + c]) > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < k; j++) std::swap(A[(size_t)c * k + j], A[(size_t)piv * k + j]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < k; r++) {
      const double f = A[(size_t)r * k + c] / A[(size_t)c * k + c];
      for (int j = c; j < k; j++) A[(size_t)r * k + j] -= f * A[(size_t)c * k + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = k - 1; r >= 0; r--) {
    double v = b[r];
    for (int j = r + 1; j < k; j++) v -= A[(size_t)r * k + j] * b[j];
    b[r] = v / A[(size_t)r * k + r];
  }
  return true;
}

// Device gather X[col * ld + idx] of host lists; returns the values on the host.
rbws_status gather_host(rbws_problem p, const double* X, int64_t ld, const std::vector<int>& col,
                        const std::vector<int64_t>& idx, std::vector<double>& out) {
  const int L = (int)idx.size();
  out.assign(L, 0.0);
  if (!L) return RBWS_OK;
  int err = 0;
  int* dc = (int*)p->buf("l1_gcol", sizeof(int) * L, &err);
  int64_t* di = err ? nullptr : (int64_t*)p->buf("l1_gidx", sizeof(int64_t) * L, &err);
  double* dv = err ? nullptr : (double*)p->buf("l1_gval", sizeof(double) * L, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(dc, col.data(), sizeof(int) * L, cudaMemcpyHostToDevice, p->cur));
  CK(cudaMemcpyAsync(di, idx.data(), sizeof(int64_t) * L, cudaMemcpyHostToDevice, p->cur));
  launch_gather(X, ld, dc, di, L, dv, p->cur);
  p->launches += 1;
  CK(cudaMemcpyAsync(out.data(), dv, sizeof(double) * L, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

// One DEIM step on the device vector in slot k of V (ld n): with V's k points,
// c solves V[pts] c = v[pts]; slot k becomes rho = v - V c; returns the point of
// the largest |rho| and rho there (slot k is left unscaled).
rbws_status deim_device(rbws_problem p, double* V, int k, const std::vector<int64_t>& pts, std::vector<double>& c,
                        int64_t* x, double* sval, double* d_sval) {
  const int64_t n = p->n;
  c.assign(k, 0.0);
  if (k > 0) {
    std::vector<int> col;
    std::vector<int64_t> idx;
    for (int i = 0; i < k; i++)  // V_j at point i (j < k), then v at the points
      for (int j = 0; j <= k; j++) col.push_back(j), idx.push_back(pts[i]);
    std::vector<double> g;
    CKI(gather_host(p, V, n, col, idx, g));
    std::vector<double> A((size_t)k * k);
    for (int i = 0; i < k; i++) {
      for (int j = 0; j < k; j++) A[(size_t)i * k + j] = g[(size_t)i * (k + 1) + j];
      c[i] = g[(size_t)i * (k + 1) + k];
    }
    if (!small_solve(k, A, c)) {
      set_error("L1ROC: singular DEIM interpolation matrix");
      return RBWS_ERR_STATE;
    }
    int err = 0;
    double* dc = (double*)p->buf("l1_coef", sizeof(double) * k, &err);
    if (err) return (rbws_status)err;
    CK(cudaMemcpyAsync(dc, c.data(), sizeof(double) * k, cudaMemcpyHostToDevice, p->cur));
    launch_sub_combination(n, k, V, dc, V + (int64_t)k * n, p->cur);
    p->launches += 1;
  }
  int err = 0;
  const int chunks = 256;
  double* sv = (double*)p->buf("l1_amax_v", sizeof(double) * chunks, &err);
  int64_t* si = err ? nullptr : (int64_t*)p->buf("l1_amax_i", sizeof(int64_t) * chunks, &err);
  int64_t* dx = err ? nullptr : (int64_t*)p->buf("l1_amax_x", sizeof(int64_t), &err);
  if (err) return (rbws_status)err;
  launch_argmax_abs(n, V + (int64_t)k * n, sv, si, chunks, dx, d_sval, p->cur);
  p->launches += 4;
  CK(cudaMemcpyAsync(x, dx, sizeof(int64_t), cudaMemcpyDeviceToHost, p->cur));
  CK(cudaMemcpyAsync(sval, d_sval, sizeof(double), cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

// P A_q W (first Nc columns of d_W) and P f at the nodes pts: [Q][M][Nc], [M].
rbws_status colloc_matrices(rbws_problem p, int Nc, const std::vector<int64_t>& pts, const std::vector<double>& rows,
                            std::vector<double>& PAWq, std::vector<double>& Pf) {
  const int M = (int)pts.size(), Q = p->Q;
  const int64_t nx = p->nx, ny = p->ny, nz = p->nz;
  static const int off[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  std::vector<int> col;
  std::vector<int64_t> idx;
  std::vector<int> cls(M);
  for (int i = 0; i < M; i++) {
    const int64_t x = pts[i];
    const int ix = (int)(x % nx), iy = (int)((x / nx) % ny), iz = (int)(x / (nx * ny));
    cls[i] = (p->az.cls[iz] * p->ay.ncls() + p->ay.cls[iy]) * p->ax.ncls() + p->ax.cls[ix];
    for (int j = 0; j < Nc; j++)
      for (int o = 0; o < 7; o++) {
        const int jx = ix + off[o][0], jy = iy + off[o][1], jz = iz + off[o][2];
        const bool in = jx >= 0 && jx < nx && jy >= 0 && jy < ny && jz >= 0 && jz < nz;
        col.push_back(j);
        idx.push_back(in ? ((int64_t)jz * ny + jy) * nx + jx : -1);
      }
  }
  std::vector<double> g;
  CKI(gather_host(p, p->d_W, p->n, col, idx, g));
  const int ncls = p->ax.ncls() * p->ay.ncls() * p->az.ncls();
  PAWq.assign((size_t)Q * M * Nc, 0.0);
  for (int q = 0; q < Q; q++)
    for (int i = 0; i < M; i++) {
      const double* row = &rows[((size_t)q * ncls + cls[i]) * 27];
      for (int j = 0; j < Nc; j++) {
        double v = 0.0;
        for (int o = 0; o < 7; o++) {
          const double a = row[(off[o][2] + 1) * 9 + (off[o][1] + 1) * 3 + off[o][0] + 1];
          v += a * g[((size_t)i * Nc + j) * 7 + o];
        }
        PAWq[((size_t)q * M + i) * Nc + j] = v;
      }
    }
  Pf.assign(M, 1.0);
  if (p->d_f) {
    std::vector<int> c0(M, 0);
    CKI(gather_host(p, p->d_f, 0, c0, pts, Pf));
  }
  return RBWS_OK;
}

// Uploads P A_q W and P f into the problem's L1ROC state (device).
rbws_status colloc_upload(rbws_problem p, int Nc, const std::vector<double>& PAWq, const std::vector<double>& Pf) {
  int err = 0;
  double* a = (double*)p->buf("l1_PAWq", sizeof(double) * PAWq.size(), &err);
  double* f = err ? nullptr : (double*)p->buf("l1_Pf", sizeof(double) * Pf.size(), &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(a, PAWq.data(), sizeof(double) * PAWq.size(), cudaMemcpyHostToDevice, p->cur));
  CK(cudaMemcpyAsync(f, Pf.data(), sizeof(double) * Pf.size(), cudaMemcpyHostToDevice, p->cur));
  (void)Nc;
  return RBWS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* rbws_last_error(void) { return g_last_error.c_str(); }

void rbws_options_default(rbws_options* o) {
  if (!o) return;
  o->max_iters = 20000;
  o->precond = RBWS_PREC_JACOBI;
  o->precision = RBWS_FP64;
  o->max_restarts = 3;
  o->inner_tol = 0.0;
  o->max_outer = 10;
  o->check_every = 0;
  o->stream = nullptr;
  o->profile = nullptr;
  o->relres_hist = nullptr;
  o->hist_len = 0;
  o->wait_cycles = 0;
  o->ru_mode = 0;
  o->persistent = 0;
}

rbws_status rbws_problem_create(const rbws_grid* grid, const rbws_blocks* blocks,
                                const uint8_t* subdomain_map, int32_t Q, const double* f_host,
                                int device, rbws_problem* out) {
  return rbws_problem_create_ex(grid, blocks, subdomain_map, Q, f_host, nullptr, device, out);
}

// Device-side set-up shared by the problem constructors: streams, events, the class maps and
// keys, the Geo view, f and its norm.  p holds the host description (grid, axes, classes);
// on failure p is destroyed.
static rbws_status problem_setup(rbws_problem p, const double* f_host, rbws_problem* out) {
  const int device = p->device;
  auto fail = [&](cudaError_t e, const char* w) {
    cuda_fail(e, w);
    rbws_problem_destroy(p);
    return RBWS_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return fail(e, "cudaSetDevice");
  if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail(e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&p->ev, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e, "cudaEventCreate");
  std::vector<uint8_t> cls;
  cls.insert(cls.end(), p->ax.cls.begin(), p->ax.cls.end());
  cls.insert(cls.end(), p->ay.cls.begin(), p->ay.cls.end());
  cls.insert(cls.end(), p->az.cls.begin(), p->az.cls.end());
  std::vector<int8_t> keys;
  keys.insert(keys.end(), p->ax.key.begin(), p->ax.key.end());
  keys.insert(keys.end(), p->ay.key.begin(), p->ay.key.end());
  keys.insert(keys.end(), p->az.key.begin(), p->az.key.end());
  if ((e = cudaMalloc(&p->d_cls, cls.size())) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->d_keys, keys.size())) != cudaSuccess) return fail(e, "cudaMalloc");
  cudaMemcpy(p->d_cls, cls.data(), cls.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_keys, keys.data(), keys.size(), cudaMemcpyHostToDevice);
  if (!p->h_segq.empty()) {
    if ((e = cudaMalloc(&p->d_segq, p->h_segq.size())) != cudaSuccess) return fail(e, "cudaMalloc");
    cudaMemcpy(p->d_segq, p->h_segq.data(), p->h_segq.size(), cudaMemcpyHostToDevice);
  }
  if (p->field) {
    if ((e = cudaMalloc(&p->d_frows, sizeof(double) * p->h_frows.size())) != cudaSuccess)
      return fail(e, "cudaMalloc");
    cudaMemcpy(p->d_frows, p->h_frows.data(), sizeof(double) * p->h_frows.size(), cudaMemcpyHostToDevice);
  }
  Geo& g = p->geo;
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.ncx = p->ax.ncls();
  g.ncy = p->ay.ncls();
  g.ncz = p->az.ncls();
  g.n = p->n;
  g.cx = p->d_cls;
  g.cy = p->d_cls + p->nx;
  g.cz = p->d_cls + p->nx + p->ny;
  std::vector<double> fw;
  if (!f_host && (p->neumann[0] || p->neumann[1] || p->neumann[2])) {
    // a unit source: the right-hand side is each node's relative control volume
    fw.resize(p->n);
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++)
          fw[((int64_t)k * p->ny + j) * p->nx + i] = (p->neumann[0] && i == p->nx - 1 ? 0.5 : 1.0) *
                                                     (p->neumann[1] && j == p->ny - 1 ? 0.5 : 1.0) *
                                                     (p->neumann[2] && k == p->nz - 1 ? 0.5 : 1.0);
    f_host = fw.data();
    p->default_f = true;
  }
  if (f_host) {
    if ((e = cudaMalloc(&p->d_f, sizeof(double) * p->n)) != cudaSuccess) return fail(e, "cudaMalloc f");
    cudaMemcpy(p->d_f, f_host, sizeof(double) * p->n, cudaMemcpyHostToDevice);
    double s = 0.0;
    for (int64_t i = 0; i < p->n; i++) s += f_host[i] * f_host[i];
    p->fnorm = std::sqrt(s);
  } else {
    p->fnorm = std::sqrt((double)p->n);
  }
  if ((e = cudaMalloc(&p->d_ones, sizeof(double) * p->n)) != cudaSuccess) return fail(e, "cudaMalloc");
  fill(p->d_ones, p->n, 1.0, p->stream);
  if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return fail(e, "set-up");
  for (auto& te : p->tev)
    if ((e = cudaEventCreate(&te)) != cudaSuccess) return fail(e, "cudaEventCreate");
  for (auto& te : p->mgev)
    if ((e = cudaEventCreate(&te)) != cudaSuccess) return fail(e, "cudaEventCreate");
  p->cur = p->stream;
  if (!(p->fnorm > 0.0)) {
    set_error("rbws_problem_create: f must be nonzero");
    rbws_problem_destroy(p);
    return RBWS_ERR_INVALID_ARG;
  }
  *out = p;
  return RBWS_OK;
}

rbws_status rbws_problem_create_ex(const rbws_grid* grid, const rbws_blocks* blocks,
                                   const uint8_t* subdomain_map, int32_t Q, const double* f_host,
                                   const rbws_axes* axes, int device, rbws_problem* out) {
  if (!out || !grid) {
    set_error("rbws_problem_create: null argument");
    return RBWS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  rbws_axes ax_def{{1.0, 1.0, 1.0}, {0, 0, 0}, 0};
  const rbws_axes& axs = axes ? *axes : ax_def;
  for (int a = 0; a < 3; a++)
    if (!(axs.kappa_scale[a] > 0.0) || !std::isfinite(axs.kappa_scale[a]) ||
        (axs.neumann_hi[a] != 0 && axs.neumann_hi[a] != 1)) {
      set_error("rbws_problem_create: kappa_scale must be positive and neumann_hi 0 or 1");
      return RBWS_ERR_INVALID_ARG;
    }
  if ((blocks == nullptr) == (subdomain_map == nullptr)) {
    set_error("rbws_problem_create: give exactly one of blocks / subdomain_map");
    return RBWS_ERR_INVALID_ARG;
  }
  const int dims[3] = {grid->nx, grid->ny, grid->nz};
  for (int d : dims)
    if (d < 2 || d > kMaxAxis) {
      set_error("rbws_problem_create: each axis needs 2..1024 interior nodes");
      return RBWS_ERR_INVALID_ARG;
    }
  std::vector<int> segx, segy, segz;
  std::vector<uint8_t> segq;
  if (subdomain_map) {
    if (Q < 1 || Q > kMaxQ) {
      set_error("rbws_problem_create: need 1 <= Q <= 64");
      return RBWS_ERR_INVALID_ARG;
    }
    const std::string why = map_segments(grid->nx, grid->ny, grid->nz, subdomain_map, Q, segx, segy, segz, segq);
    if (!why.empty()) {
      set_error("rbws_problem_create: " + why);
      return why.compare(0, 9, "map value") == 0 ? RBWS_ERR_INVALID_ARG : RBWS_ERR_UNSUPPORTED;
    }
    const int64_t ncls = (int64_t)make_axis_segments(segx, segx.back() + 1, axs.neumann_hi[0]).ncls() *
                         make_axis_segments(segy, segy.back() + 1, axs.neumann_hi[1]).ncls() *
                         make_axis_segments(segz, segz.back() + 1, axs.neumann_hi[2]).ncls();
    if (ncls > kMaxClasses) {
      set_error("rbws_problem_create: the map has " + std::to_string(ncls) + " coefficient classes (at most " +
                std::to_string(kMaxClasses) + ")");
      return RBWS_ERR_UNSUPPORTED;
    }
  } else {
    if (blocks->bx < 1 || blocks->by < 1 || blocks->bz < 1 || blocks->bx > 16 || blocks->by > 16 ||
        blocks->bz > 16 || Q != blocks->bx * blocks->by * blocks->bz || Q > kMaxQ) {
      set_error("rbws_problem_create: need 1 <= b <= 16 per axis and Q = bx*by*bz <= 64");
      return RBWS_ERR_INVALID_ARG;
    }
    if (blocks->bx > grid->nx || blocks->by > grid->ny || blocks->bz > grid->nz) {
      set_error("rbws_problem_create: more blocks than nodes along an axis");
      return RBWS_ERR_INVALID_ARG;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("rbws_problem_create: CUDA device " + std::to_string(device) + " not available");
    return RBWS_ERR_CUDA;
  }
  rbws_problem p = new rbws_problem_s();
  p->device = device;
  p->nx = grid->nx;
  p->ny = grid->ny;
  p->nz = grid->nz;
  if (subdomain_map) {
    p->bx = segx.back() + 1;
    p->by = segy.back() + 1;
    p->bz = segz.back() + 1;
    p->h_map.assign(subdomain_map, subdomain_map + (int64_t)grid->nx * grid->ny * grid->nz);
  } else {
    p->bx = blocks->bx;
    p->by = blocks->by;
    p->bz = blocks->bz;
  }
  p->Q = Q;
  p->n = (int64_t)p->nx * p->ny * p->nz;
  for (int a = 0; a < 3; a++) {
    p->kscale[a] = axs.kappa_scale[a];
    p->neumann[a] = axs.neumann_hi[a];
  }
  // 1/h^2 per axis (h = 1/(n+1), or 1/n with a Neumann face) times the tensor's entry
  auto inv_h2 = [&](int n, int a) {
    const double cells = p->neumann[a] ? (double)n : (double)(n + 1);
    return p->kscale[a] * (cells * cells);
  };
  p->sx = inv_h2(p->nx, 0);
  p->sy = inv_h2(p->ny, 1);
  p->sz = inv_h2(p->nz, 2);
  if (subdomain_map) {
    p->ax = make_axis_segments(segx, p->bx, p->neumann[0]);
    p->ay = make_axis_segments(segy, p->by, p->neumann[1]);
    p->az = make_axis_segments(segz, p->bz, p->neumann[2]);
  } else {
    p->ax = make_axis(p->nx, p->bx, p->neumann[0]);
    p->ay = make_axis(p->ny, p->by, p->neumann[1]);
    p->az = make_axis(p->nz, p->bz, p->neumann[2]);
  }
  p->h_segq = std::move(segq);
  return problem_setup(p, f_host, out);
}

// One class per node along an axis (a face-field problem): class i for node i.
static AxisClasses identity_axis(int n) {
  AxisClasses a;
  a.n = n;
  a.b = n;
  a.cls.resize(n);
  for (int i = 0; i < n; i++) a.cls[i] = (uint8_t)i;
  a.key.assign((size_t)3 * n, 0);  // unused: the tables come from the face fields
  return a;
}

extern "C" rbws_status rbws_problem_create_field(const rbws_grid* grid, int32_t Q, const double* kfx,
                                                 const double* kfy, const double* kfz, const double* f_host,
                                                 int device, rbws_problem* out) {
  if (!out || !grid || !kfx || !kfy || !kfz) {
    set_error("rbws_problem_create_field: null argument");
    return RBWS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (nx < 2 || ny < 2 || nz < 2 || nx > 256 || ny > 256 || nz > 256 || Q < 1 || Q > kMaxQ) {
    set_error("rbws_problem_create_field: need 2 <= n <= 256 per axis and 1 <= Q <= 64");
    return RBWS_ERR_INVALID_ARG;
  }
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t sfx = (int64_t)nz * ny * (nx + 1), sfy = (int64_t)nz * (ny + 1) * nx, sfz = (int64_t)(nz + 1) * ny * nx;
  for (const auto& arr : {std::make_pair(kfx, sfx), std::make_pair(kfy, sfy), std::make_pair(kfz, sfz)})
    for (int64_t t = 0; t < (int64_t)Q * arr.second; t++)
      if (!(arr.first[t] >= 0.0) || !std::isfinite(arr.first[t])) {
        set_error("rbws_problem_create_field: face coefficients must be finite and >= 0");
        return RBWS_ERR_INVALID_ARG;
      }
  // a node whose six faces are zero in every term has a zero row for every mu
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        bool pos = false;
        for (int q = 0; q < Q && !pos; q++) {
          const double* fx = kfx + q * sfx + ((int64_t)k * ny + j) * (nx + 1) + i;
          const double* fy = kfy + q * sfy + ((int64_t)k * (ny + 1) + j) * nx + i;
          const double* fz = kfz + q * sfz + ((int64_t)k * ny + j) * nx + i;
          pos = fx[0] > 0.0 || fx[1] > 0.0 || fy[0] > 0.0 || fy[nx] > 0.0 || fz[0] > 0.0 || fz[(int64_t)ny * nx] > 0.0;
        }
        if (!pos) {
          set_error("rbws_problem_create_field: node (" + std::to_string(i) + ", " + std::to_string(j) + ", " +
                    std::to_string(k) + ") has no positive face coefficient in any term");
          return RBWS_ERR_INVALID_ARG;
        }
      }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("rbws_problem_create_field: CUDA device " + std::to_string(device) + " not available");
    return RBWS_ERR_CUDA;
  }
  rbws_problem p = new rbws_problem_s();
  p->device = device;
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->Q = Q;
  p->n = n;
  p->field = true;
  const double ihx = (double)(nx + 1) * (nx + 1), ihy = (double)(ny + 1) * (ny + 1), ihz = (double)(nz + 1) * (nz + 1);
  p->sx = ihx;
  p->sy = ihy;
  p->sz = ihz;
  p->ax = identity_axis(nx);
  p->ay = identity_axis(ny);
  p->az = identity_axis(nz);
  p->h_faces.reserve((size_t)Q * (sfx + sfy + sfz));
  p->h_faces.insert(p->h_faces.end(), kfx, kfx + Q * sfx);
  p->h_faces.insert(p->h_faces.end(), kfy, kfy + Q * sfy);
  p->h_faces.insert(p->h_faces.end(), kfz, kfz + Q * sfz);
  // the scaled 7-point rows of each term: -kW -kE -kS -kN -kD -kU D
  p->h_frows.assign((size_t)Q * n * 7, 0.0);
  for (int q = 0; q < Q; q++)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          const double* fx = kfx + q * sfx + ((int64_t)k * ny + j) * (nx + 1);
          const double kW = fx[i] * ihx, kE = fx[i + 1] * ihx;
          const double kS = kfy[q * sfy + ((int64_t)k * (ny + 1) + j) * nx + i] * ihy;
          const double kN = kfy[q * sfy + ((int64_t)k * (ny + 1) + j + 1) * nx + i] * ihy;
          const double kD = kfz[q * sfz + ((int64_t)k * ny + j) * nx + i] * ihz;
          const double kU = kfz[q * sfz + ((int64_t)(k + 1) * ny + j) * nx + i] * ihz;
          double* r = &p->h_frows[((size_t)q * n + ((int64_t)k * ny + j) * nx + i) * 7];
          r[0] = -kW;
          r[1] = -kE;
          r[2] = -kS;
          r[3] = -kN;
          r[4] = -kD;
          r[5] = -kU;
          r[6] = kW + kE + kS + kN + kD + kU;
        }
  return problem_setup(p, f_host, out);
}

extern "C" rbws_status rbws_dirichlet_lift(rbws_problem p, const double* g_host, void* lift_out) {
  if (!p || !g_host || !lift_out) {
    set_error("rbws_dirichlet_lift: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (!p->field) {
    set_error("rbws_dirichlet_lift: the problem was not made by rbws_problem_create_field");
    return RBWS_ERR_UNSUPPORTED;
  }
  cudaSetDevice(p->device);
  const size_t nb = (size_t)2 * ((size_t)p->nz * p->ny + (size_t)p->nz * p->nx + (size_t)p->ny * p->nx);
  int err = 0;
  double* gb = (double*)p->buf("lift_g", sizeof(double) * nb, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(gb, g_host, sizeof(double) * nb, cudaMemcpyHostToDevice, p->stream));
  launch_dirichlet_lift(p->geo, p->Q, p->d_frows, gb, (double*)lift_out, p->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return RBWS_OK;
}

extern "C" rbws_status rbws_affine_sources(rbws_problem p, const void* F, int32_t K, const double* theta,
                                           int32_t B, void* f_out) {
  if (!p || !F || !theta || !f_out || K < 1 || K > 64 || B < 1) {
    set_error("rbws_affine_sources: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  cudaSetDevice(p->device);
  int err = 0;
  double* th = (double*)p->buf("aff_theta", sizeof(double) * (size_t)B * K, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(th, theta, sizeof(double) * (size_t)B * K, cudaMemcpyHostToDevice, p->stream));
  launch_affine_sources(p->n, K, (const double*)F, th, B, (double*)f_out, p->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->stream));
  return RBWS_OK;
}

void rbws_problem_destroy(rbws_problem p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (auto& kv : p->bufs)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  cudaFree(p->d_cls);
  cudaFree(p->d_keys);
  cudaFree(p->d_segq);
  cudaFree(p->d_frows);
  p->mg.reset();
  cudaFree(p->d_f);
  cudaFree(p->d_ones);
  cudaFree(p->d_W);
  cudaFree(p->d_W32);
  cudaFree(p->d_ANq);
  cudaFree(p->d_fN);
  cudaFree(p->l1.d_PAWq);
  cudaFree(p->l1.d_Pf);
  cudaFree(p->d_w32);
  cudaFree(p->d_w16);
  cudaFree(p->d_cscale);
  if (p->h_small) cudaFreeHost(p->h_small);
  if (p->ev) cudaEventDestroy(p->ev);
  for (auto& e : p->tev)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->mgev)
    if (e) cudaEventDestroy(e);
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

rbws_status rbws_problem_info(rbws_problem p, int64_t* n_dof, int32_t* Q, int32_t* N) {
  if (!p) {
    set_error("rbws_problem_info: null problem");
    return RBWS_ERR_INVALID_ARG;
  }
  if (n_dof) *n_dof = p->n;
  if (Q) *Q = p->Q;
  if (N) *N = p->N;
  return RBWS_OK;
}

rbws_status rbws_apply_operator(rbws_problem p, const double* mu, int32_t B, const void* x, void* y,
                                int32_t precision, void* stream) {
  if (!p || !mu || !x || !y || B < 1 || B > 65535 ||
      (precision != RBWS_FP64 && precision != RBWS_FP32_IR)) {
    set_error("rbws_apply_operator: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, stream);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_apply"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, precision == RBWS_FP32_IR ? &c32 : nullptr));
  Tile t = choose_tile(p->nx);
  if (precision == RBWS_FP64)
    launch_apply<double>(p->geo, t, c64, B, (const double*)x, p->n, (double*)y, p->cur);
  else
    launch_apply<float>(p->geo, t, c32, B, (const float*)x, p->n, (float*)y, p->cur);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_update_ff(rbws_problem p, const double* mu, int32_t B, const void* u0, const void* d, void* u_out,
                           void* r_out) {
  if (!p || !mu || !u0 || !d || !u_out || !r_out || B < 1 || B > 65535) {
    set_error("rbws_update_ff: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  const Tile t = choose_tile_v4(p->nx, p->ny);
  if (t.tx == 0) {
    set_error("rbws_update_ff: needs nx % 4 == 0 (the 4-node tiles)");
    return RBWS_ERR_UNSUPPORTED;
  }
  StreamGuard sg(p, nullptr);
  cudaStream_t s = p->cur;
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_ff"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, &c32));
  int err = 0;
  const size_t vb = sizeof(float) * (size_t)B * p->n;
  float* dd = (float*)p->buf("ffu_d", vb, &err);
  int* upd = err ? nullptr : (int*)p->buf("ffu_upd", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  CGArgs<float> a{};
  CKI(make_cg_args<float>(p, B, t, c32, dd, &a, "ffu_", 4));
  a.upd = upd;
  a.u64 = (double*)u0;
  FFState ff{};
  ff.uh = (float*)p->buf("ffu_uh", vb, &err);
  if (!err) ff.ul = (float*)p->buf("ffu_ul", vb, &err);
  if (!err) ff.rh = (float*)p->buf("ffu_rh", vb, &err);
  if (!err) ff.rl = (float*)p->buf("ffu_rl", vb, &err);
  float* cff = err ? nullptr : (float*)p->buf("ffu_coef", sizeof(float) * 2 * kCoefStride * (size_t)B * p->geo.ncls(), &err);
  if (!err) ff.part = (double*)p->buf("ffu_part", sizeof(double) * (size_t)B * a.P, &err);
  int* ones = err ? nullptr : (int*)p->buf("ffu_ones", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  ff.coef = cff;
  ff.f = p->d_f;
  ff.f_stride = 0;
  std::vector<int> one(B, 1);
  CK(cudaMemcpyAsync(upd, one.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ones, one.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  launch_coef_ff(c64, (int64_t)B * p->geo.ncls(), cff, s);
  launch_ru_ff(a, t, ff, true, s);  // u = u0, r = f - A u0
  CK(cudaMemcpyAsync(dd, d, vb, cudaMemcpyDeviceToDevice, s));
  launch_ru_ff(a, t, ff, false, s);  // r -= A d, u += d
  CGArgs<float> out = a;
  out.u64 = (double*)u_out;
  launch_ff_to64(out, ff, ones, s);
  FFState rv = ff;
  rv.uh = ff.rh;
  rv.ul = ff.rl;
  out.u64 = (double*)r_out;
  launch_ff_to64(out, rv, ones, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return RBWS_OK;
}

rbws_status rbws_apply_operator_interleaved(rbws_problem p, const double* mu, int32_t B, const void* x, void* y,
                                            int32_t precision, void* stream) {
  if (!p || !mu || !x || !y || B < 1 || B > 65535 || (precision != RBWS_FP64 && precision != RBWS_FP32_IR)) {
    set_error("rbws_apply_operator_interleaved: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, stream);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_apply"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, precision == RBWS_FP32_IR ? &c32 : nullptr));
  int err = 0;
  const size_t nc = (size_t)p->geo.ncls() * kCoefStride * B;
  void* cI = p->buf("coef_il", (precision == RBWS_FP64 ? sizeof(double) : sizeof(float)) * nc, &err);
  if (err) return (rbws_status)err;
  if (precision == RBWS_FP64)
    launch_apply_interleaved<double>(p->geo, c64, B, (double*)cI, (const double*)x, (double*)y, p->cur);
  else
    launch_apply_interleaved<float>(p->geo, c32, B, (float*)cI, (const float*)x, (float*)y, p->cur);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_autotune_layout(rbws_problem p, int32_t B, int32_t precision, double* planar_ms,
                                 double* interleaved_ms, int32_t* layout_out) {
  if (!p || B < 1 || B > 65535 || (precision != RBWS_FP64 && precision != RBWS_FP32_IR)) {
    set_error("rbws_autotune_layout: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  cudaStream_t s = p->cur;
  std::vector<double> ones((size_t)B * p->Q, 1.0);
  double* d_mu = nullptr;
  CKI(upload_mu(p, ones.data(), B, &d_mu, "mu_tune"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  const bool f32 = precision == RBWS_FP32_IR;
  CKI(coef_tables(p, d_mu, B, &c64, f32 ? &c32 : nullptr));
  const size_t el = f32 ? sizeof(float) : sizeof(double);
  int err = 0;
  void* x = p->buf("lay_x", el * (size_t)B * p->n, &err);
  void* y = err ? nullptr : p->buf("lay_y", el * (size_t)B * p->n, &err);
  void* cI = err ? nullptr : p->buf("coef_il", el * (size_t)p->geo.ncls() * kCoefStride * B, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemsetAsync(x, 0, el * (size_t)B * p->n, s));
  const Tile t = choose_tile(p->nx);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](bool il) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {  // the first call is a warm-up
      cudaEventRecord(e0, s);
      if (il) {
        if (f32) launch_apply_interleaved<float>(p->geo, c32, B, (float*)cI, (const float*)x, (float*)y, s);
        else launch_apply_interleaved<double>(p->geo, c64, B, (double*)cI, (const double*)x, (double*)y, s);
      } else {
        if (f32) launch_apply<float>(p->geo, t, c32, B, (const float*)x, p->n, (float*)y, s);
        else launch_apply<double>(p->geo, t, c64, B, (const double*)x, p->n, (double*)y, s);
      }
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);
    }
    return (double)best;
  };
  const double tp = timed(false), ti = timed(true);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  if (planar_ms) *planar_ms = tp;
  if (interleaved_ms) *interleaved_ms = ti;
  if (layout_out) *layout_out = ti < tp ? 1 : 0;
  return RBWS_OK;
}

rbws_status rbws_apply_preconditioner(rbws_problem p, const double* mu, int32_t B, int32_t precond,
                                      const void* x, void* y, void* stream) {
  if (!p || !mu || !x || !y || x == y || B < 1 || B > 65535) {
    set_error("rbws_apply_preconditioner: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (precond != RBWS_PREC_JACOBI && precond != RBWS_PREC_MG) {
    set_error("rbws_apply_preconditioner: only the Jacobi and multigrid preconditioners act alone");
    return RBWS_ERR_UNSUPPORTED;
  }
  StreamGuard sg(p, stream);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_precond"));
  double* c64 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, nullptr));
  if (precond == RBWS_PREC_JACOBI) {
    MGLevel L{p->nx, p->ny, p->nz, p->n, p->geo.ncx, p->geo.ncy, p->geo.ncz, p->geo.cx, p->geo.cy, p->geo.cz,
              (const void*)c64, kCoefStride};
    launch_diag_inverse(L, B, (const double*)x, (double*)y, p->cur);
    p->launches += 1;
  } else {
    MGBatch m;
    CKI(mg_batch(p, d_mu, B, c64, 0, nullptr, &m));
    p->launches += launch_mg_vcycle(m, (const double*)x, (double*)y, -1, p->cur);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_apply_mg32(rbws_problem p, const double* mu, int32_t B, const void* x, void* y, void* stream) {
  if (!p || !mu || !x || !y || x == y || B < 1 || B > 65535) {
    set_error("rbws_apply_mg32: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, stream);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_mg32"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, &c32));
  Tile t = choose_tile_v4(p->nx, p->ny);
  const bool v4 = t.tx > 0;
  if (!v4) t = choose_tile(p->nx);
  int err = 0;
  float* d = (float*)p->buf("mg32_u", sizeof(float) * (size_t)B * p->n, &err);
  if (err) return (rbws_status)err;
  CGArgs<float> a{};
  CKI(make_cg_args<float>(p, B, t, c32, d, &a, "m32_", v4 ? 4 : 1, 0));
  a.precond = RBWS_PREC_MG;
  std::vector<InstState> h(B);
  for (auto& e : h) e = InstState{ST_ACTIVE, 0, 0, 0, 0.0, 0.0, 0ull};
  CK(cudaMemcpyAsync(a.st, h.data(), sizeof(InstState) * B, cudaMemcpyHostToDevice, p->cur));
  CK(cudaMemsetAsync(a.active, 0, 4 * sizeof(int), p->cur));  // the third counter: the TMA error flag
  MGBatch mgb;
  CKI(mg_fp32_batch(p, d_mu, B, c32, v4, t, &a, &mgb));
  p->launches += launch_mg_vcycle(mgb, x, y, -1, p->cur);
  CK(cudaGetLastError());
  int counts[3];
  CK(cudaMemcpyAsync(counts, a.active, sizeof(counts), cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  if (counts[2]) {
    set_error("rbws_apply_mg32: a TMA stage wait ran out of time");
    return RBWS_ERR_DEVICE_TIMEOUT;
  }
  return RBWS_OK;
}

rbws_status rbws_apply_operator_static(rbws_problem p, const double* mu, int32_t B, const void* x,
                                       void* y, int32_t precision, void* stream) {
  if (!p || !mu || !x || !y || B < 1 || B > 65535 ||
      (precision != RBWS_FP64 && precision != RBWS_FP32_IR)) {
    set_error("rbws_apply_operator_static: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->field) {  // its per-node tables would not fit the static array's layout
    set_error("rbws_apply_operator_static: not available for a face-field problem");
    return RBWS_ERR_UNSUPPORTED;
  }
  StreamGuard sg(p, stream);
  const int8_t* kx = p->d_keys;
  const int8_t* ky = kx + p->ax.key.size();
  const int8_t* kz = ky + p->ay.key.size();
  return (rbws_status)apply_operator_static(p->device, p->geo, kx, ky, kz, p->bx, p->by, p->d_segq, p->sx,
                                            p->sy, p->sz, p->Q, mu, B, x, y, precision, p->cur,
                                            choose_tile(p->nx));
}

rbws_status rbws_set_basis(rbws_problem p, int32_t N, const double* W, const double* ANq,
                           const double* fN) {
  if (!p || N < 1 || N > 160 || !W || !ANq || !fN) {
    set_error("rbws_set_basis: invalid argument (1 <= N <= 160)");
    return RBWS_ERR_INVALID_ARG;
  }
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  cudaFree(p->d_W);
  cudaFree(p->d_W32);
  cudaFree(p->d_ANq);
  cudaFree(p->d_fN);
  p->d_W = p->d_ANq = p->d_fN = nullptr;
  p->d_W32 = nullptr;
  p->l1.N = p->l1.M = 0;  // collocation data belongs to the basis it was built with
  p->N = 0;
  CK(cudaMalloc(&p->d_W, sizeof(double) * (size_t)N * p->n));
  CK(cudaMalloc(&p->d_ANq, sizeof(double) * (size_t)p->Q * N * N));
  CK(cudaMalloc(&p->d_fN, sizeof(double) * (size_t)N));
  CK(cudaMemcpy(p->d_W, W, sizeof(double) * (size_t)N * p->n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_ANq, ANq, sizeof(double) * (size_t)p->Q * N * N, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_fN, fN, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice));
  p->h_ANq.assign(ANq, ANq + (size_t)p->Q * N * N);
  p->h_fN.assign(fN, fN + N);
  p->N = N;
  return RBWS_OK;
}

rbws_status rbws_get_basis(rbws_problem p, double* W, double* ANq, double* fN) {
  if (!p) {
    set_error("rbws_get_basis: null problem");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->N <= 0) {
    set_error("rbws_get_basis: no basis");
    return RBWS_ERR_NO_BASIS;
  }
  cudaSetDevice(p->device);
  CK(cudaStreamSynchronize(p->cur));
  if (W) CK(cudaMemcpy(W, p->d_W, sizeof(double) * (size_t)p->N * p->n, cudaMemcpyDeviceToHost));
  if (ANq) std::memcpy(ANq, p->h_ANq.data(), sizeof(double) * p->h_ANq.size());
  if (fN) std::memcpy(fN, p->h_fN.data(), sizeof(double) * p->h_fN.size());
  return RBWS_OK;
}

rbws_status rbws_reduced_solve(rbws_problem p, const double* mu, int32_t B, double* c_out) {
  if (!p || !mu || !c_out || B < 1) {
    set_error("rbws_reduced_solve: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->N <= 0) {
    set_error("rbws_reduced_solve: no basis");
    return RBWS_ERR_NO_BASIS;
  }
  StreamGuard sg(p, nullptr);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_rs"));
  int err = 0;
  double* C = (double*)p->buf("C", sizeof(double) * (size_t)B * p->N, &err);
  int* info = err ? nullptr : (int*)p->buf("info", sizeof(int) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  launch_reduced_solve(p->N, p->Q, p->d_ANq, p->d_fN, d_mu, B, C, info, nullptr, p->cur);
  CK(cudaGetLastError());
  std::vector<int> h(B);
  CK(cudaMemcpyAsync(c_out, C, sizeof(double) * (size_t)B * p->N, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaMemcpyAsync(h.data(), info, sizeof(int) * B, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  for (int b = 0; b < B; b++)
    if (h[b]) {
      set_error("rbws_reduced_solve: A_N(mu) not positive definite");
      return RBWS_ERR_NOT_SPD;
    }
  return RBWS_OK;
}

namespace {

// Algorithm 5's greedy loop with Galerkin RB (the residual or the L1 indicator).  f_train
// (device [n_train][n], or nullptr for the problem's f): a right-hand side per training
// parameter, with norms f_norms (device [n_train]); snapshots then solve A(mu_t) u = f_t and the
// residual indicator uses f_t and W^T f_t.
rbws_status greedy_impl(rbws_problem p, const double* mu_train, int32_t n_train, int32_t n_max,
                        double greedy_tol, double snapshot_tol, int32_t indicator, const double* f_train,
                        const double* f_norms, int32_t* selected_out, double* eta_hist_out, int32_t* n_out) {
  cudaStream_t s = p->cur;
  const int64_t n = p->n;
  const int Q = p->Q;
  int err = 0;
  // Drop any previous basis; the new one is built in place.
  cudaStreamSynchronize(s);
  cudaFree(p->d_W);
  cudaFree(p->d_W32);
  cudaFree(p->d_ANq);
  cudaFree(p->d_fN);
  p->d_W = p->d_ANq = p->d_fN = nullptr;
  p->d_W32 = nullptr;
  p->l1.N = p->l1.M = 0;  // collocation data belongs to the basis it was built with
  p->N = 0;
  CK(cudaMalloc(&p->d_W, sizeof(double) * (size_t)n_max * n));
  CK(cudaMalloc(&p->d_ANq, sizeof(double) * (size_t)Q * n_max * n_max));
  CK(cudaMalloc(&p->d_fN, sizeof(double) * (size_t)n_max));
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu_train, n_train, &d_mu, "mu_train"));
  double* usnap = (double*)p->buf("g_usnap", sizeof(double) * n, &err);
  double* w = err ? nullptr : (double*)p->buf("g_w", sizeof(double) * n, &err);
  double* V = err ? nullptr : (double*)p->buf("g_V", sizeof(double) * (size_t)Q * n, &err);
  double* dots = err ? nullptr : (double*)p->buf("g_dots", sizeof(double) * (size_t)(Q + 2) * (n_max + 1), &err);
  const int scratch_len = 256 * (n_max + 2);
  double* scratch = err ? nullptr : (double*)p->buf("g_scratch", sizeof(double) * scratch_len, &err);
  double* eye = err ? nullptr : (double*)p->buf("g_eye", sizeof(double) * (size_t)Q * Q, &err);
  double* dR = err ? nullptr : (double*)p->buf("g_R", sizeof(double) * (size_t)n_max * n_max, &err);
  double* FNt = nullptr;  // [n_max][n_train]: W^T f_t of the training right-hand sides
  double* tscratch = nullptr;
  const int tscratch_len = 256 * (n_train + 2);
  if (!err && f_train) {
    FNt = (double*)p->buf("g_FNt", sizeof(double) * (size_t)n_max * n_train, &err);
    if (!err) tscratch = (double*)p->buf("g_tscratch", sizeof(double) * tscratch_len, &err);
  }
  if (err) return (rbws_status)err;
  std::vector<double> Rh((size_t)n_max * n_max, 0.0);  // u_k = sum_j R[j][k] w_j (Gram-Schmidt factor)
  {
    std::vector<double> I((size_t)Q * Q, 0.0);
    for (int q = 0; q < Q; q++) I[(size_t)q * Q + q] = 1.0;
    CK(cudaMemcpyAsync(eye, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  const double* fvec = p->d_f ? p->d_f : p->d_ones;
  std::vector<double> ANq((size_t)Q * n_max * n_max, 0.0), fN(n_max, 0.0);
  std::vector<char> taken(n_train, 0);
  std::vector<double> eta(n_train);
  std::vector<double> hist(n_max, NAN);
  std::vector<int32_t> sel(n_max, -1);
  rbws_options o;
  rbws_options_default(&o);
  o.max_iters = 1000000;
  o.precond = RBWS_PREC_JACOBI;
  int N = 0, next = 0;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_train, ((int64_t)1 << 28) / n));
  while (N < n_max) {
    // snapshot u(mu_next) by Jacobi-PCG from zero (with its own right-hand side if given)
    std::vector<InstState> st;
    CK(cudaMemsetAsync(usnap, 0, sizeof(double) * n, s));
    if (f_train) {
      p->rhs = {};
      p->rhs.f = f_train + (int64_t)next * n;
      p->rhs.norms = f_norms + next;
    }
    const rbws_status rs = solve_fp64(p, d_mu + (int64_t)next * Q, 1, snapshot_tol, o, usnap, st);
    p->rhs = {};
    if (rs != RBWS_OK) return rs;
    // A snapshot whose true residual stalls above snapshot_tol at the rounding
    // floor of the FP64 residual (large, high-contrast grids) is still used if
    // that residual is below 1e-9.
    if (st[0].status != ST_CONVERGED && !(st[0].status == ST_MAX_ITERS && st[0].relres < 1e-9)) {
      set_error("rbws_offline_greedy: snapshot solve did not converge (relative residual " +
                std::to_string(st[0].relres) + ")");
      return RBWS_ERR_STATE;
    }
    // w = (I - W W^T)^2 u; the coefficients of both passes form column N of R
    CK(cudaMemcpyAsync(w, usnap, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    for (int pass = 0; pass < 2 && N > 0; pass++) {
      launch_multi_dot(n, N, p->d_W, n, w, dots, scratch, scratch_len, s);
      launch_sub_combination(n, N, p->d_W, dots, w, s);
      std::vector<double> cf(N);
      CK(cudaMemcpyAsync(cf.data(), dots, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int j = 0; j < N; j++) Rh[(size_t)j * n_max + N] += cf[j];
    }
    launch_multi_dot(n, 1, w, n, w, dots, scratch, scratch_len, s);
    launch_multi_dot(n, 1, usnap, n, usnap, dots + 1, scratch, scratch_len, s);
    double nn[2];
    CK(cudaMemcpyAsync(nn, dots, sizeof(nn), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double wn = std::sqrt(nn[0]), un = std::sqrt(nn[1]);
    if (!(wn >= 1e-10 * un)) break;  // no new direction
    Rh[(size_t)N * n_max + N] = wn;
    double* wN = p->d_W + (int64_t)N * n;
    CK(cudaMemcpyAsync(wN, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(dots, &wn, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale_inv(n, dots, wN, s);
    // V[q] = A_q w_N, then the new row/column of A_N^q and the new entry of f_N
    double* c64 = nullptr;
    CKI(coef_tables(p, eye, Q, &c64, nullptr));
    launch_apply<double>(p->geo, choose_tile(p->nx), c64, Q, wN, 0, V, s);
    for (int q = 0; q < Q; q++)
      launch_multi_dot(n, N + 1, p->d_W, n, V + (int64_t)q * n, dots + (int64_t)q * (N + 1), scratch,
                       scratch_len, s);
    launch_multi_dot(n, 1, wN, n, fvec, dots + (int64_t)Q * (N + 1), scratch, scratch_len, s);
    if (f_train)  // column N of the training set's reduced right-hand sides: FNt[N][t] = w_N . f_t
      launch_multi_dot(n, n_train, f_train, n, wN, FNt + (int64_t)N * n_train, tscratch, tscratch_len, s);
    CK(cudaGetLastError());
    std::vector<double> hd((size_t)Q * (N + 1) + 1);
    CK(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < Q; q++)
      for (int j = 0; j <= N; j++) {
        const double a = hd[(size_t)q * (N + 1) + j];  // w_j^T A_q w_N
        ANq[((size_t)q * n_max + j) * n_max + N] = a;
        ANq[((size_t)q * n_max + N) * n_max + j] = a;
      }
    fN[N] = hd[(size_t)Q * (N + 1)];
    sel[N] = next;
    taken[next] = 1;
    N++;
    // publish the packed reduced operators for the reduced solves
    p->h_ANq.assign((size_t)Q * N * N, 0.0);
    for (int q = 0; q < Q; q++)
      for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
          p->h_ANq[((size_t)q * N + i) * N + j] = ANq[((size_t)q * n_max + i) * n_max + j];
    p->h_fN.assign(fN.begin(), fN.begin() + N);
    CK(cudaMemcpyAsync(p->d_ANq, p->h_ANq.data(), sizeof(double) * p->h_ANq.size(),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_fN, p->h_fN.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    p->N = N;
    // indicator over the training set
    if (indicator == RBWS_INDICATOR_L1) {
      // ||R^{-1} c(mu)||_1: reduced solves only, no full-order work
      CK(cudaMemcpyAsync(dR, Rh.data(), sizeof(double) * Rh.size(), cudaMemcpyHostToDevice, s));
      double* Cd = (double*)p->buf("g_C", sizeof(double) * (size_t)n_train * N, &err);
      int* info = err ? nullptr : (int*)p->buf("g_info", sizeof(int) * (size_t)n_train, &err);
      double* etad = err ? nullptr : (double*)p->buf("g_eta", sizeof(double) * (size_t)n_train, &err);
      if (err) return (rbws_status)err;
      launch_reduced_solve(N, Q, p->d_ANq, p->d_fN, d_mu, n_train, Cd, info, nullptr, s);
      launch_l1_indicator(N, n_max, dR, Cd, info, n_train, etad, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(eta.data(), etad, sizeof(double) * n_train, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    } else {
      for (int64_t b0 = 0; b0 < n_train; b0 += chunk) {
        const int Bc = (int)std::min<int64_t>(chunk, n_train - b0);
        double* U = (double*)p->buf("g_U", sizeof(double) * (size_t)Bc * n, &err);
        double* etad = err ? nullptr : (double*)p->buf("g_eta", sizeof(double) * (size_t)Bc, &err);
        if (err) return (rbws_status)err;
        if (f_train) {  // the chunk's own right-hand sides and their reduced projections
          p->rhs.f = f_train + b0 * n;
          p->rhs.stride = n;
          p->rhs.norms = f_norms + b0;
          p->rhs.fN = FNt + b0;
          p->rhs.fN_sb = 1;
          p->rhs.fN_sj = n_train;
        }
        rbws_status rs = galerkin_start(p, d_mu + b0 * Q, Bc, U);
        double* cc = nullptr;
        if (rs == RBWS_OK) rs = coef_tables(p, d_mu + b0 * Q, Bc, &cc, nullptr);
        if (rs == RBWS_OK) rs = residual_norms(p, cc, Bc, U, nullptr, etad);
        p->rhs = {};
        if (rs != RBWS_OK) return rs;
        CK(cudaMemcpyAsync(eta.data() + b0, etad, sizeof(double) * Bc, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      }
    }
    double best = -1.0;
    next = -1;
    for (int t = 0; t < n_train; t++)
      if (!taken[t] && eta[t] > best) {
        best = eta[t];
        next = t;
      }
    hist[N - 1] = next >= 0 ? best : NAN;
    if (next < 0 || best < greedy_tol) break;
  }
  if (N == 0) {
    set_error("rbws_offline_greedy: no basis vector was added");
    return RBWS_ERR_STATE;
  }
  if (selected_out) std::copy(sel.begin(), sel.begin() + n_max, selected_out);
  if (eta_hist_out) std::copy(hist.begin(), hist.end(), eta_hist_out);
  if (n_out) *n_out = N;
  // compact A_N^q to [Q][N][N] on the device (already done above)
  return RBWS_OK;
}

}  // namespace

rbws_status rbws_offline_greedy(rbws_problem p, const double* mu_train, int32_t n_train,
                                int32_t n_max, double greedy_tol, double snapshot_tol,
                                int32_t indicator, int32_t* selected_out, double* eta_hist_out,
                                int32_t* n_out) {
  if (!p || !mu_train || n_train < 1 || n_max < 1 || n_max > 160 || !(snapshot_tol > 0.0) ||
      (indicator != RBWS_INDICATOR_RESIDUAL && indicator != RBWS_INDICATOR_L1)) {
    set_error("rbws_offline_greedy: invalid argument (1 <= n_max <= 160, snapshot_tol > 0, indicator 0 or 1)");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  return greedy_impl(p, mu_train, n_train, n_max, greedy_tol, snapshot_tol, indicator, nullptr, nullptr,
                     selected_out, eta_hist_out, n_out);
}

namespace {

// Norms ||f_b|| (device [B]) of caller right-hand sides; RBWS_ERR_INVALID_ARG if one is zero.
rbws_status rhs_norms(rbws_problem p, const double* f, int B, const char* tag, double** out) {
  int err = 0;
  double* nrm = (double*)p->buf(tag, sizeof(double) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  launch_row_norms(p->n, B, f, p->n, nrm, p->cur);
  std::vector<double> h(B);
  CK(cudaMemcpyAsync(h.data(), nrm, sizeof(double) * B, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  for (int b = 0; b < B; b++)
    if (!(h[b] > 0.0) || !std::isfinite(h[b])) {
      set_error("right-hand side " + std::to_string(b) + " is zero or not finite");
      return RBWS_ERR_INVALID_ARG;
    }
  *out = nrm;
  return RBWS_OK;
}

}  // namespace

rbws_status rbws_offline_greedy_rhs(rbws_problem p, const double* mu_train, const void* f_train, int32_t n_train,
                                    int32_t n_max, double greedy_tol, double snapshot_tol, int32_t* selected_out,
                                    double* eta_hist_out, int32_t* n_out) {
  if (!p || !mu_train || !f_train || n_train < 1 || n_max < 1 || n_max > 160 || !(snapshot_tol > 0.0)) {
    set_error("rbws_offline_greedy_rhs: invalid argument (1 <= n_max <= 160, snapshot_tol > 0)");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  double* nrm = nullptr;
  CKI(rhs_norms(p, (const double*)f_train, n_train, "g_fnorms", &nrm));
  const rbws_status rc = greedy_impl(p, mu_train, n_train, n_max, greedy_tol, snapshot_tol, RBWS_INDICATOR_RESIDUAL,
                                     (const double*)f_train, nrm, selected_out, eta_hist_out, n_out);
  p->rhs = {};
  return rc;
}

rbws_status rbws_solve_batch_rhs(rbws_problem p, const double* mu, int32_t B, const void* f, double tol,
                                 int32_t warm, const rbws_options* opt, void* u_out, int32_t* iters_out,
                                 double* relres_out, int32_t* status_out) {
  rbws_options o;
  rbws_options_default(&o);
  if (opt) o = *opt;
  if (!p || !mu || !f || !u_out || !iters_out || B < 1 || B > 65535) {
    set_error("rbws_solve_batch_rhs: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  CKI(check_solve_options(o, tol, warm));
  if ((warm != RBWS_WARM_ZERO && warm != RBWS_WARM_GALERKIN) || o.precond == RBWS_PREC_MSRB) {
    set_error("rbws_solve_batch_rhs: per-instance right-hand sides take the zero or Galerkin start and "
              "no MSRB preconditioner");
    return RBWS_ERR_UNSUPPORTED;
  }
  StreamGuard sg(p, o.stream);
  double* nrm = nullptr;
  CKI(rhs_norms(p, (const double*)f, B, "rhs_norms", &nrm));
  p->rhs = {};
  p->rhs.f = (const double*)f;
  p->rhs.stride = p->n;
  p->rhs.norms = nrm;
  std::vector<InstState> st;
  const rbws_status rc = solve_batch_impl(p, mu, B, tol, warm, o, (double*)u_out, st);
  p->rhs = {};
  if (rc != RBWS_OK) return rc;
  int warn = 0;
  for (int b = 0; b < B; b++) {
    iters_out[b] = st[b].iters;
    if (relres_out) relres_out[b] = st[b].relres;
    const int sb = st[b].status == ST_CONVERGED ? 0 : (st[b].status == ST_BREAKDOWN ? 2 : 1);
    if (status_out) status_out[b] = sb;
    warn |= sb != 0;
  }
  return warn ? RBWS_WARN_NOT_CONVERGED : RBWS_OK;
}

rbws_status rbws_gaussian_source_ex(rbws_problem p, const double* params, int32_t B, void* f_out) {
  if (!p || !params || !f_out || B < 1 || B > 65535) {
    set_error("rbws_gaussian_source: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  for (int b = 0; b < B; b++) {
    const double* pr = params + 6 * b;
    if (!(pr[3] > 0.0) || !std::isfinite(pr[3]) || !std::isfinite(pr[0]) || !std::isfinite(pr[1]) ||
        !std::isfinite(pr[2]) || !std::isfinite(pr[4]) || !std::isfinite(pr[5])) {
      set_error("rbws_gaussian_source: the width must be positive and every parameter finite");
      return RBWS_ERR_INVALID_ARG;
    }
  }
  StreamGuard sg(p, nullptr);
  int err = 0;
  double* d_prm = (double*)p->buf("gauss_prm", sizeof(double) * 6 * (size_t)B, &err);
  if (err) return (rbws_status)err;
  CK(cudaMemcpyAsync(d_prm, params, sizeof(double) * 6 * B, cudaMemcpyHostToDevice, p->cur));
  launch_gaussian_source(p->nx, p->ny, p->nz, p->neumann, d_prm, B, (double*)f_out, p->cur);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_gaussian_source(rbws_problem p, const double* params, int32_t B, void* f_out) {
  if (!p || !params || !f_out || B < 1 || B > 65535) {
    set_error("rbws_gaussian_source: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  // exp(-|x - c|^2 / (2 s^2)): width 2 s^2, amplitude 1, offset 0
  std::vector<double> p6((size_t)B * 6);
  for (int b = 0; b < B; b++) {
    const double* pr = params + 4 * b;
    if (!(pr[3] > 0.0)) {
      set_error("rbws_gaussian_source: the width must be positive and the centre finite");
      return RBWS_ERR_INVALID_ARG;
    }
    double* q = &p6[(size_t)6 * b];
    q[0] = pr[0], q[1] = pr[1], q[2] = pr[2], q[3] = 2.0 * pr[3] * pr[3], q[4] = 1.0, q[5] = 0.0;
  }
  return rbws_gaussian_source_ex(p, p6.data(), B, f_out);
}

rbws_status rbws_offline_l1roc(rbws_problem p, const double* mu_train, int32_t n_train, int32_t n_max,
                               double snapshot_tol, int32_t* selected_out, double* eta_hist_out, int32_t* n_out) {
  if (!p || !mu_train || n_train < 1 || n_max < 1 || n_max > kL1RocMaxN || !(snapshot_tol > 0.0)) {
    set_error("rbws_offline_l1roc: invalid argument (1 <= n_max <= 64, snapshot_tol > 0)");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  cudaStream_t s = p->cur;
  const int64_t n = p->n;
  const int Q = p->Q;
  int err = 0;
  cudaStreamSynchronize(s);
  cudaFree(p->d_W);
  cudaFree(p->d_W32);
  cudaFree(p->d_ANq);
  cudaFree(p->d_fN);
  p->d_W = p->d_ANq = p->d_fN = nullptr;
  p->d_W32 = nullptr;
  p->N = 0;
  p->l1.N = p->l1.M = 0;
  CK(cudaMalloc(&p->d_W, sizeof(double) * (size_t)(n_max + 1) * n));  // one spare slot for DEIM
  CK(cudaMalloc(&p->d_ANq, sizeof(double) * (size_t)Q * n_max * n_max));
  CK(cudaMalloc(&p->d_fN, sizeof(double) * (size_t)n_max));
  colloc_ls_prepare();
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu_train, n_train, &d_mu, "mu_train"));
  double* R = (double*)p->buf("l1_R", sizeof(double) * (size_t)(n_max + 1) * n, &err);  // residual DEIM basis
  double* r = err ? nullptr : (double*)p->buf("l1_r", sizeof(double) * n, &err);
  double* d_s = err ? nullptr : (double*)p->buf("l1_s", sizeof(double), &err);
  double* dT = err ? nullptr : (double*)p->buf("l1_T", sizeof(double) * (size_t)n_max * n_max, &err);
  double* Cd = err ? nullptr : (double*)p->buf("l1_C", sizeof(double) * (size_t)n_train * n_max, &err);
  int* info = err ? nullptr : (int*)p->buf("l1_info", sizeof(int) * (size_t)n_train, &err);
  double* etad = err ? nullptr : (double*)p->buf("l1_eta", sizeof(double) * (size_t)n_train, &err);
  double* rel = err ? nullptr : (double*)p->buf("l1_rel", sizeof(double), &err);
  if (err) return (rbws_status)err;
  const std::vector<double> rows = fine_rows(p);
  std::vector<int64_t> pts_s, pts_r, pts;
  std::vector<double> T((size_t)n_max * n_max, 0.0), PAWq, Pf;
  std::vector<int32_t> sel(n_max, -1);
  std::vector<double> hist(n_max, NAN), eta(n_train);
  std::vector<char> taken(n_train, 0);
  rbws_options o;
  rbws_options_default(&o);
  o.max_iters = 1000000;
  o.precond = RBWS_PREC_JACOBI;
  int N = 0, nr = 0, next = 0;
  double fmax = 1.0;
  if (p->d_f) {
    int64_t xi;
    double* scratch = (double*)p->buf("l1_fmax", sizeof(double), &err);
    if (err) return (rbws_status)err;
    CK(cudaMemcpyAsync(R, p->d_f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    std::vector<double> dummy;
    CKI(deim_device(p, R, 0, {}, dummy, &xi, &fmax, scratch));
    fmax = std::fabs(fmax);
  }
  while (N < n_max) {
    // snapshot u(mu_next) by Jacobi-PCG from zero, into slot N of W
    double* wN = p->d_W + (int64_t)N * n;
    std::vector<InstState> st;
    CK(cudaMemsetAsync(wN, 0, sizeof(double) * n, s));
    CKI(solve_fp64(p, d_mu + (int64_t)next * Q, 1, snapshot_tol, o, wN, st));
    if (st[0].status != ST_CONVERGED && !(st[0].status == ST_MAX_ITERS && st[0].relres < 1e-9)) {
      set_error("rbws_offline_l1roc: snapshot solve did not converge (relative residual " +
                std::to_string(st[0].relres) + ")");
      return RBWS_ERR_STATE;
    }
    // the snapshot's largest entry (for the breakdown test), then DEIM against W
    int64_t xu;
    double umax, sN;
    std::vector<double> dummy, c;
    CKI(deim_device(p, wN, 0, {}, dummy, &xu, &umax, d_s));  // slot N seen alone: max |u|
    int64_t x;
    {
      // deim_device with k = N reads slot N as v and leaves rho there
      std::vector<int64_t> ps(pts_s.begin(), pts_s.end());
      CKI(deim_device(p, p->d_W, N, ps, c, &x, &sN, d_s));
    }
    if (!(std::fabs(sN) > 1e-10 * std::fabs(umax))) break;  // the snapshot adds nothing new
    std::vector<int64_t> new_pts{x};
    if (N > 0) {
      // the RB residual of the new parameter with the current space, then its DEIM point
      launch_colloc_ls((int)pts.size(), N, Q, (const double*)p->buf("l1_PAWq", 0, &err),
                       (const double*)p->buf("l1_Pf", 0, &err), d_mu + (int64_t)next * Q, 1, Cd, info, s);
      launch_lift(n, N, p->d_W, Cd, 1, r, s);
      double* cc = nullptr;
      CKI(coef_tables(p, d_mu + (int64_t)next * Q, 1, &cc, nullptr));
      double* rslot = R + (int64_t)nr * n;
      CKI(residual_norms(p, cc, 1, r, rslot, rel));
      p->launches += 2;
      double sr;
      int64_t xr;
      std::vector<double> cr;
      CKI(deim_device(p, R, nr, pts_r, cr, &xr, &sr, d_s));
      if (std::fabs(sr) > 1e-10 * fmax) {
        launch_scale_inv(n, d_s, rslot, s);
        p->launches += 1;
        pts_r.push_back(xr);
        nr++;
        new_pts.push_back(xr);
      }
    }
    // the new basis vector: rho / rho[x] (d_s was overwritten by the residual's DEIM)
    CK(cudaMemcpyAsync(d_s, &sN, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale_inv(n, d_s, wN, s);
    p->launches += 1;
    for (int i = 0; i < N; i++) T[(size_t)i * n_max + N] = c[i];
    T[(size_t)N * n_max + N] = sN;
    pts_s.push_back(x);
    for (int64_t q : new_pts)
      if (std::find(pts.begin(), pts.end(), q) == pts.end()) pts.push_back(q);
    sel[N] = next;
    taken[next] = 1;
    N++;
    CKI(colloc_matrices(p, N, pts, rows, PAWq, Pf));
    CKI(colloc_upload(p, N, PAWq, Pf));
    bool all = true;
    for (int t = 0; t < n_train; t++) all = all && taken[t];
    if (all) break;
    // L1 indicator over the training set: collocation solves, then ||T^-1 c||_1
    CK(cudaMemcpyAsync(dT, T.data(), sizeof(double) * T.size(), cudaMemcpyHostToDevice, s));
    launch_colloc_ls((int)pts.size(), N, Q, (const double*)p->buf("l1_PAWq", 0, &err),
                     (const double*)p->buf("l1_Pf", 0, &err), d_mu, n_train, Cd, info, s);
    launch_l1_indicator(N, n_max, dT, Cd, info, n_train, etad, s);
    p->launches += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(eta.data(), etad, sizeof(double) * n_train, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double best = -1.0;
    next = -1;
    for (int t = 0; t < n_train; t++)
      if (!taken[t] && eta[t] > best) {
        best = eta[t];
        next = t;
      }
    hist[N - 1] = best;
    if (next < 0) break;
  }
  if (N == 0) {
    set_error("rbws_offline_l1roc: no basis vector was added");
    return RBWS_ERR_STATE;
  }
  // Galerkin data of the same basis (W^T A_q W, W^T f), so that every warm mode works with it
  {
    double* V = (double*)p->buf("g_V", sizeof(double) * (size_t)Q * n, &err);
    double* dots = err ? nullptr : (double*)p->buf("g_dots", sizeof(double) * (size_t)(Q + 1) * (n_max + 1), &err);
    const int scratch_len = 256 * (n_max + 2);
    double* scratch = err ? nullptr : (double*)p->buf("g_scratch", sizeof(double) * scratch_len, &err);
    double* eye = err ? nullptr : (double*)p->buf("g_eye", sizeof(double) * (size_t)Q * Q, &err);
    if (err) return (rbws_status)err;
    std::vector<double> I((size_t)Q * Q, 0.0);
    for (int q = 0; q < Q; q++) I[(size_t)q * Q + q] = 1.0;
    CK(cudaMemcpyAsync(eye, I.data(), sizeof(double) * I.size(), cudaMemcpyHostToDevice, s));
    double* c64 = nullptr;
    CKI(coef_tables(p, eye, Q, &c64, nullptr));
    const double* fvec = p->d_f ? p->d_f : p->d_ones;
    std::vector<double> A((size_t)Q * N * N), fN(N), hd((size_t)Q * N);
    for (int j = 0; j < N; j++) {
      launch_apply<double>(p->geo, choose_tile(p->nx), c64, Q, p->d_W + (int64_t)j * n, 0, V, s);
      for (int q = 0; q < Q; q++)
        launch_multi_dot(n, N, p->d_W, n, V + (int64_t)q * n, dots + (int64_t)q * N, scratch, scratch_len, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int q = 0; q < Q; q++)
        for (int i = 0; i < N; i++) A[((size_t)q * N + i) * N + j] = hd[(size_t)q * N + i];
    }
    launch_multi_dot(n, N, p->d_W, n, fvec, dots, scratch, scratch_len, s);
    CK(cudaMemcpyAsync(fN.data(), dots, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // symmetrise the rounding (A_N^q is symmetric)
    for (int q = 0; q < Q; q++)
      for (int i = 0; i < N; i++)
        for (int j = 0; j < i; j++) {
          double& a = A[((size_t)q * N + i) * N + j];
          double& b = A[((size_t)q * N + j) * N + i];
          a = b = 0.5 * (a + b);
        }
    p->h_ANq = A;
    p->h_fN = fN;
    CK(cudaMemcpyAsync(p->d_ANq, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->d_fN, fN.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    p->launches += 2 * N + N * Q + 2;
  }
  p->N = N;
  // the online L1ROC data of the final basis
  p->l1.N = N;
  p->l1.M = (int)pts.size();
  p->l1.pts = pts;
  p->l1.T.assign((size_t)N * N, 0.0);
  for (int i = 0; i < N; i++)
    for (int j = 0; j < N; j++) p->l1.T[(size_t)i * N + j] = T[(size_t)i * n_max + j];
  cudaFree(p->l1.d_PAWq);
  cudaFree(p->l1.d_Pf);
  p->l1.d_PAWq = p->l1.d_Pf = nullptr;
  CK(cudaMalloc(&p->l1.d_PAWq, sizeof(double) * PAWq.size()));
  CK(cudaMalloc(&p->l1.d_Pf, sizeof(double) * Pf.size()));
  CK(cudaMemcpyAsync(p->l1.d_PAWq, PAWq.data(), sizeof(double) * PAWq.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->l1.d_Pf, Pf.data(), sizeof(double) * Pf.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (selected_out) std::copy(sel.begin(), sel.end(), selected_out);
  if (eta_hist_out) std::copy(hist.begin(), hist.end(), eta_hist_out);
  if (n_out) *n_out = N;
  return RBWS_OK;
}

rbws_status rbws_l1roc_info(rbws_problem p, int32_t* M_out, int64_t* points_out, double* T_out) {
  if (!p) {
    set_error("rbws_l1roc_info: null problem");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->l1.N <= 0) {
    set_error("rbws_l1roc_info: no L1ROC basis (run rbws_offline_l1roc)");
    return RBWS_ERR_NO_BASIS;
  }
  if (M_out) *M_out = p->l1.M;
  if (points_out) std::copy(p->l1.pts.begin(), p->l1.pts.end(), points_out);
  if (T_out) std::copy(p->l1.T.begin(), p->l1.T.end(), T_out);
  return RBWS_OK;
}

rbws_status rbws_rb_residuals(rbws_problem p, const double* mu, int32_t B, int32_t n_use, double* relres_out) {
  if (!p || !mu || !relres_out || B < 1 || B > 65535) {
    set_error("rbws_rb_residuals: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->N <= 0 || !p->d_ANq) {
    set_error("rbws_rb_residuals: no reduced basis");
    return RBWS_ERR_NO_BASIS;
  }
  if (n_use < 1 || n_use > p->N) {
    set_error("rbws_rb_residuals: n_use must be in 1..N");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_rbres"));
  const int N = p->N, n = n_use, Q = p->Q;
  int err = 0;
  double* ANn = (double*)p->buf("rbres_ANn", sizeof(double) * (size_t)Q * n * n, &err);
  double* C = err ? nullptr : (double*)p->buf("rbres_C", sizeof(double) * (size_t)B * n, &err);
  int* info = err ? nullptr : (int*)p->buf("rbres_info", sizeof(int) * (size_t)B, &err);
  double* u = err ? nullptr : (double*)p->buf("rbres_u", sizeof(double) * (size_t)B * p->n, &err);
  double* rel = err ? nullptr : (double*)p->buf("rbres_rel", sizeof(double) * (size_t)B, &err);
  if (err) return (rbws_status)err;
  // the leading n x n block of each A_N^q (the reduced matrices of the first n vectors: nested spaces)
  for (int q = 0; q < Q; q++)
    CK(cudaMemcpy2DAsync(ANn + (size_t)q * n * n, sizeof(double) * n, p->d_ANq + (size_t)q * N * N,
                         sizeof(double) * N, sizeof(double) * n, n, cudaMemcpyDeviceToDevice, p->cur));
  launch_reduced_solve(n, Q, ANn, p->d_fN, d_mu, B, C, info, nullptr, p->cur);
  launch_lift(p->n, n, p->d_W, C, B, u, p->cur);
  p->launches += 2;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &coef64, &coef32));
  CKI(residual_norms(p, coef64, B, u, nullptr, rel));
  std::vector<int> h(B);
  CK(cudaMemcpyAsync(relres_out, rel, sizeof(double) * B, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaMemcpyAsync(h.data(), info, sizeof(int) * B, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  for (int b = 0; b < B; b++)
    if (h[b] != 0) {
      set_error("reduced matrix of the first n_use vectors is not positive definite for instance " +
                std::to_string(b));
      return RBWS_ERR_NOT_SPD;
    }
  return RBWS_OK;
}

rbws_status rbws_l1roc_coefficients(rbws_problem p, const double* mu, int32_t B, double* c_out) {
  if (!p || !mu || !c_out || B < 1 || B > 65535) {
    set_error("rbws_l1roc_coefficients: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_l1roc"));
  double* C = nullptr;
  CKI(l1roc_coefficients(p, d_mu, B, &C));
  CK(cudaMemcpyAsync(c_out, C, sizeof(double) * (size_t)B * p->l1.N, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_surrogate_set_params(rbws_problem p, int32_t hidden, const float* params,
                                      const float* coef_scale, double mu_lo, double mu_hi) {
  if (!p || !params || hidden < 1 || hidden > 4096 || !(mu_lo > 0.0) || !(mu_hi > mu_lo)) {
    set_error("rbws_surrogate_set_params: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->N <= 0) {
    set_error("rbws_surrogate_set_params: the network predicts reduced coefficients; set a basis first");
    return RBWS_ERR_NO_BASIS;
  }
  StreamGuard sg(p, nullptr);
  cudaDeviceSynchronize();
  CKI(net_alloc(p, hidden, p->N));
  CK(cudaMemcpy(p->d_w32, params, sizeof(float) * p->net_P, cudaMemcpyHostToDevice));
  std::vector<float> one(p->N, 1.0f);
  CK(cudaMemcpy(p->d_cscale, coef_scale ? coef_scale : one.data(), sizeof(float) * p->N,
                cudaMemcpyHostToDevice));
  launch_to_bf16(p->d_w32, p->d_w16, p->net_P, p->cur);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(p->cur));
  p->net_lo = mu_lo;
  p->net_hi = mu_hi;
  return RBWS_OK;
}

rbws_status rbws_surrogate_get_params(rbws_problem p, int32_t* hidden, float* params, float* coef_scale) {
  if (!p) {
    set_error("rbws_surrogate_get_params: null problem");
    return RBWS_ERR_INVALID_ARG;
  }
  if (!p->d_w32) {
    set_error("rbws_surrogate_get_params: no surrogate");
    return RBWS_ERR_NO_BASIS;
  }
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (hidden) *hidden = p->net_H;
  if (params) CK(cudaMemcpy(params, p->d_w32, sizeof(float) * p->net_P, cudaMemcpyDeviceToHost));
  if (coef_scale) CK(cudaMemcpy(coef_scale, p->d_cscale, sizeof(float) * p->net_N, cudaMemcpyDeviceToHost));
  return RBWS_OK;
}

rbws_status rbws_surrogate_forward(rbws_problem p, const double* mu, int32_t B, int32_t corrected,
                                   double* c_out) {
  if (!p || !mu || !c_out || B < 1) {
    set_error("rbws_surrogate_forward: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  StreamGuard sg(p, nullptr);
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, B, &d_mu, "mu_net"));
  int err = 0;
  double* C = (double*)p->buf("net_C", sizeof(double) * (size_t)B * (p->N > 0 ? p->N : 1), &err);
  if (err) return (rbws_status)err;
  CKI(net_predict(p, d_mu, B, C, corrected != 0));
  CK(cudaMemcpyAsync(c_out, C, sizeof(double) * (size_t)B * p->N, cudaMemcpyDeviceToHost, p->cur));
  CK(cudaStreamSynchronize(p->cur));
  return RBWS_OK;
}

rbws_status rbws_surrogate_loss_grad(rbws_problem p, const float* x, const float* t, int32_t B,
                                     double* loss_out, float* grad_out) {
  if (!p || !x || !t || B < 1) {
    set_error("rbws_surrogate_loss_grad: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (!p->d_w32) {
    set_error("rbws_surrogate_loss_grad: no surrogate");
    return RBWS_ERR_NO_BASIS;
  }
  StreamGuard sg(p, nullptr);
  const NetLayout L = net_layout(p->Q, p->net_H, p->net_N);
  NetBufs nb{};
  CKI(net_bufs(p, L, B, &nb));
  int err = 0;
  float* tt = (float*)p->buf("net_t", sizeof(float) * (size_t)B * L.N, &err);
  float* g = err ? nullptr : (float*)p->buf("net_grad", sizeof(float) * L.P, &err);
  if (err) return (rbws_status)err;
  cudaStream_t s = p->cur;
  CK(cudaMemcpyAsync(nb.x, x, sizeof(float) * (size_t)B * L.p, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(tt, t, sizeof(float) * (size_t)B * L.N, cudaMemcpyHostToDevice, s));
  net_forward(p, L, B, nb.x, nb, s);
  launch_mlp_loss(nb.Y, tt, B * L.N, 1.0f / (float)(B * L.N), nb.dY, nb.loss, s);
  net_backward(p, L, B, nb.x, nb, g, s);
  CK(cudaGetLastError());
  float lh = 0.f;
  CK(cudaMemcpyAsync(&lh, nb.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  if (grad_out) CK(cudaMemcpyAsync(grad_out, g, sizeof(float) * L.P, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (loss_out) *loss_out = lh;
  return RBWS_OK;
}

rbws_status rbws_train_surrogate(rbws_problem p, const double* mu, int32_t n, const double* targets,
                                 int32_t hidden, int32_t epochs, int32_t batch, double lr, double mu_lo,
                                 double mu_hi, uint64_t seed, double* final_loss_out) {
  if (!p || !mu || n < 1 || hidden < 1 || hidden > 4096 || epochs < 0 || batch < 1 || batch > n ||
      !(lr > 0.0) || !(mu_lo > 0.0) || !(mu_hi > mu_lo)) {
    set_error("rbws_train_surrogate: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->N <= 0) {
    set_error("rbws_train_surrogate: the targets are reduced coefficients; build or set a basis first");
    return RBWS_ERR_NO_BASIS;
  }
  StreamGuard sg(p, nullptr);
  cudaStream_t s = p->cur;
  cudaStreamSynchronize(s);
  CKI(net_alloc(p, hidden, p->N));
  p->net_lo = mu_lo;
  p->net_hi = mu_hi;
  const NetLayout L = net_layout(p->Q, hidden, p->N);
  const int N = p->N;
  int err = 0;
  double* d_mu = nullptr;
  CKI(upload_mu(p, mu, n, &d_mu, "mu_train_net"));
  double* C = (double*)p->buf("net_Cdata", sizeof(double) * (size_t)n * N, &err);
  float* X = err ? nullptr : (float*)p->buf("net_Xdata", sizeof(float) * (size_t)n * L.p, &err);
  float* T = err ? nullptr : (float*)p->buf("net_Tdata", sizeof(float) * (size_t)n * N, &err);
  float* g = err ? nullptr : (float*)p->buf("net_grad", sizeof(float) * L.P, &err);
  float* m1 = err ? nullptr : (float*)p->buf("net_m1", sizeof(float) * L.P, &err);
  float* m2 = err ? nullptr : (float*)p->buf("net_m2", sizeof(float) * L.P, &err);
  int* step = err ? nullptr : (int*)p->buf("net_step", sizeof(int), &err);
  int64_t* seg_end = err ? nullptr : (int64_t*)p->buf("net_seg_end", sizeof(int64_t) * 8, &err);
  float* seg_bound = err ? nullptr : (float*)p->buf("net_seg_bound", sizeof(float) * 8, &err);
  int* info = err ? nullptr : (int*)p->buf("info", sizeof(int) * (size_t)n, &err);
  if (err) return (rbws_status)err;
  // targets: reduced Galerkin coefficients of the method itself, or the caller's
  if (targets) {
    CK(cudaMemcpyAsync(C, targets, sizeof(double) * (size_t)n * N, cudaMemcpyHostToDevice, s));
  } else {
    launch_reduced_solve(N, p->Q, p->d_ANq, p->d_fN, d_mu, n, C, info, nullptr, s);
    p->launches += 1;
  }
  launch_rms_scale(C, n, N, p->d_cscale, s);
  launch_scale_targets(C, p->d_cscale, n, N, T, s);
  launch_mlp_inputs(d_mu, n, L.p, mu_lo, mu_hi, X, s);
  // initial parameters: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) per layer (weights and biases)
  {
    int64_t ends[8];
    float bounds[8];
    for (int l = 0; l < 4; l++) {
      ends[2 * l] = L.b[l];
      ends[2 * l + 1] = l < 3 ? L.W[l + 1] : L.P;
      bounds[2 * l] = bounds[2 * l + 1] = (float)(1.0 / std::sqrt((double)L.in[l]));
    }
    CK(cudaMemcpyAsync(seg_end, ends, sizeof(ends), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(seg_bound, bounds, sizeof(bounds), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    launch_init_params(p->d_w32, p->d_w16, L.P, seg_end, seg_bound, 8, seed, s);
  }
  CK(cudaMemsetAsync(m1, 0, sizeof(float) * L.P, s));
  CK(cudaMemsetAsync(m2, 0, sizeof(float) * L.P, s));
  CK(cudaMemsetAsync(step, 0, sizeof(int), s));
  p->launches += 4;
  CK(cudaGetLastError());
  const int steps = n / batch;  // minibatches in a fixed order; the remainder is not used
  NetBufs nb{};
  CKI(net_bufs(p, L, batch, &nb));
  float* losses = (float*)p->buf("net_losses", sizeof(float) * (size_t)steps, &err);
  if (err) return (rbws_status)err;
  double final_loss = NAN;
  if (epochs > 0) {
    // one epoch as a CUDA graph: forward, loss, backward, Adam for each minibatch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t before = p->launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < steps; k++) {
      const float* xb = X + (int64_t)k * batch * L.p;
      const float* tb = T + (int64_t)k * batch * N;
      net_forward(p, L, batch, xb, nb, s);
      launch_mlp_loss(nb.Y, tb, batch * N, 1.0f / (float)(batch * N), nb.dY, losses + k, s);
      net_backward(p, L, batch, xb, nb, g, s);
      launch_adam(p->d_w32, p->d_w16, g, m1, m2, L.P, (float)lr, step, s);
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) return (rbws_status)cuda_fail(ce, "capture of a training epoch");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      return (rbws_status)cuda_fail(ce, "cudaGraphInstantiate");
    }
    const int64_t per_epoch = p->launches - before + 3 * steps;  // + loss, adam (2) per step
    p->launches = before;
    for (int e = 0; e < epochs && ce == cudaSuccess; e++) {
      ce = cudaGraphLaunch(exec, s);
      p->launches += per_epoch;
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return (rbws_status)cuda_fail(ce, "training");
    std::vector<float> hl(steps);
    CK(cudaMemcpy(hl.data(), losses, sizeof(float) * steps, cudaMemcpyDeviceToHost));
    double acc = 0.0;
    for (float v : hl) acc += v;
    final_loss = acc / steps;
  }
  if (final_loss_out) *final_loss_out = final_loss;
  return RBWS_OK;
}

rbws_status rbws_solve_batch(rbws_problem p, const double* mu, int32_t B, double tol, int32_t warm,
                             const rbws_options* opt, void* u_out, int32_t* iters_out,
                             double* relres_out, int32_t* status_out) {
  rbws_options o;
  rbws_options_default(&o);
  if (opt) o = *opt;
  if (!p || !mu || !u_out || !iters_out || B < 1 || B > 65535) {
    set_error("rbws_solve_batch: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  CKI(check_solve_options(o, tol, warm));
  StreamGuard sg(p, o.stream);
  std::vector<InstState> st;
  CKI(solve_batch_impl(p, mu, B, tol, warm, o, (double*)u_out, st));
  if (o.profile) o.profile->launches = p->launches;
  int warn = 0;
  for (int b = 0; b < B; b++) {
    iters_out[b] = st[b].iters;
    if (relres_out) relres_out[b] = st[b].relres;
    const int s = st[b].status == ST_CONVERGED ? 0 : (st[b].status == ST_BREAKDOWN ? 2 : 1);
    if (status_out) status_out[b] = s;
    warn |= s != 0;
  }
  return warn ? RBWS_WARN_NOT_CONVERGED : RBWS_OK;
}

rbws_status rbws_autotune(rbws_problem p, int32_t B, const char* cache_path, int32_t* tx_out,
                          int32_t* ty_out, int32_t* zc_out, int32_t* schedule_out, double* ms_out) {
  if (!p || B < 1 || B > 65535) {
    set_error("rbws_autotune: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  if (p->nx % 4) {
    set_error("rbws_autotune: the tuned FP32 kernels need nx % 4 == 0");
    return RBWS_ERR_UNSUPPORTED;
  }
  char key[128];
  std::snprintf(key, sizeof(key), "%dx%dx%d/B%d/fp32", p->nx, p->ny, p->nz, B);
  // cache: one line per entry, "key tx ty zc ms"
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char k[128];
      int tx, ty, zc, sched;
      double ms;
      while (std::fscanf(f, "%127s %d %d %d %lf %d", k, &tx, &ty, &zc, &ms, &sched) == 6)
        if (!std::strcmp(k, key)) p->tuned32[B] = {tx, ty, zc, ms, sched};
      std::fclose(f);
      auto it = p->tuned32.find(B);
      if (it != p->tuned32.end()) {
        if (tx_out) *tx_out = it->second.tx;
        if (ty_out) *ty_out = it->second.ty;
        if (zc_out) *zc_out = it->second.zc;
        if (schedule_out) *schedule_out = it->second.sched;
        if (ms_out) *ms_out = it->second.ms;
        return RBWS_OK;
      }
    }
  }
  StreamGuard sg(p, nullptr);
  cudaStream_t s = p->cur;
  // synthetic instances: mu = 1 (coefficients do not change the timing)
  std::vector<double> ones((size_t)B * p->Q, 1.0);
  double* d_mu = nullptr;
  CKI(upload_mu(p, ones.data(), B, &d_mu, "mu_tune"));
  double* c64 = nullptr;
  float* c32 = nullptr;
  CKI(coef_tables(p, d_mu, B, &c64, &c32));
  int err = 0;
  float* d = (float*)p->buf("ir_d", sizeof(float) * (size_t)B * p->n, &err);
  if (err) return (rbws_status)err;
  rbws_problem_s::Tuned best{0, 0, 0, 1e30, 0};
  (void)0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tx : {32, 16, 8, 4}) {
    if (4 * tx > p->nx) continue;
    for (int ty : {4, 8, 16, 32, 64}) {
      if (tx * ty < 64 || tx * ty > 256 || ty > std::max(4, p->ny)) continue;
      for (int zc : {8, 16, 32, 64}) {
        if (zc > p->nz && zc != 8) continue;
        CGArgs<float> a{};
        int rc = make_cg_args<float>(p, B, Tile{tx, ty}, c32, d, &a, "f_", 4, zc);
        if (rc) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return (rbws_status)rc;
        }
        a.tol = 1e-300;
        a.max_iters = 1 << 30;
        a.precond = RBWS_PREC_JACOBI;
        a.ru = 1;
        fill((double*)a.fnorm, B, 1.0, s);
        const size_t vb = sizeof(float) * (size_t)B * p->n;
        cudaMemsetAsync(a.u, 0, vb, s);
        fill_f(a.r, (int64_t)B * p->n, 1.f, s);
        fill_f(a.s, (int64_t)B * p->n, 1.f, s);
        fill_f(a.p0, (int64_t)B * p->n, 1.f, s);
        double* alpha = (double*)p->buf("ir_alpha", sizeof(double) * 2 * (size_t)B, &err);
        if (err) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return (rbws_status)err;
        }
        a.alpha = alpha;
        int* terr = a.active + 2;
        cudaMemsetAsync(terr, 0, sizeof(int), s);
        tma_prepare();
        for (int sched = 0; sched < 4; sched++) {
          if (sched >= 2 && !tma_supported(p->geo, Tile{tx, ty})) continue;
          float ta = 0.f, tb = 0.f;
          for (int rep = 0; rep < 3; rep++) {
            launch_tune_prep(a, s);
            cudaEventRecord(e0, s);
            if (sched == 1) launch_cg_a32_v4(a, Tile{tx, ty}, 0, s);
            else if (sched == 2) launch_cg_a_tma(a, Tile{tx, ty}, 0, terr, s);
            else if (sched == 3) launch_cg_a_s_tma(a, Tile{tx, ty}, 0, terr, s);
            else launch_cg_a_v4(a, Tile{tx, ty}, 0, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t1 = 0.f;
            cudaEventElapsedTime(&t1, e0, e1);
            launch_tune_prep(a, s);
            cudaEventRecord(e0, s);
            if (sched == 1) launch_cg_b32_v4(a, Tile{tx, ty}, 0, s);
            else if (sched == 3) launch_cg_b_s_tma(a, Tile{tx, ty}, 0, terr, s);
            else launch_cg_b_v4(a, Tile{tx, ty}, 0, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float t2 = 0.f;
            cudaEventElapsedTime(&t2, e0, e1);
            if (rep > 0) {  // the first repetition warms caches and code
              ta += t1;
              tb += t2;
            }
          }
          cudaError_t ce = cudaGetLastError();
          if (ce != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return (rbws_status)cuda_fail(ce, "rbws_autotune");
          }
          const double ms = 0.5 * (ta + tb);
          if (ms < best.ms) best = {tx, ty, std::min(zc, p->nz), ms, sched};
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!best.tx) {
    set_error("rbws_autotune: no candidate tile fits this grid");
    return RBWS_ERR_UNSUPPORTED;
  }
  p->tuned32[B] = best;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s %d %d %d %.6f %d\n", key, best.tx, best.ty, best.zc, best.ms, best.sched);
      std::fclose(f);
    }
  }
  if (tx_out) *tx_out = best.tx;
  if (ty_out) *ty_out = best.ty;
  if (zc_out) *zc_out = best.zc;
  if (schedule_out) *schedule_out = best.sched;
  if (ms_out) *ms_out = best.ms;
  return RBWS_OK;
}

rbws_status rbws_solve_requests(int32_t n_req, const rbws_problem* probs, const double* const* mu,
                                void* const* u_out, double tol, int32_t warm, const rbws_options* opt,
                                int32_t* iters_out, double* relres_out, int32_t* status_out,
                                double* latency_ms_out) {
  rbws_options o;
  rbws_options_default(&o);
  if (opt) o = *opt;
  if (n_req < 1 || !probs || !mu || !u_out || !iters_out) {
    set_error("rbws_solve_requests: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  for (int r = 0; r < n_req; r++)
    if (!probs[r] || !mu[r] || !u_out[r]) {
      set_error("rbws_solve_requests: null problem, parameter or output for request " + std::to_string(r));
      return RBWS_ERR_INVALID_ARG;
    }
  CKI(check_solve_options(o, tol, warm));
  if (o.stream || o.profile || o.relres_hist) {
    set_error("rbws_solve_requests: runs each grid on its problem's own stream; stream, profile and "
              "relres_hist must be NULL");
    return RBWS_ERR_INVALID_ARG;
  }
  // group the requests by problem (one batched solve per grid)
  std::vector<rbws_problem> groups;
  std::vector<std::vector<int>> members;
  for (int r = 0; r < n_req; r++) {
    size_t g = 0;
    while (g < groups.size() && groups[g] != probs[r]) g++;
    if (g == groups.size()) {
      groups.push_back(probs[r]);
      members.emplace_back();
    }
    members[g].push_back(r);
  }
  const size_t G = groups.size();
  std::vector<int> rc(G, RBWS_OK);
  std::vector<std::string> msg(G);
  std::vector<std::vector<InstState>> st(G);
  std::vector<unsigned long long> t0(G, 0);
  if (persistent_ok(o)) {
    // one persistent cooperative launch for the batches of every grid: each problem's
    // start on its own stream, then the launch on the first problem's stream after them
    int nxmin = groups[0]->nx;
    for (size_t g = 1; g < G; g++) nxmin = std::min(nxmin, groups[g]->nx);
    const Tile t = choose_tile(nxmin);  // one CTA shape for every grid
    std::vector<Fp64Batch> fbs(G);
    std::vector<CGArgs<double>> args;
    std::vector<double*> ubuf(G, nullptr);
    std::vector<unsigned long long*> stamps(G, nullptr);
    cudaStream_t s0 = groups[0]->stream;
    for (size_t g = 0; g < G; g++) {
      rbws_problem p = groups[g];
      const std::vector<int>& mem = members[g];
      const int B = (int)mem.size();
      StreamGuard sg(p, nullptr);
      int err = 0;
      ubuf[g] = (double*)p->buf("req_u", sizeof(double) * (size_t)B * p->n, &err);
      stamps[g] = err ? nullptr : (unsigned long long*)p->buf("req_t0", 8, &err);
      if (err) return (rbws_status)err;
      launch_stamp(stamps[g], p->cur);
      std::vector<double> hmu((size_t)B * p->Q);
      for (int k = 0; k < B; k++) std::memcpy(&hmu[(size_t)k * p->Q], mu[mem[k]], sizeof(double) * p->Q);
      double* d_mu = nullptr;
      CKI(warm_start(p, hmu.data(), B, warm, o, ubuf[g], &d_mu));
      CKI(prepare_fp64(p, d_mu, B, tol, o, ubuf[g], &fbs[g], t));
      args.push_back(fbs[g].a);
      if (g > 0) {
        CK(cudaEventRecord(p->ev, p->cur));
        CK(cudaStreamWaitEvent(s0, p->ev, 0));
      }
    }
    cudaSetDevice(groups[0]->device);
    CKI(run_persistent(groups[0], args, t, o, s0));
    for (size_t g = 0; g < G; g++) {
      rbws_problem p = groups[g];
      const std::vector<int>& mem = members[g];
      st[g].resize(mem.size());
      for (size_t k = 0; k < mem.size(); k++)
        CK(cudaMemcpyAsync(u_out[mem[k]], ubuf[g] + k * p->n, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, s0));
      CK(cudaMemcpyAsync(st[g].data(), fbs[g].a.st, sizeof(InstState) * mem.size(), cudaMemcpyDeviceToHost, s0));
      CK(cudaMemcpyAsync(&t0[g], stamps[g], 8, cudaMemcpyDeviceToHost, s0));
    }
    CK(cudaStreamSynchronize(s0));
  } else {
  auto run_group = [&](size_t g) {
    rbws_problem p = groups[g];
    const std::vector<int>& mem = members[g];
    const int B = (int)mem.size();
    StreamGuard sg(p, nullptr);
    int err = 0;
    double* u = (double*)p->buf("req_u", sizeof(double) * (size_t)B * p->n, &err);
    unsigned long long* d_t0 = err ? nullptr : (unsigned long long*)p->buf("req_t0", 8, &err);
    if (err) {
      rc[g] = err;
      msg[g] = rbws_last_error();
      return;
    }
    std::vector<double> hmu((size_t)B * p->Q);
    for (int k = 0; k < B; k++) std::memcpy(&hmu[(size_t)k * p->Q], mu[mem[k]], sizeof(double) * p->Q);
    launch_stamp(d_t0, p->cur);
    rbws_options og = o;
    int r = solve_batch_impl(p, hmu.data(), B, tol, warm, og, u, st[g]);
    if (r == RBWS_OK) {
      for (int k = 0; k < B && r == RBWS_OK; k++) {
        cudaError_t e = cudaMemcpyAsync(u_out[mem[k]], u + (size_t)k * p->n, sizeof(double) * p->n,
                                        cudaMemcpyDeviceToDevice, p->cur);
        if (e != cudaSuccess) r = cuda_fail(e, "rbws_solve_requests: copy out");
      }
      cudaError_t e = cudaMemcpyAsync(&t0[g], d_t0, 8, cudaMemcpyDeviceToHost, p->cur);
      if (r == RBWS_OK && e != cudaSuccess) r = cuda_fail(e, "rbws_solve_requests: stamp");
      e = cudaStreamSynchronize(p->cur);
      if (r == RBWS_OK && e != cudaSuccess) r = cuda_fail(e, "rbws_solve_requests");
    }
    rc[g] = r;
    if (r != RBWS_OK) msg[g] = rbws_last_error();
  };
  // every grid's batch runs on its own stream, driven by its own host thread
  std::vector<std::thread> th;
  for (size_t g = 1; g < G; g++) th.emplace_back(run_group, g);
  run_group(0);
  for (auto& t : th) t.join();
  for (size_t g = 0; g < G; g++)
    if (rc[g] != RBWS_OK) {
      set_error(msg[g]);
      return (rbws_status)rc[g];
    }
  }
  unsigned long long start = t0[0];
  for (size_t g = 1; g < G; g++) start = std::min(start, t0[g]);
  int warn = 0;
  for (size_t g = 0; g < G; g++)
    for (size_t k = 0; k < members[g].size(); k++) {
      const int r = members[g][k];
      const InstState& s = st[g][k];
      iters_out[r] = s.iters;
      if (relres_out) relres_out[r] = s.relres;
      const int code = s.status == ST_CONVERGED ? 0 : (s.status == ST_BREAKDOWN ? 2 : 1);
      if (status_out) status_out[r] = code;
      if (latency_ms_out) latency_ms_out[r] = s.t_done > start ? (double)(s.t_done - start) * 1e-6 : 0.0;
      warn |= code != 0;
    }
  return warn ? RBWS_WARN_NOT_CONVERGED : RBWS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint: the offline products (reduced basis, reduced operators, the
// surrogate network) and the problem description, so a later process can
// solve online without repeating the offline stage.
//
// File layout (little endian): "RBWSPRB1", u32 version (2, 3 or 4), i32 nx ny
// nz bx by bz Q has_f N net_H net_N has_map, f64 mu_lo mu_hi, u64 payload
// bytes, then the payload: the axes (rbws_axes, version >= 3), the face arrays
// kfx | kfy | kfz (f64, if has_map = 2: a face-field problem, version 4), the
// subdomain map [n] (u8, if has_map = 1; bx by bz are then ignored), f [n] (if
// has_f), W [N][n], ANq [Q][N][N], fN [N] (f64), network parameters [P] and
// coefficient scales [net_N] (f32), then u64 FNV-1a of the payload.
// ---------------------------------------------------------------------------
namespace {

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
};

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t nx, ny, nz, bx, by, bz, Q, has_f, N, net_H, net_N, has_map;
  double mu_lo, mu_hi;
  uint64_t payload;
};

}  // namespace

extern "C" rbws_status rbws_save(rbws_problem p, const char* path) {
  if (!p || !path) {
    set_error("rbws_save: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  cudaSetDevice(p->device);
  CK(cudaDeviceSynchronize());
  const int64_t n = p->n;
  const int N = p->N;
  CkptHeader h{};
  std::memcpy(h.magic, "RBWSPRB1", 8);
  // 3: the payload starts with the axes (kappa_scale[3], neumann_hi[3], a zero int32);
  // 4: a face-field problem (has_map = 2), its face arrays following the axes
  h.version = p->field ? 4 : 3;
  h.nx = p->nx;
  h.ny = p->ny;
  h.nz = p->nz;
  h.bx = p->bx;
  h.by = p->by;
  h.bz = p->bz;
  h.Q = p->Q;
  h.has_f = p->d_f != nullptr && !p->default_f;
  h.has_map = p->field ? 2 : !p->h_map.empty();
  h.N = N;
  h.net_H = p->d_w32 ? p->net_H : 0;
  h.net_N = p->d_w32 ? p->net_N : 0;
  h.mu_lo = p->net_lo;
  h.mu_hi = p->net_hi;
  std::vector<double> f(h.has_f ? n : 0), W((size_t)N * n);
  if (h.has_f) CK(cudaMemcpy(f.data(), p->d_f, sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (N > 0) CK(cudaMemcpy(W.data(), p->d_W, sizeof(double) * W.size(), cudaMemcpyDeviceToHost));
  std::vector<float> params(h.net_H ? p->net_P : 0), scale(h.net_N);
  if (h.net_H) {
    CK(cudaMemcpy(params.data(), p->d_w32, sizeof(float) * params.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(scale.data(), p->d_cscale, sizeof(float) * scale.size(), cudaMemcpyDeviceToHost));
  }
  const size_t szA = sizeof(double) * (N > 0 ? p->h_ANq.size() : 0), szF = sizeof(double) * (N > 0 ? N : 0);
  rbws_axes axes{{p->kscale[0], p->kscale[1], p->kscale[2]}, {p->neumann[0], p->neumann[1], p->neumann[2]}, 0};
  h.payload = sizeof(axes) + sizeof(double) * p->h_faces.size() + p->h_map.size() +
              sizeof(double) * (f.size() + W.size()) + szA + szF + sizeof(float) * (params.size() + scale.size());
  FILE* fp = std::fopen(path, "wb");
  if (!fp) {
    set_error(std::string("rbws_save: cannot open ") + path);
    return RBWS_ERR_INVALID_ARG;
  }
  Fnv fnv;
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
  auto put = [&](const void* d, size_t bytes) {
    if (!bytes || !ok) return;
    ok = std::fwrite(d, 1, bytes, fp) == bytes;
    fnv.add(d, bytes);
  };
  put(&axes, sizeof(axes));
  put(p->h_faces.data(), sizeof(double) * p->h_faces.size());
  put(p->h_map.data(), p->h_map.size());
  put(f.data(), sizeof(double) * f.size());
  put(W.data(), sizeof(double) * W.size());
  if (N > 0) {
    put(p->h_ANq.data(), szA);
    put(p->h_fN.data(), szF);
  }
  put(params.data(), sizeof(float) * params.size());
  put(scale.data(), sizeof(float) * scale.size());
  if (ok) ok = std::fwrite(&fnv.h, sizeof(fnv.h), 1, fp) == 1;
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) {
    set_error(std::string("rbws_save: write failed for ") + path);
    return RBWS_ERR_STATE;
  }
  return RBWS_OK;
}

extern "C" rbws_status rbws_load(const char* path, int device, rbws_problem* out) {
  if (!path || !out) {
    set_error("rbws_load: invalid argument");
    return RBWS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) {
    set_error(std::string("rbws_load: cannot open ") + path);
    return RBWS_ERR_INVALID_ARG;
  }
  CkptHeader h{};
  auto fail = [&](const char* why) {
    std::fclose(fp);
    set_error(std::string("rbws_load: ") + why + " (" + path + ")");
    return RBWS_ERR_STATE;
  };
  if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, "RBWSPRB1", 8) != 0) return fail("not a checkpoint");
  if (h.version < 2 || h.version > 4) return fail("unsupported version");
  const bool field = h.has_map == 2;
  if (h.nx < 2 || h.ny < 2 || h.nz < 2 || h.nx > kMaxAxis || h.ny > kMaxAxis || h.nz > kMaxAxis ||
      h.N < 0 || h.N > 160 || h.Q < 1 || h.Q > kMaxQ || (h.has_map != 0 && h.has_map != 1 && !field) ||
      (field && (h.version < 4 || h.nx > 256 || h.ny > 256 || h.nz > 256)) ||
      (!h.has_map && h.Q != h.bx * h.by * h.bz) || h.net_H < 0 || h.net_H > 4096 ||
      (h.net_H > 0 && h.net_N != h.N))
    return fail("corrupt header");
  const int64_t n = (int64_t)h.nx * h.ny * h.nz;
  const int64_t P = h.net_H ? (int64_t)h.net_H * h.Q + h.net_H + 2 * ((int64_t)h.net_H * h.net_H + h.net_H) +
                                  (int64_t)h.N * h.net_H + h.N
                            : 0;
  const uint64_t nfaces = field ? (uint64_t)h.Q * ((uint64_t)h.nz * h.ny * (h.nx + 1) +
                                                   (uint64_t)h.nz * (h.ny + 1) * h.nx +
                                                   (uint64_t)(h.nz + 1) * h.ny * h.nx)
                                 : 0;
  const uint64_t expect = (h.version >= 3 ? sizeof(rbws_axes) : 0) + sizeof(double) * nfaces +
                          (h.has_map == 1 ? (uint64_t)n : 0) +
                          sizeof(double) * ((h.has_f ? n : 0) + (uint64_t)h.N * n + (uint64_t)h.Q * h.N * h.N + h.N) +
                          sizeof(float) * (P + h.net_N);
  if (h.payload != expect) return fail("payload size does not match the header");
  std::vector<uint8_t> map(h.has_map == 1 ? n : 0);
  std::vector<double> faces(nfaces);
  std::vector<double> f(h.has_f ? n : 0), W((size_t)h.N * n), ANq((size_t)h.Q * h.N * h.N), fN(h.N);
  std::vector<float> params(P), scale(h.net_N);
  Fnv fnv;
  bool ok = true;
  auto get = [&](void* d, size_t bytes) {
    if (!bytes || !ok) return;
    ok = std::fread(d, 1, bytes, fp) == bytes;
    if (ok) fnv.add(d, bytes);
  };
  rbws_axes axes{{1.0, 1.0, 1.0}, {0, 0, 0}, 0};
  if (h.version >= 3) get(&axes, sizeof(axes));
  get(faces.data(), sizeof(double) * faces.size());
  get(map.data(), map.size());
  get(f.data(), sizeof(double) * f.size());
  get(W.data(), sizeof(double) * W.size());
  get(ANq.data(), sizeof(double) * ANq.size());
  get(fN.data(), sizeof(double) * fN.size());
  get(params.data(), sizeof(float) * params.size());
  get(scale.data(), sizeof(float) * scale.size());
  uint64_t sum = 0;
  if (!ok || std::fread(&sum, sizeof(sum), 1, fp) != 1) return fail("truncated file");
  std::fclose(fp);
  if (sum != fnv.h) {
    set_error(std::string("rbws_load: checksum mismatch (") + path + ")");
    return RBWS_ERR_STATE;
  }
  rbws_grid g{h.nx, h.ny, h.nz};
  rbws_blocks bl{h.bx, h.by, h.bz};
  rbws_problem p = nullptr;
  rbws_status rc;
  if (field) {
    const double* kfx = faces.data();
    const double* kfy = kfx + (size_t)h.Q * h.nz * h.ny * (h.nx + 1);
    const double* kfz = kfy + (size_t)h.Q * h.nz * (h.ny + 1) * h.nx;
    rc = rbws_problem_create_field(&g, h.Q, kfx, kfy, kfz, h.has_f ? f.data() : nullptr, device, &p);
  } else {
    rc = rbws_problem_create_ex(&g, h.has_map ? nullptr : &bl, h.has_map ? map.data() : nullptr, h.Q,
                                h.has_f ? f.data() : nullptr, &axes, device, &p);
  }
  if (rc != RBWS_OK) return rc;
  if (h.N > 0 && (rc = rbws_set_basis(p, h.N, W.data(), ANq.data(), fN.data())) != RBWS_OK) {
    rbws_problem_destroy(p);
    return rc;
  }
  if (h.net_H > 0 &&
      (rc = rbws_surrogate_set_params(p, h.net_H, params.data(), scale.data(), h.mu_lo, h.mu_hi)) != RBWS_OK) {
    rbws_problem_destroy(p);
    return rc;
  }
  *out = p;
  return RBWS_OK;
}
