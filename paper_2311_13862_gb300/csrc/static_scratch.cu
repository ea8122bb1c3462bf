// static_scratch.cu -- rbws_apply_operator_static: the operator apply for
// callers that cannot allocate device memory after start-up.
//
// Such callers include services that run inside a fixed device-memory budget
// shared with another framework's caching allocator, and latency-sensitive
// code that cannot accept the implicit device synchronisation that
// cudaMalloc / cudaFree may perform.  rbws_apply_operator allocates its
// scratch (the device copy of mu and the per-instance coefficient tables) on
// first use; this variant keeps that scratch in one file-scope device array
// instead, so a call allocates nothing.
//
// The array is kStaticScratchBytes (4 MiB) and exists on every GPU that loads
// the library until the process exits.  Every call shares it and it keeps the
// last call's contents; a call overwrites everything it reads, so nothing has
// to start at zero.  Two calls whose GPU work overlaps (two threads, two
// problems on one device, or two streams) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace rbws {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)4 << 20;
constexpr int kMaxDevices = 64;

// Device-side scratch.  In host code this name is only a stand-in for the
// symbol; kernels must be given the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// cuCtxGetCurrent through the runtime's driver entry-point query (the library links
// only the CUDA runtime).
typedef int (*CtxGetCurrentFn)(void**);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};
void* g_scratch_ctx[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
// Set up once per device: the address is looked up with cudaGetSymbolAddress
// the first time and kept together with the context it belongs to.  If the
// caller has torn that context down since (cudaDeviceReset), the module is
// loaded again in the new context and the address is looked up again.
// Returns nullptr and sets the error on failure.
void* scratch_address(int device) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("rbws_apply_operator_static: device index out of range");
    return nullptr;
  }
  void* ctx = nullptr;
  CtxGetCurrentFn cur = ctx_get_current();
  if (cur && cur(&ctx) != 0) ctx = nullptr;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device] || !cur || ctx != g_scratch_ctx[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) {
      cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      return nullptr;
    }
    g_scratch_addr[device] = ptr;
    g_scratch_ctx[device] = ctx;
  }
  return g_scratch_addr[device];
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Needed scratch bytes for B instances: mu [B][Q] FP64, FP64 tables, and
// FP32 tables when the FP32 kernel is requested.
size_t static_scratch_need(int Q, int ncls, int B, bool fp32) {
  size_t need = align256(sizeof(double) * (size_t)B * Q);
  need += align256(sizeof(double) * (size_t)B * ncls * kCoefStride);
  if (fp32) need += align256(sizeof(float) * (size_t)B * ncls * kCoefStride);
  return need;
}

size_t static_scratch_capacity() { return kStaticScratchBytes; }

// The body of rbws_apply_operator_static (api.cu holds the C entry point and
// the problem struct).  g: the problem's geometry; keys: per-axis class keys
// on the device; d_first_*: sizes of the key arrays.
int apply_operator_static(int device, const Geo& g, const int8_t* kx, const int8_t* ky, const int8_t* kz,
                          int bx, int by, const uint8_t* segq, double sx, double sy, double sz, int Q,
                          const double* mu_host,
                          int B, const void* x, void* y, int precision, cudaStream_t s, Tile t) {
  const int ncls = g.ncls();
  const bool fp32 = precision == RBWS_FP32_IR;
  const size_t need = static_scratch_need(Q, ncls, B, fp32);
  if (need > kStaticScratchBytes) {
    set_error("rbws_apply_operator_static: " + std::to_string(B) + " instances need " + std::to_string(need) +
              " bytes of scratch, more than the static maximum of " + std::to_string(kStaticScratchBytes) +
              " (use fewer instances per call, or rbws_apply_operator)");
    return RBWS_ERR_INVALID_ARG;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch_address(device));
  if (!base) return RBWS_ERR_CUDA;
  double* d_mu = reinterpret_cast<double*>(base);
  double* c64 = reinterpret_cast<double*>(base + align256(sizeof(double) * (size_t)B * Q));
  float* c32 = fp32 ? reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(c64) +
                                               align256(sizeof(double) * (size_t)B * ncls * kCoefStride))
                    : nullptr;
  cudaError_t e = cudaMemcpyAsync(d_mu, mu_host, sizeof(double) * (size_t)B * Q, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "rbws_apply_operator_static: copy mu");
  launch_coef_tables(g, kx, ky, kz, bx, by, segq, sx, sy, sz, Q, d_mu, B, c64, c32, s);
  if (fp32)
    launch_apply<float>(g, t, c32, B, static_cast<const float*>(x), g.n, static_cast<float*>(y), s);
  else
    launch_apply<double>(g, t, c64, B, static_cast<const double*>(x), g.n, static_cast<double*>(y), s);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "rbws_apply_operator_static: launch");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "rbws_apply_operator_static");
  return RBWS_OK;
}

}  // namespace rbws
