// dpr1_noalloc.cu -- dpr1_eig for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or a caching allocator: code that runs inside
// another framework's memory pool, a plugin that must not grow the process's device
// footprint, or a setting where allocation is forbidden at run time.  dpr1_eig_noalloc
// runs exactly the dpr1_eig launch sequence, but its scratch memory (the workspace of
// dpr1_eig) is the file-scope device array below instead of caller-provided memory, so
// the caller only passes the inputs and the outputs.
//
// The array belongs to the library: every device that loads the library holds its
// NOALLOC_WS_BYTES until the process exits.  All calls on one device share it and it
// keeps the last call's contents; run_eig clears the status word and the counters at the
// start of each call.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on the shared array and give wrong
// results: order them on one stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/dpr1.h"
#include "dpr1_device.cuh"
#include "dpr1_internal.cuh"

namespace dpr1 {

dpr1_status run_eig(int64_t n64, const double* d, const double* z, double rho, double* lambda, double* Vt,
                    int64_t ldv, double* sigma, double* mu, double* xnorm, void* workspace, size_t wbytes,
                    const dpr1_options* opt, cudaStream_t st);

// holds the workspace of n <= DPR1_NOALLOC_MAX_N without the solves' stored-element buffers
// (run_eig uses what is left over for them)
constexpr size_t NOALLOC_WS_BYTES = 640u * 1024u;

static __device__ __align__(256) unsigned char g_noalloc_ws[NOALLOC_WS_BYTES];

// Device address of g_noalloc_ws.  In host code the name g_noalloc_ws is only a host-side
// stand-in for the symbol; its device address is looked up with cudaGetSymbolAddress, with the
// device current, at the first call in each CUDA context of a device, and cached under that
// context's unique ID (cuCtxGetId, reached through the runtime's driver entry points so the
// library needs no link against the driver).  A context that is destroyed and rebuilt (for
// example after cudaDeviceReset by the caller or another library) reloads the module, and the
// array may then sit at another address: the new context has a new ID, so the next call looks
// the address up again instead of using a stale one.  Where the context ID cannot be read, the
// address is looked up at every call.
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

static std::mutex g_mu;
static void* g_addr[64];
static unsigned long long g_ctx[64];      // context ID the cached address belongs to (0: none)
static ctx_get_current_fn g_get_current = nullptr;
static ctx_get_id_fn g_get_id = nullptr;
static bool g_entry_tried = false;

// ID of the context current on this thread, 0 if there is none or it cannot be read.
static unsigned long long current_ctx_id() {
  if (!g_entry_tried) {
    g_entry_tried = true;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      g_get_current = (ctx_get_current_fn)f1;
      g_get_id = (ctx_get_id_fn)f2;
    }
  }
  if (!g_get_current || !g_get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (g_get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
  if (g_get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

static dpr1_status noalloc_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DPR1_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long id = current_ctx_id();
  if (id != 0 && g_ctx[dev] == id) {
    *out = g_addr[dev];
    return DPR1_OK;
  }
  // first call in this context (the lookup also makes the device's primary context current)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || p == nullptr) return DPR1_ERR_CUDA;
  g_addr[dev] = p;
  g_ctx[dev] = current_ctx_id();
  *out = p;
  return DPR1_OK;
}

}  // namespace dpr1

using namespace dpr1;

extern "C" dpr1_status dpr1_eig_noalloc(int64_t n, const double* d, const double* z, double rho, double* lambda,
                                        double* Vt, int64_t ldv, double* sigma, double* mu, double* xnorm,
                                        const dpr1_options* opt, int wait, dpr1_stream_t stream) {
  if (n < 0) return DPR1_ERR_ARG;
  if (n > DPR1_NOALLOC_MAX_N) return DPR1_ERR_ARG;        // beyond the static scratch
  if (!std::isfinite(rho) || rho < 0.0) return DPR1_ERR_RHO;
  if (n == 0) return DPR1_OK;
  if (!d || !z || !lambda) return DPR1_ERR_ARG;
  if (Vt && ldv < n) return DPR1_ERR_ARG;
  size_t need = ws_layout(n, nullptr, nullptr);   // the stored-element buffers are optional
  if (need > NOALLOC_WS_BYTES) return DPR1_ERR_WORKSPACE;
  void* ws = nullptr;
  dpr1_status s = noalloc_address(&ws);
  if (s != DPR1_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  s = run_eig(n, d, z, rho, lambda, Vt, ldv, sigma, mu, xnorm, ws, NOALLOC_WS_BYTES, opt, st);
  if (s != DPR1_OK || !wait) return s;
  return dpr1_stream_status(ws, stream);
}
