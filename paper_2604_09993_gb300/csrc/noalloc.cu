// noalloc.cu — ciscvx_discretize_vjp_static: the VJP with its scratch memory in a
// fixed array that the library itself holds on every device, for callers that
// must not allocate device memory at call time.
//
// Who needs it: a model-predictive-control loop that re-linearizes and
// re-solves every few milliseconds cannot afford cudaMalloc in its loop (it
// may synchronize the whole device and its latency is unbounded), and a solver
// embedded in a host framework that owns all device memory through its own
// pool is often not allowed to allocate outside that pool.  Both can call this
// entry point with only their inputs and outputs.
//
// How: the scratch lives in g_vjp_scratch below, CISCVX_STATIC_SCRATCH_BYTES
// bytes of static device memory that every GPU loading the library keeps until
// the process exits.  Host code cannot use the array's name as a device
// address, so on its first call on a device (with that device current) the
// entry point asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result, and caches it for that device.
// That first call should therefore come before any stream capture.  The
// cached address stays valid for the life of the device's primary context: a
// cudaDeviceReset (or any teardown of that context) invalidates it, so a
// process that resets a device must not call this entry point on it again.
// No cudaMalloc, cudaFree or allocating library routine is called.  Every
// call shares the one array: two calls whose work overlaps on the GPU
// (different streams or host threads) race and corrupt each other's results,
// so callers must serialize them.  The VJP writes every scratch element
// before reading it, so nothing needs clearing between calls.
//
// Sizing: the request is sized with ciscvx_discretize_workspace_size.  For
// models whose VJP is the per-link adjoint kernel (either auxiliary model)
// the scratch is one fixed size for N.  For models with coupled links the
// coupled adjoint runs in chunks of intervals that fit the scratch, so only
// the minimum (a chunk of up to 32 intervals) has to fit.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = CISCVX_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_vjp_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_vjp_scratch on the current device (looked up once per device).
ciscvx_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return ciscvx::set_error(CISCVX_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return ciscvx::set_error(CISCVX_EUNSUPPORTED, "device index %d above %d", dev, kMaxDevices - 1);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_vjp_scratch);
    if (e != cudaSuccess || !p)
      return ciscvx::set_error(CISCVX_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                               cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CISCVX_OK;
}

}  // namespace

extern "C" ciscvx_status ciscvx_discretize_vjp_static(
    const ciscvx_model* model, int N, int n_sub, ciscvx_precision precision,
    ciscvx_u_layout layout, const double* X, const double* U, const double* s, const double* w,
    const double* rho, double* gX, double* gU, double* gs, double* L, void* stream) {
  if (!model) return ciscvx::set_error(CISCVX_EINVAL, "null model");
  size_t need = 0;
  ciscvx_status st = ciscvx_discretize_workspace_size(model, CISCVX_OP_VJP, N, n_sub, precision,
                                                      layout, &need, nullptr);
  if (st != CISCVX_OK) return st;
  if (need > kScratchBytes)
    return ciscvx::set_error(CISCVX_EUNSUPPORTED,
                             "this VJP needs at least %zu bytes of scratch; the built-in static "
                             "scratch holds %zu bytes (use ciscvx_discretize_vjp with a workspace, "
                             "or fewer intervals)",
                             need, kScratchBytes);
  void* scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != CISCVX_OK) return st;
  return ciscvx_discretize_vjp(model, N, n_sub, precision, layout, X, U, s, w, rho, gX, gU, gs, L,
                               scratch, kScratchBytes, stream);
}
