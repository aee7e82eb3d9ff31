// Allocation-free variant of the electronic reduced-density-matrix reduction.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool with the device allocator locked, host threads that
// must not call cudaMalloc because it can synchronise the device, or embedded
// integrations that only hand over pre-allocated buffers.  For them this file
// provides ttns_rho_from_root_noalloc: the caller passes the root tensor and the
// output in its own device memory, and the per-block partial sums go to a
// fixed scratch array in this file instead of a buffer allocated by the library.
//
// The scratch array is a file-scope static __device__ array of
// TTNS_NOALLOC_SCRATCH_DOUBLES doubles (1 MiB): every GPU that loads the library
// holds it until the process exits.  Its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) on the first call made
// on that device; make that first call before any stream capture.
//
// The looked-up address belongs to the device's current context: after a
// cudaDeviceReset (or any reset of the primary context) the module is loaded again
// and the remembered address is stale, so the entry point must not be used across
// such a reset within one process.
//
// All calls share the one array, so two calls whose kernels overlap on the GPU
// race on it: order them on one stream (or synchronise between them).  Each call
// overwrites every partial it reads, so nothing has to start at zero.
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/ttns.h"
#include "internal.h"

#define TTNS_NOALLOC_MAX_BLOCKS 256
#define TTNS_NOALLOC_MAX_NEL 16
#define TTNS_NOALLOC_SCRATCH_DOUBLES (TTNS_NOALLOC_MAX_BLOCKS * 2 * TTNS_NOALLOC_MAX_NEL * TTNS_NOALLOC_MAX_NEL)

namespace ttns {
cudaError_t launch_density(const double2* pool, const NodeDesc& nd, int l, const double2* rho_in, double2* xbuf,
                           double* partials, int nblocks, double* out, cudaStream_t st);
void set_last_error(const std::string& msg);
}  // namespace ttns

static __device__ __align__(256) double g_noalloc_partials[TTNS_NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" ttns_status ttns_rho_from_root_noalloc(const double* d_root, long long rows, int n_el, double* d_rho,
                                                  void* cuda_stream) {
  if (!d_root || !d_rho) {
    ttns::set_last_error("ttns_rho_from_root_noalloc: NULL device pointer");
    return TTNS_E_INVALID;
  }
  if (n_el < 1 || n_el > TTNS_NOALLOC_MAX_NEL) {
    ttns::set_last_error("ttns_rho_from_root_noalloc: n_el must be in 1..16 (the fixed scratch holds 256 blocks of "
                         "16 x 16 complex partial sums)");
    return TTNS_E_INVALID;
  }
  if (rows < 1 || rows * n_el >= (1LL << 24)) {
    ttns::set_last_error("ttns_rho_from_root_noalloc: rows must be >= 1 with rows * n_el < 2^24");
    return TTNS_E_INVALID;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    ttns::set_last_error(std::string("ttns_rho_from_root_noalloc: scratch address: ") + cudaGetErrorString(e));
    return TTNS_E_CUDA;
  }
  ttns::NodeDesc nd{};
  nd.nl = 2;
  nd.dims[0] = (int)rows;
  nd.dims[1] = n_el;
  nd.strides[0] = n_el;
  nd.strides[1] = 1;
  nd.size = (int)(rows * n_el);
  nd.off = 0;
  nd.inv_dims[0] = 1.0f / (float)nd.dims[0];
  nd.inv_dims[1] = 1.0f / (float)nd.dims[1];
  nd.inv_strides[0] = 1.0f / (float)nd.strides[0];
  nd.inv_strides[1] = 1.0f;
  long long nb = rows / 64;
  if (nb < 1) nb = 1;
  if (nb > TTNS_NOALLOC_MAX_BLOCKS) nb = TTNS_NOALLOC_MAX_BLOCKS;
  e = ttns::launch_density(reinterpret_cast<const double2*>(d_root), nd, 1, nullptr, nullptr, scratch, (int)nb, d_rho,
                           static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    ttns::set_last_error(std::string("ttns_rho_from_root_noalloc: launch: ") + cudaGetErrorString(e));
    return TTNS_E_CUDA;
  }
  return TTNS_OK;
}
