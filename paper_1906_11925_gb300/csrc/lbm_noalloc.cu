// Static device scratch for the entry point that allocates nothing
// (lbm_get_populations_noalloc in lbm_host.cpp).
//
// lbm_get_populations stages the float64 populations in a buffer it obtains
// with cudaMalloc and releases with cudaFree on every call.  Some callers
// cannot allow that: an application whose device memory is owned by its own
// pool allocator (a framework's caching allocator, a server running under a
// fixed memory budget) must not see allocations outside the pool, and
// cudaFree synchronises the whole device, stalling every other stream.  For
// them the same gather writes into the file-scope array below instead.
//
// The array is a fixed 8 MiB (kNoAllocMaxValues float64 values) that every GPU
// loading this library holds until the process exits.  In host code its name
// is only a host-side stand-in: the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, and cached for
// the life of the process.  A device reset (cudaDeviceReset) unloads the
// module and would leave the cached address stale, so the library assumes the
// device is not reset while it is loaded.
#include <mutex>

#include "lbm_internal.h"

namespace hemelb_gb300 {

namespace {

constexpr size_t kNoAllocMaxValues = size_t(1) << 20;  // 8 MiB of float64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxValues];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

}  // namespace

size_t noalloc_max_values() { return kNoAllocMaxValues; }

cudaError_t noalloc_scratch(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace hemelb_gb300
