// Allocation-free overlap: ps_overlap_noalloc (see include/ps.h).
//
// The paper has no counterpart of this entry point.  It exists for callers
// that cannot allocate device memory: cudaMalloc and cudaFree synchronise the
// whole device and fail once another allocator (a framework's caching
// allocator, a fixed budget set at start-up) owns the memory, so code on a
// latency-critical path or inside such a framework must get by with the
// buffers it already has.  The two-pass reduction needs a few kilobytes of
// partial sums; here they live in one file-scope device array instead of a
// per-handle cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <sstream>

#include "ps_internal.h"

namespace ps {

// Partial sums of the first pass (two doubles per block) for every call.
// Every GPU that loads the library holds this array until the process ends.
constexpr int kNoallocPartials = 1216;
static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocPartials];

namespace {

// Device address of g_noalloc_partials on each device, looked up once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in, never a device address.
struct SymbolCache {
    std::mutex mu;
    double *addr[64] = {};
};

SymbolCache &cache() {
    static SymbolCache c;
    return c;
}

int partials_on_current_device(double **out, std::string *err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return PS_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        *err = "device index " + std::to_string(dev) + " is outside the 64-entry scratch address cache";
        return PS_ERR_UNSUPPORTED;
    }
    SymbolCache &c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    if (!c.addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress (overlap scratch): ") + cudaGetErrorString(e);
            return PS_ERR_CUDA;
        }
        c.addr[dev] = static_cast<double *>(p);
    }
    *out = c.addr[dev];
    return PS_OK;
}

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" int ps_overlap_noalloc(int n, int dtype, const void *psi0_dev, const void *psi_dev, void *stream,
                                  double *out_dev) {
    if (n < 1 || n > kMaxN) {
        std::ostringstream os;
        os << "ps_overlap_noalloc: n = " << n << " is outside [1, " << kMaxN
           << "]; its fixed scratch of " << kNoallocPartials << " partial sums serves states up to 2^" << kMaxN
           << " amplitudes";
        set_error(os.str());
        return PS_ERR_ARG;
    }
    if (dtype != PS_C64 && dtype != PS_C128) {
        set_error("ps_overlap_noalloc: dtype must be PS_C64 or PS_C128");
        return PS_ERR_ARG;
    }
    if (!psi0_dev || !psi_dev || !out_dev) {
        set_error("ps_overlap_noalloc: null state or output pointer");
        return PS_ERR_ARG;
    }
    if (((uintptr_t)psi0_dev | (uintptr_t)psi_dev) & 15) {
        set_error("ps_overlap_noalloc: state buffers must be 16-byte aligned");
        return PS_ERR_ARG;
    }
    if (reduce_blocks() > kNoallocPartials) {
        set_error("ps_overlap_noalloc: reduction grid larger than the fixed scratch");
        return PS_ERR_UNSUPPORTED;
    }
    double *partials = nullptr;
    std::string err;
    if (int rc = partials_on_current_device(&partials, &err)) {
        set_error(err);
        return rc;
    }
    // Every partial sum is written by the first pass before the second pass
    // reads it, so nothing in the scratch needs clearing between calls.
    const int e = launch_reduce(dtype, 1, psi0_dev, psi_dev, n, partials, out_dev, stream);
    if (e != 0) {
        std::ostringstream os;
        os << "ps_overlap_noalloc: reduction launch: " << cudaGetErrorString((cudaError_t)e);
        set_error(os.str());
        return PS_ERR_CUDA;
    }
    return PS_OK;
}
