// Morton sort that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they run: code that lives inside
// a framework whose caching allocator owns the device memory (a foreign
// allocation breaks its accounting), latency-bound loops where cudaMalloc or
// cudaFree would stall (cudaFree waits for the whole device), and processes
// that reserve a fixed memory budget up front.  For them this file keeps the
// sort's scratch in one statically sized device array that every GPU loading
// the library holds until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "ls_internal.h"
#include "ls_kernels.h"

namespace {

constexpr long long kMaxPoints = 1LL << 18;        // largest n accepted
constexpr size_t kScratchBytes = 3932160;           // >= ls_morton_scratch_bytes(kMaxPoints) (3.75 MiB)
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code its name is only a host-side stand-in for
// the symbol, never a device address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch on the current device, looked up once per
// device (on the first call made with that device current).
ls_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ls_fail(LS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return ls_fail(LS_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ls_fail(LS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                            cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LS_OK;
}

}  // namespace

extern "C" ls_status ls_morton_sort_noalloc(const float *pts, int64_t n, const float *origin, float cell,
                                            int32_t *perm, uint32_t *keys_out, ls_stream stream)
{
    if (n < 0 || (n > 0 && (!pts || !perm)) || !origin) return ls_fail(LS_ERR_INVALID_ARG, "NULL argument");
    if (!(cell > 0.0f) || !std::isfinite(cell)) return ls_fail(LS_ERR_INVALID_ARG, "cell must be positive");
    if (n > kMaxPoints)
        return ls_fail(LS_ERR_INVALID_ARG, "ls_morton_sort_noalloc sorts at most 262144 points (2^18); use "
                                           "ls_morton_sort for more");
    if (n == 0) return LS_OK;
    const size_t need = align256((size_t)n * 4) + lsk::sort_scratch_bytes(n);
    if (need > kScratchBytes) return ls_fail(LS_ERR_INVALID_ARG, "static scratch too small for this n");
    void *base = nullptr;
    ls_status st = scratch_address(&base);
    if (st != LS_OK) return st;
    // Nothing in the scratch has to start at zero: the key pass writes every
    // key, and each radix pass overwrites its histograms and prefix sums before
    // reading them.
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *keys = keys_out ? keys_out : (uint32_t *)base;
    void *sort_ws = (char *)base + align256((size_t)n * 4);
    cudaError_t e = lsk::morton_keys(pts, n, origin, cell, keys, perm, s);
    if (e == cudaSuccess) e = lsk::radix_sort_pairs(keys, perm, n, 30, sort_ws, s);
    if (e != cudaSuccess) return ls_fail(LS_ERR_CUDA, std::string("morton sort kernels: ") + cudaGetErrorString(e));
    return LS_OK;
}
