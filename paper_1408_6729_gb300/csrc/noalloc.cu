// noalloc.cu -- bsps_sort_keys for callers that cannot allocate device memory.
//
// The regular entry points take a caller-owned workspace.  Some callers have no
// way to provide one: code whose device memory is owned by another runtime or
// framework with no allocation hook exposed to it, or latency-critical code
// that must never call cudaMalloc (which can synchronize the device).  For them,
// the library carries its own scratch: one file-scope __device__ array of
// BSPS_NOALLOC_SCRATCH_BYTES, held by every GPU that loads this library until
// the process exits.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so its device address is looked up once per device with
// cudaGetSymbolAddress and cached.
#include <mutex>

#include "kernels.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[BSPS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_of_device[kMaxDevices] = {};

// Device address of the scratch on the current device (set up on first use).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BSPS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_of_device[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BSPS_ERR_CUDA;
        g_scratch_of_device[dev] = p;
    }
    *out = g_scratch_of_device[dev];
    return BSPS_OK;
}

} // namespace

extern "C" int bsps_sort_keys_noalloc(const void *d_keys_in, void *d_keys_out, int64_t n, int32_t dtype,
                                      const bsps_params *prm, int64_t *d_bucket_sizes, void *stream) {
    size_t need = 0;
    const int rc = bsps_workspace_size(n, dtype, prm, 0, &need);
    if (rc) return rc;
    if (need > (size_t)BSPS_NOALLOC_SCRATCH_BYTES) return BSPS_ERR_TOO_LARGE;
    void *ws = nullptr;
    const int ra = scratch_address(&ws);
    if (ra) return ra;
    return bsps_sort_keys(d_keys_in, d_keys_out, n, dtype, prm, d_bucket_sizes, ws,
                          (size_t)BSPS_NOALLOC_SCRATCH_BYTES, stream);
}

extern "C" int bsps_noalloc_read_stats(bsps_stats *stats, void *stream) {
    if (!stats) return BSPS_ERR_INVALID_ARG;
    void *ws = nullptr;
    const int ra = scratch_address(&ws);
    if (ra) return ra;
    return bsps_read_stats(ws, stats, stream);
}
