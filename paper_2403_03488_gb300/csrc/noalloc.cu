// BM3D for callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc: a plug-in living inside a
// host application that owns the whole device-memory budget (a camera or
// video pipeline with a fixed memory pool), or a caller in a latency-critical
// loop that cannot afford an allocation, which may block until the device is
// idle.  For them this file keeps the BM3D workspace in a fixed-size array of
// device memory that is part of the library itself: it is reserved when the
// library's device code is loaded on a GPU and stays reserved until the
// process exits.
#include <mutex>

#include "common.cuh"

// The scratch array.  In host code its name is only a host-side stand-in; the
// device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DN_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up on the
// first call per device).
dn_status scratch_for_current_device(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return DN_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return DN_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return DN_ECUDA;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return DN_OK;
}

}  // namespace

extern "C" dn_status denoise_bm3d_noalloc(const float *noisy, float *out, int B, int C, int H, int W,
                                          const float *sigma, const dn_bm3d_params *p, dn_stream_t stream)
{
    try {
        const size_t need = dn_bm3d_workspace_bytes(B, C, H, W, p);
        if (need == 0) return DN_EINVAL;
        if (need > (size_t)DN_NOALLOC_SCRATCH_BYTES) return DN_ENOMEM;
        void *ws = nullptr;
        DN_TRY(scratch_for_current_device(&ws));
        return denoise_bm3d(noisy, out, B, C, H, W, sigma, p, ws, (size_t)DN_NOALLOC_SCRATCH_BYTES, stream);
    } catch (...) {
        return DN_ECUDA;
    }
}
