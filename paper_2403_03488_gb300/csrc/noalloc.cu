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
#include "common.cuh"

// The scratch array.  In host code its name is only a host-side stand-in; the
// device address is looked up on every call with cudaGetSymbolAddress (a host
// lookup in the current context, so a device reset or a new primary context
// never leaves a stale address behind).
static __device__ __align__(256) unsigned char g_noalloc_scratch[DN_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array in the current context.  Under lazy
// module loading the first lookup on a device loads the library's device code
// there, which is when the array is reserved.
dn_status scratch_for_current_device(void **out)
{
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return DN_ECUDA;
    *out = ptr;
    return DN_OK;
}

}  // namespace

extern "C" size_t dn_noalloc_scratch_bytes(void) { return (size_t)DN_NOALLOC_SCRATCH_BYTES; }

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
