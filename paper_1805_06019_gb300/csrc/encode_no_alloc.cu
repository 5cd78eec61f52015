// rlfc_encode_no_alloc: the GPU encoder with its device scratch taken from a
// fixed array compiled into the library instead of cudaMalloc.
//
// Some callers cannot allocate device memory while they encode: code running
// under a custom or capped device allocator that must not see foreign
// cudaMalloc calls, processes whose device memory is fully reserved up front,
// or callers that must avoid the device-wide synchronisation cudaMalloc and
// cudaFree can cause.  This entry point serves them for light fields whose
// encoder scratch fits in kScratchBytes.
//
// The array lives in this translation unit only.  Under lazy module loading
// (the CUDA default since 12.2) its module, and with it kScratchBytes of
// device memory, is loaded on a device the first time this entry point runs
// there and then held until the process exits; with CUDA_MODULE_LOADING=EAGER
// every context that loads the library reserves the array at creation, even
// one that only decodes or renders.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "rlfc_internal.h"

namespace rlfc {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB

static __device__ __align__(256) uint8_t g_encode_scratch[kScratchBytes];

// Device address of the scratch array in the current context.  Host code may
// not use the array's name as a device pointer, so the address is looked up
// with the device current, on every call: it allocates nothing and costs
// little next to the encode, and a cached address would go stale if the
// caller reset the device or the primary context was created again.
int scratch_on_current_device(uint8_t **out)
{
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_encode_scratch);
    if (e != cudaSuccess)
        return cuda_fail(e, "no-alloc encoder: scratch address");
    *out = static_cast<uint8_t *>(ptr);
    return RLFC_OK;
}

}  // namespace
}  // namespace rlfc

using namespace rlfc;

extern "C" RLFC_API int rlfc_encode_no_alloc(const rlfc_enc_params *p, const uint8_t *d_rgb,
                                             void *cuda_stream, void *host_out, size_t capacity,
                                             size_t *nbytes)
{
    if (!p || !d_rgb || !nbytes) {
        set_error("null argument");
        return RLFC_E_INVALID_ARG;
    }
    *nbytes = 0;
    const size_t need = encode_scratch_bound(p);
    if (need == 0) {
        set_error("encoder parameters out of range (or a block size other than 4)");
        return p->B != 4 ? RLFC_E_UNSUPPORTED : RLFC_E_INVALID_ARG;
    }
    if (need > kScratchBytes) {
        set_error("light field needs " + std::to_string(need) + " bytes of encoder scratch; the no-alloc "
                  "encoder has " + std::to_string(kScratchBytes) + " (use rlfc_encode)");
        return RLFC_E_RANGE;
    }
    uint8_t *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != RLFC_OK)
        return rc;
    try {
        std::vector<uint8_t> out;
        // the buffers are carved from the first `need` bytes only, so an
        // encode that would use more than its bound fails instead of
        // reaching past what the size check above admitted
        rc = encode_gpu(p, d_rgb, (cudaStream_t)cuda_stream, out, scratch, need);
        if (rc != RLFC_OK)
            return rc;
        *nbytes = out.size();
        if (!host_out || capacity < out.size()) {
            set_error("output buffer too small: the stream has " + std::to_string(out.size()) + " bytes");
            return RLFC_E_RANGE;
        }
        std::memcpy(host_out, out.data(), out.size());
        return RLFC_OK;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return RLFC_E_OOM;
    }
}
