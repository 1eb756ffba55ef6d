// he_static.cu -- he_mul_rescale_static: HE Mul + rescale whose workspace is a
// fixed scratch array in the library's own device memory, for callers that
// cannot allocate device memory or keep a workspace between calls (a host
// application whose device memory is entirely owned by another allocator, or
// a thin foreign-language binding with no device allocator of its own).
//
// The scratch is a file-scope __device__ array of HE_STATIC_SCRATCH_BYTES
// (one instance per device).  In host code its name is only a stand-in, not a
// device address, so every call looks the address up with
// cudaGetSymbolAddress for the current device (cheap once the module is
// loaded, and never stale, even after the device's context was torn down
// and recreated).  The first lookup on a device may load this file's device
// module, so the first call on a device should be made outside any stream
// capture.  Nothing here calls cudaMalloc, cudaFree or any allocating routine.
//
// Nothing in the scratch has to start at zero: every word the HE Mul pipeline
// reads from its workspace is written earlier in the same call.
//
// All calls on one device share the one scratch array: two calls whose
// executions overlap (different streams, or different host threads without
// ordering between their streams) race on it and give wrong results.  Calls
// issued to the same stream are ordered and safe.
#include "he_internal.h"

using namespace he;

namespace {

constexpr size_t kScratchWords = (size_t)HE_STATIC_SCRATCH_BYTES / sizeof(u64);
static_assert((size_t)HE_STATIC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");

static __device__ __align__(256) u64 g_scratch[kScratchWords];

// Device address of the scratch on the current device.
int scratch_address(void **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HE_ECUDA;
    *out = p;
    return HE_OK;
}

}  // namespace

extern "C" int he_mul_rescale_static(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk,
                                     int level, uint64_t *out, void *stream)
{
    if (!c || !c->device || !ct1 || !ct2 || !evk || !out) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (he_workspace_bytes(c, level) > (size_t)HE_STATIC_SCRATCH_BYTES) return HE_ENOMEM;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HE_ECUDA;
    if (dev != c->device_id) return HE_EINVAL;  // the context's tables live on another device
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != HE_OK) return rc;
    return he_mul_rescale(c, ct1, ct2, evk, level, out, ws, (size_t)HE_STATIC_SCRATCH_BYTES, stream);
}
