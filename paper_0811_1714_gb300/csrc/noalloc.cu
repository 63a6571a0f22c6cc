// noalloc.cu -- gf2_mul_noalloc: the product for callers that cannot
// allocate device memory (see include/gf2.h).  The paper has no
// counterpart; the arithmetic is gf2_mul's, unchanged.
//
// The scratch is one file-scope __device__ array of
// GF2_NOALLOC_SCRATCH_BYTES, part of the library's device image, so every
// GPU that loads the library holds it until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it names a
// stand-in, not device memory): its device address is looked up here, once
// per device and CUDA context with that device current, by
// cudaGetSymbolAddress, and only that address is handed on.
#include "common.cuh"

#include <cuda.h>

#include <mutex>

namespace gf2 {
int mul_with_scratch(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts *opts,
                     void *scratch, size_t scratch_bytes, void *stream);
}

namespace {

constexpr size_t kScratchBytes = (size_t)GF2_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The buffer's device address belongs to the CUDA context it was looked up
// in: after a cudaDeviceReset, or with another context current, it has to
// be looked up again.  So the cache is keyed by (device, current context).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);

CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
        cudaGetLastError();
    });
    return fn;
}

struct SetUp {
    int dev = -1;
    CUcontext ctx = nullptr;
    void *ptr = nullptr;
};
constexpr int kSlots = 64;
std::mutex g_setup_mu;
SetUp g_setup[kSlots];   // (device, context) -> device address of the buffer
int g_next_slot = 0;

// Set-up on the current device: the buffer's device address, once per
// (device, context).
int scratch_for_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ECUDA;
    }
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    bool keyed = get && get(&ctx) == CUDA_SUCCESS && ctx;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (keyed)
        for (const SetUp &e : g_setup)
            if (e.ptr && e.dev == dev && e.ctx == ctx) {
                *out = e.ptr;
                return GF2_OK;
            }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return GF2_ECUDA;
    }
    // no context was current before the lookup, which made the device's
    // primary context current: key the address by that one
    if (!keyed) keyed = get && get(&ctx) == CUDA_SUCCESS && ctx;
    if (keyed) {
        SetUp &slot = g_setup[g_next_slot];
        g_next_slot = (g_next_slot + 1) % kSlots;
        slot.dev = dev;
        slot.ctx = ctx;
        slot.ptr = p;
    }
    *out = p;
    return GF2_OK;
}

}  // namespace

extern "C" int gf2_mul_noalloc(gf2_mat *C, const gf2_mat *A, const gf2_mat *B,
                               const gf2_opts *opts, void *cuda_stream)
{
    if (!C || !A || !B) return GF2_EINVAL;
    if (A->device == GF2_HOST || B->device == GF2_HOST || C->device == GF2_HOST) return GF2_EINVAL;
    void *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    return gf2::mul_with_scratch(C, A, B, opts, scratch, kScratchBytes, cuda_stream);
}
