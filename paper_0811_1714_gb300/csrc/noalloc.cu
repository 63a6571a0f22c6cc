// noalloc.cu -- gf2_mul_noalloc: the product for callers that cannot
// allocate device memory (see include/gf2.h).  The paper has no
// counterpart; the arithmetic is gf2_mul's, unchanged.
//
// The scratch is one file-scope __device__ array of
// GF2_NOALLOC_SCRATCH_BYTES, part of the library's device image, so every
// GPU that loads the library holds it until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it names a
// stand-in, not device memory): its device address is looked up here, once
// per device with that device current, by cudaGetSymbolAddress, and only
// that address is handed on.
#include "common.cuh"

#include <mutex>

namespace gf2 {
int mul_with_scratch(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts *opts,
                     void *scratch, size_t scratch_bytes, void *stream);
}

namespace {

constexpr size_t kScratchBytes = (size_t)GF2_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices];   // device address of the buffer, per device (null: not set up)

// Set-up on the current device: the buffer's device address, once.
int scratch_for_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GF2_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GF2_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
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
