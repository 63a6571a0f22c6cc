// tc_status.cu -- the device status word of the tensor-core base cases'
// bounded waits, and the failure-detection self test: a wait that nothing can
// satisfy, bounded like every wait of the product kernels, which records
// GF2_ETIMEOUT instead of hanging.
#include "common.cuh"
#include "tcgen05.cuh"

namespace gf2 {
namespace {

__device__ unsigned int g_tc_status;   // -GF2_ETIMEOUT after an expired wait

// One wait that nothing can satisfy (an mbarrier nobody arrives on), bounded
// by `limit` clock cycles; it records GF2_ETIMEOUT in the status word exactly
// like the product kernels do.
__global__ void wait_selftest_kernel(unsigned long long limit, unsigned int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(tc::smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (!tc::mbar_try_wait(tc::smem_u32(&bar), 0)) {
            if ((unsigned long long)(clock64() - t0) > limit) {
                atomicExch(status, (unsigned int)(-GF2_ETIMEOUT));
                break;
            }
        }
    }
}

}  // namespace

int wait_selftest_launch(long long limit, cudaStream_t s)
{
    unsigned int *st = nullptr;
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&st, g_tc_status));
    wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)limit, st);
    note_launch();
    return check_launch();
}

int tc_status_address(unsigned int **p)
{
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)p, g_tc_status));
    return GF2_OK;
}

int tc_status_read_and_clear(unsigned int *out, cudaStream_t s)
{
    unsigned int *p = nullptr;
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&p, g_tc_status));
    unsigned int v = 0;
    GF2_CUDA_TRY(cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, s));
    GF2_CUDA_TRY(cudaStreamSynchronize(s));
    GF2_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof v, s));
    *out = v;
    return GF2_OK;
}

}  // namespace gf2
