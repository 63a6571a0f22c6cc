// tc_fp8.cu -- tensor-core base case (placeholder until the tcgen05 kernel lands).
#include "common.cuh"

namespace gf2 {

bool tc_fp8_available() { return false; }

int tc_fp8_launch(const TcLaunch &, cudaStream_t) { return GF2_EUNSUPPORTED; }

}  // namespace gf2
