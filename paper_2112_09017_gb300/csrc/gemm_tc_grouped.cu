// Grouped tensor-core launches of the batched solves (many problems per launch, a tile table):
// the instantiations for three BF16 planes (a translation unit of its own so that they compile in parallel).
#include "gemm_tc_kernel.cuh"

namespace polar {

cudaError_t tc_dispatch_grouped3(const TcGroupLaunch& g, cudaStream_t s) { return dispatch_grouped<3>(g, s); }

}  // namespace polar
