// Grouped tensor-core launches of the batched solves: the instantiations for one and two BF16 planes
// (a translation unit of its own so that they compile in parallel).
#include "gemm_tc_kernel.cuh"

namespace polar {

cudaError_t tc_dispatch_grouped1(const TcGroupLaunch& g, cudaStream_t s) { return dispatch_grouped<1>(g, s); }

cudaError_t tc_dispatch_grouped2(const TcGroupLaunch& g, cudaStream_t s) { return dispatch_grouped<2>(g, s); }

}  // namespace polar
