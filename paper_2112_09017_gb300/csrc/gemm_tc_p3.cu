// Single-CTA tensor-core products with three BF16 planes: every epilogue kind and operand layout
// (instantiated in a translation unit of its own so that the kernels compile in parallel).
#include "gemm_tc_kernel.cuh"

namespace polar {

cudaError_t tc_dispatch_single3(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                                int64_t ntiles, cudaStream_t s) {
  return dispatch_p<3>(ma, mb, a, tm, tn, ntiles, s);
}

}  // namespace polar
