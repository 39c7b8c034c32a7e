// CTA-pair tensor-core products (cta_group::2, 256 x 256 tiles, three BF16 planes): every epilogue kind
// and operand layout (a translation unit of its own so that the kernels compile in parallel).
#include "gemm_tc_kernel.cuh"

namespace polar {

cudaError_t tc_dispatch_pair3(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm2, int64_t tn,
                              int64_t ntiles, cudaStream_t s) {
  return dispatch_pair(ma, mb, a, tm2, tn, ntiles, s);
}

}  // namespace polar
