// FP8 E4M3 tensor-core products (tcgen05.mma.kind::f8f6f4, one plane of codes, K-major operands, per-tile
// power-of-two scales applied at the promotion of every 128-K slice): the STORE, GRAM and NS epilogues
// (a translation unit of its own so that the kernels compile in parallel).
#include "gemm_tc_kernel.cuh"

namespace polar {

cudaError_t tc_dispatch_fp8(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                            int64_t ntiles, cudaStream_t s) {
  switch (a.epi) {
    case TC_EPI_GRAM: return launch_t<FP8, false, false, TC_EPI_GRAM>(ma, mb, a, tm, tn, ntiles, s);
    case TC_EPI_NS: return launch_t<FP8, false, false, TC_EPI_NS>(ma, mb, a, tm, tn, ntiles, s);
    default: return launch_t<FP8, false, false, TC_EPI_STORE>(ma, mb, a, tm, tn, ntiles, s);
  }
}

}  // namespace polar
