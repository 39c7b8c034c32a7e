// polar_gemm_noalloc: the general product of polar_gemm without any device
// allocation.
//
// polar_gemm keeps the BF16 planes of its operands in a scratch buffer that it
// grows with cudaMalloc (and cudaFree). Some callers cannot allow that: a process
// whose device memory is entirely owned by another allocator (for example a
// framework's caching allocator that reserved the pool up front), or a
// latency-critical loop that must not take the device-wide synchronisation a
// cudaFree may imply. For them this entry point keeps the planes in one static
// device array of fixed size, POLAR_NOALLOC_SCRATCH_BYTES, instead.
//
// The array lives on every GPU that loads this part of the library, from then
// until the process exits. Its device address is looked up once per device
// (cudaGetSymbolAddress, with that device current) by the first call made on
// that device, so that first call should come before any stream capture.
// Every call shares the array: two calls whose work overlaps on the GPU (other
// streams, other threads) race on it. Each call rewrites every plane element
// it reads; padding between rows is never read (the TMA tensor maps stop at
// the matrix edge and fill zeros beyond), so nothing has to be cleared.
#include <mutex>

#include "internal.cuh"

using namespace polar;

namespace {

static __device__ __align__(256) uint16_t g_noalloc_scratch[POLAR_NOALLOC_SCRATCH_BYTES / 2];

// Per-device address of the array. Only a successful lookup is kept: a failed one
// (its error cleared from the runtime's last-error slot) is retried by the next call.
struct ScratchAddr {
  std::mutex mu;
  void* ptr = nullptr;
};
ScratchAddr g_addr[64];

polar_status_t scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return POLAR_ECUDA;
  }
  ScratchAddr& s = g_addr[dev];
  std::lock_guard<std::mutex> lk(s.mu);
  if (!s.ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return POLAR_ECUDA;
    }
    s.ptr = p;
  }
  *out = s.ptr;
  return POLAR_OK;
}

int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" polar_status_t polar_gemm_noalloc(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                             float* C, int64_t ldc, int prec, polar_stream_t stream) {
  if (M < 0 || N < 0 || K < 0) return POLAR_EINVAL;
  if (M == 0 || N == 0) return POLAR_OK;
  if (!C || ldc < N) return POLAR_EINVAL;
  if (K > 0 && (!A || !B)) return POLAR_EINVAL;
  const int64_t a_rows = transA ? K : M, a_cols = transA ? M : K;
  const int64_t b_rows = transB ? N : K, b_cols = transB ? K : N;
  if (K > 0 && (lda < a_cols || ldb < b_cols)) return POLAR_EINVAL;
  // the same device check and precision resolution as polar_gemm, in the same order
  if (!device_is_sm103()) { cudaGetLastError(); return POLAR_ECUDA; }
  prec = resolve_precision(prec, M < N ? M : N);
  const int P = product_planes(prec);
  if (P == 0 && prec != POLAR_FP32) return prec == POLAR_TF32X3 ? POLAR_ENOTSUP : POLAR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0 || P == 0) {  // no scratch needed: the FP32 product reads its operands directly
    SimtArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = K ? A : C; g.lda = K ? lda : ldc; g.a_kmajor = transA ? 0 : 1;
    g.B = K ? B : C; g.ldb = K ? ldb : ldc; g.b_kmajor = transB ? 1 : 0;
    g.C = C; g.ldc = ldc; g.alpha = K ? alpha : 0.f; g.beta = beta;
    return launch_simt_gemm(g, SIMT_EPI_STORE, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
  }
  const int64_t lpa = up(a_cols, 64), lpb = up(b_cols, 64);
  const int64_t sa = up(a_rows * lpa, 64), sb = up(b_rows * lpb, 64);
  if ((uint64_t)P * (uint64_t)(sa + sb) * 2u > (uint64_t)POLAR_NOALLOC_SCRATCH_BYTES) return POLAR_ENOMEM;
  if (!tc_available()) return POLAR_ENOTSUP;
  void* base = nullptr;
  polar_status_t r = scratch_address(&base);
  if (r != POLAR_OK) return r;
  uint16_t* pa = static_cast<uint16_t*>(base);
  uint16_t* pb = pa + P * sa;
  if (launch_scale_split(A, lda, a_rows, a_cols, nullptr, false, nullptr, 0, pa, lpa, sa, P, s) != cudaSuccess ||
      launch_scale_split(B, ldb, b_rows, b_cols, nullptr, false, nullptr, 0, pb, lpb, sb, P, s) != cudaSuccess)
    return POLAR_ECUDA;
  TcArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.a.planes = pa; g.a.rows = a_rows; g.a.cols = a_cols; g.a.ld = lpa; g.a.plane_stride = sa; g.a.kmajor = transA ? 0 : 1;
  g.b.planes = pb; g.b.rows = b_rows; g.b.cols = b_cols; g.b.ld = lpb; g.b.plane_stride = sb; g.b.kmajor = transB ? 1 : 0;
  g.nplanes = P;
  g.epi = TC_EPI_STORE;
  g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta;
  return launch_tc_gemm(g, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}
