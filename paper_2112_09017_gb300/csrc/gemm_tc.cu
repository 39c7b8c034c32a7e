// Host side of the split-BF16 tensor-core products (tcgen05, sm_103a): tensor maps over the
// operands' BF16 planes, argument checks, the choice between single-CTA tiles and CTA-pair
// tiles, and the launches (the kernels themselves are in gemm_tc_kernel.cuh).
#include <cuda.h>
#include <stdlib.h>

#include <mutex>

#include "gemm_tc_kernel.cuh"

namespace polar {

__device__ unsigned int g_tc_error;      // timeouts of launches without a plan state or error word
__device__ unsigned int g_tc_error_out;  // tc_take_error's copy of the word it cleared

namespace {

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    else
      cudaGetLastError();
  });
  return fn;
}

// 3-D map (columns, rows, planes) over an operand's planes; the box is one stage's slice.
bool make_map(CUtensorMap* map, const TcOperand& op, int nplanes, bool mn_major, int mn_box) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.cols, (cuuint64_t)op.rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld * 2, (cuuint64_t)op.plane_stride * 2};
  cuuint32_t box[3];
  cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMapSwizzle swz;
  if (mn_major) {
    box[0] = 64; box[1] = BK; box[2] = (cuuint32_t)nplanes;
    swz = CU_TENSOR_MAP_SWIZZLE_128B;
  } else {
    box[0] = BK; box[1] = (cuuint32_t)mn_box; box[2] = (cuuint32_t)nplanes;
    swz = BK == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : BK == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  }
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(op.planes), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D map over one plane of FP8 E4M3 codes (columns = K, rows, one plane), K-major, 128-byte rows of
// the box with the 128-byte swizzle (the layout of the FP8 kernel's stages).
bool make_map_u8(CUtensorMap* map, const TcOperand& op, int mn_box) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)op.cols, (cuuint64_t)op.rows, 1};
  const uint64_t plane = ((uint64_t)op.ld * (uint64_t)op.rows + 15) / 16 * 16;
  cuuint64_t strides[2] = {(cuuint64_t)op.ld, (cuuint64_t)plane};
  cuuint32_t box[3] = {128, (cuuint32_t)mn_box, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint16_t*>(op.planes), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Device address of g_tc_error on the current device (looked up once per device), the error word
// of launches that have neither a plan state nor an error word of their own.
unsigned int* default_error_word() {
  static std::mutex mu;
  static unsigned int* word[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!word[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_error) == cudaSuccess) word[dev] = static_cast<unsigned int*>(p);
    else cudaGetLastError();
  }
  return word[dev];
}

}  // namespace

__global__ void tc_take_error_kernel() { g_tc_error_out = atomicExch(&g_tc_error, 0u); }

cudaError_t tc_take_error(cudaStream_t s, unsigned int* out) {
  tc_take_error_kernel<<<1, 1, 0, s>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyFromSymbolAsync(out, g_tc_error_out, sizeof(unsigned int), 0, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

// Whether a launch of `planes`-plane products runs as CTA pairs: three planes (the pair kernels'
// instantiations) and at least one 256 x 256 pair tile for every pair of SMs, so that the pairs'
// halved shared-memory operand traffic is not paid for with idle SMs. POLAR_TC_CTA_PAIR in the
// environment overrides the size rule: 0 never, 1 whenever the planes allow it.
bool use_pair(int planes, int64_t M, int64_t N, bool tri) {
  if (planes != 3) return false;
  const char* e = getenv("POLAR_TC_CTA_PAIR");
  const int mode = (e && (e[0] == '0' || e[0] == '1')) ? e[0] - '0' : -1;
  if (mode >= 0) return mode == 1;
  const int64_t tm2 = (M + 2 * BM - 1) / (2 * BM), tn = (N + BN - 1) / BN;
  const int64_t tiles = tri ? pair_tri_tiles(tn) : tm2 * tn;
  return tiles >= sm_count() / 2;
}

int tc_gram_partials(int64_t n, int planes) {
  const int64_t tm = (n + BM - 1) / BM, tn = (n + BN - 1) / BN;
  if (use_pair(planes, n, n, true)) return (int)(pair_tri_tiles(tn) * 2 * EPI_WARPS);
  return (int)(tri_tiles(tm, tn) * EPI_WARPS);
}

int tc_gram_partials_max(int64_t n) {
  const int64_t tm = (n + BM - 1) / BM, tn = (n + BN - 1) / BN;
  const int64_t a = tri_tiles(tm, tn) * EPI_WARPS, b = pair_tri_tiles(tn) * 2 * EPI_WARPS;
  return (int)(a > b ? a : b);
}

// k-stages per promoted slice. Each slice accumulates passes x K/16 MMAs with
// round-toward-zero before its round-to-nearest promotion; 64 of K for three
// planes (24 MMAs), 128 for two and 256 for one keep the promotion work below the
// MMA time of a slice. POLAR_TC_SLICE_STAGES (1..16) overrides it for tuning.
int default_slice_stages(int planes) {
  static int env = [] {
    const char* e = getenv("POLAR_TC_SLICE_STAGES");
    int x = e ? atoi(e) : 0;
    return (x >= 1 && x <= 16) ? x : 0;
  }();
  if (env) return env;
  static_assert(BK == 16 || BK == 32, "slice lengths are multiples of the k-stage width");
  return (planes == 3 ? 64 : planes == 2 ? 128 : 256) / BK;
}

// Test hook for the bounded waits: with POLAR_TEST_WITHHOLD_TMA=1 in the environment
// the producer issues no copies, so the consumers' waits expire after about one
// second and the launch reports a timeout instead of computing.
int withhold_tma() {
  const char* e = getenv("POLAR_TEST_WITHHOLD_TMA");
  return (e && e[0] == '1') ? 1 : 0;
}

cudaError_t launch_tc_gemm(const TcArgs& a_in, cudaStream_t s) {
  TcArgs a = a_in;
  if (a.slice_stages <= 0) a.slice_stages = default_slice_stages(a.nplanes);
  a.withhold_tma = withhold_tma();
  if (!a.st && !a.err_out) a.err_out = default_error_word();
  if (a.nplanes < 1 || a.nplanes > 3 || a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaErrorInvalidValue;
  const TcOperand* ops[2] = {&a.a, &a.b};
  for (const TcOperand* o : ops)
    if (!o->planes || !aligned(o->planes, 16) || o->ld % 8 || o->plane_stride % 8) return cudaErrorInvalidValue;
  const bool ns = a.epi == TC_EPI_NS || a.epi == TC_EPI_NS_STEP;
  const bool clen = a.epi == TC_EPI_CLENSHAW;
  if (ns || clen || a.epi == TC_EPI_GRAM || a.epi == TC_EPI_PLANES) {
    if (!a.out_planes || !aligned(a.out_planes, 16) || a.ldo % 8 || a.out_plane_stride % 8) return cudaErrorInvalidValue;
    if (a.out_nplanes < 1 || a.out_nplanes > 3) return cudaErrorInvalidValue;
  }
  if ((a.epi == TC_EPI_GRAM || a.epi == TC_EPI_NS_STEP) && !a.partials) return cudaErrorInvalidValue;
  if (clen && (!a.triangular || a.M != a.N)) return cudaErrorInvalidValue;
  if ((ns || clen) &&
      (!a.x_planes || !aligned(a.x_planes, 16) || a.ldxp % 8 || a.x_plane_stride % 8 || a.out_nplanes != 3))
    return cudaErrorInvalidValue;
  if (a.triangular && a.M != a.N) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  const bool pair = use_pair(a.nplanes, a.M, a.N, a.triangular != 0);
  if (!make_map(&ma, a.a, a.nplanes, !a.a.kmajor, BM)) return cudaErrorInvalidValue;
  if (!make_map(&mb, a.b, a.nplanes, !a.b.kmajor, pair ? BN / 2 : BN)) return cudaErrorInvalidValue;
  if (pair) {   // 256 x 256 pair tiles; each CTA stages 128 of the tile's columns of B
    const int64_t tm2 = (a.M + 2 * BM - 1) / (2 * BM), tn2 = (a.N + BN - 1) / BN;
    return tc_dispatch_pair3(ma, mb, a, tm2, tn2, a.triangular ? pair_tri_tiles(tn2) : tm2 * tn2, s);
  }
  const int64_t tm = (a.M + BM - 1) / BM, tn = (a.N + BN - 1) / BN;
  const int64_t ntiles = a.triangular ? tri_tiles(tm, tn) : tm * tn;
  switch (a.nplanes) {
    case 1: return tc_dispatch_single1(ma, mb, a, tm, tn, ntiles, s);
    case 2: return tc_dispatch_single2(ma, mb, a, tm, tn, ntiles, s);
    default: return tc_dispatch_single3(ma, mb, a, tm, tn, ntiles, s);
  }
}

cudaError_t launch_tc_gemm_fp8(const TcArgs& a_in, cudaStream_t s) {
  TcArgs a = a_in;
  a.slice_stages = 1;                 // one 128-K block per slice: its scale is applied at the promotion
  if (a.a_uni && a.b_uni && a.fp8_run <= 0) a.fp8_run = 8;   // tiles under one scale: 1024 K per slice
  if (!a.a_uni || !a.b_uni) a.a_uni = a.b_uni = nullptr;
  a.withhold_tma = withhold_tma();
  if (!a.st && !a.err_out) a.err_out = default_error_word();
  if (a.M <= 0 || a.N <= 0 || a.K <= 0 || !a.a_exp || !a.b_exp || a.lde_a < (a.K + 127) / 128 ||
      a.lde_b < (a.K + 127) / 128)
    return cudaErrorInvalidValue;
  if (!a.a.kmajor || !a.b.kmajor) return cudaErrorInvalidValue;
  const TcOperand* ops[2] = {&a.a, &a.b};
  for (const TcOperand* o : ops)
    if (!o->planes || !aligned(o->planes, 16) || o->ld % 16 || o->ld < o->cols) return cudaErrorInvalidValue;
  if (a.epi != TC_EPI_STORE && a.epi != TC_EPI_GRAM && a.epi != TC_EPI_NS) return cudaErrorInvalidValue;
  if (a.epi != TC_EPI_STORE) {
    if (!a.out_planes || !aligned(a.out_planes, 16) || a.ldo % 8 || a.out_plane_stride % 8 || a.out_nplanes != 3)
      return cudaErrorInvalidValue;
  }
  if (a.epi == TC_EPI_GRAM && (!a.partials || !a.triangular)) return cudaErrorInvalidValue;
  if (a.epi == TC_EPI_NS && (!a.x_planes || !aligned(a.x_planes, 16) || a.ldxp % 8 || a.x_plane_stride % 8))
    return cudaErrorInvalidValue;
  if (a.triangular && a.M != a.N) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map_u8(&ma, a.a, BM) || !make_map_u8(&mb, a.b, BN)) return cudaErrorInvalidValue;
  const int64_t tm = (a.M + BM - 1) / BM, tn = (a.N + BN - 1) / BN;
  return tc_dispatch_fp8(ma, mb, a, tm, tn, a.triangular ? tri_tiles(tm, tn) : tm * tn, s);
}

}  // namespace polar

// ---------------------------------------------------------------- grouped launches

namespace polar {

bool tc_make_entry_maps(TcGroupEntry* e) {
  const TcArgs& a = e->args;
  return make_map(reinterpret_cast<CUtensorMap*>(e->map_a), a.a, a.nplanes, !a.a.kmajor, BM) &&
         make_map(reinterpret_cast<CUtensorMap*>(e->map_b), a.b, a.nplanes, !a.b.kmajor, BN);
}

cudaError_t launch_tc_gemm_grouped(const TcGroupLaunch& g_in, cudaStream_t s) {
  TcGroupLaunch g = g_in;
  if (g.nplanes < 1 || g.nplanes > 3 || !g.tiles || !g.entries) return cudaErrorInvalidValue;
  if (g.slice_stages <= 0) g.slice_stages = default_slice_stages(g.nplanes);
  g.withhold_tma = withhold_tma();
  switch (g.nplanes) {
    case 1: return tc_dispatch_grouped1(g, s);
    case 2: return tc_dispatch_grouped2(g, s);
    default: return tc_dispatch_grouped3(g, s);
  }
}

}  // namespace polar
