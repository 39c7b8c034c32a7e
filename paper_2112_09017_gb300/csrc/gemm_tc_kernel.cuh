// Split-BF16 GEMM / SYRK on the 5th-generation tensor cores (tcgen05, sm_103a): the kernels
// and their launch templates. The host side (tensor maps, argument checks, the choice of
// kernel) is gemm_tc.cu; the instantiations are spread over gemm_tc_*.cu so that they
// compile in parallel.
//
// The products of the Newton-Schulz step (Eq. NewtonSchulz: G = X^T X and
// X' = 1.5 X - 0.5 X G) and U^T A for H, with FP32 operands given as P BF16
// planes (x = x_0 + x_1 + x_2). Each k-slice of every plane of both operands is
// staged once in shared memory and all plane-pair passes are issued on it
// (P = 3: hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid), accumulating into one
// FP32 TMEM accumulator, so the split costs tensor-pipe time but not extra
// global or L2 traffic per pass.
//
// The tensor cores add into their FP32 accumulator with round-toward-zero
// (inside one MMA and across MMAs), so a long accumulation drifts toward zero
// by about half an ulp per step. The kernel therefore accumulates each short
// k-slice (64 of K for three planes) into a fresh TMEM buffer, issuing the
// small plane pairs first and hi*hi last in every k-stage (the truncations of
// the small passes happen at 2^-8 of the result's scale), and the epilogue warps
// add every slice into FP32 registers with round-to-nearest ("promotion").
//
// Structure (one CTA per SM, persistent over output tiles of 128 x 256; or CTA pairs, below):
//   warp 0      TMA producer: cp.async.bulk.tensor 3-D loads (columns, rows,
//               planes) into a ring of shared-memory stages, mbarrier tx count
//   warp 1      TMEM allocator and MMA issuer: tcgen05.mma kind::f16 M128 N256
//               K16 into two alternating 256-column slice buffers; commits free
//               the stage and publish the slice
//   warps 2..9  epilogue: two warps per TMEM lane quarter, 128 columns each;
//               tcgen05.ld of every slice, running sums in registers, then the
//               fused output step of the tile:
//                 STORE  C = alpha acc + beta C   (optionally upper triangle)
//                 NS     X_{k+1} = c1 X_k + c3 acc (1.5, -0.5, or the preconditioning
//                        coefficients of Algorithm 1), X_k read from its three
//                        BF16 planes (an exact FP32 encoding), written as planes
//                 CLENSHAW alpha acc + beta Z + diag I on the upper-triangle tiles,
//                        each entry also stored at its mirror position (a product of
//                        two commuting symmetric matrices), Z read from three planes
//                 NS_STEP NS, plus float64 per-warp sums of (X_{k+1} - X_k)^2 and
//                        X_{k+1}^2 (the step size of the inverse iteration)
//                 PLANES the product itself as BF16 planes (an operand of the next product)
//                 GRAM   BF16 planes of G's upper triangle (upper-triangle tiles;
//                        a mirror pass fills the lower one) and float64
//                        partials of ||G - I||_F^2 per tile and warp
// Operands are K-major (stored MN x K, 64-byte swizzle, 32-element k-stages)
// or MN-major (stored K x MN, 128-byte swizzle, 64-element MN chunks); three
// 72 KiB stages for three planes. (16-element stages, six of 36 KiB, keep more
// bytes in flight but measured slower: twice the per-stage barrier work.)
// CTA pairs (cta_group::2, clusters of two CTAs on neighbouring SMs, three planes):
// the pair computes a 256 x 256 tile with M = 256 MMAs issued by one thread of
// the even CTA. Each CTA stages its own 128 rows of A and its own 128 columns of B
// (48 KiB stages instead of 72 KiB), the MMAs read the peer's half of B across the
// pair, and each CTA's TMEM holds its 128 rows of the accumulator. Per SM this
// halves the B operand's shared-memory reads and TMA writes, the limit of the
// single-CTA form (about 90 % of the tensor pipe), and cuts the operand panels
// read from L2 by a third. Both CTAs' copies complete on the even CTA's stage
// barriers; its MMA commits arrive on both CTAs' barriers (multicast); the odd
// CTA's epilogue warps free an accumulator buffer by arriving on the even CTA's
// barrier.
// Every mbarrier wait is bounded (about one second); on expiry the kernel
// records an error flag, lets its copies and MMAs drain, frees TMEM and returns.
#pragma once

#include <cuda.h>
#include <math.h>
#include <stdlib.h>

#include "device_util.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace polar {
namespace {

constexpr int BM = 128, BN = 256, BK = 32;   // two K=16 MMA steps per k-stage
constexpr int NTHREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr uint32_t A_PLANE = BM * BK * 2;  // 8 KiB per plane per stage
constexpr uint32_t B_PLANE = BN * BK * 2;  // 16 KiB (128 x 256 tiles)
// MN-major operands: 64-column chunks of BK rows x 128 bytes (128-byte swizzle)
constexpr uint32_t MN_CHUNK = 64 * BK * 2;
// K-major operands: rows of BK elements (BK * 2 bytes), swizzle of that width, 8-row groups
constexpr uint32_t KM_SBO = 8 * BK * 2;
constexpr uint32_t KM_SWZ = BK == 16 ? 6 : BK == 32 ? 4 : 2;   // descriptor codes: 32, 64, 128-byte swizzle
constexpr uint32_t TMEM_COLS = 512;        // two 128 x 256 FP32 slice accumulators

// Tile width TN: 256 (one epilogue group of eight warps, two 256-column TMEM slice buffers)
// or 128 (two epilogue groups of four warps taking alternate tiles, two 128-column slice
// buffers each, so that one group's output step overlaps the next tile's MMAs).
// CG = 2: CTA pairs; each CTA stages TN / 2 of the tile's B columns. P = FP8 (below): one plane of
// FP8 E4M3 codes, 128-element (128-byte) k-stages, K-major operands only.
constexpr int FP8 = 8;
template <int P, int TN = BN, int CG = 1>
struct Cfg {
  static constexpr int TNL = TN / CG;                     // B columns staged by one CTA
  static constexpr int BKE = P == FP8 ? 128 : BK;         // elements of K per k-stage
  static constexpr int STAGES = P == FP8 ? 4
                              : CG == 2 ? (P == 3 ? 4 : (P == 2 ? 6 : 12))
                              : TN == BN ? (P == 3 ? 6 : (P == 2 ? 9 : 16)) * 16 / BK : (P == 3 ? 4 : (P == 2 ? 6 : 12));
  static constexpr int NBUF = TN == BN ? 2 : 4;          // TMEM slice buffers of TN columns
  static constexpr int GROUP_WARPS = TN == BN ? EPI_WARPS : EPI_WARPS / 2;
  static constexpr uint32_t A_BYTES = P == FP8 ? BM * 128 : P * A_PLANE;
  static constexpr uint32_t B_BYTES = P == FP8 ? TNL * 128 : P * TNL * BK * 2;
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t NBARS = 2 * STAGES + 2 * NBUF + 1;
  static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024 + 8 * NBARS + 16;
};

// Instruction descriptor: D = F32, A = B = BF16, M = m (128, or 256 for a CTA pair), N = tn,
// majors as given.
__host__ __device__ constexpr uint32_t make_idesc(bool a_mn, bool b_mn, int tn = BN, int m = BM) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(tn >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// FP8: D = F32, A = B = E4M3 (format code 0), both K-major, M = 128, N = tn.
__host__ __device__ constexpr uint32_t make_idesc_f8(int tn = BN) {
  return (1u << 4) | ((uint32_t)(tn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Plane pairs of the split product in issue order for `np` planes: the smallest
// terms first, hi*hi last (6 passes: (1,1) (0,2) (2,0) (0,1) (1,0) (0,0)).
__host__ __device__ constexpr int pass_a(int np, int i) {
  return ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 0 ? 1
       : ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 2 ? 2
       : ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 4 ? 1 : 0;
}
__host__ __device__ constexpr int pass_b(int np, int i) {
  return ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 0 ? 1
       : ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 1 ? 2
       : ((np == 1 ? 5 : np == 2 ? 3 : 0) + i) == 3 ? 1 : 0;
}

__host__ __device__ __forceinline__ int passes_for(int planes) { return planes == 1 ? 1 : (planes == 2 ? 3 : 6); }

// ---------------------------------------------------------------- tile schedule

__host__ __device__ __forceinline__ int64_t tri_tiles(int64_t tm, int64_t tn) {
  // column bj of 256 holds row-tiles bi <= 2 bj + 1 (rows of 128), clipped to tm
  return (tn - 1) * tn + ((2 * tn) < tm ? 2 * tn : tm);
}

__device__ __forceinline__ void tile_coords(int64_t t, int64_t tm, int64_t tn, bool tri, int64_t& bi, int64_t& bj) {
  if (tri) {
    int64_t j = (int64_t)((sqrt(4.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (j > 0 && j * (j + 1) > t) --j;
    while ((j + 1) * (j + 2) <= t) ++j;
    bj = j;
    bi = t - j * (j + 1);
  } else {
    const int64_t G = 16;
    int64_t group = t / (G * tn);
    int64_t first = group * G;
    int64_t rows = (tm - first) < G ? (tm - first) : G;
    int64_t in = t % (G * tn);
    bi = first + in % rows;
    bj = in / rows;
  }
}

// Pair tiles of 256 x 256: rectangular ones rastered in groups of 8 tile rows (2048 rows, as the
// single-CTA groups of 16 x 128); triangular ones (bi2 <= bj) column by column.
__host__ __device__ __forceinline__ int64_t pair_tri_tiles(int64_t t) { return t * (t + 1) / 2; }

__device__ __forceinline__ void pair_tile_coords(int64_t t, int64_t tm2, int64_t tn, bool tri, int64_t& bi2,
                                                 int64_t& bj) {
  if (tri) {
    int64_t j = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (j > 0 && j * (j + 1) / 2 > t) --j;
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    bj = j;
    bi2 = t - j * (j + 1) / 2;
  } else {
    const int64_t G = 8;
    int64_t group = t / (G * tn);
    int64_t first = group * G;
    int64_t rows = (tm2 - first) < G ? (tm2 - first) : G;
    int64_t in = t % (G * tn);
    bi2 = first + in % rows;
    bj = in / rows;
  }
}

// ---------------------------------------------------------------- epilogue pieces

// Three BF16 planes of two values at once: each plane is the round-to-nearest-even
// BF16 of what the previous planes left (cvt.rn.bf16x2.f32 packs b into the low
// half and a into the high half, so element 0 lands at the lower address).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t (&w)[3]) {
  float r0 = x0, r1 = x1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(r1), "f"(r0));
    w[q] = h;
    r0 = r0 - __uint_as_float(h << 16);
    r1 = r1 - __uint_as_float(h & 0xffff0000u);
  }
}

// The three-plane split of 32 consecutive values (np planes, 64 bytes each, 16-byte stores) and also the
// mirrored entries: value j goes to row (c0 + j),
// column r of every plane (lanes hold consecutive r, so each store is 64 contiguous bytes).
__device__ __forceinline__ void store_planes32_mirror(uint16_t* base, uint16_t* tbase, int64_t ld, int64_t pstride,
                                                      int np, const float* x) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    uint32_t w[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t t[3];
      split2(x[8 * v + 2 * i], x[8 * v + 2 * i + 1], t);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        w[q][i] = t[q];
        if (q < np) {
          tbase[q * pstride + (int64_t)(8 * v + 2 * i) * ld] = (uint16_t)(t[q] & 0xffffu);
          tbase[q * pstride + (int64_t)(8 * v + 2 * i + 1) * ld] = (uint16_t)(t[q] >> 16);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q < np) reinterpret_cast<uint4*>(base + q * pstride)[v] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
}

// 4 x 4 transpose of 32-bit words across the four lanes of an aligned lane quad (lane c = lane & 3):
// lane c holds x[j] = M[c][j] before and x[i] = M[i][c] after (two exchange rounds).
__device__ __forceinline__ void quad_transpose(uint32_t (&x)[4], int c) {
  {
    const bool hi = (c & 2) != 0;
    const uint32_t s0 = hi ? x[0] : x[2], s1 = hi ? x[1] : x[3];
    const uint32_t r0 = __shfl_xor_sync(0xffffffffu, s0, 2), r1 = __shfl_xor_sync(0xffffffffu, s1, 2);
    if (hi) { x[0] = r0; x[1] = r1; } else { x[2] = r0; x[3] = r1; }
  }
  {
    const bool odd = (c & 1) != 0;
    const uint32_t s0 = odd ? x[0] : x[1], s1 = odd ? x[2] : x[3];
    const uint32_t r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
    if (odd) { x[0] = r0; x[2] = r1; } else { x[1] = r0; x[3] = r1; }
  }
}

// The three-plane split of 32 consecutive values with the lanes' rows exchanged first: each lane holds 32 values of its own row;
// a lane quad (lanes 4g..4g+3) transposes its 16-byte quads so that store i of lane 4g + c writes
// quad c of row 4g + i. Every store instruction then covers 8 rows x 64 contiguous bytes instead of
// 32 rows x 16 bytes. base: plane 0 at row 4g (of the lane's quad), column c0 + 8c; mask bit i:
// row 4g + i may be written. Every lane of the warp must call it (the exchange is warp-wide); the
// values are split in place (x is left holding the last remainders). Each plane is the
// round-to-nearest-even BF16 of what the previous planes left (cvt.rn.bf16x2.f32).
__device__ __forceinline__ void store_planes32_t(uint16_t* base, int64_t ld, int64_t pstride, int np, float* x,
                                                 int c, unsigned mask) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q >= np) break;
    uint32_t w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint32_t h;
      asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x[2 * k + 1]), "f"(x[2 * k]));
      w[k] = h;
      x[2 * k] = x[2 * k] - __uint_as_float(h << 16);
      x[2 * k + 1] = x[2 * k + 1] - __uint_as_float(h & 0xffff0000u);
    }
    uint32_t o[4][4];   // o[i][wp]: word wp of quad c of row 4g + i
#pragma unroll
    for (int wp = 0; wp < 4; ++wp) {
      uint32_t y[4] = {w[wp], w[4 + wp], w[8 + wp], w[12 + wp]};
      quad_transpose(y, c);
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i][wp] = y[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (mask & (1u << i))
        *reinterpret_cast<uint4*>(base + q * pstride + i * ld) = make_uint4(o[i][0], o[i][1], o[i][2], o[i][3]);
  }
}

__device__ __forceinline__ void store_planes1(uint16_t* base, int64_t pstride, int np, float x) {
  uint32_t t[3];
  split2(x, 0.0f, t);
  for (int q = 0; q < np; ++q) base[q * pstride] = (uint16_t)(t[q] & 0xffffu);
}

// ---------------------------------------------------------------- the kernel
//
// The three roles are separate non-inlined functions so that the register
// pressure of the epilogue (128 running sums per thread) does not make the
// single-thread producer and MMA loops spill: a spilled loop variable reloaded
// from local memory (which mostly misses the small L1 left beside the stages)
// stalls the thread that feeds the tensor pipe.

struct Bars {
  uint32_t full0, empty0, tfull0, tempty0, drain;  // shared addresses; stage s at + 8 s
};

// What one output tile needs: its operand maps, origin, K-stage count, the
// epilogue arguments of its problem and the index of its residual partials.
struct TileCtx {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  int64_t bi, bj, nk;
  const TcArgs* args;
  int64_t part;  // partials slot base: tile index within its problem x EPI_WARPS
  int sl;        // k-stages per promoted slice for this tile (its problem's, else the launch's)
};

// One problem: tiles enumerated by tile_coords (CG = 1), or pair tiles by pair_tile_coords, each CTA
// of the pair taking its 128 rows (CG = 2). Tiles t0, t0 + dt, ... belong to this CTA (or pair).
template <int CG>
struct SingleSrc {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  const TcArgs* args;
  int64_t tm, tn, ntiles, nk;   // CG = 2: tm counts 256-row blocks
  int64_t t0, dt;
  uint32_t rank;                // CG = 2: this CTA's rank in its pair
  bool tri;
  __device__ __forceinline__ bool get(int64_t t, TileCtx& c) const {
    if (CG == 2) {
      int64_t bi2;
      pair_tile_coords(t, tm, tn, tri, bi2, c.bj);
      c.bi = 2 * bi2 + rank;
      c.part = (2 * t + rank) * EPI_WARPS;
    } else {
      tile_coords(t, tm, tn, tri, c.bi, c.bj);
      c.part = t * EPI_WARPS;
    }
    c.ma = ma;
    c.mb = mb;
    c.nk = nk;
    c.args = args;
    c.sl = args->slice_stages > 0 ? args->slice_stages : 1;
    if (args->a_uni) {
      // FP8: a tile whose A block and B blocks each keep one exponent along K has one scale per
      // epilogue half, so its K blocks accumulate fp8_run at a time before the promotion
      const int64_t nb = (args->N + 127) / 128, j0 = c.bj * (BN / 128);
      bool u = args->a_uni[c.bi] != 0;
#pragma unroll
      for (int h = 0; h < BN / 128; ++h)
        if (j0 + h < nb) u = u && args->b_uni[j0 + h] != 0;
      if (u) c.sl = args->fp8_run;
    }
    return true;
  }
};

// Many problems: tiles from a table; tiles of stopped problems are skipped (every
// role reads the same status, which no launch-concurrent code changes).
struct GroupSrc {
  const TcTile* tiles;
  const TcGroupEntry* entries;
  int64_t ntiles;
  int64_t t0, dt;
  int sl_default;   // slice length of problems whose entry leaves it 0
  __device__ __forceinline__ bool get(int64_t t, TileCtx& c) const {
    const TcTile d = tiles[t];
    const TcGroupEntry* e = entries + d.prob;
    if (e->args.st && e->args.st->status != ST_RUNNING) return false;
    c.ma = reinterpret_cast<const CUtensorMap*>(e->map_a);
    c.mb = reinterpret_cast<const CUtensorMap*>(e->map_b);
    c.bi = d.bi;
    c.bj = d.bj;
    c.nk = (e->args.K + BK - 1) / BK;
    c.args = &e->args;
    c.sl = e->args.slice_stages > 0 ? e->args.slice_stages : sl_default;
    c.part = (int64_t)d.local * EPI_WARPS;
    return true;
  }
};

template <int P, bool A_MN, bool B_MN, int TN, int CG, class Src>
__device__ __noinline__ void role_producer(const Src& src, uint32_t smem_base, Bars br, volatile int* abort_flag,
                                           int withhold) {
  using C = Cfg<P, TN, CG>;
  constexpr int S = C::STAGES;
  if (withhold) return;  // test hook: no copies are issued, the consumers' bounded waits expire
  // CTA pairs: both CTAs' copies of a stage complete on the even CTA's barrier, which the even
  // CTA arms for both; the odd CTA stages the tile's second 128 columns of B
  const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
  const bool arms = rank == 0;
  int stage = 0;
  uint32_t phase = 0;
  uint32_t armed = 0, armed_phase = 0;  // bit s: stage s was armed / the parity it was armed with
  bool ok = true;
  const CUtensorMap* last_a = nullptr;
  for (int64_t t = src.t0; t < src.ntiles && ok; t += src.dt) {
    TileCtx c;
    if (!src.get(t, c)) continue;
    if (c.ma != last_a) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(c.ma)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(c.mb)) : "memory");
      last_a = c.ma;
    }
    const int m0 = (int)(c.bi * BM), n0 = (int)(c.bj * TN + rank * C::TNL);
    for (int64_t kb = 0; kb < c.nk; ++kb) {
      if (!mbar_wait(br.empty0 + 8 * stage, phase ^ 1u, abort_flag)) { ok = false; break; }
      const uint32_t fb = br.full0 + 8 * stage;
      if (arms) {
        mbar_expect_tx(fb, CG * C::STAGE_BYTES);
        armed |= 1u << stage;
        armed_phase = (armed_phase & ~(1u << stage)) | (phase << stage);
      }
      const uint32_t fbx = CG == 2 ? mapa_shared(fb, 0) : fb;   // the barrier the copies complete on
      const uint32_t a_dst = smem_base + stage * C::STAGE_BYTES;
      const uint32_t b_dst = a_dst + C::A_BYTES;
      const int k0 = (int)(kb * C::BKE);
      if (A_MN) {
#pragma unroll
        for (int cc = 0; cc < BM / 64; ++cc) {
          if (CG == 2) tma_load_3d_pair(a_dst + cc * P * MN_CHUNK, c.ma, fbx, m0 + 64 * cc, k0, 0);
          else tma_load_3d(a_dst + cc * P * MN_CHUNK, c.ma, fb, m0 + 64 * cc, k0, 0);
        }
      } else {
        if (CG == 2) tma_load_3d_pair(a_dst, c.ma, fbx, k0, m0, 0);
        else tma_load_3d(a_dst, c.ma, fb, k0, m0, 0);
      }
      if (B_MN) {
#pragma unroll
        for (int cc = 0; cc < C::TNL / 64; ++cc) {
          if (CG == 2) tma_load_3d_pair(b_dst + cc * P * MN_CHUNK, c.mb, fbx, n0 + 64 * cc, k0, 0);
          else tma_load_3d(b_dst + cc * P * MN_CHUNK, c.mb, fb, n0 + 64 * cc, k0, 0);
        }
      } else {
        if (CG == 2) tma_load_3d_pair(b_dst, c.mb, fbx, k0, n0, 0);
        else tma_load_3d(b_dst, c.mb, fb, k0, n0, 0);
      }
      if (++stage == S) { stage = 0; phase ^= 1u; }
    }
  }
  // every copy this thread started lands before the CTA can exit (a pair's odd CTA: its copies
  // complete on the even CTA's barriers, which the even CTA drains before the pair's exit barrier)
  for (int s2 = 0; s2 < S; ++s2)
    if (armed & (1u << s2)) mbar_drain(br.full0 + 8 * s2, (armed_phase >> s2) & 1u);
}

// The NP-plane passes on one k-stage: descriptors are the stage-0 bases plus
// compile-time offsets (the start-address field is the low 14 bits, address / 16).
// FP8: the stage's 128 K-elements as four K = 32 MMAs on E4M3 codes (32 bytes of every row each).
template <int TN>
__device__ __forceinline__ void issue_stage_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t first_acc) {
  constexpr uint32_t idesc = make_idesc_f8(TN);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk)
    tc_mma_f8(d_tmem, a_desc + ((kk * 32) >> 4), b_desc + ((kk * 32) >> 4), idesc, kk == 0 ? first_acc : 1u);
}

template <int P, bool A_MN, bool B_MN, int NP, int TN = BN, int CG = 1>
__device__ __forceinline__ void issue_stage(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t first_acc) {
  constexpr uint32_t idesc = make_idesc(A_MN, B_MN, TN, BM * CG);
  constexpr uint32_t B_PL = (TN / CG) * BK * 2;
#pragma unroll
  for (int ps = 0; ps < passes_for(NP); ++ps) {
#pragma unroll
    for (int kk = 0; kk < BK / 16; ++kk) {
      const uint32_t aoff = A_MN ? pass_a(NP, ps) * MN_CHUNK + kk * 2048 : pass_a(NP, ps) * A_PLANE + kk * 32;
      const uint32_t boff = B_MN ? pass_b(NP, ps) * MN_CHUNK + kk * 2048 : pass_b(NP, ps) * B_PL + kk * 32;
      const uint32_t acc = (ps == 0 && kk == 0) ? first_acc : 1u;
      if (CG == 2) tc_mma_pair(d_tmem, a_desc + (aoff >> 4), b_desc + (boff >> 4), idesc, acc);
      else tc_mma(d_tmem, a_desc + (aoff >> 4), b_desc + (boff >> 4), idesc, acc);
    }
  }
}

template <int P, bool A_MN, bool B_MN, int TN, int CG, class Src>
__device__ __noinline__ void role_mma(const Src& src, uint32_t smem_base, uint32_t tmem_base, Bars br,
                                      volatile int* abort_flag, int pu) {
  using C = Cfg<P, TN, CG>;
  constexpr int S = C::STAGES;
  // FP8 operands: K-major rows of 128 bytes, 128-byte swizzle, 8-row groups of 1024 bytes
  const uint64_t a_desc0 = P == FP8 ? smem_desc(smem_base, 16, 1024, 2)
                         : A_MN ? smem_desc(smem_base, P * MN_CHUNK, 1024, 2)
                                : smem_desc(smem_base, 16, KM_SBO, KM_SWZ);
  const uint64_t b_desc0 = P == FP8 ? smem_desc(smem_base + C::A_BYTES, 16, 1024, 2)
                         : B_MN ? smem_desc(smem_base + C::A_BYTES, P * MN_CHUNK, 1024, 2)
                                : smem_desc(smem_base + C::A_BYTES, 16, KM_SBO, KM_SWZ);
  int stage = 0;
  uint32_t phase = 0;
  // slice buffers: one pair for TN = 256; with TN = 128 a pair per epilogue group, the groups
  // taking alternate tiles (each pair keeps its own position and phase)
  int gbuf[2] = {0, 0};
  uint32_t gphase[2] = {0u, 0u};
  int64_t ntile = 0;
  bool ok = true;
  for (int64_t t = src.t0; t < src.ntiles && ok; t += src.dt) {
    TileCtx c;
    if (!src.get(t, c)) continue;
    const int grp = TN == BN ? 0 : (int)(ntile++ & 1);
    int& buf = gbuf[grp];
    uint32_t& buf_phase = gphase[grp];
    int kin = 0;  // k-stage index within the current slice
    for (int64_t kb = 0; kb < c.nk; ++kb) {
      // c.sl k-stages into a fresh slice buffer, then published to the epilogue
      const bool slice_start = kin == 0;
      const bool slice_end = kin == c.sl - 1 || kb == c.nk - 1;
      const int bslot = 2 * grp + buf;
      if (slice_start && !mbar_wait(br.tempty0 + 8 * bslot, buf_phase ^ 1u, abort_flag)) { ok = false; break; }
      if (!mbar_wait(br.full0 + 8 * stage, phase, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(bslot * TN);
      const uint64_t soff = (uint64_t)((stage * C::STAGE_BYTES) >> 4);
      const uint32_t first_acc = slice_start ? 0u : 1u;
      if constexpr (P == FP8) {
        issue_stage_f8<TN>(d_tmem, a_desc0 + soff, b_desc0 + soff, first_acc);
      } else {
        if (pu == P) issue_stage<P, A_MN, B_MN, P, TN, CG>(d_tmem, a_desc0 + soff, b_desc0 + soff, first_acc);
        else if (pu == 2)
          issue_stage<P, A_MN, B_MN, (P >= 2 ? 2 : P), TN, CG>(d_tmem, a_desc0 + soff, b_desc0 + soff, first_acc);
        else issue_stage<P, A_MN, B_MN, 1, TN, CG>(d_tmem, a_desc0 + soff, b_desc0 + soff, first_acc);
      }
      // the stage is free in both CTAs of a pair, the slice is ready in both CTAs' TMEM
      if (CG == 2) tc_commit_pair(br.empty0 + 8 * stage, 3);
      else tc_commit(br.empty0 + 8 * stage);
      if (slice_end) {
        if (CG == 2) tc_commit_pair(br.tfull0 + 8 * bslot, 3);
        else tc_commit(br.tfull0 + 8 * bslot);
        if (++buf == 2) { buf = 0; buf_phase ^= 1u; }
        kin = 0;
      } else {
        ++kin;
      }
      if (++stage == S) { stage = 0; phase ^= 1u; }
    }
  }
  // every MMA issued so far completes before TMEM is released
  if (CG == 2) tc_commit_pair(br.drain, 1);
  else tc_commit(br.drain);
  mbar_drain(br.drain, 0);
}

template <int EPI, int TN, int CG, class Src>
__device__ __noinline__ void role_epilogue(const Src& src, uint32_t tmem_base, Bars br, volatile int* abort_flag,
                                           int warp, int lane) {
  const int q = warp & 3;                              // TMEM lane quarter this warp may access
  const int half = TN == BN ? (warp - 2) >> 2 : 0;     // TN = 256: which 128 of the tile's columns
  const int grp = TN == BN ? 0 : (warp - 2) >> 2;      // TN = 128: the group (alternate tiles)
  const int gw = TN == BN ? warp - 2 : (warp - 2) & 3; // this warp's partials slot within the tile
  const int row_in_tile = q * 32 + lane;
  const uint32_t t_lane = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 128);
  int buf = 0;
  uint32_t buf_phase = 0;
  int64_t ntile = 0;
  for (int64_t t = src.t0; t < src.ntiles; t += src.dt) {
    TileCtx ctx;
    if (!src.get(t, ctx)) continue;
    if (TN != BN && (int)(ntile++ & 1) != grp) continue;   // the other group's tile
    const TcArgs& p = *ctx.args;
    const int64_t nslices = (ctx.nk + ctx.sl - 1) / ctx.sl;
    constexpr bool NS = EPI == TC_EPI_NS || EPI == TC_EPI_NS_STEP;
    constexpr bool STEP = EPI == TC_EPI_NS_STEP;
    constexpr bool CLEN = EPI == TC_EPI_CLENSHAW;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
    int e_sum = 0;
    bool ok = true;
    for (int64_t sl = 0; sl < nslices; ++sl) {
      const int bslot = 2 * grp + buf;
      if (!mbar_wait(br.tfull0 + 8 * bslot, buf_phase, abort_flag)) { ok = false; break; }
      tc_fence_after();
      if (p.a_exp) {
        // FP8 operands: the slice is one 128-K block, scaled by its tiles' powers of two (exact), or,
        // in a tile whose blocks keep one exponent along K, several blocks under that one scale. Lane
        // l holds the exponent sum of slice 32 j + l, fetched once per 32 slices; a half tile past N
        // has no exponent (its columns are not stored).
        if ((sl & 31) == 0) {
          const int64_t bcol = ctx.bj * (TN / 128) + half, s2 = ctx.sl > 1 ? 0 : sl + lane;
          e_sum = (s2 < nslices && bcol * 128 < p.N)
                      ? (int)p.a_exp[ctx.bi * p.lde_a + s2] + (int)p.b_exp[bcol * p.lde_b + s2]
                      : 0;
        }
        const float sc = ldexpf(1.0f, __shfl_sync(0xffffffffu, e_sum, (int)(sl & 31)));
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float v[16];
          tmem_ld16(t_lane + (uint32_t)(bslot * TN + c * 16), v);
          fma16_packed(&acc[c * 16], v, sc);   // round-to-nearest promotion of the scaled slice
        }
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float v[16];
          tmem_ld16(t_lane + (uint32_t)(bslot * TN + c * 16), v);
          add16_packed(&acc[c * 16], v);   // round-to-nearest promotion
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        // a pair's buffer is free once both CTAs' epilogue warps have read it: they arrive on the
        // even CTA's barrier, whose MMA thread reuses the buffer
        if (CG == 2) mbar_arrive_cluster(mapa_shared(br.tempty0 + 8 * bslot, 0));
        else mbar_arrive(br.tempty0 + 8 * bslot);
      }
      if (++buf == 2) { buf = 0; buf_phase ^= 1u; }
      if ((NS || CLEN) && sl == (nslices > 1 ? nslices - 2 : 0)) {
        // the output step reads this row's 128 columns of X_k's (or Z's) three planes: pull them into L2 now
        const int64_t r = ctx.bi * BM + row_in_tile;
        const int64_t c0 = ctx.bj * TN + half * 128;
        if (r < p.M && c0 < p.N) {
          const uint16_t* xr = p.x_planes + r * p.ldxp + c0;
#pragma unroll
          for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int l = 0; l < 2; ++l)
              asm volatile("prefetch.global.L2 [%0];" ::"l"(xr + q * p.x_plane_stride + 64 * l));
        }
      }
    }
    if (!ok) return;
    const bool tri = p.triangular != 0;
    // update coefficients of this step (1.5, -0.5 for Newton-Schulz; a, -4/27 a^3 while preconditioning)
    const float c1 = (NS && p.st) ? p.st->upd_c1 : 1.5f;
    const float c3 = (NS && p.st) ? p.st->upd_c3 : -0.5f;
    const int64_t r = ctx.bi * BM + row_in_tile;
    const bool row_ok = r < p.M;
    const int lq = lane & 3;                      // this lane's place in its quad (store_planes32_t)
    const int64_t r4 = r - lq;                    // the quad's first row
    double part = 0.0;
    float d2 = 0.f, x2 = 0.f;  // NS_STEP: sum (x' - x)^2 and sum x'^2 over this thread's row chunk
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t c0 = ctx.bj * TN + half * 128 + c * 32;
      float* v = &acc[c * 32];
      if (c0 >= p.N) continue;                    // the same for every lane of the warp
      const bool full_chunk = c0 + 32 <= p.N;
      // rows of this lane's quad that exist (store_planes32_t writes rows r4 .. r4 + 3)
      unsigned rows4 = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) rows4 |= (r4 + i < p.M) ? (1u << i) : 0u;
      if (NS) {
        // X_{k+1} = c1 X_k + c3 X_k G: X_k from its three planes (exact), result as planes. A chunk
        // that ends past column N still moves whole 32-value rows when the pitch holds them: the
        // columns from N to the pitch are zero in X_k (the library zeroes its plane buffers and
        // never writes a non-zero there), the product is zero there (the operand maps stop at N),
        // so the padding stays zero and no element-by-element path is needed.
        const uint16_t* xr = p.x_planes + r * p.ldxp + c0;
        uint16_t* pr = p.out_planes + r * p.ldo + c0;
        if (full_chunk || (c0 + 32 <= p.ldxp && c0 + 32 <= p.ldo)) {
          // every lane takes part (rows past M read zeros and are not stored)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            uint4 h = make_uint4(0u, 0u, 0u, 0u), m = h, l = h;
            if (row_ok) {
              h = *reinterpret_cast<const uint4*>(xr + 8 * i);
              m = *reinterpret_cast<const uint4*>(xr + p.x_plane_stride + 8 * i);
              l = *reinterpret_cast<const uint4*>(xr + 2 * p.x_plane_stride + 8 * i);
            }
            const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, mw[4] = {m.x, m.y, m.z, m.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int w = e >> 1, sh = (e & 1) * 16;
              const float x = (bf16_to_f32_dev((uint16_t)(hw[w] >> sh)) + bf16_to_f32_dev((uint16_t)(mw[w] >> sh))) +
                              bf16_to_f32_dev((uint16_t)(lw[w] >> sh));
              const float xn = c1 * x + c3 * v[8 * i + e];
              if (STEP) {
                d2 = fmaf(xn - x, xn - x, d2);
                x2 = fmaf(xn, xn, x2);
              }
              v[8 * i + e] = xn;
            }
          }
          store_planes32_t(p.out_planes + r4 * p.ldo + c0 + 8 * lq, p.ldo, p.out_plane_stride, p.out_nplanes, v, lq,
                           rows4);
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (c0 + j < p.N) {
              const float x = (bf16_to_f32_dev(xr[j]) + bf16_to_f32_dev(xr[p.x_plane_stride + j])) +
                              bf16_to_f32_dev(xr[2 * p.x_plane_stride + j]);
              const float xn = c1 * x + c3 * v[j];
              if (STEP) {
                d2 = fmaf(xn - x, xn - x, d2);
                x2 = fmaf(xn, xn, x2);
              }
              store_planes1(pr + j, p.out_plane_stride, p.out_nplanes, xn);
            }
          }
        }
      } else if (EPI == TC_EPI_GRAM) {
        // planes of G for the chunks that reach the diagonal or lie above it, as whole 32-value rows;
        // the strictly lower triangle is written afterwards by the mirror pass from the upper one
        // (launch_mirror_planes3, or the batched solves' own), which also overwrites what a chunk
        // crossing the diagonal stores below it. Columns past N hold zeros (the operand maps stop at N)
        // and land in the pitch's padding, which no operand map reads.
        uint16_t* pr = p.out_planes + r * p.ldo + c0;
        float s_off = 0.f, s_diag = 0.f;
        if (!row_ok || c0 + 31 < r) {
          // a row past M, or a chunk entirely below the diagonal: no terms
        } else if (r < c0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) s_off = fmaf(v[j], v[j], s_off);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t cc = c0 + j;
            if (cc == r) {
              float d = v[j] - 1.0f;
              s_diag = fmaf(d, d, s_diag);
            } else if (cc > r && cc < p.N) {
              s_off = fmaf(v[j], v[j], s_off);
            }
          }
        }
        if (c0 + 32 <= p.ldo) {
          // rows of the quad whose chunk reaches the diagonal or lies above it
          unsigned upper4 = 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) upper4 |= (c0 + 31 >= r4 + i) ? (1u << i) : 0u;
          store_planes32_t(p.out_planes + r4 * p.ldo + c0 + 8 * lq, p.ldo, p.out_plane_stride, p.out_nplanes, v, lq,
                           rows4 & upper4);
        } else if (row_ok && c0 + 31 >= r) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < p.N) store_planes1(pr + j, p.out_plane_stride, p.out_nplanes, v[j]);
        }
        part += 2.0 * (double)s_off + (double)s_diag;
      } else if (CLEN) {
        if (!row_ok) continue;
        // Clenshaw step on the upper triangle, mirrored: alpha acc + beta Z + diag I, Z from its three planes
        const uint16_t* zr = p.x_planes + r * p.ldxp + c0;
        uint16_t* pr = p.out_planes + r * p.ldo + c0;
        uint16_t* pt = p.out_planes + c0 * p.ldo + r;
        if (full_chunk && r < c0) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            uint4 h = *reinterpret_cast<const uint4*>(zr + 8 * i);
            uint4 m = *reinterpret_cast<const uint4*>(zr + p.x_plane_stride + 8 * i);
            uint4 l = *reinterpret_cast<const uint4*>(zr + 2 * p.x_plane_stride + 8 * i);
            const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, mw[4] = {m.x, m.y, m.z, m.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int w = e >> 1, sh = (e & 1) * 16;
              const float z = (bf16_to_f32_dev((uint16_t)(hw[w] >> sh)) + bf16_to_f32_dev((uint16_t)(mw[w] >> sh))) +
                              bf16_to_f32_dev((uint16_t)(lw[w] >> sh));
              v[8 * i + e] = fmaf(p.alpha, v[8 * i + e], p.beta * z);
            }
          }
          store_planes32_mirror(pr, pt, p.ldo, p.out_plane_stride, p.out_nplanes, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t cc = c0 + j;
            if (cc < p.N && r <= cc) {
              const float z = (bf16_to_f32_dev(zr[j]) + bf16_to_f32_dev(zr[p.x_plane_stride + j])) +
                              bf16_to_f32_dev(zr[2 * p.x_plane_stride + j]);
              float o = fmaf(p.alpha, v[j], p.beta * z);
              if (r == cc) o += p.diag;
              else store_planes1(pt + j * p.ldo, p.out_plane_stride, p.out_nplanes, o);
              store_planes1(pr + j, p.out_plane_stride, p.out_nplanes, o);
            }
          }
        }
      } else if (EPI == TC_EPI_PLANES) {
        // the product itself as three BF16 planes (an operand of the next product); columns past N
        // hold zeros (the operand maps stop at N) and land in the pitch's padding
        uint16_t* pr = p.out_planes + r * p.ldo + c0;
        if (c0 + 32 <= p.ldo) {
          store_planes32_t(p.out_planes + r4 * p.ldo + c0 + 8 * lq, p.ldo, p.out_plane_stride, p.out_nplanes, v, lq,
                           rows4);
        } else if (row_ok) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < p.N) store_planes1(pr + j, p.out_plane_stride, p.out_nplanes, v[j]);
        }
      } else {  // STORE
        if (!row_ok) continue;
        float* cr = p.C + r * p.ldc + c0;
        if (full_chunk && !(tri && r > c0) && (reinterpret_cast<uintptr_t>(cr) & 15u) == 0) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float4 o = make_float4(p.alpha * v[4 * i], p.alpha * v[4 * i + 1], p.alpha * v[4 * i + 2],
                                   p.alpha * v[4 * i + 3]);
            if (p.beta != 0.0f) {
              const float4 c = reinterpret_cast<const float4*>(cr)[i];
              o = make_float4(fmaf(p.beta, c.x, o.x), fmaf(p.beta, c.y, o.y), fmaf(p.beta, c.z, o.z),
                              fmaf(p.beta, c.w, o.w));
            }
            reinterpret_cast<float4*>(cr)[i] = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (c0 + j < p.N && !(tri && r > c0 + j)) {
              float o = p.alpha * v[j];
              if (p.beta != 0.0f) o = fmaf(p.beta, cr[j], o);
              cr[j] = o;
            }
          }
        }
      }
    }
    if (EPI == TC_EPI_GRAM) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      if (lane == 0) {
        p.partials[ctx.part + gw] = part;
        if (TN != BN) p.partials[ctx.part + 4 + gw] = 0.0;   // a 128-wide tile fills four of its eight slots
      }
    }
    if (STEP) {
      double a = d2, b = x2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        p.partials[2 * (ctx.part + gw)] = a;
        p.partials[2 * (ctx.part + gw) + 1] = b;
        if (TN != BN) {
          p.partials[2 * (ctx.part + 4 + gw)] = 0.0;
          p.partials[2 * (ctx.part + 4 + gw) + 1] = 0.0;
        }
      }
    }
  }
}

// Shared prologue/epilogue of both launch forms; `Src` supplies the tiles.
template <int P, bool A_MN, bool B_MN, int EPI, int TN, int CG, class Src>
__device__ __forceinline__ void tc_body(const Src& src, DevState* st, int* err_word, unsigned int* err_out,
                                        const int* planes_dyn, int withhold) {
  using C = Cfg<P, TN, CG>;
  constexpr int S = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * C::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + C::NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t smem_base = smem_u32(smem);
  Bars br;
  br.full0 = smem_u32(&bars[0]);
  br.empty0 = smem_u32(&bars[S]);
  br.tfull0 = smem_u32(&bars[2 * S]);
  br.tempty0 = smem_u32(&bars[2 * S + C::NBUF]);
  br.drain = smem_u32(&bars[2 * S + 2 * C::NBUF]);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(br.full0 + 8 * s, 1);
      mbar_init(br.empty0 + 8 * s, 1);
    }
    for (int a = 0; a < C::NBUF; ++a) {
      mbar_init(br.tfull0 + 8 * a, 1);
      mbar_init(br.tempty0 + 8 * a, C::GROUP_WARPS * CG);   // a pair: both CTAs' epilogue warps
    }
    mbar_init(br.drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    // a pair allocates collectively: one warp of each CTA, the same columns in both
    if (CG == 2) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (CG == 2) cluster_sync_all();   // the peer's barriers are initialised before any copy or arrive
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) role_producer<P, A_MN, B_MN, TN, CG>(src, smem_base, br, abort_flag, withhold);
  } else if (warp == 1) {
    if (lane == 0 && (CG == 1 || cluster_rank() == 0)) {   // a pair's MMAs come from its even CTA
      const int pu = planes_dyn ? min(max(*planes_dyn, 1), P) : P;
      role_mma<P, A_MN, B_MN, TN, CG>(src, smem_base, tmem_base, br, abort_flag, pu);
    }
  } else {
    role_epilogue<EPI, TN, CG>(src, tmem_base, br, abort_flag, warp, lane);
  }

  tc_fence_before();
  __syncthreads();
  // a pair: neither CTA leaves (or frees TMEM) while the other's MMAs, copies or arrives may still
  // touch its shared memory or TMEM
  if (CG == 2) cluster_sync_all();
  if (*abort_flag && threadIdx.x == 0 && err_word) atomicOr(err_word, 1);
  if (*abort_flag && threadIdx.x == 0) {
    if (st) {
      atomicOr(&st->err_flags, 1u);
      st->status = ST_TIMEOUT;  // later launches of this solve return at once
    } else if (err_out) {
      atomicOr(err_out, 1u);   // the launch's error word (the host passes the device-wide one by default)
    }
  }
  if (warp == 1) {
    tc_fence_after();
    if (CG == 2)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
  }
}

template <int P, bool A_MN, bool B_MN, int EPI>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ TcArgs p, int64_t tm, int64_t tn, int64_t ntiles) {
  if (p.st && p.st->status != ST_RUNNING) return;
  if (p.planes_dyn && *p.planes_dyn <= 0) return;   // a schedule's launch for a phase that is not current
  SingleSrc<1> src;
  src.ma = &tmA;
  src.mb = &tmB;
  src.args = &p;
  src.tm = tm;
  src.tn = tn;
  src.ntiles = ntiles;
  src.nk = (p.K + Cfg<P>::BKE - 1) / Cfg<P>::BKE;
  src.t0 = blockIdx.x;
  src.dt = gridDim.x;
  src.rank = 0;
  src.tri = p.triangular != 0;
  tc_body<P, A_MN, B_MN, EPI, BN, 1>(src, p.st, nullptr, p.err_out, p.planes_dyn, p.withhold_tma);
}

// CTA pairs: clusters of two; pair tiles t0 = cluster index, dt = number of clusters. Both CTAs read
// the same state words, so both return early or neither does.
template <int P, bool A_MN, bool B_MN, int EPI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ TcArgs p, int64_t tm2, int64_t tn, int64_t ntiles) {
  if (p.st && p.st->status != ST_RUNNING) return;
  if (p.planes_dyn && *p.planes_dyn <= 0) return;
  SingleSrc<2> src;
  src.ma = &tmA;
  src.mb = &tmB;
  src.args = &p;
  src.tm = tm2;
  src.tn = tn;
  src.ntiles = ntiles;
  src.nk = (p.K + BK - 1) / BK;
  src.t0 = blockIdx.x / 2;
  src.dt = gridDim.x / 2;
  src.rank = cluster_rank();
  src.tri = p.triangular != 0;
  tc_body<P, A_MN, B_MN, EPI, BN, 2>(src, p.st, nullptr, p.err_out, p.planes_dyn, p.withhold_tma);
}

template <int P, bool A_MN, bool B_MN, int EPI, int TN>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_grouped_kernel(const __grid_constant__ TcGroupLaunch g) {
  if (g.done && *g.done) return;
  GroupSrc src;
  src.tiles = g.tiles;
  src.entries = g.entries;
  src.ntiles = g.ntiles;
  src.t0 = blockIdx.x;
  src.dt = gridDim.x;
  src.sl_default = g.slice_stages > 0 ? g.slice_stages : 1;
  tc_body<P, A_MN, B_MN, EPI, TN, 1>(src, nullptr, g.err, nullptr, g.planes_dyn, g.withhold_tma);
}

inline int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int P, bool A_MN, bool B_MN, int EPI>
cudaError_t launch_t(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                     int64_t ntiles, cudaStream_t s) {
  auto k = tc_gemm_kernel<P, A_MN, B_MN, EPI>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P>::SMEM);
  if (e != cudaSuccess) return e;
  int64_t grid = ntiles < sm_count() ? ntiles : sm_count();
  k<<<(unsigned)grid, NTHREADS, Cfg<P>::SMEM, s>>>(ma, mb, a, tm, tn, ntiles);
  return cudaGetLastError();
}

// Clusters of two that can be resident at once for a pair kernel (one CTA per SM).
inline int max_active_pairs(const void* kernel, int smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * (sm_count() / 2)), 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 2;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = sm_count() / 2;
  }
  return n;
}

template <int P, bool A_MN, bool B_MN, int EPI>
cudaError_t launch_pair_t(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm2, int64_t tn,
                          int64_t ntiles, cudaStream_t s) {
  auto k = tc_gemm_pair_kernel<P, A_MN, B_MN, EPI>;
  constexpr int smem = (int)Cfg<P, BN, 2>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  static const int pairs = max_active_pairs(reinterpret_cast<const void*>(k), smem);
  const int64_t np = ntiles < pairs ? ntiles : pairs;
  k<<<(unsigned)(2 * np), NTHREADS, smem, s>>>(ma, mb, a, tm2, tn, ntiles);
  return cudaGetLastError();
}

// The pair kernels exist for three planes (the BF16X6 products of the solve).
cudaError_t dispatch_pair(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm2, int64_t tn,
                          int64_t ntiles, cudaStream_t s) {
  const bool amn = !a.a.kmajor, bmn = !a.b.kmajor;
  switch (a.epi) {
    case TC_EPI_NS:
      if (!amn && bmn) return launch_pair_t<3, false, true, TC_EPI_NS>(ma, mb, a, tm2, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_GRAM:
      if (amn && bmn) return launch_pair_t<3, true, true, TC_EPI_GRAM>(ma, mb, a, tm2, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_NS_STEP:
      if (!amn && bmn) return launch_pair_t<3, false, true, TC_EPI_NS_STEP>(ma, mb, a, tm2, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_CLENSHAW:
      if (amn && bmn) return launch_pair_t<3, true, true, TC_EPI_CLENSHAW>(ma, mb, a, tm2, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_PLANES:
      if (!amn && bmn) return launch_pair_t<3, false, true, TC_EPI_PLANES>(ma, mb, a, tm2, tn, ntiles, s);
      return cudaErrorInvalidValue;
    default:
      if (amn && bmn) return launch_pair_t<3, true, true, TC_EPI_STORE>(ma, mb, a, tm2, tn, ntiles, s);
      if (!amn && bmn) return launch_pair_t<3, false, true, TC_EPI_STORE>(ma, mb, a, tm2, tn, ntiles, s);
      if (amn && !bmn) return launch_pair_t<3, true, false, TC_EPI_STORE>(ma, mb, a, tm2, tn, ntiles, s);
      return launch_pair_t<3, false, false, TC_EPI_STORE>(ma, mb, a, tm2, tn, ntiles, s);
  }
}

template <int P>
cudaError_t dispatch_p(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                       int64_t ntiles, cudaStream_t s) {
  const bool amn = !a.a.kmajor, bmn = !a.b.kmajor;
  switch (a.epi) {
    case TC_EPI_NS:
      if (!amn && bmn) return launch_t<P, false, true, TC_EPI_NS>(ma, mb, a, tm, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_GRAM:
      if (amn && bmn) return launch_t<P, true, true, TC_EPI_GRAM>(ma, mb, a, tm, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_NS_STEP:
      if (!amn && bmn) return launch_t<P, false, true, TC_EPI_NS_STEP>(ma, mb, a, tm, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_CLENSHAW:
      if (amn && bmn) return launch_t<P, true, true, TC_EPI_CLENSHAW>(ma, mb, a, tm, tn, ntiles, s);
      return cudaErrorInvalidValue;
    case TC_EPI_PLANES:
      if (!amn && bmn) return launch_t<P, false, true, TC_EPI_PLANES>(ma, mb, a, tm, tn, ntiles, s);
      return cudaErrorInvalidValue;
    default:
      if (amn && bmn) return launch_t<P, true, true, TC_EPI_STORE>(ma, mb, a, tm, tn, ntiles, s);
      if (!amn && bmn) return launch_t<P, false, true, TC_EPI_STORE>(ma, mb, a, tm, tn, ntiles, s);
      if (amn && !bmn) return launch_t<P, true, false, TC_EPI_STORE>(ma, mb, a, tm, tn, ntiles, s);
      return launch_t<P, false, false, TC_EPI_STORE>(ma, mb, a, tm, tn, ntiles, s);
  }
}


template <int P, bool A_MN, bool B_MN, int EPI, int TN>
cudaError_t launch_grouped_t(const TcGroupLaunch& g, cudaStream_t s) {
  auto k = tc_gemm_grouped_kernel<P, A_MN, B_MN, EPI, TN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<P, TN>::SMEM);
  if (e != cudaSuccess) return e;
  int64_t grid = g.ntiles < sm_count() ? g.ntiles : sm_count();
  if (grid < 1) return cudaSuccess;
  k<<<(unsigned)grid, NTHREADS, Cfg<P, TN>::SMEM, s>>>(g);
  return cudaGetLastError();
}

template <int P, int TN>
cudaError_t dispatch_grouped_tn(const TcGroupLaunch& g, cudaStream_t s) {
  if (g.epi == TC_EPI_NS && !g.a_mn && g.b_mn) return launch_grouped_t<P, false, true, TC_EPI_NS, TN>(g, s);
  if (g.epi == TC_EPI_GRAM && g.a_mn && g.b_mn) return launch_grouped_t<P, true, true, TC_EPI_GRAM, TN>(g, s);
  if (g.epi == TC_EPI_STORE && g.a_mn && g.b_mn) return launch_grouped_t<P, true, true, TC_EPI_STORE, TN>(g, s);
  return cudaErrorInvalidValue;
}

template <int P>
cudaError_t dispatch_grouped(const TcGroupLaunch& g, cudaStream_t s) {
  if (g.tile_n == 128) return dispatch_grouped_tn<P, 128>(g, s);
  if (g.tile_n == 0 || g.tile_n == BN) return dispatch_grouped_tn<P, BN>(g, s);
  return cudaErrorInvalidValue;
}


}  // namespace

// One function per translation unit that instantiates a group of the kernels above.
cudaError_t tc_dispatch_single1(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                                int64_t ntiles, cudaStream_t s);
cudaError_t tc_dispatch_single2(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                                int64_t ntiles, cudaStream_t s);
cudaError_t tc_dispatch_single3(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                                int64_t ntiles, cudaStream_t s);
cudaError_t tc_dispatch_pair3(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm2, int64_t tn,
                              int64_t ntiles, cudaStream_t s);
cudaError_t tc_dispatch_fp8(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int64_t tm, int64_t tn,
                            int64_t ntiles, cudaStream_t s);
cudaError_t tc_dispatch_grouped1(const TcGroupLaunch& g, cudaStream_t s);
cudaError_t tc_dispatch_grouped2(const TcGroupLaunch& g, cudaStream_t s);
cudaError_t tc_dispatch_grouped3(const TcGroupLaunch& g, cudaStream_t s);

}  // namespace polar
