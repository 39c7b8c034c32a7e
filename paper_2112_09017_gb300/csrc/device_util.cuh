// Device helpers shared by the kernels of libpolar.so.
#pragma once

#include <stdint.h>

namespace polar {

// Round-to-nearest-even BF16 bit pattern of a float32 (NaN stays NaN).
__device__ __forceinline__ uint16_t bf16_rne_bits_dev(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7fffu + lsb) >> 16);
}

__device__ __forceinline__ float bf16_to_f32_dev(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

// Plane q of the split x = x_0 + x_1 + x_2 (each the BF16 rounding of what the
// previous planes left), for q < NP; planes[q] receives the bit pattern.
template <int NP>
__device__ __forceinline__ void split_planes_dev(float x, uint16_t (&planes)[3]) {
  float rem = x;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    uint16_t b = bf16_rne_bits_dev(rem);
    planes[q] = b;
    rem = rem - bf16_to_f32_dev(b);
  }
}

// The strictly lower triangle of a symmetric n x n matrix kept as three BF16 planes (pitch ldp,
// plane stride ps) from its upper triangle: 64 x 64 blocks (bi <= bj) of the upper triangle, taken
// t0, t0 + dt, ... in column order, read with 16-byte accesses into shared memory (`tile`, at least
// 3 x 64 x 66 halves) and written transposed with 16-byte accesses (diagonal blocks element by
// element below their diagonal). Columns from n up to the next multiple of 8 are padding: they may
// be written with zeros. All threads of the block take part (blockDim.x a multiple of 32).
__device__ __forceinline__ void mirror3_tiles(uint16_t* P, int64_t ldp, int64_t ps, int64_t n, int64_t t0, int64_t dt,
                                              uint16_t* tile) {
  constexpr int LD = 66;   // halves per shared row: 33 words, so column reads of eight rows miss each other's banks
  const int64_t nt = (n + 63) / 64, ntri = nt * (nt + 1) / 2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int64_t t = t0; t < ntri; t += dt) {
    int64_t bj = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (bj * (bj + 1) / 2 > t) --bj;
    while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
    const int64_t bi = t - bj * (bj + 1) / 2;
    const int64_t i0 = bi * 64, j0 = bj * 64;
    __syncthreads();
    for (int u = tid; u < 3 * 512; u += nthr) {   // rows i0.., columns j0.. of the upper block
      const int q = u >> 9, rr = (u >> 3) & 63, cv = u & 7;
      const int64_t i = i0 + rr, j = j0 + 8 * cv;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (i < n && j < n) v = *reinterpret_cast<const uint4*>(P + q * ps + i * ldp + j);
      uint32_t* d = reinterpret_cast<uint32_t*>(tile + (q * 64 + rr) * LD + 8 * cv);
      d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __syncthreads();
    for (int u = tid; u < 3 * 512; u += nthr) {   // rows j0.. of the lower block, columns i0..
      const int q = u >> 9, jj = (u >> 3) & 63, iv = u & 7;
      const int64_t j = j0 + jj, i = i0 + 8 * iv;
      if (j >= n || i >= n) continue;
      const uint16_t* col = tile + (q * 64 + 8 * iv) * LD + jj;
      uint16_t* dst = P + q * ps + j * ldp + i;
      if (bi < bj) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) w[e] = (uint32_t)col[(2 * e) * LD] | ((uint32_t)col[(2 * e + 1) * LD] << 16);
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (i + e < j && i + e < n) dst[e] = col[e * LD];
      }
    }
  }
}

}  // namespace polar
