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

}  // namespace polar
