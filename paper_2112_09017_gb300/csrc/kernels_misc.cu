// Bandwidth-bound kernels of the Newton-Schulz polar path:
//  - ||A||_F with float64 accumulation (the Frobenius scaling of Sec. III.D,
//    first step of Algorithm 1), in a fixed reduction order;
//  - X_0 = A / ||A||_F fused with the BF16 plane split of X_0;
//  - the residual finalize and stop rule ||G - I||_F / sqrt(n) <= tol;
//  - H = (C + C^T) / 2 from C = U^T A with the symmetry check;
//  - mirror of an upper-triangle Gram to the full symmetric matrix.
#include <cuda_fp16.h>
#include <math.h>

#include "device_util.cuh"
#include "internal.cuh"

namespace polar {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint16_t bf16_rne_bits(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
  uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7fffu + lsb) >> 16);
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

// Fixed-order block sum of one double per thread (result valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

__global__ void frob_partials_kernel(const float* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                                     double* __restrict__ partials) {
  double acc = 0.0;
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    const float* row = A + r * lda;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      double v = (double)row[c];
      acc = fma(v, v, acc);
    }
  }
  double t = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void norm_finalize_kernel(const double* __restrict__ partials, int nparts, DevState* st,
                                     double inv_sqrt_n, int planes_first, int fp8_first) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  double t = block_sum(acc);
  if (threadIdx.x == 0) {
    double nrm = sqrt(t);
    st->normA = nrm;
    st->inv_sqrt_n = inv_sqrt_n;
    st->iters = 0;
    st->hist_len = 0;
    st->err_flags = 0;
    st->planes_next = planes_first;   // 0 with fp8_first: the FP8 phase of schedule 2
    st->fp8_on = fp8_first;
    st->sym_err = 0.0;
    st->upd_c1 = 1.5f;
    st->upd_c3 = -0.5f;
    for (int i = 0; i < 4; ++i) st->ring[i] = 0.0;
    st->status = (isfinite(nrm) && nrm > 0.0) ? ST_RUNNING : ST_NONFINITE;
  }
}

// dst = src * (1/||A||_F as float32 divisor) and/or BF16 planes of the same values.
__global__ void scale_split_kernel(const float* __restrict__ src, int64_t lds, int64_t m, int64_t n,
                                   const DevState* __restrict__ st, int scale, float* __restrict__ dst,
                                   int64_t ldd, uint16_t* __restrict__ planes, int64_t ldp,
                                   int64_t plane_stride, int nplanes) {
  if (st && st->status != ST_RUNNING) return;
  float s = scale ? (float)st->normA : 1.0f;
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      float x = src[r * lds + c];
      if (scale) x = __fdiv_rn(x, s);
      if (dst) dst[r * ldd + c] = x;
      float rem = x;
      for (int p = 0; p < nplanes; ++p) {
        uint16_t b = bf16_rne_bits(rem);
        planes[p * plane_stride + r * ldp + c] = b;
        rem = rem - bf16_bits_to_float(b);
      }
    }
  }
}

__global__ void split_flat_kernel(const float* __restrict__ x, int64_t count, int nplanes,
                                  uint16_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float rem = x[i];
    for (int p = 0; p < nplanes; ++p) {
      uint16_t b = bf16_rne_bits(rem);
      out[p * count + i] = b;
      rem = rem - bf16_bits_to_float(b);
    }
  }
}

// Sums the Gram partials in a fixed order and applies the stop rule for step k.
__global__ void residual_finalize_kernel(const double* __restrict__ partials, int nparts, DevState* st,
                                         StopRule rule, int k, int planes_this) {
  if (st->status != ST_RUNNING) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partials[i];
  double t = block_sum(acc);
  if (threadIdx.x != 0) return;
  double r = sqrt(t) * st->inv_sqrt_n;
  if (k < POLAR_HIST) {
    st->res_hist[k] = r;
    st->planes_hist[k] = (unsigned char)(planes_this < 0 ? st->planes_next : planes_this);
    st->hist_len = k + 1;
  }
  double r2 = (k >= 2) ? st->ring[(k - 2) & 3] : 0.0;
  st->ring[k & 3] = r;
  st->iters = k;
  const bool testing = k >= rule.n_pre;  // Algorithm 1: no stop test during preconditioning
  if (!isfinite(r)) {
    st->status = ST_NONFINITE;
  } else if (testing && r <= rule.tol) {
    st->status = ST_CONVERGED;
  } else if (testing && k >= rule.n_pre + 2 && r > rule.stagnation * r2 && r < rule.stag_floor) {
    st->status = ST_NOT_CONVERGED;
  } else if (k >= rule.max_iter) {
    st->status = ST_NOT_CONVERGED;
  } else {
    if (rule.sched == 2) {  // FP8 operands while r > fp8_switch (once ended, for good), then as schedule 1
      if (st->fp8_on && !(r > rule.fp8_switch)) st->fp8_on = 0;
      st->planes_next = st->fp8_on ? 0 : (r > rule.switch_residual ? 1 : 2);
    } else {
      st->planes_next = rule.sched == 1 ? (r > rule.switch_residual ? 1 : 2) : rule.planes_fixed;
    }
    // Eq. RogueMatrix (X <- a X - (4/27) a^3 X G) while preconditioning, then Eq. NewtonSchulz
    // (X <- 1.5 X - 0.5 X G): the coefficients of update k
    float c1, c3;
    update_coeffs(rule, k, c1, c3);
    st->upd_c1 = c1;
    st->upd_c3 = c3;
  }
}

// H = (C + C^T)/2 through 32x32 shared-memory tiles; float64 partials of
// ||(C - C^T)/2||^2 and ||C||^2 per block (grid-stride over tiles, fixed order).
__global__ void symmetrize_kernel(const float* __restrict__ C, int64_t ldc, int64_t n, float* __restrict__ H,
                                  int64_t ldh, double* __restrict__ partials) {
  __shared__ float ta[32][33];
  __shared__ float tb[32][33];
  int64_t nt = (n + 31) / 32;
  int64_t ntiles = nt * nt;
  double skew = 0.0, full = 0.0;
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int64_t bi = t / nt, bj = t % nt;
    int64_t i0 = bi * 32, j0 = bj * 32;
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      int64_t i = i0 + yy, j = j0 + tx;
      ta[yy][tx] = (i < n && j < n) ? C[i * ldc + j] : 0.0f;
      int64_t i2 = j0 + yy, j2 = i0 + tx;  // tile (bj, bi)
      tb[yy][tx] = (i2 < n && j2 < n) ? C[i2 * ldc + j2] : 0.0f;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      int64_t i = i0 + yy, j = j0 + tx;
      if (i < n && j < n) {
        float c = ta[yy][tx], ct = tb[tx][yy];
        H[i * ldh + j] = 0.5f * (c + ct);
        double d = 0.5 * ((double)c - (double)ct);
        skew = fma(d, d, skew);
        full = fma((double)c, (double)c, full);
      }
    }
  }
  double s1 = block_sum(skew);
  double s2 = block_sum(full);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s1;
    partials[2 * blockIdx.x + 1] = s2;
  }
}

__global__ void sym_finalize_kernel(const double* __restrict__ partials, int blocks, DevState* st) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < blocks; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  double s1 = block_sum(a);
  double s2 = block_sum(b);
  if (threadIdx.x == 0) st->sym_err = s2 > 0.0 ? sqrt(s1 / s2) : 0.0;
}

template <typename T>
__global__ void mirror_kernel(T* __restrict__ C, int64_t ldc, int64_t plane_stride, int nplanes, int64_t n,
                              const DevState* __restrict__ st, const int* __restrict__ planes_dyn) {
  if (st && st->status != ST_RUNNING) return;
  if (planes_dyn) nplanes = *planes_dyn;
  __shared__ T tile[32][33];
  int64_t nt = (n + 31) / 32;
  int64_t ntri = nt * (nt + 1) / 2;  // tiles (bi <= bj) of the upper triangle
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int p = 0; p < nplanes; ++p) {
    T* Cp = C + p * plane_stride;
    for (int64_t t = blockIdx.x; t < ntri; t += gridDim.x) {
      // column-major enumeration of the upper triangle: t = bj (bj + 1) / 2 + bi
      int64_t bj = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while (bj * (bj + 1) / 2 > t) --bj;
      while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
      int64_t bi = t - bj * (bj + 1) / 2;
      int64_t i0 = bi * 32, j0 = bj * 32;
      __syncthreads();
      for (int yy = ty; yy < 32; yy += 8) {
        int64_t i = i0 + yy, j = j0 + tx;
        tile[yy][tx] = (i < n && j < n) ? Cp[i * ldc + j] : T(0);
      }
      __syncthreads();
      // write C[j][i] = C[i][j] for i < j: row (j0 + yy), column (i0 + tx)
      for (int yy = ty; yy < 32; yy += 8) {
        int64_t j = j0 + yy, i = i0 + tx;
        if (i < n && j < n && i < j) Cp[j * ldc + i] = tile[tx][yy];
      }
    }
  }
}

// The lower triangle of G's three planes from its upper triangle (the Gram epilogue writes the
// upper one); skipped once the solve has stopped.
__global__ void mirror_planes3_kernel(uint16_t* __restrict__ P, int64_t ldp, int64_t ps, int64_t n,
                                      const DevState* __restrict__ st) {
  if (st && st->status != ST_RUNNING) return;
  __shared__ uint16_t tile[3 * 64 * 66];
  mirror3_tiles(P, ldp, ps, n, blockIdx.x, gridDim.x, tile);
}

// Three BF16 planes that came from an FP32 value sum back to it exactly:
// hi + mid has at most 16 significant bits and (hi + mid) + lo at most 24.
__global__ void planes_to_f32_kernel(const uint16_t* __restrict__ P, int64_t ldp, int64_t ps, int64_t m, int64_t n,
                                     float* __restrict__ dst, int64_t ldd) {
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      const int64_t i = r * ldp + c;
      dst[r * ldd + c] = (bf16_bits_to_float(P[i]) + bf16_bits_to_float(P[ps + i])) + bf16_bits_to_float(P[2 * ps + i]);
    }
}

__global__ void copy2d_kernel(const float* __restrict__ src, int64_t lds, float* __restrict__ dst, int64_t ldd,
                              int64_t m, int64_t n) {
  for (int64_t r = blockIdx.x; r < m; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) dst[r * ldd + c] = src[r * lds + c];
}

// X_0[i][j] = A[j][i] / ||A A^T||_F (Algorithm 2) as three BF16 planes, through 32 x 32 shared tiles.
__global__ void transpose_scale_split_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                             const DevState* __restrict__ st, uint16_t* __restrict__ P, int64_t ldp,
                                             int64_t ps) {
  if (st->status != ST_RUNNING) return;
  __shared__ float t[32][33];
  const float sc = (float)st->normA;
  const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < tr * tc; b += gridDim.x) {
    const int64_t r0 = (b / tc) * 32, c0 = (b % tc) * 32;
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t r = r0 + yy, c = c0 + tx;
      t[yy][tx] = (r < rows && c < cols) ? A[r * lda + c] : 0.0f;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t i = c0 + yy, j = r0 + tx;  // X_0 row i (a column of A), column j
      if (i < cols && j < rows) {
        float rem = __fdiv_rn(t[tx][yy], sc);
        for (int q = 0; q < 3; ++q) {
          const uint16_t bq = bf16_rne_bits(rem);
          P[q * ps + i * ldp + j] = bq;
          rem = rem - bf16_bits_to_float(bq);
        }
      }
    }
  }
}

// Clenshaw set-up: out(i, j) = s1 (alpha_map S(i, j) + beta_map [i = j]) + s0 [i = j], with S the
// symmetric matrix whose upper triangle is A's. Each 32 x 32 output tile reads the upper-triangle
// tile that holds its entries (itself above the diagonal, its transpose below) through shared memory.
__global__ void cheb_affine_split_kernel(const float* __restrict__ A, int64_t lda, int64_t n, double am, double bm,
                                         double s1, double s0, uint16_t* __restrict__ P, int64_t ldp, int64_t ps,
                                         int nplanes) {
  __shared__ float t[32][33];
  const int64_t nt = (n + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t b = blockIdx.x; b < nt * nt; b += gridDim.x) {
    const int64_t bi = b / nt, bj = b % nt;
    const int64_t si = bi < bj ? bi : bj, sj = bi < bj ? bj : bi;  // source tile in the upper triangle
    __syncthreads();
    if (s1 != 0.0) {
      for (int yy = ty; yy < 32; yy += 8) {
        const int64_t r = si * 32 + yy, c = sj * 32 + tx;
        t[yy][tx] = (r < n && c < n) ? A[r * lda + c] : 0.0f;
      }
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t i = bi * 32 + yy, j = bj * 32 + tx;
      if (i >= n || j >= n) continue;
      // entry (i, j) of S: A(min, max); within the source tile at (yy, tx) or transposed
      const bool upper = bi < bj || (bi == bj && yy <= tx);
      const double a = s1 != 0.0 ? (double)(upper ? t[yy][tx] : t[tx][yy]) : 0.0;
      const bool d = i == j;
      const float v = (float)(s1 * (am * a + (d ? bm : 0.0)) + (d ? s0 : 0.0));
      float rem = v;
      for (int q = 0; q < nplanes; ++q) {
        const uint16_t bq = bf16_rne_bits(rem);
        P[q * ps + i * ldp + j] = bq;
        rem = rem - bf16_bits_to_float(bq);
      }
    }
  }
}

// FP8 E4M3 with a power-of-two scale per 128 x 128 tile. One tile per block pass: the tile's
// amax (a block reduction), s = 2^t with t the smallest exponent such that amax <= 448 s
// (amax = m 2^e, m in [0.5, 1): t = e - 9, or e - 8 when m > 0.875, since 448 = 0.875 2^9),
// then s * e4m3(x / s) with round-to-nearest-even and saturation (cvt.rn.satfinite), exact
// in BF16 and FP32. An all-zero or non-finite tile keeps s = 1.
template <bool FROM_PLANES, bool TO_BF16>
__global__ void quantize_e4m3_kernel(const void* __restrict__ src, int64_t lds, int64_t sps, int64_t rows,
                                     int64_t cols, void* __restrict__ dst, int64_t ldd, const DevState* st) {
  if (st && (st->status != ST_RUNNING || !st->fp8_on)) return;
  __shared__ float red[kThreads / 32];
  const int64_t tr = (rows + 127) / 128, tc = (cols + 127) / 128;
  for (int64_t b = blockIdx.x; b < tr * tc; b += gridDim.x) {
    const int64_t r0 = (b / tc) * 128, c0 = (b % tc) * 128;
    float v[64];
    float amax = 0.0f;
#pragma unroll 8
    for (int i = 0; i < 64; ++i) {
      const int e = threadIdx.x + kThreads * i;   // 128 x 128 entries, 256 threads
      const int64_t gr = r0 + (e >> 7), gc = c0 + (e & 127);
      float x = 0.0f;
      if (gr < rows && gc < cols) {
        if (FROM_PLANES) {
          const uint16_t* p = reinterpret_cast<const uint16_t*>(src) + gr * lds + gc;
          x = (bf16_bits_to_float(p[0]) + bf16_bits_to_float(p[sps])) + bf16_bits_to_float(p[2 * sps]);
        } else {
          x = reinterpret_cast<const float*>(src)[gr * lds + gc];
        }
      }
      v[i] = x;
      amax = fmaxf(amax, fabsf(x));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    amax = red[0];
    for (int w = 1; w < kThreads / 32; ++w) amax = fmaxf(amax, red[w]);
    int t = 0;
    if (amax > 0.0f && isfinite(amax)) {
      int e;
      const float m = frexpf(amax, &e);
      t = e - 9 + (m > 0.875f ? 1 : 0);
    }
#pragma unroll 8
    for (int i = 0; i < 64; ++i) {
      const int e = threadIdx.x + kThreads * i;
      const int64_t gr = r0 + (e >> 7), gc = c0 + (e & 127);
      if (gr >= rows || gc >= cols) continue;
      uint16_t q8;
      asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(q8) : "f"(0.0f), "f"(ldexpf(v[i], -t)));
      uint32_t h2;
      asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(q8));
      const float q = ldexpf(__half2float(__ushort_as_half((unsigned short)(h2 & 0xffffu))), t);
      if (TO_BF16) reinterpret_cast<uint16_t*>(dst)[gr * ldd + gc] = (uint16_t)(__float_as_uint(q) >> 16);
      else reinterpret_cast<float*>(dst)[gr * ldd + gc] = q;
    }
  }
}

__global__ void inverse_init_kernel(DevState* st) {
  st->upd_c1 = 2.0f;   // X' = X (2I - A X) = 2 X - X (A X)
  st->upd_c3 = -1.0f;
}

// Algorithm 2's test after update k: delta = ||X' - X||_F / ||X'||_F against eps = u 2^k, u = 2^-24.
__global__ void inverse_finalize_kernel(const double* __restrict__ partials, int npairs, DevState* st, int k,
                                        int max_iter) {
  if (st->status != ST_RUNNING) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  const double sa = block_sum(a);
  const double sb = block_sum(b);
  if (threadIdx.x != 0) return;
  const double delta = sb > 0.0 ? sqrt(sa / sb) : INFINITY;
  if (k < POLAR_HIST) {
    st->res_hist[k] = delta;
    st->hist_len = k + 1;
  }
  st->ring[k & 3] = delta;
  st->iters = k + 1;
  const double eps = ldexp(1.0, k - 24);
  if (!isfinite(delta)) st->status = ST_NONFINITE;
  else if (delta <= eps) st->status = ST_CONVERGED;
  else if (k + 1 >= max_iter) st->status = ST_NOT_CONVERGED;
}

int grid_rows(int64_t m) { return (int)(m < 4096 ? (m > 0 ? m : 1) : 4096); }

}  // namespace

int precond_steps(double s_minus, double s0) {
  // Algorithm 1, first loop: s <- a s (1 - 4/27 a^2 s^2) until s >= s_minus (Eqs. a_def, RogueScalar)
  const double a = 1.5 * sqrt(3.0) - s_minus;
  double s = s0;
  int k = 0;
  while (s < s_minus && k < 1000) {
    s = a * s * (1.0 - (4.0 / 27.0) * a * a * s * s);
    ++k;
  }
  return k;
}

int frob_partials_blocks(int64_t m, int64_t n) {
  (void)n;
  return (int)(m < 2048 ? m : 2048);
}

cudaError_t launch_frob_partials(const float* A, int64_t m, int64_t n, int64_t lda, double* partials, int blocks,
                                 cudaStream_t s) {
  frob_partials_kernel<<<blocks, kThreads, 0, s>>>(A, m, n, lda, partials);
  return cudaGetLastError();
}

cudaError_t launch_norm_finalize(const double* partials, int nparts, DevState* st, double inv_sqrt_n,
                                 int planes_first, int fp8_first, cudaStream_t s) {
  norm_finalize_kernel<<<1, kThreads, 0, s>>>(partials, nparts, st, inv_sqrt_n, planes_first, fp8_first);
  return cudaGetLastError();
}

cudaError_t launch_scale_split(const float* src, int64_t lds, int64_t m, int64_t n, const DevState* st, bool scale,
                               float* dst, int64_t ldd, uint16_t* planes, int64_t ldp, int64_t plane_stride,
                               int nplanes, cudaStream_t s) {
  scale_split_kernel<<<grid_rows(m), kThreads, 0, s>>>(src, lds, m, n, st, scale ? 1 : 0, dst, ldd, planes, ldp,
                                                        plane_stride, nplanes);
  return cudaGetLastError();
}

cudaError_t launch_split_flat(const float* x, int64_t count, int nplanes, uint16_t* out, cudaStream_t s) {
  int64_t blocks = (count + kThreads - 1) / kThreads;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  split_flat_kernel<<<(int)blocks, kThreads, 0, s>>>(x, count, nplanes, out);
  return cudaGetLastError();
}

cudaError_t launch_residual_finalize(const double* partials, int nparts, DevState* st, StopRule rule, int k,
                                     int planes_this, cudaStream_t s) {
  residual_finalize_kernel<<<1, kThreads, 0, s>>>(partials, nparts, st, rule, k, planes_this);
  return cudaGetLastError();
}

int symmetrize_blocks(int64_t n) {
  int64_t nt = (n + 31) / 32;
  int64_t t = nt * nt;
  return (int)(t < 1024 ? t : 1024);
}

cudaError_t launch_symmetrize(const float* C, int64_t ldc, int64_t n, float* H, int64_t ldh, double* partials,
                              int blocks, cudaStream_t s) {
  symmetrize_kernel<<<blocks, kThreads, 0, s>>>(C, ldc, n, H, ldh, partials);
  return cudaGetLastError();
}

cudaError_t launch_sym_finalize(const double* partials, int blocks, DevState* st, cudaStream_t s) {
  sym_finalize_kernel<<<1, kThreads, 0, s>>>(partials, blocks, st);
  return cudaGetLastError();
}

static int mirror_blocks(int64_t n) {
  int64_t nt = (n + 31) / 32;
  int64_t t = nt * (nt + 1) / 2;
  return (int)(t < 4096 ? t : 4096);
}

cudaError_t launch_mirror_f32(float* C, int64_t ldc, int64_t n, const DevState* st, cudaStream_t s) {
  mirror_kernel<float><<<mirror_blocks(n), kThreads, 0, s>>>(C, ldc, 0, 1, n, st, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_mirror_planes(uint16_t* P, int64_t ldp, int64_t plane_stride, int nplanes, int64_t n,
                                 const DevState* st, const int* planes_dyn, cudaStream_t s) {
  mirror_kernel<uint16_t><<<mirror_blocks(n), kThreads, 0, s>>>(P, ldp, plane_stride, nplanes, n, st, planes_dyn);
  return cudaGetLastError();
}

cudaError_t launch_mirror_planes3(uint16_t* P, int64_t ldp, int64_t plane_stride, int64_t n, const DevState* st,
                                  cudaStream_t s) {
  const int64_t nt = (n + 63) / 64, ntri = nt * (nt + 1) / 2;
  mirror_planes3_kernel<<<(unsigned)(ntri < 2048 ? ntri : 2048), kThreads, 0, s>>>(P, ldp, plane_stride, n, st);
  return cudaGetLastError();
}

cudaError_t launch_planes_to_f32(const uint16_t* planes, int64_t ldp, int64_t plane_stride, int64_t m, int64_t n,
                                 float* dst, int64_t ldd, cudaStream_t s) {
  planes_to_f32_kernel<<<grid_rows(m), kThreads, 0, s>>>(planes, ldp, plane_stride, m, n, dst, ldd);
  return cudaGetLastError();
}

cudaError_t launch_transpose_scale_split(const float* A, int64_t lda, int64_t rows, int64_t cols, const DevState* st,
                                         uint16_t* planes, int64_t ldp, int64_t plane_stride, cudaStream_t s) {
  const int64_t tiles = ((rows + 31) / 32) * ((cols + 31) / 32);
  transpose_scale_split_kernel<<<(int)(tiles < 8192 ? tiles : 8192), kThreads, 0, s>>>(A, lda, rows, cols, st, planes,
                                                                                       ldp, plane_stride);
  return cudaGetLastError();
}

cudaError_t launch_cheb_affine_split(const float* A, int64_t lda, int64_t n, double alpha_map, double beta_map,
                                     double s1, double s0, uint16_t* planes, int64_t ldp, int64_t plane_stride,
                                     int nplanes, cudaStream_t s) {
  const int64_t tiles = ((n + 31) / 32) * ((n + 31) / 32);
  cheb_affine_split_kernel<<<(int)(tiles < 8192 ? tiles : 8192), kThreads, 0, s>>>(
      A, lda, n, alpha_map, beta_map, s1, s0, planes, ldp, plane_stride, nplanes);
  return cudaGetLastError();
}

// FP8 operands of the E4M3 tensor-core products: per 128 x 128 tile of src (rows x cols; float32, or
// three BF16 planes summed), the exponent t of quantize_e4m3_kernel (the smallest power of two 2^t with
// max|x| <= 448 2^t, 0 for a zero tile) and the E4M3 codes of x / 2^t (round to nearest even,
// saturating). Codes go to codes[r * ldc + c], or transposed to codes[c * ldc + r]; t to
// exps[tile_r * lde + tile_c], or transposed to exps[tile_c * lde + tile_r]. Skipped while st is not
// RUNNING or its FP8 phase is over.
//
// Each thread takes four 4 x 4 blocks of the tile (rows 4 rb .. 4 rb + 3, rb = warp + 8 k; columns
// 4 lane .. 4 lane + 3), so every load instruction of a warp reads 128 consecutive values of one row.
// Codes are packed four to a word: as they are for the row-major output; for the transposed output
// each 4 x 4 block of codes is transposed in registers and its four column words go to shared memory
// (output row c at words 32 c .. 32 c + 31, row block rb at word rb ^ (c / 4): the 32 lanes of a store
// hit 32 different banks), from where quads of words leave as 16-byte rows of the transposed tile.
__device__ __forceinline__ uint32_t e4m3x4(float x0, float x1, float x2, float x3) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(x1), "f"(x0));   // x0 in the low byte
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(x3), "f"(x2));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

template <bool FROM_PLANES>
__global__ void __launch_bounds__(kThreads) quantize_codes_kernel(
    const void* __restrict__ src, int64_t lds, int64_t sps, int64_t rows, int64_t cols, uint8_t* __restrict__ codes,
    int64_t ldc, int8_t* __restrict__ exps, int64_t lde, int transpose, int vec_in, int vec_out,
    const DevState* st) {
  if (st && (st->status != ST_RUNNING || !st->fp8_on)) return;
  __shared__ __align__(16) uint32_t sT[128 * 32];
  __shared__ float red[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t tr = (rows + 127) / 128, tc = (cols + 127) / 128;
  for (int64_t b = blockIdx.x; b < tr * tc; b += gridDim.x) {
    const int64_t bi = b / tc, bj = b % tc, r0 = bi * 128, c0 = bj * 128;
    const int64_t gc = c0 + 4 * lane;
    float v[4][4][4];   // [row block k][row in block][column in block]
    float amax = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t gr = r0 + 4 * (wid + 8 * k) + i;
        float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (gr < rows) {
          if (FROM_PLANES) {
            const uint16_t* pp = reinterpret_cast<const uint16_t*>(src) + gr * lds + gc;
            if (vec_in && gc + 3 < cols) {
              const uint2 h = *reinterpret_cast<const uint2*>(pp);
              const uint2 m = *reinterpret_cast<const uint2*>(pp + sps);
              const uint2 l = *reinterpret_cast<const uint2*>(pp + 2 * sps);
              const uint32_t hw[2] = {h.x, h.y}, mw[2] = {m.x, m.y}, lw[2] = {l.x, l.y};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int sh = (j & 1) * 16;
                x[j] = (bf16_bits_to_float((uint16_t)(hw[j >> 1] >> sh)) +
                        bf16_bits_to_float((uint16_t)(mw[j >> 1] >> sh))) +
                       bf16_bits_to_float((uint16_t)(lw[j >> 1] >> sh));
              }
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (gc + j < cols)
                  x[j] = (bf16_bits_to_float(pp[j]) + bf16_bits_to_float(pp[j + sps])) +
                         bf16_bits_to_float(pp[j + 2 * sps]);
            }
          } else {
            const float* pf = reinterpret_cast<const float*>(src) + gr * lds + gc;
            if (vec_in && gc + 3 < cols) {
              const float4 f = *reinterpret_cast<const float4*>(pf);
              x[0] = f.x; x[1] = f.y; x[2] = f.z; x[3] = f.w;
            } else {
#pragma unroll
              for (int j = 0; j < 4; ++j)
                if (gc + j < cols) x[j] = pf[j];
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          v[k][i][j] = x[j];
          amax = fmaxf(amax, fabsf(x[j]));
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    __syncthreads();   // the previous tile's readers are done with red and sT
    if (lane == 0) red[wid] = amax;
    __syncthreads();
    amax = red[0];
    for (int w = 1; w < kThreads / 32; ++w) amax = fmaxf(amax, red[w]);
    int t = 0;
    if (amax > 0.0f && isfinite(amax)) {
      int e;
      const float m = frexpf(amax, &e);
      t = e - 9 + (m > 0.875f ? 1 : 0);
    }
    if (threadIdx.x == 0) exps[transpose ? bj * lde + bi : bi * lde + bj] = (int8_t)t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int rb = wid + 8 * k;
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        w[i] = e4m3x4(ldexpf(v[k][i][0], -t), ldexpf(v[k][i][1], -t), ldexpf(v[k][i][2], -t),
                      ldexpf(v[k][i][3], -t));
      if (!transpose) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t gr = r0 + 4 * rb + i;
          if (gr >= rows) continue;
          uint8_t* cp = codes + gr * ldc + gc;
          if (vec_out && gc + 3 < cols) {
            *reinterpret_cast<uint32_t*>(cp) = w[i];
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (gc + j < cols) cp[j] = (uint8_t)(w[i] >> (8 * j));
          }
        }
      } else {
        // column j of the block: bytes j of the four row words
        const uint32_t a = __byte_perm(w[0], w[1], 0x5140), bb = __byte_perm(w[2], w[3], 0x5140);
        const uint32_t c = __byte_perm(w[0], w[1], 0x7362), d = __byte_perm(w[2], w[3], 0x7362);
        const uint32_t tcol[4] = {__byte_perm(a, bb, 0x5410), __byte_perm(a, bb, 0x7632), __byte_perm(c, d, 0x5410),
                                  __byte_perm(c, d, 0x7632)};
#pragma unroll
        for (int j = 0; j < 4; ++j) sT[(4 * lane + j) * 32 + (rb ^ lane)] = tcol[j];
      }
    }
    if (transpose) {
      __syncthreads();
      // output row oc (source column c0 + oc), 16 source rows 16 s .. 16 s + 15 per quad of words
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = threadIdx.x + kThreads * u;
        const int oc = idx >> 3, sq = idx & 7, g = oc >> 2;
        if (c0 + oc >= cols) continue;
        const uint4 x = *reinterpret_cast<const uint4*>(&sT[oc * 32 + 4 * (sq ^ (g >> 2))]);
        // word e of the quad holds row block 4 sq + (e ^ (g & 3)): undo the swizzle's order
        uint32_t o[4] = {x.x, x.y, x.z, x.w}, tmp;
        if (g & 1) { tmp = o[0]; o[0] = o[1]; o[1] = tmp; tmp = o[2]; o[2] = o[3]; o[3] = tmp; }
        if (g & 2) { tmp = o[0]; o[0] = o[2]; o[2] = tmp; tmp = o[1]; o[1] = o[3]; o[3] = tmp; }
        const int64_t gr0 = r0 + 16 * sq;
        uint8_t* cp = codes + (c0 + oc) * ldc + gr0;
        if (vec_out && gr0 + 15 < rows) {
          *reinterpret_cast<uint4*>(cp) = make_uint4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (gr0 + e < rows) cp[e] = (uint8_t)(o[e >> 2] >> (8 * (e & 3)));
        }
      }
    }
  }
}

// uni[r] = 1 when exps[r * lde + k] is the same for every k < nk (block rows r < nr).
__global__ void uniform_exps_kernel(const int8_t* __restrict__ exps, int64_t lde, int64_t nr, int64_t nk,
                                    uint8_t* __restrict__ uni, const DevState* st) {
  if (st && (st->status != ST_RUNNING || !st->fp8_on)) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int8_t* e = exps + r * lde;
  const int8_t e0 = e[0];
  uint8_t u = 1;
  for (int64_t k = 1; k < nk; ++k) u &= (uint8_t)(e[k] == e0);
  uni[r] = u;
}

cudaError_t launch_quantize_codes(const void* src, bool from_planes, int64_t lds, int64_t sps, int64_t rows,
                                  int64_t cols, uint8_t* codes, int64_t ldc, int8_t* exps, int64_t lde, bool transpose,
                                  uint8_t* uni, const DevState* st, cudaStream_t s) {
  const int64_t tiles = ((rows + 127) / 128) * ((cols + 127) / 128);
  if (tiles <= 0) return cudaSuccess;
  const int grid = (int)(tiles < 8192 ? tiles : 8192);
  const uintptr_t sa = reinterpret_cast<uintptr_t>(src), ca = reinterpret_cast<uintptr_t>(codes);
  // vector accesses: 16-byte float4 (8-byte uint2 for the planes) rows and 4-byte (transposed: 16-byte)
  // code words, where the base and the pitches keep every one aligned
  const int vec_in = from_planes ? (sa % 8 == 0 && lds % 4 == 0 && sps % 4 == 0) : (sa % 16 == 0 && lds % 4 == 0);
  const int vec_out = transpose ? (ca % 16 == 0 && ldc % 16 == 0) : (ca % 4 == 0 && ldc % 4 == 0);
  if (from_planes)
    quantize_codes_kernel<true><<<grid, kThreads, 0, s>>>(src, lds, sps, rows, cols, codes, ldc, exps, lde,
                                                         transpose ? 1 : 0, vec_in, vec_out, st);
  else
    quantize_codes_kernel<false><<<grid, kThreads, 0, s>>>(src, lds, sps, rows, cols, codes, ldc, exps, lde,
                                                          transpose ? 1 : 0, vec_in, vec_out, st);
  if (uni) {
    const int64_t tr = (rows + 127) / 128, tc = (cols + 127) / 128;
    const int64_t nr = transpose ? tc : tr, nk = transpose ? tr : tc;
    uniform_exps_kernel<<<(int)((nr + kThreads - 1) / kThreads), kThreads, 0, s>>>(exps, lde, nr, nk, uni, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_quantize_e4m3_planes(const uint16_t* src, int64_t ldp, int64_t sps, int64_t rows, int64_t cols,
                                        uint16_t* dst, int64_t ldd, const DevState* st, cudaStream_t s) {
  const int64_t tiles = ((rows + 127) / 128) * ((cols + 127) / 128);
  quantize_e4m3_kernel<true, true><<<(int)(tiles < 8192 ? tiles : 8192), kThreads, 0, s>>>(src, ldp, sps, rows, cols,
                                                                                          dst, ldd, st);
  return cudaGetLastError();
}

cudaError_t launch_quantize_e4m3_f32(const float* src, int64_t lds, int64_t rows, int64_t cols, float* dst,
                                     int64_t ldd, cudaStream_t s) {
  const int64_t tiles = ((rows + 127) / 128) * ((cols + 127) / 128);
  quantize_e4m3_kernel<false, false><<<(int)(tiles < 8192 ? tiles : 8192), kThreads, 0, s>>>(src, lds, 0, rows, cols,
                                                                                            dst, ldd, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_inverse_init(DevState* st, cudaStream_t s) {
  inverse_init_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_inverse_finalize(const double* partials, int npairs, DevState* st, int k, int max_iter,
                                    cudaStream_t s) {
  inverse_finalize_kernel<<<1, kThreads, 0, s>>>(partials, npairs, st, k, max_iter);
  return cudaGetLastError();
}

cudaError_t launch_copy2d(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t m, int64_t n,
                          cudaStream_t s) {
  copy2d_kernel<<<grid_rows(m), kThreads, 0, s>>>(src, lds, dst, ldd, m, n);
  return cudaGetLastError();
}

}  // namespace polar
