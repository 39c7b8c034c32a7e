// Plain-form float32 products on the SIMT cores (every multiply-add an FFMA).
//
// One register-tiled kernel serves the three products of the iteration
// (Eq. NewtonSchulz): the Gram G = X^T X (upper-triangle tiles; the lower
// half is mirrored afterwards), the update X' = 1.5 X - 0.5 X G, and
// C = U^T A for H, plus the general C = alpha op(A) op(B) + beta C.
//
// Tile 128 x 128 x 16, 256 threads, 8 x 8 accumulators per thread in two
// 4 x 4 quadrants (rows ty*4 and 64 + ty*4, columns tx*4 and 64 + tx*4), two
// shared-memory buffers with register prefetch of the next k-slice. Each
// 16-wide k-slice is summed into a fresh register tile before it is added to
// the running sums (blocked summation).
#include "internal.cuh"

namespace polar {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256, PAD = 4;

struct Smem {
  float a[2][BK][BM + PAD];
  float b[2][BK][BN + PAD];
};

// Loads the (tile_rows x BK) slice of an operand into 8 registers.
// kmajor: stored (MN x K) row-major; else stored (K x MN).
// Register j of thread t holds element (mn, k) as listed by slot_coords().
__device__ __forceinline__ void slot_coords(bool kmajor, int f, int& mn, int& kk) {
  if (kmajor) { mn = f >> 2; kk = (f & 3) * 4; }   // 128 rows x 4 float4 along K
  else        { kk = f >> 5; mn = (f & 31) * 4; }  // 16 rows x 32 float4 along MN
}

__device__ __forceinline__ void load_slice(const float* __restrict__ P, int64_t ld, bool kmajor, int64_t mn0,
                                           int64_t MN, int64_t k0, int64_t K, bool vec, float (&r)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int f = t + NT * h;
    int mn, kk;
    slot_coords(kmajor, f, mn, kk);
    int64_t gm = mn0 + mn, gk = k0 + kk;
    if (kmajor) {
      // 4 consecutive k of row gm
      const float* p = P + gm * ld + gk;
      if (vec && gm < MN && gk + 3 < K) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p));
        r[4 * h + 0] = v.x; r[4 * h + 1] = v.y; r[4 * h + 2] = v.z; r[4 * h + 3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) r[4 * h + j] = (gm < MN && gk + j < K) ? __ldg(p + j) : 0.0f;
      }
    } else {
      // 4 consecutive mn of row gk
      const float* p = P + gk * ld + gm;
      if (vec && gk < K && gm + 3 < MN) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p));
        r[4 * h + 0] = v.x; r[4 * h + 1] = v.y; r[4 * h + 2] = v.z; r[4 * h + 3] = v.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) r[4 * h + j] = (gk < K && gm + j < MN) ? __ldg(p + j) : 0.0f;
      }
    }
  }
}

__device__ __forceinline__ void store_slice(float (*dst)[BM + PAD], bool kmajor, const float (&r)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int f = t + NT * h;
    int mn, kk;
    slot_coords(kmajor, f, mn, kk);
    if (kmajor) {
#pragma unroll
      for (int j = 0; j < 4; ++j) dst[kk + j][mn] = r[4 * h + j];
    } else {
      *reinterpret_cast<float4*>(&dst[kk][mn]) = make_float4(r[4 * h], r[4 * h + 1], r[4 * h + 2], r[4 * h + 3]);
    }
  }
}

// Tile coordinates: grouped raster (8 tile-rows per group) for L2 reuse, or the
// column-major upper triangle (bi <= bj) for the Gram.
__device__ __forceinline__ void tile_of(int64_t t, int64_t tm, int64_t tn, bool tri, int64_t& bi, int64_t& bj) {
  if (tri) {
    int64_t j = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (j * (j + 1) / 2 > t) --j;
    while ((j + 1) * (j + 2) / 2 <= t) ++j;
    bj = j;
    bi = t - j * (j + 1) / 2;
  } else {
    const int64_t G = 8;
    int64_t group = t / (G * tn);
    int64_t first = group * G;
    int64_t rows = (tm - first) < G ? (tm - first) : G;
    int64_t in = t % (G * tn);
    bi = first + in % rows;
    bj = in / rows;
  }
}

template <int EPI>
__global__ void __launch_bounds__(NT) simt_gemm_kernel(SimtArgs p, bool vec_a, bool vec_b, bool vec_c) {
  if (p.st && p.st->status != ST_RUNNING) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);

  const int64_t tm = (p.M + BM - 1) / BM, tn = (p.N + BN - 1) / BN;
  int64_t bi, bj;
  tile_of(blockIdx.x, tm, tn, p.triangular != 0, bi, bj);
  const int64_t m0 = bi * BM, n0 = bj * BN;
  const bool akm = p.a_kmajor != 0, bkm = p.b_kmajor != 0;

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  float ra[8], rb[8];
  const int64_t nk = (p.K + BK - 1) / BK;
  load_slice(p.A, p.lda, akm, m0, p.M, 0, p.K, vec_a, ra);
  load_slice(p.B, p.ldb, bkm, n0, p.N, 0, p.K, vec_b, rb);
  store_slice(sm.a[0], akm, ra);
  store_slice(sm.b[0], bkm, rb);
  __syncthreads();

  for (int64_t kt = 0; kt < nk; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < nk) {
      load_slice(p.A, p.lda, akm, m0, p.M, (kt + 1) * BK, p.K, vec_a, ra);
      load_slice(p.B, p.ldb, bkm, n0, p.N, (kt + 1) * BK, p.K, vec_b, rb);
    }
    // each k-slice sums into a fresh tile first (blocked summation: the rounding
    // error of the running sums grows with K / 16 additions, not K)
    float part[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) part[i][j] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
      float4 a0 = *reinterpret_cast<const float4*>(&sm.a[cur][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&sm.a[cur][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&sm.b[cur][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&sm.b[cur][kk][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) part[i][j] = fmaf(a[i], b[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] += part[i][j];
    if (kt + 1 < nk) {
      store_slice(sm.a[cur ^ 1], akm, ra);
      store_slice(sm.b[cur ^ 1], bkm, rb);
    }
    __syncthreads();
  }

  // Epilogue.
  double part = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= p.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t c0 = n0 + h * 64 + tx * 4;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = acc[i][4 * h + j];
      if (EPI == SIMT_EPI_STORE) {
        float* dst = p.C + r * p.ldc + c0;
        if (vec_c && c0 + 3 < p.N) {
          float4 o;
          if (p.beta != 0.0f) {
            float4 old = *reinterpret_cast<const float4*>(dst);
            o = make_float4(p.alpha * v[0] + p.beta * old.x, p.alpha * v[1] + p.beta * old.y,
                            p.alpha * v[2] + p.beta * old.z, p.alpha * v[3] + p.beta * old.w);
          } else {
            o = make_float4(p.alpha * v[0], p.alpha * v[1], p.alpha * v[2], p.alpha * v[3]);
          }
          *reinterpret_cast<float4*>(dst) = o;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c0 + j < p.N) dst[j] = p.alpha * v[j] + (p.beta != 0.0f ? p.beta * dst[j] : 0.0f);
        }
      } else if (EPI == SIMT_EPI_NS) {
        // X_{k+1} = c1 X_k + c3 X_k G (1.5, -0.5; or Algorithm 1's preconditioning coefficients)
        const float c1 = p.st ? p.st->upd_c1 : 1.5f, c3 = p.st ? p.st->upd_c3 : -0.5f;
        const float* xo = p.Xold + r * p.ldx + c0;
        float* dst = p.C + r * p.ldc + c0;
        if (vec_c && c0 + 3 < p.N) {
          float4 x = *reinterpret_cast<const float4*>(xo);
          *reinterpret_cast<float4*>(dst) =
              make_float4(c1 * x.x + c3 * v[0], c1 * x.y + c3 * v[1], c1 * x.z + c3 * v[2], c1 * x.w + c3 * v[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c0 + j < p.N) dst[j] = c1 * xo[j] + c3 * v[j];
        }
      } else {  // GRAM: store the tile; residual weights 2 above the diagonal, 1 on it
        float* dst = p.C + r * p.ldc + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t c = c0 + j;
          if (c < p.N) {
            dst[j] = v[j];
            if (r < c) {
              double d = (double)v[j];
              part += 2.0 * d * d;
            } else if (r == c) {
              double d = (double)v[j] - 1.0;
              part += d * d;
            }
          }
        }
      }
    }
  }
  if (EPI == SIMT_EPI_GRAM) {
    __shared__ double red[NT / 32];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      p.partials[blockIdx.x] = t;
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

int simt_gram_tiles(int64_t n) {
  int64_t t = (n + BN - 1) / BN;
  return (int)(t * (t + 1) / 2);
}

cudaError_t launch_simt_gemm(const SimtArgs& a, int epi, cudaStream_t s) {
  const int64_t tm = (a.M + BM - 1) / BM, tn = (a.N + BN - 1) / BN;
  int64_t tiles = a.triangular ? tn * (tn + 1) / 2 : tm * tn;
  if (tiles <= 0) return cudaSuccess;
  const bool vec_a = aligned16(a.A) && (a.lda % 4 == 0);
  const bool vec_b = aligned16(a.B) && (a.ldb % 4 == 0);
  const bool vec_c = aligned16(a.C) && (a.ldc % 4 == 0) &&
                     (epi != SIMT_EPI_NS || (aligned16(a.Xold) && a.ldx % 4 == 0));
  const size_t smem = sizeof(Smem);
  cudaError_t e = cudaSuccess;
  switch (epi) {
    case SIMT_EPI_STORE:
      cudaFuncSetAttribute(simt_gemm_kernel<SIMT_EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      simt_gemm_kernel<SIMT_EPI_STORE><<<(unsigned)tiles, NT, smem, s>>>(a, vec_a, vec_b, vec_c);
      break;
    case SIMT_EPI_NS:
      cudaFuncSetAttribute(simt_gemm_kernel<SIMT_EPI_NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      simt_gemm_kernel<SIMT_EPI_NS><<<(unsigned)tiles, NT, smem, s>>>(a, vec_a, vec_b, vec_c);
      break;
    default:
      cudaFuncSetAttribute(simt_gemm_kernel<SIMT_EPI_GRAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      simt_gemm_kernel<SIMT_EPI_GRAM><<<(unsigned)tiles, NT, smem, s>>>(a, vec_a, vec_b, vec_c);
      break;
  }
  e = cudaGetLastError();
  return e;
}

}  // namespace polar
