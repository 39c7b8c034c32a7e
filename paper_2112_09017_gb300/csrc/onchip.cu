// Batched small problems (n <= 128, m <= 256) solved entirely on one SM each: the
// whole Newton-Schulz loop of Sec. III.D (Eq. NewtonSchulz with the residual stop
// rule; Algorithm 1's preconditioning steps when asked) in one CTA per problem, with
// no global-memory traffic between iterations.
//
//   shared memory  the three BF16 planes of X_k, rows padded to 16 and columns to 128,
//                  in 64-column chunks of 128-byte rows with the 128-byte swizzle: the
//                  same bytes are the MN-major operands of the Gram (K = rows of X)
//                  and the K-major operand of the update (N = rows of X)
//   TMEM           two Gram accumulators (columns 0 and 128), the planes of G as the
//                  A operand of the update (two BF16 per 32-bit column, from column
//                  256), and the update accumulator (columns 0 .. m, once the Gram's
//                  have been read)
//   Gram           G = X^T X in 64-row slices into alternating accumulators, each
//                  promoted by the workers with round-to-nearest adds (the tensor-core
//                  accumulator itself truncates)
//   update         P^T = G X^T (G is symmetric): A = G from TMEM (M = 128 lanes = the
//                  columns of X), B = X, N = the rows of X; then
//                  X_{k+1}(r, i) = c1 X_k(r, i) + c3 P^T(i, r), split back into the
//                  planes in place
// Warps 0-7 (workers, two per TMEM lane quarter, one per half of the columns) load
// X_0, promote accumulators, evaluate the residual and the stop rule, write G into
// TMEM and X back into shared memory; warp 8 allocates TMEM and one of its threads
// issues the MMAs. Every mbarrier wait is bounded (about one second); on expiry the
// problem reports a timeout, the MMAs in flight drain and TMEM is freed.
#include <cuda.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "device_util.cuh"
#include "internal.cuh"
#include "stop_rule.cuh"
#include "tc_ptx.cuh"

namespace polar {
namespace {

constexpr int OC_WORKER_WARPS = 8;
constexpr int OC_WORKERS = OC_WORKER_WARPS * 32;
constexpr int OC_THREADS = OC_WORKERS + 32;
constexpr uint32_t OC_TMEM_COLS = 512;
constexpr uint32_t OC_G_COL = 256;          // first TMEM column of G's planes
constexpr int64_t OC_MAX_M = 256, OC_MAX_N = 128;

// Plane pairs (A plane, B plane) of the split product, smallest terms first; P planes
// use the last passes_for(P) entries.
__constant__ int kOcPassA[6] = {1, 0, 2, 0, 1, 0};
__constant__ int kOcPassB[6] = {1, 2, 0, 1, 0, 0};

struct OcCtl {
  uint64_t full[2];    // MMA -> workers: accumulator ready
  uint64_t empty[2];   // workers -> MMA: accumulator read
  uint64_t ops;        // workers -> MMA: operands ready (X in shared memory, or G in TMEM)
  uint64_t drain;
  int abort;           // a bounded wait expired
  int decision;        // 0: keep iterating, 1: stop, 2: abort
  uint32_t tmem_base;
  int pad;
  float c1, c3;
  double red[OC_WORKER_WARPS];
};

__host__ __device__ __forceinline__ uint32_t oc_rows(int64_t m) { return (uint32_t)((m + 15) / 16 * 16); }

size_t oc_smem_bytes(int64_t max_m) { return (size_t)6 * oc_rows(max_m) * 128 + sizeof(OcCtl) + 1024; }
static_assert(6 * 256 * 128 + sizeof(OcCtl) + 1024 > 232448 / 2 && 6 * 256 * 128 + sizeof(OcCtl) + 1024 <= 232448,
              "one CTA per SM and within the opt-in shared memory of a CTA");

// Byte offset of element (r, c) in a plane: chunk c / 64, row r, 16-byte unit swizzled by r % 8.
__device__ __forceinline__ uint32_t oc_off(uint32_t r, uint32_t c, uint32_t ch) {
  return (c >> 6) * ch + r * 128u + ((((c & 63u) >> 3) ^ (r & 7u)) << 4) + ((c & 7u) << 1);
}

__device__ __forceinline__ void oc_sync_workers() { asm volatile("bar.sync 1, %0;" ::"n"(OC_WORKERS) : "memory"); }

__device__ __forceinline__ void oc_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Instruction descriptor: D = F32, A = B = BF16, M = 128, N = n, majors as given.
__device__ __forceinline__ uint32_t oc_idesc(bool a_mn, bool b_mn, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) | ((n >> 3) << 17) |
         ((128u >> 4) << 24);
}

struct OcBars {
  uint32_t full, empty, ops, drain;
};

template <int P>
__device__ __noinline__ void oc_mma(uint32_t xbase, uint32_t ch, uint32_t mp, uint32_t np, uint32_t tmem, OcBars br,
                                    volatile OcCtl* ctl, int withhold) {
  volatile int* abort_flag = &ctl->abort;
  constexpr int NPASS = P == 3 ? 6 : (P == 2 ? 3 : 1);
  constexpr int P0 = 6 - NPASS;
  const uint32_t idesc_g = oc_idesc(true, true, np);
  const uint32_t idesc_u = oc_idesc(false, false, mp);
  const uint32_t ks_g = mp / 16, ks_u = np / 16;
  uint32_t ph_ops = 0, use0 = 0, use1 = 0;
  bool issued = false;
  while (true) {
    // X_k is in shared memory
    if (!mbar_wait(br.ops, ph_ops, abort_flag)) break;
    ph_ops ^= 1u;
    if (ctl->decision != 0) break;
    tc_fence_after();
    bool ok = true;
    for (uint32_t s = 0; 4 * s < ks_g; ++s) {
      const uint32_t b = s & 1u;
      if (!mbar_wait(br.empty + 8 * b, ((b ? use1 : use0) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const uint32_t k_end = 4 * s + 4 < ks_g ? 4 * s + 4 : ks_g;
      if (!withhold) {
        for (int ps = 0; ps < NPASS; ++ps) {
          const uint32_t qa = (uint32_t)kOcPassA[P0 + ps], qb = (uint32_t)kOcPassB[P0 + ps];
          for (uint32_t kk = 4 * s; kk < k_end; ++kk) {
            const uint64_t ad = smem_desc(xbase + 2 * qa * ch + kk * 2048, ch, 1024, 2);
            const uint64_t bd = smem_desc(xbase + 2 * qb * ch + kk * 2048, ch, 1024, 2);
            tc_mma(tmem + 128 * b, ad, bd, idesc_g, (ps == 0 && kk == 4 * s) ? 0u : 1u);
          }
        }
        tc_commit(br.full + 8 * b);
        issued = true;
      }
      if (b) ++use1; else ++use0;
    }
    if (!ok) break;
    // G is in TMEM (or the workers stopped)
    if (!mbar_wait(br.ops, ph_ops, abort_flag)) break;
    ph_ops ^= 1u;
    if (ctl->decision != 0) break;
    tc_fence_after();
    if (!mbar_wait(br.empty, (use0 & 1u) ^ 1u, abort_flag) || !mbar_wait(br.empty + 8, (use1 & 1u) ^ 1u, abort_flag))
      break;
    tc_fence_after();
    if (!withhold) {
      for (int ps = 0; ps < NPASS; ++ps) {
        const uint32_t qa = (uint32_t)kOcPassA[P0 + ps], qb = (uint32_t)kOcPassB[P0 + ps];
        for (uint32_t kk = 0; kk < ks_u; ++kk) {
          const uint32_t at = tmem + OC_G_COL + 64 * qa + 8 * kk;
          const uint64_t bd = smem_desc(xbase + (2 * qb + (kk >> 2)) * ch + (kk & 3u) * 32, 16, 1024, 2);
          tc_mma_ts(tmem, at, bd, idesc_u, (ps == 0 && kk == 0) ? 0u : 1u);
        }
      }
      tc_commit(br.full);
      tc_commit(br.full + 8);
      issued = true;
    }
    ++use0;
    ++use1;
  }
  // every MMA issued has completed before the CTA frees TMEM
  if (issued) {
    tc_commit(br.drain);
    mbar_drain(br.drain, 0);
  }
}

template <int P>
__device__ __noinline__ void oc_workers(const OcTask& tk, uint8_t* xs, uint32_t ch, uint32_t mp, uint32_t np,
                                        uint32_t tmem, OcBars br, volatile OcCtl* ctl, const StopRule& rule,
                                        double tol, int warp, int lane) {
  const int tid = warp * 32 + lane;
  const int h = warp >> 2;                            // half of the columns this warp reads
  const uint32_t i = (uint32_t)((warp & 3) * 32 + lane);   // TMEM lane: a row of G, a column of X
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
  const int64_t m = tk.m, n = tk.n;
  DevState* st = tk.st;
  volatile int* abort_flag = &ctl->abort;
  uint32_t use0 = 0, use1 = 0;
  const uint32_t nslices = (mp / 16 + 3) / 4;
  int k = 0;
  for (;; ++k) {
    // X_k complete in shared memory: hand it to the tensor cores
    oc_fence_async();
    oc_sync_workers();
    if (tid == 0) mbar_arrive(br.ops);
    // ---- Gram: promote its slices
    float g[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) g[j] = 0.0f;
    for (uint32_t s = 0; s < nslices; ++s) {
      const uint32_t b = s & 1u;
      bool ok = !*abort_flag && mbar_wait(br.full + 8 * b, (b ? use1 : use0) & 1u, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
        if (64u * h < np) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tmem + lane_addr + 128u * b + 64u * h + 16u * c, v);
            add16_packed(&g[16 * c], v);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(br.empty + 8 * b);
      if (b) ++use1; else ++use0;
    }
    // ---- residual ||G - I||_F^2 over the n x n block, fixed-order reduction
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      const int64_t jj = 64 * h + j;
      if (jj >= n) g[j] = 0.0f;   // columns beyond n (stale accumulator columns)
      if ((int64_t)i < n && jj < n) {
        const double d = (double)g[j] - ((int64_t)i == jj ? 1.0 : 0.0);
        part = fma(d, d, part);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if (lane == 0) ctl->red[warp] = part;
    oc_sync_workers();
    if (tid == 0) {
      int dec = 2;
      if (!*abort_flag) {
        double sum = 0.0;
        for (int w = 0; w < OC_WORKER_WARPS; ++w) sum += ctl->red[w];
        const double r = sqrt(sum) * st->inv_sqrt_n;
        const bool running = batched_step_rule(*st, rule, tol, r, k, P);
        ctl->c1 = st->upd_c1;
        ctl->c3 = st->upd_c3;
        dec = running ? 0 : 1;
      }
      ctl->decision = dec;
    }
    oc_sync_workers();
    const int dec = ctl->decision;
    if (dec != 0) {
      if (tid == 0) mbar_arrive(br.ops);   // lets the MMA thread see the decision
      break;
    }
    // ---- G's planes into TMEM as the update's A operand (two BF16 per column, low half first)
    if (64u * h < np) {
#pragma unroll
      for (int qp = 0; qp < P; ++qp) {
        uint32_t w[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint16_t b0 = bf16_rne_bits_dev(g[2 * j]), b1 = bf16_rne_bits_dev(g[2 * j + 1]);
          g[2 * j] -= bf16_to_f32_dev(b0);
          g[2 * j + 1] -= bf16_to_f32_dev(b1);
          w[j] = (uint32_t)b0 | ((uint32_t)b1 << 16);
        }
        tmem_st32(tmem + lane_addr + OC_G_COL + 64u * qp + 32u * h, w);
      }
      tmem_st_wait();
    }
    tc_fence_before();
    oc_sync_workers();
    if (tid == 0) mbar_arrive(br.ops);
    // ---- update: P^T = G X^T, then X_{k+1} = c1 X_k + c3 P in place
    bool ok = !*abort_flag && mbar_wait(br.full, use0 & 1u, abort_flag) && mbar_wait(br.full + 8, use1 & 1u, abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
    if (ok) {
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (128u * h + 16u * c < mp) {
          float v[16];
          tmem_ld16(tmem + lane_addr + 128u * h + 16u * c, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[16 * c + e] = v[e];
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(br.empty);
      mbar_arrive(br.empty + 8);
    }
    ++use0;
    ++use1;
    if (ok && (int64_t)i < n) {
      const float c1 = ctl->c1, c3 = ctl->c3;
#pragma unroll
      for (int rr = 0; rr < 128; ++rr) {
        const int64_t r = 128 * h + rr;
        if (r < m) {
          const uint32_t o = oc_off((uint32_t)r, i, ch);
          uint16_t* p0 = reinterpret_cast<uint16_t*>(xs + o);
          uint16_t* p1 = reinterpret_cast<uint16_t*>(xs + 2 * ch + o);
          uint16_t* p2 = reinterpret_cast<uint16_t*>(xs + 4 * ch + o);
          const float x = (bf16_to_f32_dev(*p0) + bf16_to_f32_dev(*p1)) + bf16_to_f32_dev(*p2);
          const float xn = c1 * x + c3 * acc[rr];
          uint16_t qv[3];
          split_planes_dev<3>(xn, qv);
          *p0 = qv[0];
          *p1 = qv[1];
          *p2 = qv[2];
        }
      }
    }
  }
  if (ctl->decision != 1) return;
  // ---- the final iterate's planes to global memory, where the H product and U read them
  uint16_t* dst = tk.xp[k & 1];
  for (uint32_t u = (uint32_t)tid; u < 3u * (uint32_t)m * 16u; u += OC_WORKERS) {
    const uint32_t q = u / ((uint32_t)m * 16u), rem = u % ((uint32_t)m * 16u), r = rem >> 4, c8 = (rem & 15u) * 8u;
    if (c8 >= n) continue;
    const uint4 v = *reinterpret_cast<const uint4*>(xs + 2 * q * ch + oc_off(r, c8, ch));
    uint16_t* d = dst + q * tk.xps + r * tk.ldp + c8;
    if (c8 + 8 <= n) {
      *reinterpret_cast<uint4*>(d) = v;
    } else {
      const uint16_t* e = reinterpret_cast<const uint16_t*>(&v);
      for (uint32_t t = 0; c8 + t < n; ++t) d[t] = e[t];
    }
  }
}

template <int P>
__global__ void __launch_bounds__(OC_THREADS, 1)
    onchip_ns_kernel(const OcTask* __restrict__ tasks, StopRule rule, const double* tol_dev, int* err_word,
                     int withhold) {
  extern __shared__ uint8_t oc_smem[];
  const OcTask tk = tasks[blockIdx.x];
  // nothing in this kernel has written the status yet, so every thread sees the same value
  if (tk.st->status != ST_RUNNING) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(oc_smem);
  const uint32_t xbase = (raw + 1023u) & ~1023u;     // swizzle atoms need 1024-byte alignment
  uint8_t* xs = oc_smem + (xbase - raw);
  const uint32_t mp = oc_rows(tk.m), np = oc_rows(tk.n), ch = mp * 128u;
  volatile OcCtl* ctl = reinterpret_cast<volatile OcCtl*>(xs + 6 * ch);
  OcBars br;
  br.full = smem_u32((const void*)&ctl->full[0]);
  br.empty = smem_u32((const void*)&ctl->empty[0]);
  br.ops = smem_u32((const void*)&ctl->ops);
  br.drain = smem_u32((const void*)&ctl->drain);
  if (threadIdx.x == 0) {
    mbar_init(br.full, 1);
    mbar_init(br.full + 8, 1);
    mbar_init(br.empty, OC_WORKER_WARPS);
    mbar_init(br.empty + 8, OC_WORKER_WARPS);
    mbar_init(br.ops, 1);
    mbar_init(br.drain, 1);
    ctl->abort = 0;
    ctl->decision = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    oc_fence_async();
  }
  if (warp == OC_WORKER_WARPS) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)&ctl->tmem_base)),
                 "n"(OC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  } else {
    // X_0's three planes into shared memory, zero beyond m x n
    const int64_t m = tk.m, n = tk.n;
    for (uint32_t u = threadIdx.x; u < 3u * mp * 16u; u += OC_WORKERS) {
      const uint32_t q = u / (mp * 16u), rem = u % (mp * 16u), r = rem >> 4, c8 = (rem & 15u) * 8u;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r < m && c8 < n) {
        const uint16_t* src = tk.x0 + q * tk.xps + r * tk.ldp + c8;
        if (c8 + 8 <= n) {
          v = *reinterpret_cast<const uint4*>(src);
        } else {
          uint16_t* e = reinterpret_cast<uint16_t*>(&v);
          for (uint32_t t = 0; c8 + t < n; ++t) e[t] = src[t];
        }
      }
      *reinterpret_cast<uint4*>(xs + 2 * q * ch + oc_off(r, c8, ch)) = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  if (warp == OC_WORKER_WARPS) {
    if (lane == 0) oc_mma<P>(xbase, ch, mp, np, tmem, br, ctl, withhold);
  } else {
    const double tol = (tol_dev && *tol_dev > 0) ? *tol_dev : rule.tol;
    oc_workers<P>(tk, xs, ch, mp, np, tmem, br, ctl, rule, tol, warp, lane);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && ctl->decision == 2) {
    atomicOr(&tk.st->err_flags, 1u);
    tk.st->status = ST_TIMEOUT;
    if (err_word) atomicOr(err_word, 1);
  }
  if (warp == OC_WORKER_WARPS) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(OC_TMEM_COLS) : "memory");
  }
}

template <int P>
cudaError_t launch_p(const OcTask* tasks, int ntasks, const StopRule& rule, const double* tol_dev, int* err_word,
                     int withhold, cudaStream_t s) {
  // sized for the largest problem whatever the batch holds: more than half an SM's shared
  // memory keeps one CTA per SM, so no CTA waits for another's 512 TMEM columns
  const size_t smem = oc_smem_bytes(OC_MAX_M);
  auto k = onchip_ns_kernel<P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<ntasks, OC_THREADS, smem, s>>>(tasks, rule, tol_dev, err_word, withhold);
  return cudaGetLastError();
}

}  // namespace

bool onchip_fits(int64_t m, int64_t n) { return n >= 1 && m >= n && m <= OC_MAX_M && n <= OC_MAX_N; }

// Test hook for the bounded waits of this kernel: with POLAR_TEST_WITHHOLD_MMA=1 in the
// environment the MMA thread issues nothing, so the workers' waits expire after about
// one second and the problems report a timeout.
int onchip_withhold() {
  const char* e = getenv("POLAR_TEST_WITHHOLD_MMA");
  return (e && e[0] == '1') ? 1 : 0;
}

cudaError_t launch_onchip_ns(const OcTask* tasks, int ntasks, const StopRule& rule, const double* tol_dev,
                             int* err_word, int P, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const int withhold = onchip_withhold();
  switch (P) {
    case 1: return launch_p<1>(tasks, ntasks, rule, tol_dev, err_word, withhold, s);
    case 2: return launch_p<2>(tasks, ntasks, rule, tol_dev, err_word, withhold, s);
    case 3: return launch_p<3>(tasks, ntasks, rule, tol_dev, err_word, withhold, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace polar
