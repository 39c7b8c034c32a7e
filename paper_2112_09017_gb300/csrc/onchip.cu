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
// Sixteen warps, four per TMEM lane quarter taking 16-wide chunks of columns or rows in
// turn, load X_0, promote accumulators, evaluate the residual and the stop rule, write
// G into TMEM and X back into shared memory; warp 0 allocates TMEM and thread 0 issues
// the MMAs once a barrier has published their operands. Every mbarrier wait is bounded (about one second); on expiry the
// problem reports a timeout, the MMAs in flight drain and TMEM is freed.
#include <cuda.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "device_util.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace polar {
namespace {

constexpr int OC_WARPS = 16;          // four per TMEM lane quarter
constexpr int OC_THREADS = OC_WARPS * 32;
constexpr uint32_t OC_TMEM_COLS = 512;
constexpr uint32_t OC_G_COL = 256;          // first TMEM column of G's planes
constexpr int64_t OC_MAX_M = 256, OC_MAX_N = 128;

// Plane pairs (A plane, B plane) of the split product, smallest terms first:
// (1,1) (0,2) (2,0) (0,1) (1,0) (0,0); P planes use the last 6, 3 or 1 of them.
__host__ __device__ constexpr uint32_t oc_pass_a(int i) { return i == 0 ? 1u : i == 2 ? 2u : i == 4 ? 1u : 0u; }
__host__ __device__ constexpr uint32_t oc_pass_b(int i) { return i == 0 ? 1u : i == 1 ? 2u : i == 3 ? 1u : 0u; }

// The stop rule of the batched finalize on squares: with v = ||G - I||_F^2 = n r^2,
// r <= tol is v <= n tol^2 and r > s r_{k-2} is v > s^2 v_{k-2} (one FP64 compare each
// instead of a square root on the critical path).
struct OcRule {
  double v_tol, stag2, v_floor;
  int n_pre, max_iter;
  float pre_c1, pre_c3;
};

struct OcCtl {
  uint64_t full[2];    // tcgen05.commit -> all warps: accumulator ready
  uint64_t drain;
  int abort;           // a bounded wait expired
  int decision;        // 0: keep iterating, 1: stop, 2: abort
  int status;          // the problem's status after the step
  double v;            // ||G - I||_F^2 of the step
  OcRule dr;
  uint32_t tmem_base;
  int pad;
  float c1, c3;
  double red[OC_WARPS];
};

__host__ __device__ __forceinline__ uint32_t oc_rows(int64_t m) { return (uint32_t)((m + 15) / 16 * 16); }

size_t oc_smem_bytes(int64_t max_m) { return (size_t)6 * oc_rows(max_m) * 128 + sizeof(OcCtl) + 1024; }
static_assert(6 * 256 * 128 + sizeof(OcCtl) + 1024 > 232448 / 2 && 6 * 256 * 128 + sizeof(OcCtl) + 1024 <= 232448,
              "one CTA per SM and within the opt-in shared memory of a CTA");

// Byte offset of element (r, c) in a plane: chunk c / 64, row r, 16-byte unit swizzled by r % 8.
__device__ __forceinline__ uint32_t oc_off(uint32_t r, uint32_t c, uint32_t ch) {
  return (c >> 6) * ch + r * 128u + ((((c & 63u) >> 3) ^ (r & 7u)) << 4) + ((c & 7u) << 1);
}

__device__ __forceinline__ void oc_sync_workers() { asm volatile("bar.sync 1, %0;" ::"n"(OC_THREADS) : "memory"); }

// 8 consecutive 32-bit columns of this thread's TMEM lane (completed by tmem_st_wait).
__device__ __forceinline__ void oc_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

__device__ __forceinline__ void oc_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Instruction descriptor: D = F32, A = B = BF16, M = 128, N = n, majors as given.
__device__ __forceinline__ uint32_t oc_idesc(bool a_mn, bool b_mn, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) | ((n >> 3) << 17) |
         ((128u >> 4) << 24);
}

struct OcBars {
  uint32_t full, drain;
};

// TMEM loads without the wait, and the wait tied to the loaded registers so that no use
// is scheduled before it (tcgen05.wait::ld covers every earlier load of the thread).
__device__ __forceinline__ void oc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void oc_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Two floats to BF16 with round-to-nearest-even: lo in the low half, hi in the high half.
__device__ __forceinline__ uint32_t oc_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float oc_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float oc_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// The three-plane split of a pair (each value the sum of its planes exactly): planes of
// x0 in the low halves of w[0..2], of x1 in the high halves.
__device__ __forceinline__ void oc_split2(float x0, float x1, uint32_t (&w)[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    w[q] = oc_bf16x2(x0, x1);
    x0 -= oc_lo(w[q]);
    x1 -= oc_hi(w[q]);
  }
}

// MMA issue, by one thread: the Gram's 64-row slice s of X into accumulator s % 2, and the
// update P^T = G X^T into columns 0 .. mp, each completed on its full barrier. Plane q of
// X is read through MN-major descriptors (chunk stride ch, 8-row groups of 1024 bytes)
// and K-major ones (rows of 128 bytes), built per MMA from the plane's address.
template <int P>
struct OcIssuer {
  static constexpr int NPASS = P == 3 ? 6 : (P == 2 ? 3 : 1);
  static constexpr int P0 = 6 - NPASS;
  // descriptor high word: stride between 8-row groups 1024 bytes, version 1, 128-byte swizzle
  static constexpr uint32_t HI = (1024u >> 4) | (1u << 14) | (2u << 29);
  uint32_t xbase, ch, tmem, full, idesc_g, idesc_u, ks_g, ks_u;

  __device__ __forceinline__ void init(uint32_t xbase_, uint32_t ch_, uint32_t mp, uint32_t np, uint32_t tmem_,
                                       uint32_t full_) {
    xbase = xbase_;
    ch = ch_;
    tmem = tmem_;
    full = full_;
    idesc_g = oc_idesc(true, true, np);
    idesc_u = oc_idesc(false, false, mp);
    ks_g = mp / 16;
    ks_u = np / 16;
  }

  __device__ __forceinline__ static uint64_t desc(uint32_t addr, uint32_t lbo) {
    return ((uint64_t)HI << 32) | ((addr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16);
  }

  __device__ __forceinline__ void gram_slice(uint32_t s) {
    const uint32_t b = s & 1u;
    const uint32_t k_end = 4 * s + 4 < ks_g ? 4 * s + 4 : ks_g;
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps) {
      const uint32_t a0 = xbase + 2 * oc_pass_a(P0 + ps) * ch, b0 = xbase + 2 * oc_pass_b(P0 + ps) * ch;
      for (uint32_t kk = 4 * s; kk < k_end; ++kk)   // 16 rows of X: 2048 bytes
        tc_mma(tmem + 128 * b, desc(a0 + kk * 2048, ch), desc(b0 + kk * 2048, ch), idesc_g,
               (ps == 0 && kk == 4 * s) ? 0u : 1u);
    }
    tc_commit(full + 8 * b);
  }

  __device__ __forceinline__ void update() {
#pragma unroll
    for (int ps = 0; ps < NPASS; ++ps) {
      const uint32_t b0 = xbase + 2 * oc_pass_b(P0 + ps) * ch;
      for (uint32_t kk = 0; kk < ks_u; ++kk)   // 16 columns of X: 32 bytes within its 64-column chunk
        tc_mma_ts(tmem, tmem + OC_G_COL + 64 * oc_pass_a(P0 + ps) + 8 * kk, desc(b0 + (kk >> 2) * ch + (kk & 3u) * 32, 16),
                  idesc_u, (ps == 0 && kk == 0) ? 0u : 1u);
    }
    tc_commit(full);
    tc_commit(full + 8);
  }
};

// The whole loop for one problem, all warps. The four warps of a TMEM lane quarter take
// 16-wide chunks in turn: chunk c of the Gram's columns and of the update's rows belongs
// to warp sub = c % 4 of the quarter. Thread 0 issues the MMAs as soon as a barrier has
// published their operands (X_k in shared memory, G in TMEM, an accumulator read).
template <int P>
__device__ __noinline__ void oc_solve(const OcTask& tk, uint8_t* xs, uint32_t xbase, uint32_t ch, uint32_t mp,
                                      uint32_t np, uint32_t tmem, OcBars br, volatile OcCtl* ctl,
                                      int warp, int lane, int withhold) {
  const int tid = warp * 32 + lane;
  const uint32_t sub = (uint32_t)warp >> 2;
  const uint32_t i = (uint32_t)((warp & 3) * 32 + lane);           // TMEM lane: a row of G, a column of X
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
  const int64_t m = tk.m, n = tk.n;
  DevState* st = tk.st;
  volatile int* abort_flag = &ctl->abort;
  // byte offset of column i in a plane for each of the 8 row phases of the swizzle
  uint32_t colo[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) colo[e] = (i >> 6) * ch + ((((i & 63u) >> 3) ^ (uint32_t)e) << 4) + ((i & 7u) << 1);
  OcIssuer<P> iss;
  const bool issuer = tid == 0 && !withhold;
  if (issuer) iss.init(xbase, ch, mp, np, tmem, br.full);
  bool issued = false;
  const double inv_sqrt_n = tid == 32 ? st->inv_sqrt_n : 0.0;
  double v_km1 = 0.0, v_km2 = 0.0;                                 // thread 0: sums of squares of steps k-1, k-2
  uint32_t use0 = 0, use1 = 0;                                     // completions awaited on full[0], full[1]
  const uint32_t nslices = (mp / 16 + 3) / 4;
  const uint32_t gch = np / 16, uch = mp / 16;                     // 16-wide chunks of G's columns, X's rows
  int k = 0;
  for (;; ++k) {
    // X_k complete in shared memory (and the last accumulator read): the first two Gram slices
    oc_fence_async();
    tc_fence_before();
    oc_sync_workers();
    if (issuer && !*abort_flag) {
      tc_fence_after();
      iss.gram_slice(0);
      if (nslices > 1) iss.gram_slice(1);
      issued = true;
    }
    // ---- Gram: promote this warp's chunks (at most two) of every slice
    float g[2][16];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 16; ++e) g[t][e] = 0.0f;
    for (uint32_t s = 0; s < nslices; ++s) {
      const uint32_t b = s & 1u;
      bool ok = !*abort_flag && mbar_wait(br.full + 8 * b, (b ? use1 : use0) & 1u, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        tc_fence_after();
        uint32_t v[2][16];
#pragma unroll
        for (int t = 0; t < 2; ++t)
          if (sub + 4 * t < gch) oc_ld16(tmem + lane_addr + 128u * b + 16u * (sub + 4 * t), v[t]);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (sub + 4 * t < gch) {
            oc_wait16(v[t]);
            float f[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) f[e] = __uint_as_float(v[t][e]);
            add16_packed(g[t], f);
          }
        }
      }
      if (b) ++use1; else ++use0;
      if (s + 2 < nslices) {
        // every warp has read slice s: its accumulator takes slice s + 2
        tc_fence_before();
        oc_sync_workers();
        if (issuer && !*abort_flag) {
          tc_fence_after();
          iss.gram_slice(s + 2);
        }
      }
    }
    // ---- residual ||G - I||_F^2 over the n x n block (float per thread, at most 32 terms;
    // FP64 is slow on this part), and G's planes into TMEM as the update's A operand (two
    // BF16 per column, low half first) whatever the decision
    float part32 = 0.0f;
    bool stored = false;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const uint32_t c = sub + 4 * t;
      if (c < gch) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int64_t jj = 16 * c + e;
          if (jj >= n) g[t][e] = 0.0f;   // columns beyond n
          if ((int64_t)i < n && jj < n) {
            const float d = g[t][e] - ((int64_t)i == jj ? 1.0f : 0.0f);
            part32 = fmaf(d, d, part32);
          }
        }
#pragma unroll
        for (int qp = 0; qp < P; ++qp) {
          uint32_t w[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            w[j] = oc_bf16x2(g[t][2 * j], g[t][2 * j + 1]);
            g[t][2 * j] -= oc_lo(w[j]);
            g[t][2 * j + 1] -= oc_hi(w[j]);
          }
          oc_st8(tmem + lane_addr + OC_G_COL + 64u * qp + 8u * c, w);
        }
        stored = true;
      }
    }
    if (stored) tmem_st_wait();
    double part = (double)part32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if (lane == 0) ctl->red[warp] = part;
    tc_fence_before();
    oc_sync_workers();
    // ---- the stop rule: warp 0 sums the warps' partials in a fixed order and thread 0
    // decides on the sum of squares v = n r^2 against squared thresholds, then issues the
    // update at once; thread 32 records r and the outcome while the update runs
    if (warp == 0) {
      double v = lane < OC_WARPS ? ctl->red[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        int dec = 2, status = ST_TIMEOUT;
        if (!*abort_flag) {
          const bool testing = k >= ctl->dr.n_pre;
          if (!isfinite(v)) status = ST_NONFINITE;
          else if (testing && v <= ctl->dr.v_tol) status = ST_CONVERGED;
          else if (testing && k >= ctl->dr.n_pre + 2 && v > ctl->dr.stag2 * v_km2 && v < ctl->dr.v_floor) status = ST_NOT_CONVERGED;
          else if (k >= ctl->dr.max_iter) status = ST_NOT_CONVERGED;
          else status = ST_RUNNING;
          dec = status == ST_RUNNING ? 0 : 1;
          ctl->c1 = k < ctl->dr.n_pre ? ctl->dr.pre_c1 : 1.5f;
          ctl->c3 = k < ctl->dr.n_pre ? ctl->dr.pre_c3 : -0.5f;
          ctl->status = status;
          ctl->v = v;
        }
        ctl->decision = dec;
        v_km2 = v_km1;
        v_km1 = v;
        if (dec == 0 && issuer) {
          tc_fence_after();
          iss.update();
        }
      }
    }
    oc_sync_workers();
    if (tid == 32 && ctl->decision != 2) {
      // the record of step k, as the batched finalize keeps it
      const double r = sqrt(ctl->v) * inv_sqrt_n;
      if (k < POLAR_HIST) {
        st->res_hist[k] = r;
        st->planes_hist[k] = (unsigned char)P;
        st->hist_len = k + 1;
      }
      st->ring[k & 3] = r;
      st->iters = k;
      if (ctl->status != ST_RUNNING) st->status = ctl->status;
      else {
        st->upd_c1 = ctl->c1;
        st->upd_c3 = ctl->c3;
      }
    }
    if (ctl->decision != 0) break;
    // ---- update: P^T = G X^T, then X_{k+1} = c1 X_k + c3 P in place, this warp's 16-row
    // chunks one at a time from TMEM with the next in flight
    bool ok = !*abort_flag && mbar_wait(br.full, use0 & 1u, abort_flag) && mbar_wait(br.full + 8, use1 & 1u, abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    ++use0;
    ++use1;
    if (ok && sub < uch) {
      tc_fence_after();
      const float c1 = ctl->c1, c3 = ctl->c3;
      const bool active = (int64_t)i < n;
      uint32_t cur[16], nxt[16];
      oc_ld16(tmem + lane_addr + 16u * sub, cur);
      oc_wait16(cur);
      for (uint32_t c = sub; c < uch; c += 4) {
        const bool more = c + 4 < uch;
        if (more) oc_ld16(tmem + lane_addr + 16u * (c + 4), nxt);
        const uint32_t rb = 16u * c;
        if (active && rb < (uint32_t)m) {
          uint8_t* row = xs + rb * 128u;
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            uint8_t* a0 = row + e * 128 + colo[e & 7];
            uint8_t* a1 = row + (e + 1) * 128 + colo[(e + 1) & 7];
            const bool v0 = rb + e < (uint32_t)m, v1 = rb + e + 1 < (uint32_t)m;
            float x0 = 0.0f, x1 = 0.0f;
            if (v0)
              x0 = (bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a0)) +
                    bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a0 + 2 * ch))) +
                   bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a0 + 4 * ch));
            if (v1)
              x1 = (bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a1)) +
                    bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a1 + 2 * ch))) +
                   bf16_to_f32_dev(*reinterpret_cast<uint16_t*>(a1 + 4 * ch));
            const float xn0 = c1 * x0 + c3 * __uint_as_float(cur[e]);
            const float xn1 = c1 * x1 + c3 * __uint_as_float(cur[e + 1]);
            uint32_t w[3];
            oc_split2(xn0, xn1, w);
            if (v0) {
#pragma unroll
              for (int q = 0; q < 3; ++q) *reinterpret_cast<uint16_t*>(a0 + 2 * q * ch) = (uint16_t)w[q];
            }
            if (v1) {
#pragma unroll
              for (int q = 0; q < 3; ++q) *reinterpret_cast<uint16_t*>(a1 + 2 * q * ch) = (uint16_t)(w[q] >> 16);
            }
          }
        }
        if (more) {
          oc_wait16(nxt);
#pragma unroll
          for (int e = 0; e < 16; ++e) cur[e] = nxt[e];
        }
      }
    }
  }
  // everything issued has completed before the CTA frees TMEM
  if (tid == 0 && issued) {
    tc_commit(br.drain);
    mbar_drain(br.drain, 0);
  }
  if (ctl->decision != 1) return;
  // ---- the final iterate's planes to global memory, where the H product and U read them
  uint16_t* dst = tk.xp[k & 1];
  for (uint32_t u = (uint32_t)tid; u < 3u * (uint32_t)m * 16u; u += OC_THREADS) {
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
  br.drain = smem_u32((const void*)&ctl->drain);
  if (threadIdx.x == 0) {
    mbar_init(br.full, 1);
    mbar_init(br.full + 8, 1);
    mbar_init(br.drain, 1);
    ctl->abort = 0;
    ctl->decision = 0;
    const double tol = (tol_dev && *tol_dev > 0) ? *tol_dev : rule.tol;
    const double nn = (double)tk.n;
    ctl->dr.v_tol = tol * tol * nn;
    ctl->dr.stag2 = rule.stagnation * rule.stagnation;
    ctl->dr.v_floor = rule.stag_floor * rule.stag_floor * nn;
    ctl->dr.n_pre = rule.n_pre;
    ctl->dr.max_iter = rule.max_iter;
    ctl->dr.pre_c1 = (float)rule.pre_a;
    ctl->dr.pre_c3 = (float)(-(4.0 / 27.0) * rule.pre_a * rule.pre_a * rule.pre_a);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    oc_fence_async();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32((const void*)&ctl->tmem_base)),
                 "n"(OC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // X_0's three planes into shared memory, zero beyond m x n
  {
    const int64_t m = tk.m, n = tk.n;
    for (uint32_t u = threadIdx.x; u < 3u * mp * 16u; u += OC_THREADS) {
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
  oc_solve<P>(tk, xs, xbase, ch, mp, np, tmem, br, ctl, warp, lane, withhold);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && ctl->decision == 2) {
    atomicOr(&tk.st->err_flags, 1u);
    tk.st->status = ST_TIMEOUT;
    if (err_word) atomicOr(err_word, 1);
  }
  if (warp == 0) {
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
