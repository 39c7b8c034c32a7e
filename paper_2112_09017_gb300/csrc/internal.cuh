// Internal declarations shared by the translation units of libpolar.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/polar.h"

namespace polar {

// Iteration state kept in device memory by a single-solve plan.
// Status values written by device code.
enum : int {
  ST_RUNNING = 0,
  ST_CONVERGED = 1,
  ST_NOT_CONVERGED = 2,
  ST_NONFINITE = 3,
  ST_TIMEOUT = 4,
};

struct DevState {
  double normA;          // ||A||_F
  double inv_sqrt_n;     // 1 / sqrt(n)
  int status;            // ST_*
  int iters;             // updates applied so far (the U = X_iters iterate)
  int planes_next;       // planes of the next product (schedules)
  int hist_len;
  unsigned int err_flags;// device error bits (timeouts)
  int fp8_on;            // FP8 schedule: 1 while the products take E4M3-quantized operands
  float upd_c1, upd_c3;  // the next update is X <- upd_c1 X + upd_c3 X G
  double ring[4];        // r_k at slot k % 4 (stagnation test beyond the history)
  double sym_err;        // ||skew(U^T A)||_F / ||U^T A||_F
  double res_hist[POLAR_HIST];
  unsigned char planes_hist[POLAR_HIST];
};

// Parameters of the stop rule evaluated on the device after every Gram.
struct StopRule {
  double tol;
  double stagnation;
  double stag_floor;
  double switch_residual;
  int max_iter;
  int sched;      // 0: fixed planes, 1: BF16 then BF16X3, 2: FP8 E4M3, then BF16, then BF16X3
  int planes_fixed;
  int n_pre;      // preconditioning steps (Algorithm 1) before the Newton-Schulz steps
  double pre_a;   // their coefficient a = 3 sqrt(3)/2 - s_minus
  double fp8_switch;  // schedule 2: residual below which the FP8 phase ends
};
// Number of Eq. RogueScalar steps lifting s0 to s_minus (the first loop of Algorithm 1).
int precond_steps(double s_minus, double s0);
// Coefficients of update k, X_{k+1} = c1 X_k + c3 X_k G_k: a and -(4/27) a^3 for the preconditioning
// steps of Algorithm 1 (Eq. RogueMatrix), 1.5 and -0.5 after them (Eq. NewtonSchulz); rounded to float32.
__host__ __device__ inline void update_coeffs(const StopRule& rule, int k, float& c1, float& c3) {
  if (k < rule.n_pre) {
    c1 = (float)rule.pre_a;
    c3 = (float)(-(4.0 / 27.0) * rule.pre_a * rule.pre_a * rule.pre_a);
  } else {
    c1 = 1.5f;
    c3 = -0.5f;
  }
}

// Small batched problems solved on one SM each (onchip.cu): X_0's three planes at x0
// (pitch ldp, plane stride xps, as the batched workspace stores them); the final
// iterate's planes go to xp[iters & 1]; the stop rule updates *st.
struct OcTask {
  int64_t m, n, ldp, xps;
  const uint16_t* x0;
  uint16_t* xp[2];
  DevState* st;
};
bool onchip_fits(int64_t m, int64_t n);   // n <= 128, n <= m <= 256
cudaError_t launch_onchip_ns(const OcTask* tasks, int ntasks, const StopRule& rule, const double* tol_dev,
                             int* err_word, int P, cudaStream_t s);

// ---------------------------------------------------------------------------------
// Misc kernels (kernels_misc.cu)
// Frobenius norm: per-block float64 partials, then a fixed-order final sum.
int frob_partials_blocks(int64_t m, int64_t n);
cudaError_t launch_frob_partials(const float* A, int64_t m, int64_t n, int64_t lda, double* partials,
                                 int blocks, cudaStream_t s);
cudaError_t launch_norm_finalize(const double* partials, int nparts, DevState* st, double inv_sqrt_n,
                                 int planes_first, int fp8_first, cudaStream_t s);
// dst = src / ||A||_F (if scale) or src (otherwise); optional float32 copy and BF16 planes.
cudaError_t launch_scale_split(const float* src, int64_t lds, int64_t m, int64_t n, const DevState* st,
                               bool scale, float* dst, int64_t ldd, uint16_t* planes, int64_t ldp,
                               int64_t plane_stride, int nplanes, cudaStream_t s);
// Residual finalize: fixed-order sum of Gram partials, stop rule, schedule.
cudaError_t launch_residual_finalize(const double* partials, int nparts, DevState* st, StopRule rule,
                                     int k, int planes_this, cudaStream_t s);
// H = (C + C^T)/2 from C = U^T A (n x n, ldc), and partials of ||skew C||^2, ||C||^2.
cudaError_t launch_symmetrize(const float* C, int64_t ldc, int64_t n, float* H, int64_t ldh,
                              double* partials, int blocks, cudaStream_t s);
int symmetrize_blocks(int64_t n);
cudaError_t launch_sym_finalize(const double* partials, int blocks, DevState* st, cudaStream_t s);
// C[j][i] = C[i][j] for every i < j (n x n float32), or the same on `nplanes` BF16 planes.
cudaError_t launch_mirror_f32(float* C, int64_t ldc, int64_t n, const DevState* st, cudaStream_t s);
cudaError_t launch_mirror_planes(uint16_t* P, int64_t ldp, int64_t plane_stride, int nplanes, int64_t n,
                                 const DevState* st, const int* planes_dyn, cudaStream_t s);
// The strictly lower triangle of an n x n symmetric matrix's three BF16 planes from its upper
// triangle (after a Gram launch, which writes the upper one); skipped unless st is RUNNING.
cudaError_t launch_mirror_planes3(uint16_t* P, int64_t ldp, int64_t plane_stride, int64_t n, const DevState* st,
                                  cudaStream_t s);
cudaError_t launch_copy2d(const float* src, int64_t lds, float* dst, int64_t ldd, int64_t m, int64_t n,
                          cudaStream_t s);
cudaError_t launch_split_flat(const float* x, int64_t count, int nplanes, uint16_t* out, cudaStream_t s);
// X_0 = A^T / st->normA as three BF16 planes (A rows x cols, X_0 cols x rows).
cudaError_t launch_transpose_scale_split(const float* A, int64_t lda, int64_t rows, int64_t cols, const DevState* st,
                                         uint16_t* planes, int64_t ldp, int64_t plane_stride, cudaStream_t s);
// Newton-Schulz inverse (Algorithm 2): coefficients 2, -1, and the growing-tolerance test after step k.
cudaError_t launch_inverse_init(DevState* st, cudaStream_t s);
cudaError_t launch_inverse_finalize(const double* partials, int npairs, DevState* st, int k, int max_iter,
                                    cudaStream_t s);
// dst = plane_0 + plane_1 + plane_2 (the FP32 value the three BF16 planes encode exactly)
cudaError_t launch_planes_to_f32(const uint16_t* planes, int64_t ldp, int64_t plane_stride, int64_t m, int64_t n,
                                 float* dst, int64_t ldd, cudaStream_t s);
// FP8 E4M3 with a power-of-two scale per 128 x 128 tile (the smallest s with amax / s <= 448):
// every entry becomes s * e4m3_rne(x / s), written as one BF16 plane (exact). Source: the
// three planes of an iterate (pitch ldp, plane stride sps); skipped unless st->fp8_on.
cudaError_t launch_quantize_e4m3_planes(const uint16_t* src, int64_t ldp, int64_t sps, int64_t rows, int64_t cols,
                                        uint16_t* dst, int64_t ldd, const DevState* st, cudaStream_t s);
// FP8 operands for the E4M3 tensor-core products: the E4M3 codes of every 128 x 128 tile of src (float32, or
// three BF16 planes with from_planes) divided by that tile's power of two, and the exponents, optionally
// transposed (codes and exponent table both); with uni, also one byte per 128-row block of the codes (per
// column block of src when transposed): 1 when every exponent of that block is the same. Skipped unless
// st is null or RUNNING in its FP8 phase.
cudaError_t launch_quantize_codes(const void* src, bool from_planes, int64_t lds, int64_t sps, int64_t rows,
                                  int64_t cols, uint8_t* codes, int64_t ldc, int8_t* exps, int64_t lde, bool transpose,
                                  uint8_t* uni, const DevState* st, cudaStream_t s);
// The same from a float32 matrix into a float32 matrix (library service).
cudaError_t launch_quantize_e4m3_f32(const float* src, int64_t lds, int64_t rows, int64_t cols, float* dst,
                                     int64_t ldd, cudaStream_t s);
// Clenshaw set-up (n x n): planes of s1 (alpha_map S + beta_map I) + s0 I, S the symmetric matrix
// whose upper triangle is A's, each value rounded once to float32 and split into `nplanes` planes.
cudaError_t launch_cheb_affine_split(const float* A, int64_t lda, int64_t n, double alpha_map, double beta_map,
                                     double s1, double s0, uint16_t* planes, int64_t ldp, int64_t plane_stride,
                                     int nplanes, cudaStream_t s);

// ---------------------------------------------------------------------------------
// SIMT float32 GEMM / SYRK (gemm_simt.cu)
enum SimtEpi : int { SIMT_EPI_STORE = 0, SIMT_EPI_NS = 1, SIMT_EPI_GRAM = 2 };

struct SimtArgs {
  int64_t M, N, K;
  const float* A; int64_t lda; int a_kmajor;   // a_kmajor: A stored M x K (row-major); else K x M
  const float* B; int64_t ldb; int b_kmajor;   // b_kmajor: B stored N x K; else K x N
  float* C; int64_t ldc;
  float alpha, beta;
  const float* Xold; int64_t ldx;              // NS epilogue: C = 1.5 Xold - 0.5 acc
  double* partials;                            // GRAM epilogue: one float64 per tile
  const DevState* st;                          // skip if st && st->status != RUNNING
  int triangular;                              // SYRK: upper-triangle tiles + mirror store
};
cudaError_t launch_simt_gemm(const SimtArgs& a, int epi, cudaStream_t s);
int simt_gram_tiles(int64_t n);

// ---------------------------------------------------------------------------------
// tcgen05 split-BF16 GEMM / SYRK (gemm_tc.cu)
enum TcEpi : int { TC_EPI_STORE = 0, TC_EPI_NS = 1, TC_EPI_GRAM = 2, TC_EPI_PLANES = 3, TC_EPI_NS_STEP = 4,
                   TC_EPI_CLENSHAW = 5 };

struct TcOperand {
  const uint16_t* planes;  // plane p at planes + p * plane_stride (elements)
  int64_t rows, cols;      // stored matrix shape (row-major)
  int64_t ld;              // elements; multiple of 8
  int64_t plane_stride;    // elements; multiple of 8
  int kmajor;              // 1: stored (MN x K), K contiguous; 0: stored (K x MN), MN contiguous
};

struct TcArgs {
  int64_t M, N, K;
  TcOperand a, b;
  int nplanes;             // 1..3: planes stored per operand (and passes: 1, 3, 6)
  int epi;                 // TcEpi
  int triangular;          // SYRK upper-triangle tiles + mirror store
  float* C; int64_t ldc; float alpha, beta;      // STORE; CLENSHAW: alpha acc + beta Z + diag I
  float diag;                                     // CLENSHAW: added on the diagonal
  const uint16_t* x_planes; int64_t ldxp; int64_t x_plane_stride;  // NS: three planes of X_k; CLENSHAW: of Z
  uint16_t* out_planes; int64_t ldo; int64_t out_plane_stride; int out_nplanes; // NS/GRAM plane output
  double* partials;                               // GRAM residual partials; NS_STEP step-size pairs, per tile and warp
                                                  // the pair (sum (x' - x)^2, sum x'^2)
  DevState* st;                                   // skip when not RUNNING; error flags
  int slice_stages;                               // k-stages per promoted slice (0: library default)
  const int* planes_dyn;                          // if non-null: passes use min(*planes_dyn, nplanes)
                                                  // planes (schedules); outputs keep out_nplanes;
                                                  // the launch does nothing while *planes_dyn <= 0
  int withhold_tma;                               // test hook: the producer issues no copies, so the
                                                  // bounded waits expire (set by the launcher)
  const int8_t* a_exp;                            // FP8 operands: power-of-two exponents of A's 128 x 128 tiles,
  const int8_t* b_exp;                            // a_exp[M block * lde_a + K block], b_exp[N block * lde_b +
  int64_t lde_a, lde_b;                           // K block]; each 128-K slice is promoted times 2^(ea + eb)
  const uint8_t* a_uni;                           // FP8: per 128-row block of A (of B), 1 when all its K blocks
  const uint8_t* b_uni;                           // share one exponent; a tile whose blocks all do accumulates
  int fp8_run;                                    // fp8_run K blocks per slice under its one scale
  unsigned int* err_out;                          // without st: word set to 1 when a bounded wait expired
                                                  // (null: the device-wide word read by tc_take_error)
};
cudaError_t launch_tc_gemm(const TcArgs& a, cudaStream_t s);
// The same on FP8 E4M3 codes (one byte per element; a.a and a.b K-major with plane_stride unused,
// ld in bytes a multiple of 16) with a.a_exp, a.b_exp giving every 128 x 128 tile's power-of-two
// scale: tcgen05.mma.kind::f8f6f4, one 128-K slice per promotion, each scaled exactly. Epilogues
// STORE, GRAM and NS.
cudaError_t launch_tc_gemm_fp8(const TcArgs& a, cudaStream_t s);
// Reads and clears the device-wide word that launches without st and err_out set on a
// timeout; waits for `s` and writes the old value to *out.
cudaError_t tc_take_error(cudaStream_t s, unsigned int* out);

// Grouped launch: many independent problems in one persistent launch. Each problem
// has an entry (its TMA maps and its own TcArgs: sizes, epilogue pointers, status);
// the tile table lists (problem, tile row, tile column, tile index within the problem)
// in the order CTAs take them. Tiles of problems whose status is not RUNNING are skipped.
struct TcGroupEntry {
  alignas(128) unsigned char map_a[128];  // CUtensorMap
  alignas(128) unsigned char map_b[128];
  TcArgs args;                            // per problem: M, N, K, epilogue fields, st
};
struct TcTile {
  int32_t prob, bi, bj, local;
};
struct TcGroupLaunch {
  int nplanes, epi, a_mn, b_mn;           // shared by every problem of the launch
  const TcTile* tiles;                    // device
  int64_t ntiles;
  const TcGroupEntry* entries;            // device
  const int* done;                        // device flag: nonzero -> the launch returns at once
  int* err;                               // device word: set to 1 when a bounded wait expired
  const int* planes_dyn;
  int slice_stages;
  int withhold_tma;                       // test hook, as in TcArgs
  int tile_n;                             // 256 (0 also) or 128: the tiles' width; the table must match
};
cudaError_t launch_tc_gemm_grouped(const TcGroupLaunch& g, cudaStream_t s);
// Fills entry->map_a / map_b for the operands of entry->args (host side).
bool tc_make_entry_maps(TcGroupEntry* entry);
// Residual partial slots a GRAM launch of an n x n triangle with `planes` planes writes (the CTA-pair
// and single-CTA forms tile it differently), and the largest of the two (for allocation).
int tc_gram_partials(int64_t n, int planes);
int tc_gram_partials_max(int64_t n);
bool tc_available();

// Host helpers defined in polar_api.cu and shared with the other entry points.
bool device_is_sm103(int* sms = nullptr);         // the current device is an sm_103 GPU
int resolve_precision(int prec, int64_t n);       // POLAR_AUTO -> BF16X6 for n >= 256, FP32 below
int product_planes(int prec);                     // BF16 planes of a product mode (0: FP32 or not a product mode)

// ---------------------------------------------------------------------------------
// Batched solves (batched.cu)
struct BatchedPlan;
polar_status_t batched_create(BatchedPlan** out, int count, const int64_t* m, const int64_t* n,
                              const polar_options_t& opt, int prec);
polar_status_t batched_run(BatchedPlan* bp, const float* const* A, float* const* U, float* const* H, double tol,
                           int32_t* iters_dev, double* resid_dev, cudaStream_t s);
void batched_destroy(BatchedPlan* bp);
size_t batched_workspace_bytes(const BatchedPlan* bp);

}  // namespace polar
