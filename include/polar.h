/*
 * polar.h - C ABI of the GB300 Newton-Schulz polar factorisation library (libpolar.so).
 *
 * The method (arXiv 2112.09017, Sec. III.D): the polar decomposition A = U H of an
 * m x n matrix A, m >= n (Eq. PolarDecomp), with U having orthonormal columns and H
 * symmetric positive semi-definite, is the fixed point of the Newton-Schulz iteration
 * X_{k+1} = X_k (3 I - X_k^T X_k) / 2 (Eq. NewtonSchulz) started from the Frobenius-
 * scaled X_0 = A / ||A||_F (Sec. III.D and the first step of Algorithm 1). This library
 * runs that iteration until ||X_k^T X_k - I||_F / sqrt(n) <= tol and returns U = X_k and
 * H = (U^T A + A^T U) / 2 (Algorithm 1, "Ensure": H = U^H A).
 *
 * Conventions shared by every entry point:
 *  - Matrices are row-major float32. Element (i, j) of a matrix with leading dimension ld
 *    is at p[i * ld + j]; ld >= number of columns.
 *  - Matrix pointers are DEVICE pointers (cudaMalloc'd or equivalent) unless stated.
 *    The caller owns every buffer it passes; the library never frees them.
 *  - `stream` is a cudaStream_t cast to void* (NULL = the legacy default stream).
 *  - Entry points return a polar_status_t and never abort, exit or trap. Invalid
 *    arguments are rejected before any device work with POLAR_EINVAL.
 *  - The library has no CPU fallback: without a usable sm_103 device every call that
 *    needs one returns POLAR_ECUDA.
 *  - A plan may be used by one host thread / one stream at a time.
 */
#ifndef POLAR_H
#define POLAR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define POLAR_API __attribute__((visibility("default")))
#else
#define POLAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  POLAR_OK = 0,
  POLAR_NOT_CONVERGED = 1,  /* stopped by stagnation or max_iter; U, H of the last iterate returned */
  POLAR_EINVAL = -1,        /* bad argument: null pointer, m < n, n < 1, ld too small, aliasing */
  POLAR_ENOMEM = -2,        /* device allocation failed or workspace above ws_limit */
  POLAR_ECUDA = -3,         /* CUDA runtime/driver error, or no sm_103 device */
  POLAR_ENONFINITE = -4,    /* ||A||_F is zero, Inf or NaN, or a residual became non-finite */
  POLAR_ETIMEOUT = -5,      /* a bounded device-side wait expired (kernel returned early) */
  POLAR_ENOTSUP = -6        /* precision mode or shape not implemented by the library */
} polar_status_t;

/* How the matrix products of the iteration are computed.
 *   FP32      every product in float32 FFMA on the SIMT cores (the plain form)
 *   BF16X6    float32 operands split into 3 BF16 planes, 6 tensor-core passes
 *             (hi*hi, hi*mid, mid*hi, hi*lo, lo*hi, mid*mid), float32 accumulation
 *   BF16X3    2 BF16 planes, 3 passes (hi*hi, hi*lo, lo*hi)
 *   BF16      1 BF16 plane, 1 pass
 *   SCHED_BF16_THEN_X3   BF16 while the residual is above switch_residual, then BF16X3
 *   SCHED_FP8_BF16_X3    while the residual is above fp8_switch_residual, both products take FP8 E4M3
 *             operands with a power-of-two scale per 128 x 128 tile (computed on the BF16 tensor-core
 *             path, where such values are exact); then as SCHED_BF16_THEN_X3 (single plans only)
 *   AUTO      BF16X6 for n >= 256, FP32 below
 * The schedules do not meet the 5e-6 orthogonality / backward-error target: a product made at a
 * precision u leaves a backward error of about u that the iteration never removes; BF16X6 (or the
 * FP32 form) does. TF32X3 is reserved and returns POLAR_ENOTSUP. */
typedef enum {
  POLAR_FP32 = 0,
  POLAR_BF16X6 = 1,
  POLAR_TF32X3 = 2,
  POLAR_BF16X3 = 3,
  POLAR_SCHED_BF16_THEN_X3 = 4,
  POLAR_SCHED_FP8_BF16_X3 = 5,
  POLAR_AUTO = 6,
  POLAR_BF16 = 7
} polar_precision_t;

typedef void* polar_stream_t;
typedef struct polar_plan_s* polar_plan_t;

/* One entry of a batched plan's tuning table: the problems with n_lo <= n <= n_hi and
 * aspect_lo <= m / n <= aspect_hi use the tile width and slice length given here (the first
 * matching entry wins; problems no entry matches use the plan's options). Written by the
 * library's autotuner (paper_2112_09017_gb300/autotune.py), which times the choices per size
 * bucket and keeps the fastest whose orthogonality and backward errors stay within 5e-6. */
typedef struct {
  int64_t n_lo, n_hi;
  double aspect_lo, aspect_hi;
  int tile_n;        /* width of the grouped launches' output tiles: 128 or 256 (0: the plan's) */
  int slice_stages;  /* 32-element k-stages accumulated per promoted slice, 1..8 (0: the library's) */
} polar_tune_entry_t;

typedef struct {
  double tol;              /* stop when ||X^T X - I||_F / sqrt(n) <= tol; <= 0 means 1e-6 */
  int max_iter;            /* maximum number of updates; <= 0 means 100 */
  int prec;                /* a polar_precision_t */
  double stagnation;       /* stop (NOT_CONVERGED) when r_k > stagnation * r_{k-2} ... ; <= 0 means 0.7 */
  double stag_floor;       /* ... and r_k < stag_floor; <= 0 means 1e-4 */
  double switch_residual;  /* schedules: residual below which the finer precision is used; <= 0 means 1e-2 */
  size_t ws_limit;         /* maximum workspace bytes a plan may allocate; 0 = no limit */
  int profile;             /* nonzero: time every Gram and update launch with CUDA events (info) */
  int precondition;        /* nonzero: Algorithm 1 - first the steps X <- a X (I - 4/27 a^2 X^T X),
                              a = 3 sqrt(3)/2 - s_minus (Eqs. a_def, RogueMatrix), as many as lift s0 to
                              s_minus under Eq. RogueScalar; then Newton-Schulz. Stop tests start after them */
  double s_minus;          /* preconditioning threshold; <= 0 means 0.1 */
  double s0;               /* estimate of the smallest singular value of A / ||A||_F; <= 0 means 2^-23 */
  double fp8_switch_residual; /* SCHED_FP8_BF16_X3: residual below which the FP8 phase ends; <= 0 means 0.5 */
  int batched_tile_n;      /* batched plans: width of the grouped launches' output tiles, 256 (0 means 256:
                              one epilogue group, as in the single solve) or 128 (two epilogue groups on
                              alternate tiles, so that one tile's output step can overlap the next tile's
                              products; measured no faster on the 4096-problem configuration) */
  int small_onchip;        /* batched plans with a fixed plane count: nonzero (the default) solves every
                              problem with n <= 128 and m <= 256 in one CTA that keeps X, G and the
                              accumulators on its SM for the whole loop; 0 sends them through the
                              grouped tile kernels like the others */
  const polar_tune_entry_t* tune; /* batched plans: a tuning table of n_tune entries (host memory, read
                              only during plan creation), or NULL */
  int n_tune;
} polar_options_t;

#define POLAR_HIST 128

typedef struct {
  int status;                 /* the polar_status_t of the run */
  int iters;                  /* Newton-Schulz updates applied (U = X_iters) */
  int prec;                   /* precision mode used */
  int hist_len;               /* number of valid entries in res_hist / planes_hist */
  double residual;            /* ||U^T U - I||_F / sqrt(n) as measured at the returned U (float32 Gram) */
  double normA_F;             /* ||A||_F (float64 accumulation) */
  double sym_err;             /* ||skew(U^T A)||_F / ||U^T A||_F */
  float ms_total;             /* device time of the whole solve (CUDA events), milliseconds */
  int launches;               /* kernels this run enqueued (including ones that found the run stopped) */
  int n_gram, n_update;       /* profile: Gram and update launches that did work */
  int n_precond;              /* preconditioning steps among the iters updates (0 without preconditioning) */
  float ms_gram, ms_update;   /* profile: their summed device time (CUDA events), milliseconds */
  double res_hist[POLAR_HIST];         /* r_k for k = 0 .. hist_len-1 */
  unsigned char planes_hist[POLAR_HIST];/* BF16 planes of the Gram at step k (0 = FP32 SIMT) */
} polar_info_t;

/* Fill *o with the defaults listed in polar_options_t (prec = POLAR_BF16X6). */
POLAR_API void polar_default_options(polar_options_t* o);

/* Human-readable name of a status code (static string). */
POLAR_API const char* polar_status_string(polar_status_t s);

/* Create a plan for m x n problems (m >= n >= 1) and allocate its device workspace
 * on the current CUDA device. o may be NULL for defaults. The plan owns the workspace
 * until polar_plan_destroy. Errors: EINVAL (shape, prec), ENOMEM (allocation or
 * ws_limit), ENOTSUP (reserved prec), ECUDA.
 * Paper: Algorithm 1, "Require" (an M x N matrix with M >= N; real here) and Sec. III.D
 * (the Frobenius scaling X_0 = A / ||A||_F the plan's first kernels compute). */
POLAR_API polar_status_t polar_plan_create(polar_plan_t* plan, int64_t m, int64_t n, const polar_options_t* o);

/* Bytes of device workspace the plan holds. */
POLAR_API size_t polar_plan_workspace_bytes(polar_plan_t plan);

/* Polar factorisation of A (m x n, lda >= n), writing U (m x n, ldu >= n) and
 * H (n x n, ldh >= n). tol <= 0 uses the plan's tolerance. A is read-only; U and H
 * must not overlap A or each other (EINVAL). Work is enqueued on `stream`; the call
 * returns after the solve has finished and *info (may be NULL) is filled.
 * Returns OK, NOT_CONVERGED (U, H of the last iterate are still written),
 * ENONFINITE (U and H untouched), ETIMEOUT or ECUDA.
 * Paper: Sec. III.D, Eqs. NewtonSchulz and PolarDecomp, Algorithm 1. */
POLAR_API polar_status_t polar_run(polar_plan_t plan, const float* A, int64_t lda, float* U, int64_t ldu,
                         float* H, int64_t ldh, double tol, polar_info_t* info, polar_stream_t stream);

/* Plan for `count` independent problems of sizes (m[i], n[i]) (host arrays), m[i] >= n[i] >= 1.
 * Problem i's matrices are packed row-major (ld = n[i]). Allocates every problem's workspace,
 * builds the tile tables and captures the whole solve in a CUDA graph. Errors: EINVAL (count,
 * sizes, prec), ENOTSUP (FP32, TF32X3 or the FP8 schedule), ENOMEM, ECUDA.
 * Paper: Sec. III.D and Algorithm 1, applied to each problem on its own (the paper solves one
 * matrix at a time; running many uneven problems through shared launches is this library's). */
POLAR_API polar_status_t polar_batched_plan_create(polar_plan_t* plan, int count, const int64_t* m,
                                         const int64_t* n, const polar_options_t* o);

/* Polar factorisation of every problem of a batched plan. A, U, H are HOST arrays of
 * `count` DEVICE pointers (A[i]: m_i x n_i, U[i]: m_i x n_i, H[i]: n_i x n_i, all packed);
 * the arrays must hold exactly the plan's count and the matrices the plan's sizes (the
 * library cannot check either: a short array or a smaller matrix is read or written out of
 * bounds). iters_dev[i] (int32) and resid_dev[i] (float64) are device arrays receiving each
 * problem's update count and final residual; either may be NULL. Stream-asynchronous:
 * returns after enqueueing; per-problem status goes to the device arrays (a problem
 * that did not converge reports iters = -1 - updates; a device timeout INT32_MIN).
 * Paper: Sec. III.D, Eq. NewtonSchulz and Algorithm 1 per problem (see the plan above). */
POLAR_API polar_status_t polar_batched_run(polar_plan_t plan, const float* const* A, float* const* U,
                                 float* const* H, double tol, int32_t* iters_dev, double* resid_dev,
                                 polar_stream_t stream);

/* polar_run with HOST buffers: A (m x n, lda >= n), U (m x n, ldu >= n) and H (n x n, ldh >= n) are
 * host pointers (pinned memory gives full copy speed; pageable memory works). The plan copies A
 * into device memory it owns (allocated on the first call, counted in its workspace and ws_limit),
 * runs the solve of polar_run on `stream` and copies U and H back; it returns after U and H are in
 * host memory. Same statuses as polar_run; U and H are written only for OK and NOT_CONVERGED.
 * Paper: Sec. III.D, Eqs. NewtonSchulz and PolarDecomp, Algorithm 1. */
POLAR_API polar_status_t polar_run_host(polar_plan_t plan, const float* A, int64_t lda, float* U, int64_t ldu,
                                        float* H, int64_t ldh, double tol, polar_info_t* info,
                                        polar_stream_t stream);

POLAR_API void polar_plan_destroy(polar_plan_t plan);

/* Device-side status of the stream-asynchronous products (polar_gemm, polar_syrk,
 * polar_gemm_noalloc): waits for the work enqueued on `stream`, then reads and clears the
 * current device's timeout word. Returns POLAR_ETIMEOUT when a tensor-core launch of one of
 * those calls on this device had a bounded wait expire since the previous call (its C is then
 * not fully written; the kernel returned on its own and the context stays usable), POLAR_ECUDA
 * on a CUDA error or without an sm_103 device, else POLAR_OK. The word is shared by every
 * stream of the device. The paper has no counterpart: error reporting of this library. */
POLAR_API polar_status_t polar_async_status(polar_stream_t stream);

/* C = alpha * op(A) op(B) + beta * C, op(X) = X or X^T (trans != 0), with op(A) M x K and
 * op(B) K x N, in precision `prec` (FP32, BF16, BF16X3, BF16X6, AUTO: BF16X6 when min(M, N) >= 256,
 * else FP32; the schedules return EINVAL). beta == 0 does not read C. Stream-asynchronous: a
 * device-side timeout of the product is reported by polar_async_status. Split planes live in a
 * library-owned per-device scratch buffer that grows on demand (so this call may allocate). The
 * building block of every step of the iteration (Eq. NewtonSchulz is two such products). */
POLAR_API polar_status_t polar_gemm(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                          const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                          float* C, int64_t ldc, int prec, polar_stream_t stream);

/* C = alpha * Q(op(A)) Q(op(B)) + beta * C on the FP8 tensor cores (tcgen05.mma.kind::f8f6f4), op(A) M x K and
 * op(B) K x N as in polar_gemm. Q rounds every 128 x 128 tile of its operand (tiles counted from element
 * (0, 0) of op(X)) to FP8 E4M3 with a power-of-two scale, exactly as polar_quantize_e4m3; the products of
 * the codes accumulate in float32, one 128-element block of K at a time, and each block is multiplied by
 * its two tiles' scales (exact) and added with round-to-nearest. beta == 0 does not read C. Stream-
 * asynchronous (timeouts: polar_async_status); may allocate scratch as polar_gemm. Row-major device
 * buffers, caller-owned; lda, ldb, ldc in elements. Returns POLAR_EINVAL for negative sizes, a null C,
 * null operands with K > 0 or leading dimensions below the row lengths; POLAR_ENOTSUP without tcgen05
 * FP8 support; POLAR_ENOMEM when the scratch cannot grow; POLAR_ECUDA on a CUDA error; M == 0 or
 * N == 0 is a no-op and K == 0 gives C = beta * C. The operands of the FP8 phase of
 * POLAR_SCHED_FP8_BF16_X3. The paper has no counterpart: FP8 schedules are this library's. */
POLAR_API polar_status_t polar_gemm_fp8(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                                        const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                        float* C, int64_t ldc, polar_stream_t stream);

/* C = alpha * A^T A + beta * C for A k x n (lda >= n), C n x n (ldc >= n), storing the full
 * symmetric C (each off-diagonal pair computed once and mirrored). The Gram matrix
 * X^T X of Eq. NewtonSchulz. Stream-asynchronous (timeouts: polar_async_status); may allocate
 * scratch as polar_gemm. */
POLAR_API polar_status_t polar_syrk(int64_t n, int64_t k, float alpha, const float* A, int64_t lda, float beta,
                          float* C, int64_t ldc, int prec, polar_stream_t stream);

/* Split `count` float32 values into `planes` (1..3) BF16 planes with round-to-nearest-even
 * on each remainder: out[p * count + i] holds plane p of X[i] as a BF16 bit pattern.
 * X and out are device pointers. The operand encoding of the split-precision products
 * (Sec. II: FP32 products emulated on BF16 multipliers). Stream-asynchronous. */
POLAR_API polar_status_t polar_split_bf16(const float* X, int64_t count, int planes, uint16_t* out,
                                polar_stream_t stream);

/* Newton-Schulz matrix inverse (Algorithm 2) of A (rows x cols, rows >= cols, full column rank,
 * lda >= cols) into X (cols x rows, ldx >= rows): X_0 = A^T / ||A A^T||_F, then
 * X <- X (2I - A X) (the X A = I branch; X tends to the pseudo-inverse, A^{-1} when square) until
 * ||X' - X||_F / ||X'||_F <= u 2^k after update k (u = 2^-24: the paper's doubling tolerance), or
 * max_iter (<= 0 means 100) updates. The doubling tolerance ends the loop within ~25 updates, so for
 * ill-conditioned A (kappa >~ 1e2) the result is an approximate inverse. prec: BF16X6, BF16X3 or BF16
 * (products on the tensor cores with the same promotion as polar_run); FP32 -> ENOTSUP. Device pointers;
 * allocates its workspace for the call and returns after the result is in X. *iters (updates applied)
 * and *delta (the last relative change) may be NULL. Returns OK, NOT_CONVERGED (max_iter reached),
 * ENONFINITE (A zero or non-finite), EINVAL, ENOMEM, ENOTSUP or ECUDA.
 * Paper: Sec. III.D, Algorithm 2. */
POLAR_API polar_status_t polar_ns_inverse(const float* A, int64_t rows, int64_t cols, int64_t lda, float* X,
                                          int64_t ldx, int prec, int max_iter, int32_t* iters, double* delta,
                                          polar_stream_t stream);

/* The degree + 1 first-kind Chebyshev points of [a, b] (b > a, degree >= 0), host memory:
 * x[j] = (a + b)/2 + (b - a)/2 cos(pi (j + 1/2) / (degree + 1)), j = 0..degree.
 * Paper: Sec. III.D, the matrix-function paragraph after Algorithm 2. Returns OK or EINVAL. */
POLAR_API polar_status_t polar_chebyshev_nodes(double a, double b, int degree, double* x);

/* Coefficients c_0..c_degree of the Chebyshev interpolant through g[j] = g(x[j]) at the points of
 * polar_chebyshev_nodes (host memory): c_k = 2/(degree + 1) sum_j g[j] cos(k pi (j + 1/2)/(degree + 1)),
 * c_0 halved, so that p(x) = sum_k c_k T_k((2x - a - b)/(b - a)). Returns OK, EINVAL or ENONFINITE. */
POLAR_API polar_status_t polar_chebyshev_fit(const double* g, int degree, double* coef);

/* Chebyshev matrix function F = sum_k coef[k] T_k(T), T = (2A - (a + b) I)/(b - a), of a real symmetric
 * n x n matrix A whose eigenvalues lie in [a, b] (the matrix function of Eq. MatFuncEig through the
 * polynomial of Eq. EigenvaluePolynomial), by Clenshaw summation:
 *   B_{d+1} = B_{d+2} = 0, B_k = c_k I + 2 T B_{k+1} - B_{k+2} (k = d..1), F = c_0 I + T B_1 - B_2,
 * degree - 1 matrix products for degree >= 2 on the tensor cores (split BF16 as polar_run; each product
 * of two polynomials in T is symmetric, so only its upper-triangle tiles are computed and mirrored).
 * Only the upper triangle of A (lda >= n) is read; F (ldf >= n) is written in full and is exactly
 * symmetric. A and F are device pointers, coef host memory (degree + 1 finite values, rounded to
 * float32 where they enter the device arithmetic). prec: BF16X6, BF16X3 or BF16; FP32 -> ENOTSUP.
 * Allocates its workspace for the call and returns after F is written. Returns OK, EINVAL, ENOMEM,
 * ENOTSUP, ETIMEOUT or ECUDA. Paper: Sec. III.D, the matrix-function paragraph after Algorithm 2. */
POLAR_API polar_status_t polar_chebyshev(const float* A, int64_t n, int64_t lda, double a, double b,
                                         const double* coef, int degree, float* F, int64_t ldf, int prec,
                                         polar_stream_t stream);

/* FP8 E4M3 quantization as the FP8 schedule applies it, for checking: each 128 x 128 tile of X
 * (rows x cols, ldx >= cols, float32, device) is scaled by s = 2^t, the smallest power of two with
 * max|x| <= 448 s over the tile (s = 1 for a zero tile), rounded to E4M3 with round-to-nearest-even
 * and saturation at +-448, and scaled back: Y = s * e4m3(X / s) (float32, ldy >= cols; may equal X
 * with ldy = ldx). Stream-asynchronous. The paper has no counterpart: its schedules are configuration
 * choices of this library. Returns OK, EINVAL or ECUDA. */
POLAR_API polar_status_t polar_quantize_e4m3(const float* X, int64_t rows, int64_t cols, int64_t ldx, float* Y,
                                             int64_t ldy, polar_stream_t stream);

/* Size of the static device array behind polar_gemm_noalloc (32 MiB). */
#define POLAR_NOALLOC_SCRATCH_BYTES (32u << 20)

/* polar_gemm without any device allocation. The paper has no counterpart: this is a
 * library-service entry point. polar_gemm keeps the BF16 planes of its operands in a
 * scratch buffer it grows with cudaMalloc/cudaFree; callers that must not allocate
 * (device memory owned entirely by another allocator, or a latency-critical loop that
 * cannot take the synchronisation a cudaFree implies) use this variant, whose planes
 * live in one static device array of POLAR_NOALLOC_SCRATCH_BYTES per GPU, held from
 * the first use on that GPU until the process exits.
 * Arguments, layouts, precision resolution (AUTO included), device check, results and
 * timeout reporting (polar_async_status) are those of polar_gemm. The BF16 modes need
 * P * (round64(rows_A * round64(cols_A)) + round64(rows_B * round64(cols_B))) * 2 bytes of the
 * array, P the mode's planes (3, 2, 1), rows and cols the stored shapes of A and B, round64
 * rounding up to a multiple of 64: each row is padded to 64 elements and each plane to a multiple
 * of 64 elements. A larger problem returns POLAR_ENOMEM before any device work. FP32 needs no
 * scratch. The first call on a device looks up the
 * array's address there (cudaGetSymbolAddress with that device current), so make it
 * before any stream capture. All calls share the array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams or threads) race. */
POLAR_API polar_status_t polar_gemm_noalloc(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha,
                                            const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                            float* C, int64_t ldc, int prec, polar_stream_t stream);

/* Number of SMs and compute capability of the current device; ECUDA without one. */
POLAR_API polar_status_t polar_device_query(int* sm_count, int* cc_major, int* cc_minor);

#ifdef __cplusplus
}
#endif

#endif /* POLAR_H */
