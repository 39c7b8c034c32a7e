// Batched Newton-Schulz polar factorisations: many independent problems of uneven
// sizes advance in lockstep iterations, each with its own stop rule, in grouped
// launches (one persistent tensor-core launch per product for all problems), the
// whole sequence captured once in a CUDA graph.
//
// Per iteration k (Sec. III.D, Eq. NewtonSchulz, applied to every problem):
//   grouped Gram  G_p = X_p^T X_p (BF16 split, triangle tiles stored with their
//                 mirror, residual partials)
//   finalize      r_p = ||G_p - I||_F / sqrt(n_p), the stop rule per problem
//   grouped update X_p <- 1.5 X_p - 0.5 X_p G_p for problems still running
// Problems that stopped keep their iterate; a launch returns at once when none runs.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "device_util.cuh"
#include "internal.cuh"
#include "stop_rule.cuh"

namespace polar {

namespace {

constexpr int kThreads = 256;
constexpr int kStored = 3;       // BF16 planes kept for X and G
constexpr int kEpiWarps = 8;     // residual partials per Gram tile (one per epilogue warp)
constexpr int kBM = 128;         // tile rows (the tile width is per problem)

int64_t up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Per-problem layout of the workspace (device memory).
struct BMeta {
  int64_t m, n;
  uint16_t* xp[2];   // three planes each, pitch ldp, plane stride xps
  uint16_t* gp;      // three planes, pitch ldp, plane stride gps
  uint16_t* ap;      // P planes of A
  float* C;          // n x n, U^T A
  double* partials;  // Gram partials: ntiles_gram * kEpiWarps
  int64_t ldp, xps, gps;
  int ntiles_gram;
  int pad;
};

struct BShared {     // device: shared state of the batch
  int done;          // no problem is running
  int err;           // a bounded wait of a grouped launch expired
  double tol;
  int running[POLAR_HIST + 8];  // problems still running after the finalize of step k
};

__device__ __forceinline__ double block_sum_b(double v) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// ||A_p||_F (fixed order) and the initial state of every problem: one block per problem.
__global__ void b_norm_kernel(const float* const* __restrict__ A, const BMeta* __restrict__ meta,
                              DevState* __restrict__ st, BShared* sh, int planes_first) {
  const int p = blockIdx.x;
  const BMeta& mt = meta[p];
  const float* a = A[p];
  double acc = 0.0;
  const int64_t total = mt.m * mt.n, step = blockDim.x;
  int64_t i = threadIdx.x;
  // eight loads in flight per thread; each thread still adds its elements in increasing order
  for (; i + 7 * step < total; i += 8 * step) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = a[i + j * step];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc = fma((double)v[j], (double)v[j], acc);
  }
  for (; i < total; i += step) {
    const double v = (double)a[i];
    acc = fma(v, v, acc);
  }
  const double t = block_sum_b(acc);
  if (threadIdx.x == 0) {
    DevState& s = st[p];
    const double nrm = sqrt(t);
    s.normA = nrm;
    s.inv_sqrt_n = 1.0 / sqrt((double)mt.n);
    s.iters = 0;
    s.hist_len = 0;
    s.err_flags = 0;
    s.planes_next = planes_first;
    s.sym_err = 0.0;
    s.upd_c1 = 1.5f;
    s.upd_c3 = -0.5f;
    for (int i = 0; i < 4; ++i) s.ring[i] = 0.0;
    s.status = (isfinite(nrm) && nrm > 0.0) ? ST_RUNNING : ST_NONFINITE;
    if (p == 0) {
      sh->done = 0;
      sh->err = 0;
    }
  }
}

// A block's threads as rows of `tw` lanes (the smallest of 32, 64, 128, 256 that covers n, at
// most 256), so that narrow problems keep every thread busy: thread t takes column t % tw of
// row t / tw of each group of blockDim / tw rows.
__device__ __forceinline__ int row_lanes(int64_t n) { return n > 128 ? 256 : n > 64 ? 128 : n > 32 ? 64 : 32; }

// X_0 = A_p / ||A_p||_F as three planes, and P planes of A_p (for H). Grid (count, Y).
__global__ void b_scale_split_kernel(const float* const* __restrict__ A, const BMeta* __restrict__ meta,
                                     const DevState* __restrict__ st, int P) {
  const int p = blockIdx.x;
  if (st[p].status != ST_RUNNING) return;
  const BMeta& mt = meta[p];
  const float* a = A[p];
  const float s = (float)st[p].normA;
  const int tw = row_lanes(mt.n), rpb = (int)blockDim.x / tw;
  for (int64_t r = (int64_t)blockIdx.y * rpb + threadIdx.x / tw; r < mt.m; r += (int64_t)gridDim.y * rpb) {
    for (int64_t c = threadIdx.x % tw; c < mt.n; c += tw) {
      const float av = a[r * mt.n + c];
      const int64_t o = r * mt.ldp + c;
      uint16_t q[3];
      split_planes_dev<3>(__fdiv_rn(av, s), q);
      for (int i = 0; i < kStored; ++i) mt.xp[0][i * mt.xps + o] = q[i];
      split_planes_dev<3>(av, q);
      for (int i = 0; i < P; ++i) mt.ap[i * mt.xps + o] = q[i];
    }
  }
}

// The stop rule of step k for every running problem: one warp per problem, its
// Gram partials summed in a fixed order.
__global__ void b_finalize_kernel(const BMeta* __restrict__ meta, DevState* __restrict__ st, BShared* sh,
                                  int count, StopRule rule, int k) {
  if (sh->done) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= count) return;
  DevState& s = st[warp];
  if (s.status != ST_RUNNING) return;
  const BMeta& mt = meta[warp];
  const int np = mt.ntiles_gram * kEpiWarps;
  double acc = 0.0;
  for (int i = lane; i < np; i += 32) acc += mt.partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane != 0) return;
  const double r = sqrt(acc) * s.inv_sqrt_n;
  const double tol = sh->tol > 0 ? sh->tol : rule.tol;
  float c1, c3;
  if (batched_step_rule(s, rule, tol, r, k >= 2 ? s.ring[(k - 2) & 3] : 0.0, k, s.planes_next, c1, c3)) {
    s.planes_next = rule.sched == 1 ? (r > rule.switch_residual ? 1 : 2) : rule.planes_fixed;
    atomicAdd(&sh->running[k < POLAR_HIST + 8 ? k : POLAR_HIST + 7], 1);
  }
}

// The lower triangle of every running problem's G planes from the upper one the grouped Gram
// wrote. Grid (count, Y): block (p, y) takes problem p's 64 x 64 upper blocks y, y + Y, ...
__global__ void b_mirror_kernel(const BMeta* __restrict__ meta, const DevState* __restrict__ st, const BShared* sh) {
  if (sh->done) return;
  const int p = blockIdx.x;
  if (st[p].status != ST_RUNNING) return;
  const BMeta& mt = meta[p];
  __shared__ uint16_t tile[3 * 64 * 66];
  mirror3_tiles(mt.gp, mt.ldp, mt.gps, mt.n, blockIdx.y, gridDim.y, tile);
}

__global__ void b_check_done_kernel(BShared* sh, int k) {
  if (sh->done) return;
  const int slot = k < POLAR_HIST + 8 ? k : POLAR_HIST + 7;
  if (sh->running[slot] == 0 || sh->err) sh->done = 1;
  sh->running[slot] = 0;  // ready for the next use of this slot
}

// The H entries of each problem point at the planes of its own final iterate.
__global__ void b_select_h_kernel(const TcGroupEntry* __restrict__ h2, TcGroupEntry* __restrict__ h,
                                  const DevState* __restrict__ st, int count) {
  const int p = blockIdx.x;
  if (p >= count) return;
  const int par = st[p].iters & 1;
  const uint4* src = reinterpret_cast<const uint4*>(&h2[2 * p + par]);
  uint4* dst = reinterpret_cast<uint4*>(&h[p]);
  for (int i = threadIdx.x; i < (int)(sizeof(TcGroupEntry) / 16); i += blockDim.x) dst[i] = src[i];
}

__device__ __forceinline__ bool finished_ok(int status) {
  return status == ST_CONVERGED || status == ST_NOT_CONVERGED;
}

// U_p = the planes of its final iterate summed (exact). Grid (count, Y), rows strided.
__global__ void b_u_kernel(const BMeta* __restrict__ meta, const DevState* __restrict__ st, float* const* __restrict__ U,
                           const BShared* sh) {
  const int p = blockIdx.x;
  if (sh->err || !finished_ok(st[p].status)) return;
  const BMeta& mt = meta[p];
  const uint16_t* X = mt.xp[st[p].iters & 1];
  float* u = U[p];
  const int tw = row_lanes(mt.n), rpb = (int)blockDim.x / tw;
  for (int64_t r = (int64_t)blockIdx.y * rpb + threadIdx.x / tw; r < mt.m; r += (int64_t)gridDim.y * rpb)
    for (int64_t c = threadIdx.x % tw; c < mt.n; c += tw) {
      const int64_t o = r * mt.ldp + c;
      u[r * mt.n + c] = (bf16_to_f32_dev(X[o]) + bf16_to_f32_dev(X[mt.xps + o])) + bf16_to_f32_dev(X[2 * mt.xps + o]);
    }
}

// H_p = (C_p + C_p^T) / 2 through 32 x 32 shared tiles. Grid (count, Y), tiles strided.
__global__ void b_h_kernel(const BMeta* __restrict__ meta, const DevState* __restrict__ st, float* const* __restrict__ H,
                           const BShared* sh) {
  const int p = blockIdx.x;
  if (sh->err || !finished_ok(st[p].status)) return;
  const BMeta& mt = meta[p];
  __shared__ float ta[32][33];
  __shared__ float tb[32][33];
  const int64_t n = mt.n, nt = (n + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float* h = H[p];
  for (int64_t t = blockIdx.y; t < nt * nt; t += gridDim.y) {
    const int64_t i0 = (t / nt) * 32, j0 = (t % nt) * 32;
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t i = i0 + yy, j = j0 + tx;
      ta[yy][tx] = (i < n && j < n) ? mt.C[i * n + j] : 0.0f;
      const int64_t i2 = j0 + yy, j2 = i0 + tx;
      tb[yy][tx] = (i2 < n && j2 < n) ? mt.C[i2 * n + j2] : 0.0f;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t i = i0 + yy, j = j0 + tx;
      if (i < n && j < n) h[i * n + j] = 0.5f * (ta[yy][tx] + tb[tx][yy]);
    }
  }
}

// Per-problem results: updates applied (negative, -1 - updates, when not converged;
// INT32_MIN after a device timeout) and the final residual.
__global__ void b_results_kernel(const DevState* __restrict__ st, const BShared* sh, int count, int32_t* iters_dev,
                                 double* resid_dev) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const DevState& s = st[p];
  const int it = s.iters;
  int32_t code = s.status == ST_CONVERGED ? it : -1 - it;
  double r = (it < POLAR_HIST && it < s.hist_len) ? s.res_hist[it] : s.ring[it & 3];
  if (!finished_ok(s.status)) r = NAN;
  if (sh->err) {
    code = INT32_MIN;
    r = NAN;
  }
  iters_dev[p] = code;
  resid_dev[p] = r;
}

}  // namespace

struct BatchedPlan {
  int count = 0;
  int P = 3;
  int prec = POLAR_BF16X6;
  polar_options_t opt{};
  std::vector<int64_t> m, n;
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  BMeta* meta_d = nullptr;
  DevState* st_d = nullptr;
  BShared* sh_d = nullptr;
  const float** A_tab = nullptr;   // device tables of the caller's pointers (per run)
  float** U_tab = nullptr;
  float** H_tab = nullptr;
  void** host_tab = nullptr;       // pinned staging: A, U, H pointers, then tol
  TcGroupEntry* gram_e[2] = {nullptr, nullptr};  // per parity of k
  TcGroupEntry* upd_e[2] = {nullptr, nullptr};
  TcGroupEntry* h2_e = nullptr;    // [count][2] candidates
  TcGroupEntry* h_e = nullptr;     // selected
  // tile tables of the grouped Gram and update launches, one per tile width ([0]: 256, [1]: 128);
  // each problem's width is its tuning entry's, else options.batched_tile_n
  TcTile* gram_t[2] = {nullptr, nullptr};
  TcTile* upd_t[2] = {nullptr, nullptr};
  int64_t n_gram_t[2] = {0, 0}, n_upd_t[2] = {0, 0};
  TcTile* h_t = nullptr;           // U^T A for H: 256-wide tiles for every problem
  int64_t n_h_t = 0;
  std::vector<int> tile_n_of, slice_of;   // per problem: tile width, k-stages per slice (0: default)
  OcTask* oc_tasks = nullptr;      // problems solved on one SM each (largest first)
  int n_oc = 0;
  int32_t* iters_scratch = nullptr;
  double* resid_scratch = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t* iters_cap = nullptr;    // the graph writes results here; copied out per run
  double* resid_cap = nullptr;
  cudaEvent_t tab_ev = nullptr;    // the last upload of host_tab has been consumed
};

namespace {

polar_status_t b_alloc(BatchedPlan* b, size_t bytes, void** out) {
  if (b->opt.ws_limit && b->ws_bytes + bytes > b->opt.ws_limit) return POLAR_ENOMEM;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return POLAR_ENOMEM;
  }
  b->allocs.push_back(p);
  b->ws_bytes += bytes;
  *out = p;
  return POLAR_OK;
}


// Tile table: problems by decreasing work, each problem's tiles contiguous
// (neighbouring CTAs of a wave share that problem's operand panels in L2).
void build_tiles(const std::vector<int>& order, const std::vector<int64_t>& rows, const std::vector<int64_t>& cols,
                 bool tri, int tile_n, std::vector<TcTile>& out, std::vector<int>* ntiles_of) {
  out.clear();
  for (int p : order) {
    const int64_t tm = (rows[p] + kBM - 1) / kBM, tn = (cols[p] + tile_n - 1) / tile_n;
    int local = 0;
    if (tri) {
      for (int64_t bj = 0; bj < tn; ++bj)
        for (int64_t bi = 0; bi < std::min((bj + 1) * tile_n / kBM, tm); ++bi)   // rows that reach the diagonal
          out.push_back({p, (int32_t)bi, (int32_t)bj, local++});
    } else {
      for (int64_t bi = 0; bi < tm; ++bi)
        for (int64_t bj = 0; bj < tn; ++bj) out.push_back({p, (int32_t)bi, (int32_t)bj, local++});
    }
    if (ntiles_of) (*ntiles_of)[p] = local;
  }
}

TcOperand opnd(const uint16_t* planes, int64_t rows, int64_t cols, int64_t ld, int64_t stride, int kmajor) {
  TcOperand o;
  o.planes = planes; o.rows = rows; o.cols = cols; o.ld = ld; o.plane_stride = stride; o.kmajor = kmajor;
  return o;
}

polar_status_t enqueue_all(BatchedPlan* b, cudaStream_t s) {
  const int count = b->count;
  StopRule rule;
  rule.tol = b->opt.tol;
  rule.stagnation = b->opt.stagnation;
  rule.stag_floor = b->opt.stag_floor;
  rule.switch_residual = b->opt.switch_residual;
  rule.max_iter = b->opt.max_iter;
  rule.sched = b->prec == POLAR_SCHED_BF16_THEN_X3 ? 1 : 0;
  rule.planes_fixed = b->P;
  rule.n_pre = b->opt.precondition ? precond_steps(b->opt.s_minus, b->opt.s0) : 0;
  rule.pre_a = 1.5 * sqrt(3.0) - b->opt.s_minus;
  const int planes_first = rule.sched ? 1 : b->P;
#define BK_(x) do { if ((x) != cudaSuccess) return POLAR_ECUDA; } while (0)
  b_norm_kernel<<<count, kThreads, 0, s>>>(b->A_tab, b->meta_d, b->st_d, b->sh_d, planes_first);
  BK_(cudaGetLastError());
  b_scale_split_kernel<<<dim3(count, 16), kThreads, 0, s>>>(b->A_tab, b->meta_d, b->st_d, b->P);
  BK_(cudaGetLastError());
  // the small problems' whole loops, one SM each; the grouped launches below skip them
  BK_(launch_onchip_ns(b->oc_tasks, b->n_oc, rule, &b->sh_d->tol, &b->sh_d->err, b->P, s));
  // the grouped loop, unless every problem was solved on-chip; one launch per tile width in use
  const int widths[2] = {256, 128};
  for (int k = 0; k <= b->opt.max_iter && b->n_gram_t[0] + b->n_gram_t[1] > 0; ++k) {
    for (int w = 0; w < 2; ++w) {
      if (!b->n_gram_t[w]) continue;
      TcGroupLaunch g{};
      g.tile_n = widths[w];
      g.nplanes = b->P;
      g.epi = TC_EPI_GRAM; g.a_mn = 1; g.b_mn = 1;
      g.tiles = b->gram_t[w]; g.ntiles = b->n_gram_t[w]; g.entries = b->gram_e[k & 1];
      g.done = &b->sh_d->done;
      g.err = &b->sh_d->err;
      BK_(launch_tc_gemm_grouped(g, s));
    }
    b_finalize_kernel<<<(count * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(b->meta_d, b->st_d, b->sh_d, count,
                                                                                   rule, k);
    BK_(cudaGetLastError());
    b_check_done_kernel<<<1, 1, 0, s>>>(b->sh_d, k);
    BK_(cudaGetLastError());
    if (k == b->opt.max_iter) break;
    b_mirror_kernel<<<dim3(count, 8), kThreads, 0, s>>>(b->meta_d, b->st_d, b->sh_d);
    BK_(cudaGetLastError());
    for (int w = 0; w < 2; ++w) {
      if (!b->n_upd_t[w]) continue;
      TcGroupLaunch u{};
      u.tile_n = widths[w];
      u.nplanes = b->P;
      u.epi = TC_EPI_NS; u.a_mn = 0; u.b_mn = 1;
      u.tiles = b->upd_t[w]; u.ntiles = b->n_upd_t[w]; u.entries = b->upd_e[k & 1];
      u.done = &b->sh_d->done;
      u.err = &b->sh_d->err;
      BK_(launch_tc_gemm_grouped(u, s));
    }
  }
  // H: C_p = U_p^T A_p for every problem, from the planes of its final iterate
  b_select_h_kernel<<<count, 64, 0, s>>>(b->h2_e, b->h_e, b->st_d, count);
  BK_(cudaGetLastError());
  TcGroupLaunch h{};
  h.tile_n = 256;
  h.nplanes = b->P;
  h.epi = TC_EPI_STORE; h.a_mn = 1; h.b_mn = 1;
  h.tiles = b->h_t; h.ntiles = b->n_h_t; h.entries = b->h_e;
  h.done = nullptr;
  h.err = &b->sh_d->err;
  BK_(launch_tc_gemm_grouped(h, s));
  b_u_kernel<<<dim3(count, 8), kThreads, 0, s>>>(b->meta_d, b->st_d, b->U_tab, b->sh_d);
  BK_(cudaGetLastError());
  b_h_kernel<<<dim3(count, 8), kThreads, 0, s>>>(b->meta_d, b->st_d, b->H_tab, b->sh_d);
  BK_(cudaGetLastError());
  b_results_kernel<<<(count + 127) / 128, 128, 0, s>>>(b->st_d, b->sh_d, count, b->iters_cap, b->resid_cap);
  BK_(cudaGetLastError());
#undef BK_
  return POLAR_OK;
}

}  // namespace

polar_status_t batched_create(BatchedPlan** out, int count, const int64_t* m, const int64_t* n,
                              const polar_options_t& opt, int prec) {
  BatchedPlan* b = new (std::nothrow) BatchedPlan();
  if (!b) return POLAR_ENOMEM;
  b->count = count;
  b->opt = opt;
  b->prec = prec;
  b->P = prec == POLAR_BF16X6 ? 3 : (prec == POLAR_BF16X3 || prec == POLAR_SCHED_BF16_THEN_X3) ? 2 : 1;
  b->m.assign(m, m + count);
  b->n.assign(n, n + count);
  // per-problem tile width and slice length: the first matching tuning entry, else the options
  const int tile_default = opt.batched_tile_n == 128 ? 128 : 256;
  b->tile_n_of.assign(count, tile_default);
  b->slice_of.assign(count, 0);
  for (int p = 0; p < count && opt.tune; ++p) {
    const double aspect = (double)m[p] / (double)n[p];
    for (int e = 0; e < opt.n_tune; ++e) {
      const polar_tune_entry_t& te = opt.tune[e];
      if (n[p] < te.n_lo || n[p] > te.n_hi || aspect < te.aspect_lo || aspect > te.aspect_hi) continue;
      if (te.tile_n == 128 || te.tile_n == 256) b->tile_n_of[p] = te.tile_n;
      if (te.slice_stages >= 1 && te.slice_stages <= 8) b->slice_of[p] = te.slice_stages;
      break;
    }
  }
  polar_status_t r = POLAR_OK;
  void* v = nullptr;
  auto fail = [&](polar_status_t e) {
    batched_destroy(b);
    return e;
  };
  // per-problem layout, packed into one allocation per buffer kind
  std::vector<BMeta> meta(count);
  size_t x_bytes = 0, g_bytes = 0, a_bytes = 0, c_bytes = 0;
  std::vector<int> ntg(count, 0);
  for (int p = 0; p < count; ++p) {
    BMeta& mt = meta[p];
    mt.m = m[p];
    mt.n = n[p];
    mt.ldp = up(n[p], 64);
    mt.xps = up(m[p] * mt.ldp, 64);
    mt.gps = up(n[p] * mt.ldp, 64);
    x_bytes += (size_t)kStored * mt.xps * 2;
    g_bytes += (size_t)kStored * mt.gps * 2;
    a_bytes += (size_t)b->P * mt.xps * 2;
    c_bytes += (size_t)up(n[p] * n[p], 64) * 4;
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return (double)m[x] * n[x] * n[x] > (double)m[y] * n[y] * n[y]; });
  // problems that fit one SM run their loop there (fixed plane counts only); the rest go
  // through the grouped tile kernels, which all problems share for H
  const bool oc_ok = opt.small_onchip != 0 && prec != POLAR_SCHED_BF16_THEN_X3;
  std::vector<int> order_tc, order_oc;
  for (int p : order) (oc_ok && onchip_fits(m[p], n[p]) ? order_oc : order_tc).push_back(p);
  std::vector<int> order_w[2];
  for (int p : order_tc) order_w[b->tile_n_of[p] == 256 ? 0 : 1].push_back(p);
  std::vector<TcTile> gram_t[2], upd_t[2], h_t;
  for (int w = 0; w < 2; ++w) {
    build_tiles(order_w[w], b->n, b->n, true, w == 0 ? 256 : 128, gram_t[w], &ntg);
    build_tiles(order_w[w], b->m, b->n, false, w == 0 ? 256 : 128, upd_t[w], nullptr);
  }
  build_tiles(order, b->n, b->n, false, 256, h_t, nullptr);
  size_t part_count = 0;
  for (int p = 0; p < count; ++p) part_count += (size_t)ntg[p] * kEpiWarps;

  uint8_t *xb[2], *gb, *ab, *cb;
  for (int i = 0; i < 2; ++i) {
    if ((r = b_alloc(b, x_bytes, &v)) != POLAR_OK) return fail(r);
    xb[i] = (uint8_t*)v;
    if (cudaMemset(v, 0, x_bytes) != cudaSuccess) return fail(POLAR_ECUDA);
  }
  if ((r = b_alloc(b, g_bytes, &v)) != POLAR_OK) return fail(r);
  gb = (uint8_t*)v;
  if (cudaMemset(v, 0, g_bytes) != cudaSuccess) return fail(POLAR_ECUDA);
  if ((r = b_alloc(b, a_bytes, &v)) != POLAR_OK) return fail(r);
  ab = (uint8_t*)v;
  if (cudaMemset(v, 0, a_bytes) != cudaSuccess) return fail(POLAR_ECUDA);
  if ((r = b_alloc(b, c_bytes, &v)) != POLAR_OK) return fail(r);
  cb = (uint8_t*)v;
  if ((r = b_alloc(b, std::max<size_t>(part_count, 1) * 8, &v)) != POLAR_OK) return fail(r);
  double* partials = (double*)v;
  size_t xo = 0, go = 0, ao = 0, co = 0, po = 0;
  for (int p = 0; p < count; ++p) {
    BMeta& mt = meta[p];
    mt.xp[0] = (uint16_t*)(xb[0] + xo);
    mt.xp[1] = (uint16_t*)(xb[1] + xo);
    mt.gp = (uint16_t*)(gb + go);
    mt.ap = (uint16_t*)(ab + ao);
    mt.C = (float*)(cb + co);
    mt.partials = partials + po;
    mt.ntiles_gram = ntg[p];
    xo += (size_t)kStored * mt.xps * 2;
    go += (size_t)kStored * mt.gps * 2;
    ao += (size_t)b->P * mt.xps * 2;
    co += (size_t)up(mt.n * mt.n, 64) * 4;
    po += (size_t)ntg[p] * kEpiWarps;
  }
  if ((r = b_alloc(b, sizeof(BMeta) * count, &v)) != POLAR_OK) return fail(r);
  b->meta_d = (BMeta*)v;
  if (cudaMemcpy(b->meta_d, meta.data(), sizeof(BMeta) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(POLAR_ECUDA);
  if ((r = b_alloc(b, sizeof(DevState) * count, &v)) != POLAR_OK) return fail(r);
  b->st_d = (DevState*)v;
  if (cudaMemset(v, 0, sizeof(DevState) * count) != cudaSuccess) return fail(POLAR_ECUDA);
  if (!order_oc.empty()) {
    std::vector<OcTask> tasks;
    for (int p : order_oc) {
      OcTask t;
      t.m = meta[p].m; t.n = meta[p].n; t.ldp = meta[p].ldp; t.xps = meta[p].xps;
      t.x0 = meta[p].xp[0];
      t.xp[0] = meta[p].xp[0];
      t.xp[1] = meta[p].xp[1];
      t.st = b->st_d + p;
      tasks.push_back(t);
    }
    if ((r = b_alloc(b, sizeof(OcTask) * tasks.size(), &v)) != POLAR_OK) return fail(r);
    b->oc_tasks = (OcTask*)v;
    b->n_oc = (int)tasks.size();
    if (cudaMemcpy(v, tasks.data(), sizeof(OcTask) * tasks.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(POLAR_ECUDA);
  }
  if ((r = b_alloc(b, sizeof(BShared), &v)) != POLAR_OK) return fail(r);
  b->sh_d = (BShared*)v;
  if (cudaMemset(v, 0, sizeof(BShared)) != cudaSuccess) return fail(POLAR_ECUDA);
  if ((r = b_alloc(b, sizeof(void*) * 3 * count, &v)) != POLAR_OK) return fail(r);
  b->A_tab = (const float**)v;
  b->U_tab = (float**)v + count;
  b->H_tab = (float**)v + 2 * count;
  if (cudaMallocHost((void**)&b->host_tab, sizeof(void*) * 3 * count + 16) != cudaSuccess) return fail(POLAR_ENOMEM);
  if ((r = b_alloc(b, sizeof(int32_t) * count, &v)) != POLAR_OK) return fail(r);
  b->iters_cap = (int32_t*)v;
  if ((r = b_alloc(b, sizeof(double) * count, &v)) != POLAR_OK) return fail(r);
  b->resid_cap = (double*)v;

  // group entries: Gram and update for both parities of k, H candidates per parity
  std::vector<TcGroupEntry> ge(count), ue(count), he(2 * (size_t)count);
  for (int par = 0; par < 2; ++par) {
    for (int p = 0; p < count; ++p) {
      const BMeta& mt = meta[p];
      TcGroupEntry& g = ge[p];
      memset(&g, 0, sizeof(g));
      TcArgs& a = g.args;
      a.M = mt.n; a.N = mt.n; a.K = mt.m;
      a.a = opnd(mt.xp[par], mt.m, mt.n, mt.ldp, mt.xps, 0);
      a.b = a.a;
      a.nplanes = b->P;
      a.epi = TC_EPI_GRAM; a.triangular = 1;
      a.out_planes = mt.gp; a.ldo = mt.ldp; a.out_plane_stride = mt.gps; a.out_nplanes = kStored;
      a.partials = mt.partials;
      a.st = b->st_d + p;
      a.slice_stages = b->slice_of[p];
      if (!tc_make_entry_maps(&g)) return fail(POLAR_ECUDA);
      TcGroupEntry& u = ue[p];
      memset(&u, 0, sizeof(u));
      TcArgs& c = u.args;
      c.M = mt.m; c.N = mt.n; c.K = mt.n;
      c.a = opnd(mt.xp[par], mt.m, mt.n, mt.ldp, mt.xps, 1);
      c.b = opnd(mt.gp, mt.n, mt.n, mt.ldp, mt.gps, 0);
      c.nplanes = b->P;
      c.epi = TC_EPI_NS;
      c.x_planes = mt.xp[par]; c.ldxp = mt.ldp; c.x_plane_stride = mt.xps;
      c.out_planes = mt.xp[par ^ 1]; c.ldo = mt.ldp; c.out_plane_stride = mt.xps; c.out_nplanes = kStored;
      c.st = b->st_d + p;
      c.slice_stages = b->slice_of[p];
      if (!tc_make_entry_maps(&u)) return fail(POLAR_ECUDA);
      TcGroupEntry& h = he[2 * (size_t)p + par];
      memset(&h, 0, sizeof(h));
      TcArgs& d = h.args;
      d.M = mt.n; d.N = mt.n; d.K = mt.m;
      d.a = opnd(mt.xp[par], mt.m, mt.n, mt.ldp, mt.xps, 0);
      d.b = opnd(mt.ap, mt.m, mt.n, mt.ldp, mt.xps, 0);
      d.nplanes = b->P;
      d.epi = TC_EPI_STORE;
      d.C = mt.C; d.ldc = mt.n; d.alpha = 1.f; d.beta = 0.f;
      d.st = nullptr;
      if (!tc_make_entry_maps(&h)) return fail(POLAR_ECUDA);
    }
    if ((r = b_alloc(b, sizeof(TcGroupEntry) * count, &v)) != POLAR_OK) return fail(r);
    b->gram_e[par] = (TcGroupEntry*)v;
    if ((r = b_alloc(b, sizeof(TcGroupEntry) * count, &v)) != POLAR_OK) return fail(r);
    b->upd_e[par] = (TcGroupEntry*)v;
    if (cudaMemcpy(b->gram_e[par], ge.data(), sizeof(TcGroupEntry) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->upd_e[par], ue.data(), sizeof(TcGroupEntry) * count, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(POLAR_ECUDA);
  }
  if ((r = b_alloc(b, sizeof(TcGroupEntry) * 2 * count, &v)) != POLAR_OK) return fail(r);
  b->h2_e = (TcGroupEntry*)v;
  if (cudaMemcpy(b->h2_e, he.data(), sizeof(TcGroupEntry) * 2 * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(POLAR_ECUDA);
  if ((r = b_alloc(b, sizeof(TcGroupEntry) * count, &v)) != POLAR_OK) return fail(r);
  b->h_e = (TcGroupEntry*)v;
  auto put_tiles = [&](const std::vector<TcTile>& t, TcTile** dst, int64_t* nt) -> polar_status_t {
    polar_status_t rr = b_alloc(b, sizeof(TcTile) * std::max<size_t>(t.size(), 1), &v);
    if (rr != POLAR_OK) return rr;
    *dst = (TcTile*)v;
    *nt = (int64_t)t.size();
    if (!t.empty() && cudaMemcpy(v, t.data(), sizeof(TcTile) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return POLAR_ECUDA;
    return POLAR_OK;
  };
  for (int w = 0; w < 2; ++w) {
    if ((r = put_tiles(gram_t[w], &b->gram_t[w], &b->n_gram_t[w])) != POLAR_OK) return fail(r);
    if ((r = put_tiles(upd_t[w], &b->upd_t[w], &b->n_upd_t[w])) != POLAR_OK) return fail(r);
  }
  if ((r = put_tiles(h_t, &b->h_t, &b->n_h_t)) != POLAR_OK) return fail(r);

  // capture the whole sequence once; each run uploads its pointer tables and replays it
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(POLAR_ECUDA);
  if (cudaEventCreateWithFlags(&b->tab_ev, cudaEventDisableTiming) != cudaSuccess) return fail(POLAR_ECUDA);
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return fail(POLAR_ECUDA);
  polar_status_t er = enqueue_all(b, b->cap);
  cudaGraph_t gph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->cap, &gph);
  if (er != POLAR_OK || ce != cudaSuccess || !gph) {
    if (gph) cudaGraphDestroy(gph);
    cudaGetLastError();
    b->graph = nullptr;  // the run enqueues the sequence directly instead
  } else {
    b->graph = gph;
    if (cudaGraphInstantiate(&b->exec, gph, 0) != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
    }
  }
  *out = b;
  return POLAR_OK;
}

polar_status_t batched_run(BatchedPlan* b, const float* const* A, float* const* U, float* const* H, double tol,
                           int32_t* iters_dev, double* resid_dev, cudaStream_t s) {
  const int count = b->count;
  // the previous run's upload from the pinned table must have been consumed
  if (cudaEventSynchronize(b->tab_ev) != cudaSuccess) return POLAR_ECUDA;
  for (int p = 0; p < count; ++p) {
    b->host_tab[p] = (void*)A[p];
    b->host_tab[count + p] = (void*)U[p];
    b->host_tab[2 * count + p] = (void*)H[p];
  }
  BShared shh;
  memset(&shh, 0, sizeof(shh));
  if (cudaMemcpyAsync(b->A_tab, b->host_tab, sizeof(void*) * 3 * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return POLAR_ECUDA;
  // tol is read by the finalize kernel from the shared block (0: the plan's tolerance)
  double* tol_pinned = reinterpret_cast<double*>(b->host_tab + 3 * count);
  *tol_pinned = tol > 0 ? tol : 0.0;
  if (cudaMemcpyAsync(&b->sh_d->tol, tol_pinned, sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return POLAR_ECUDA;
  if (cudaEventRecord(b->tab_ev, s) != cudaSuccess) return POLAR_ECUDA;
  if (b->exec) {
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return POLAR_ECUDA;
  } else {
    polar_status_t r = enqueue_all(b, s);
    if (r != POLAR_OK) return r;
  }
  if (iters_dev &&
      cudaMemcpyAsync(iters_dev, b->iters_cap, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return POLAR_ECUDA;
  if (resid_dev &&
      cudaMemcpyAsync(resid_dev, b->resid_cap, sizeof(double) * count, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return POLAR_ECUDA;
  return POLAR_OK;
}

void batched_destroy(BatchedPlan* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->tab_ev) cudaEventDestroy(b->tab_ev);
  for (void* p : b->allocs) cudaFree(p);
  if (b->host_tab) cudaFreeHost(b->host_tab);
  delete b;
}

size_t batched_workspace_bytes(const BatchedPlan* b) { return b ? b->ws_bytes : 0; }

}  // namespace polar
