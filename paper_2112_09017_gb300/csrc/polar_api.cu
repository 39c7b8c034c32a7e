// C ABI of libpolar.so: plans, the single-solve iteration driver, batched solves,
// and the general products. The iteration (Sec. III.D, Eq. NewtonSchulz,
// Algorithm 1 with the residual stop rule) runs entirely on the device; the host
// only enqueues kernels and reads a small status block between chunks.
#include <cuda.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

using namespace polar;

namespace {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return POLAR_ECUDA;  \
  } while (0)

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

constexpr int kStoredPlanes = 3;  // BF16 planes kept for X and G' on the tensor-core path

int planes_of(int prec) {
  switch (prec) {
    case POLAR_BF16X6: return 3;
    case POLAR_BF16X3: return 2;
    case POLAR_BF16: return 1;
    case POLAR_SCHED_BF16_THEN_X3: return 2;  // workspace for the finer phase
    case POLAR_SCHED_FP8_BF16_X3: return 2;
    default: return 0;
  }
}

bool device_ok(int* sms = nullptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int major = 0, minor = 0, count = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (sms) *sms = count;
  return major == 10 && minor == 3;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  uintptr_t x0 = (uintptr_t)a, x1 = x0 + na, y0 = (uintptr_t)b, y1 = y0 + nb;
  return x0 < y1 && y0 < x1;
}

// Per-device scratch for polar_gemm / polar_syrk plane splits.
struct Scratch {
  std::mutex mu;
  void* ptr = nullptr;
  size_t bytes = 0;
};
Scratch g_scratch[64];

polar_status_t scratch_get(size_t bytes, void** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return POLAR_ECUDA;
  Scratch& s = g_scratch[dev];
  std::lock_guard<std::mutex> lk(s.mu);
  if (s.bytes < bytes) {
    if (s.ptr) {
      CK(cudaDeviceSynchronize());
      cudaFree(s.ptr);
      s.ptr = nullptr;
      s.bytes = 0;
    }
    if (cudaMalloc(&s.ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return POLAR_ENOMEM;
    }
    s.bytes = bytes;
  }
  *out = s.ptr;
  return POLAR_OK;
}

}  // namespace

namespace polar {
bool device_is_sm103(int* sms) { return device_ok(sms); }
int resolve_precision(int prec, int64_t n) { return prec == POLAR_AUTO ? (n >= 256 ? POLAR_BF16X6 : POLAR_FP32) : prec; }
int product_planes(int prec) {
  return prec == POLAR_BF16X6 ? 3 : prec == POLAR_BF16X3 ? 2 : prec == POLAR_BF16 ? 1 : 0;
}
}  // namespace polar

struct polar_plan_s {
  bool batched = false;
  int64_t m = 0, n = 0;
  polar_options_t opt{};
  int prec = POLAR_BF16X6;
  int P = 0;  // BF16 planes (0: FP32 SIMT path)
  int sms = 0;
  // workspace
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  float* hostA = nullptr;  // polar_run_host: device copies of A, U, H (allocated on first use)
  float* hostU = nullptr;
  float* hostH = nullptr;
  float* X[2] = {nullptr, nullptr};  // FP32 path: double buffer; BF16 path: X[0] in place
  int64_t ldx = 0;
  float* G = nullptr;  // FP32 Gram, and C = U^T A at the end (both paths)
  int64_t ldg = 0;
  uint16_t* Xp[2] = {nullptr, nullptr};  // BF16 planes of X (double buffer)
  uint16_t* Gp = nullptr;                // BF16 planes of G
  uint16_t* Ap = nullptr;                // BF16 planes of A (for H)
  uint8_t* Xq = nullptr;                 // FP8 schedule: E4M3 codes of X_k (m x n, for the update), of X_k^T
  uint8_t* XqT = nullptr;                // (n x m, for the Gram) and of G (n x n), rows padded to 16 bytes,
  uint8_t* Gq = nullptr;                 // and the exponents of their 128 x 128 tiles
  int8_t* eX = nullptr;
  int8_t* eXT = nullptr;
  int8_t* eG = nullptr;
  uint8_t* uX = nullptr;                 // per 128-row block of those codes: one exponent along K
  uint8_t* uXT = nullptr;
  uint8_t* uG = nullptr;
  int64_t kpm = 0, kpn = 0;              // code row pitches: m and n rounded up to 16
  int64_t ldp = 0;                       // plane row pitch (elements)
  int64_t xps = 0, gps = 0;              // plane strides (elements)
  double* partials = nullptr;
  int nparts = 0;
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
  cudaEvent_t ev_chunk[2] = {nullptr, nullptr};
  // bookkeeping of one run
  int launches = 0;
  struct Prof { cudaEvent_t a, b; int kind, k; };  // kind 0: Gram, 1: update
  std::vector<Prof> prof;
  size_t prof_used = 0;
  // batched
  int count = 0;
  BatchedPlan* bp = nullptr;
  std::vector<polar_plan_t> subplans;
};

extern "C" {

void polar_default_options(polar_options_t* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->max_iter = 100;
  o->prec = POLAR_BF16X6;
  o->stagnation = 0.7;
  o->stag_floor = 1e-4;
  o->switch_residual = 1e-2;
  o->ws_limit = 0;
  o->profile = 0;
  o->precondition = 0;
  o->s_minus = 0.1;
  o->s0 = 0.0;
  o->small_onchip = 1;
  o->fp8_switch_residual = 0.5;
}

const char* polar_status_string(polar_status_t s) {
  switch (s) {
    case POLAR_OK: return "ok";
    case POLAR_NOT_CONVERGED: return "not converged (stagnation or max_iter)";
    case POLAR_EINVAL: return "invalid argument";
    case POLAR_ENOMEM: return "out of device memory or above ws_limit";
    case POLAR_ECUDA: return "CUDA error or no sm_103 device";
    case POLAR_ENONFINITE: return "input norm or residual is zero or non-finite";
    case POLAR_ETIMEOUT: return "a bounded device wait expired";
    case POLAR_ENOTSUP: return "not supported by the library";
  }
  return "unknown status";
}

polar_status_t polar_device_query(int* sm_count, int* cc_major, int* cc_minor) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return POLAR_ECUDA; }
  int a = 0, b = 0, c = 0;
  if (cudaDeviceGetAttribute(&a, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&c, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return POLAR_ECUDA;
  }
  if (sm_count) *sm_count = a;
  if (cc_major) *cc_major = b;
  if (cc_minor) *cc_minor = c;
  return POLAR_OK;
}

}  // extern "C"

namespace {

void normalize_options(polar_options_t& o) {
  if (!(o.tol > 0)) o.tol = 1e-6;
  if (o.max_iter <= 0) o.max_iter = 100;
  if (!(o.stagnation > 0)) o.stagnation = 0.7;
  if (!(o.stag_floor > 0)) o.stag_floor = 1e-4;
  if (!(o.switch_residual > 0)) o.switch_residual = 1e-2;
  if (!(o.s_minus > 0) || o.s_minus >= 1.0) o.s_minus = 0.1;
  if (!(o.s0 > 0)) o.s0 = 1.1920928955078125e-07;  // 2^-23, single-precision machine epsilon
  if (!(o.fp8_switch_residual > 0)) o.fp8_switch_residual = 0.5;
}

int resolve_prec(int prec, int64_t n) { return polar::resolve_precision(prec, n); }

polar_status_t plan_alloc(polar_plan_s* p, size_t bytes, void** out) {
  if (p->opt.ws_limit && p->ws_bytes + bytes > p->opt.ws_limit) return POLAR_ENOMEM;
  void* ptr = nullptr;
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return POLAR_ENOMEM;
  }
  p->allocs.push_back(ptr);
  p->ws_bytes += bytes;
  *out = ptr;
  return POLAR_OK;
}

void plan_free(polar_plan_s* p) {
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  if (p->st_host) cudaFreeHost(p->st_host);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_stop) cudaEventDestroy(p->ev_stop);
  for (auto& e : p->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (auto& pr : p->prof) {
    cudaEventDestroy(pr.a);
    cudaEventDestroy(pr.b);
  }
  p->prof.clear();
  for (auto sp : p->subplans) {
    plan_free(sp);
    delete sp;
  }
  p->subplans.clear();
  if (p->bp) {
    batched_destroy(p->bp);
    p->bp = nullptr;
  }
}

polar_status_t plan_setup(polar_plan_s* p) {
  const int64_t m = p->m, n = p->n;
  polar_status_t r;
  void* v = nullptr;
  p->P = planes_of(p->prec);
  p->ldx = round_up(n, 4);
  p->ldg = round_up(n, 4);
  if (p->P == 0) {
    for (int i = 0; i < 2; ++i) {
      if ((r = plan_alloc(p, (size_t)m * p->ldx * 4, &v)) != POLAR_OK) return r;
      p->X[i] = (float*)v;
    }
  } else {
    // X and G are kept only as three BF16 planes (an exact FP32 encoding); the
    // products read the first P of them. Pitch padding is zeroed once.
    p->ldp = round_up(n, 64);
    p->xps = round_up(m * p->ldp, 64);
    p->gps = round_up(n * p->ldp, 64);
    for (int i = 0; i < 2; ++i) {
      if ((r = plan_alloc(p, (size_t)kStoredPlanes * p->xps * 2, &v)) != POLAR_OK) return r;
      CK(cudaMemset(v, 0, (size_t)kStoredPlanes * p->xps * 2));
      p->Xp[i] = (uint16_t*)v;
    }
    if ((r = plan_alloc(p, (size_t)kStoredPlanes * p->gps * 2, &v)) != POLAR_OK) return r;
    CK(cudaMemset(v, 0, (size_t)kStoredPlanes * p->gps * 2));
    p->Gp = (uint16_t*)v;
    if ((r = plan_alloc(p, (size_t)p->P * p->xps * 2, &v)) != POLAR_OK) return r;
    CK(cudaMemset(v, 0, (size_t)p->P * p->xps * 2));
    p->Ap = (uint16_t*)v;
    if (p->prec == POLAR_SCHED_FP8_BF16_X3) {
      p->kpm = round_up(m, 16);
      p->kpn = round_up(n, 16);
      const int64_t mb = (m + 127) / 128, nb = (n + 127) / 128;
      const size_t bx = (size_t)round_up(m * p->kpn, 256), bxt = (size_t)round_up(n * p->kpm, 256),
                   bg = (size_t)round_up(n * p->kpn, 256), be = (size_t)round_up(mb * nb, 256) * 2 +
                                                                (size_t)round_up(nb * nb, 256) +
                                                                (size_t)round_up(mb, 256) + 2 * (size_t)round_up(nb, 256);
      if ((r = plan_alloc(p, bx + bxt + bg + be, &v)) != POLAR_OK) return r;
      CK(cudaMemset(v, 0, bx + bxt + bg + be));
      uint8_t* w = (uint8_t*)v;
      p->Xq = w;
      p->XqT = w + bx;
      p->Gq = w + bx + bxt;
      p->eX = (int8_t*)(w + bx + bxt + bg);
      p->eXT = p->eX + round_up(mb * nb, 256);
      p->eG = p->eXT + round_up(mb * nb, 256);
      p->uX = reinterpret_cast<uint8_t*>(p->eG + round_up(nb * nb, 256));
      p->uXT = p->uX + round_up(mb, 256);
      p->uG = p->uXT + round_up(nb, 256);
    }
  }
  if ((r = plan_alloc(p, (size_t)n * p->ldg * 4, &v)) != POLAR_OK) return r;
  p->G = (float*)v;
  int np = frob_partials_blocks(m, n);
  np = std::max(np, simt_gram_tiles(n));
  np = std::max(np, 2 * symmetrize_blocks(n));
  if (p->P) np = std::max(np, tc_gram_partials_max(n));
  p->nparts = np;
  if ((r = plan_alloc(p, (size_t)np * 8, &v)) != POLAR_OK) return r;
  p->partials = (double*)v;
  if ((r = plan_alloc(p, sizeof(DevState), &v)) != POLAR_OK) return r;
  p->st = (DevState*)v;
  CK(cudaMemset(v, 0, sizeof(DevState)));
  CK(cudaMallocHost((void**)&p->st_host, sizeof(DevState)));
  memset(p->st_host, 0, sizeof(DevState));
  CK(cudaEventCreate(&p->ev_start));
  CK(cudaEventCreate(&p->ev_stop));
  for (auto& e : p->ev_chunk) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return POLAR_OK;
}

StopRule make_rule(const polar_plan_s* p, double tol) {
  StopRule r;
  r.tol = tol;
  r.stagnation = p->opt.stagnation;
  r.stag_floor = p->opt.stag_floor;
  r.switch_residual = p->opt.switch_residual;
  r.max_iter = p->opt.max_iter;
  r.sched = p->prec == POLAR_SCHED_BF16_THEN_X3 ? 1 : p->prec == POLAR_SCHED_FP8_BF16_X3 ? 2 : 0;
  r.fp8_switch = p->opt.fp8_switch_residual;
  r.planes_fixed = p->P;
  r.n_pre = p->opt.precondition ? precond_steps(p->opt.s_minus, p->opt.s0) : 0;
  r.pre_a = 1.5 * sqrt(3.0) - p->opt.s_minus;
  return r;
}

// ---- profiling: optional event pair around each Gram / update launch ----

cudaError_t prof_begin(polar_plan_s* p, int kind, int k, cudaStream_t s, int* idx) {
  *idx = -1;
  if (!p->opt.profile) return cudaSuccess;
  if (p->prof_used == p->prof.size()) {
    polar_plan_s::Prof pr;
    cudaError_t e = cudaEventCreate(&pr.a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&pr.b);
    if (e != cudaSuccess) return e;
    p->prof.push_back(pr);
  }
  auto& pr = p->prof[p->prof_used];
  pr.kind = kind;
  pr.k = k;
  *idx = (int)p->prof_used++;
  return cudaEventRecord(pr.a, s);
}

cudaError_t prof_end(polar_plan_s* p, int idx, cudaStream_t s) {
  if (idx < 0) return cudaSuccess;
  return cudaEventRecord(p->prof[idx].b, s);
}

// ---- one Newton-Schulz step k: Gram of X_k + residual/stop rule, then the update ----

cudaError_t enqueue_gram_fp32(polar_plan_s* p, int k, const StopRule& rule, cudaStream_t s) {
  const float* Xk = p->X[k & 1];
  SimtArgs g{};
  g.M = p->n; g.N = p->n; g.K = p->m;
  g.A = Xk; g.lda = p->ldx; g.a_kmajor = 0;
  g.B = Xk; g.ldb = p->ldx; g.b_kmajor = 0;
  g.C = p->G; g.ldc = p->ldg; g.alpha = 1.f; g.beta = 0.f;
  g.partials = p->partials; g.st = p->st; g.triangular = 1;
  int pi;
  cudaError_t e = prof_begin(p, 0, k, s, &pi);
  if (e != cudaSuccess) return e;
  e = launch_simt_gemm(g, SIMT_EPI_GRAM, s);
  if (e != cudaSuccess) return e;
  if ((e = prof_end(p, pi, s)) != cudaSuccess) return e;
  e = launch_residual_finalize(p->partials, simt_gram_tiles(p->n), p->st, rule, k, 0, s);
  if (e != cudaSuccess) return e;
  p->launches += 3;
  return launch_mirror_f32(p->G, p->ldg, p->n, p->st, s);
}

cudaError_t enqueue_update_fp32(polar_plan_s* p, int k, cudaStream_t s) {
  const float* Xk = p->X[k & 1];
  float* Xn = p->X[(k + 1) & 1];
  SimtArgs u{};
  u.M = p->m; u.N = p->n; u.K = p->n;
  u.A = Xk; u.lda = p->ldx; u.a_kmajor = 1;
  u.B = p->G; u.ldb = p->ldg; u.b_kmajor = 0;
  u.C = Xn; u.ldc = p->ldx;
  u.Xold = Xk; u.ldx = p->ldx; u.st = p->st;
  int pi;
  cudaError_t e = prof_begin(p, 1, k, s, &pi);
  if (e != cudaSuccess) return e;
  e = launch_simt_gemm(u, SIMT_EPI_NS, s);
  if (e != cudaSuccess) return e;
  p->launches += 1;
  return prof_end(p, pi, s);
}

TcOperand op_planes(const uint16_t* planes, int64_t rows, int64_t cols, int64_t ld, int64_t stride, int kmajor) {
  TcOperand o;
  o.planes = planes; o.rows = rows; o.cols = cols; o.ld = ld; o.plane_stride = stride; o.kmajor = kmajor;
  return o;
}

cudaError_t enqueue_gram_tc(polar_plan_s* p, int k, const StopRule& rule, cudaStream_t s) {
  const uint16_t* Xk = p->Xp[k & 1];
  if (rule.sched == 2) {
    // FP8 phase: the E4M3 codes of X_k (per 128 x 128 tile, with the tiles' exponents) as the Gram's
    // K-major operands X_k^T, and as the update's X_k; the Gram on the FP8 tensor cores (both launches
    // are enqueued; the one for the phase that is not current returns at once)
    const int64_t mb = (p->m + 127) / 128, nb = (p->n + 127) / 128;
    cudaError_t e = launch_quantize_codes(Xk, true, p->ldp, p->xps, p->m, p->n, p->XqT, p->kpm, p->eXT, mb, true,
                                          p->uXT, p->st, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_quantize_codes(Xk, true, p->ldp, p->xps, p->m, p->n, p->Xq, p->kpn, p->eX, nb, false, p->uX,
                                   p->st, s)) != cudaSuccess)
      return e;
    TcArgs q{};
    q.M = p->n; q.N = p->n; q.K = p->m;
    q.a = op_planes((const uint16_t*)p->XqT, p->n, p->m, p->kpm, 0, 1);
    q.b = q.a;
    q.nplanes = 1;
    q.epi = TC_EPI_GRAM; q.triangular = 1;
    q.out_planes = p->Gp; q.ldo = p->ldp; q.out_plane_stride = p->gps; q.out_nplanes = kStoredPlanes;
    q.partials = p->partials; q.st = p->st;
    q.planes_dyn = &p->st->fp8_on;
    q.a_exp = p->eXT; q.lde_a = mb;
    q.b_exp = p->eXT; q.lde_b = mb;
    q.a_uni = p->uXT; q.b_uni = p->uXT;
    if ((e = launch_tc_gemm_fp8(q, s)) != cudaSuccess) return e;
    p->launches += 5;
  }
  TcArgs g{};
  g.M = p->n; g.N = p->n; g.K = p->m;
  g.a = op_planes(Xk, p->m, p->n, p->ldp, p->xps, 0);
  g.b = g.a;
  g.nplanes = p->P;
  g.epi = TC_EPI_GRAM; g.triangular = 1;
  g.out_planes = p->Gp; g.ldo = p->ldp; g.out_plane_stride = p->gps; g.out_nplanes = kStoredPlanes;
  g.partials = p->partials; g.st = p->st;
  g.planes_dyn = rule.sched ? &p->st->planes_next : nullptr;
  int pi;
  cudaError_t e = prof_begin(p, 0, k, s, &pi);
  if (e != cudaSuccess) return e;
  e = launch_tc_gemm(g, s);
  if (e != cudaSuccess) return e;
  if ((e = prof_end(p, pi, s)) != cudaSuccess) return e;
  p->launches += 2;
  // the finalize records the planes this Gram used (schedules: read on the device); then the lower
  // triangle of G's planes from the upper one the Gram epilogue wrote (skipped once stopped)
  e = launch_residual_finalize(p->partials, tc_gram_partials(p->n, p->P), p->st, rule, k, rule.sched ? -1 : p->P, s);
  if (e != cudaSuccess) return e;
  p->launches += 1;
  return launch_mirror_planes3(p->Gp, p->ldp, p->gps, p->n, p->st, s);
}

cudaError_t enqueue_update_tc(polar_plan_s* p, int k, const StopRule& rule, cudaStream_t s) {
  if (rule.sched == 2) {
    // FP8 phase: X_k's codes (made with the Gram) times the codes of G (symmetric: its rows are the
    // K-major B operand), on the FP8 tensor cores
    const int64_t nb = (p->n + 127) / 128;
    cudaError_t e = launch_quantize_codes(p->Gp, true, p->ldp, p->gps, p->n, p->n, p->Gq, p->kpn, p->eG, nb, false,
                                          p->uG, p->st, s);
    if (e != cudaSuccess) return e;
    TcArgs q{};
    q.M = p->m; q.N = p->n; q.K = p->n;
    q.a = op_planes((const uint16_t*)p->Xq, p->m, p->n, p->kpn, 0, 1);
    q.b = op_planes((const uint16_t*)p->Gq, p->n, p->n, p->kpn, 0, 1);
    q.a_exp = p->eX; q.lde_a = nb;
    q.b_exp = p->eG; q.lde_b = nb;
    q.a_uni = p->uX; q.b_uni = p->uG;
    q.nplanes = 1;
    q.epi = TC_EPI_NS;
    q.x_planes = p->Xp[k & 1]; q.ldxp = p->ldp; q.x_plane_stride = p->xps;
    q.out_planes = p->Xp[(k + 1) & 1]; q.ldo = p->ldp; q.out_plane_stride = p->xps; q.out_nplanes = kStoredPlanes;
    q.st = p->st;
    q.planes_dyn = &p->st->fp8_on;
    if ((e = launch_tc_gemm_fp8(q, s)) != cudaSuccess) return e;
    p->launches += 3;
  }
  TcArgs u{};
  u.M = p->m; u.N = p->n; u.K = p->n;
  u.a = op_planes(p->Xp[k & 1], p->m, p->n, p->ldp, p->xps, 1);
  u.b = op_planes(p->Gp, p->n, p->n, p->ldp, p->gps, 0);
  u.nplanes = p->P;
  u.epi = TC_EPI_NS;
  u.x_planes = p->Xp[k & 1]; u.ldxp = p->ldp; u.x_plane_stride = p->xps;
  u.out_planes = p->Xp[(k + 1) & 1]; u.ldo = p->ldp; u.out_plane_stride = p->xps; u.out_nplanes = kStoredPlanes;
  u.st = p->st;
  u.planes_dyn = rule.sched ? &p->st->planes_next : nullptr;
  int pi;
  cudaError_t e = prof_begin(p, 1, k, s, &pi);
  if (e != cudaSuccess) return e;
  e = launch_tc_gemm(u, s);
  if (e != cudaSuccess) return e;
  p->launches += 1;
  return prof_end(p, pi, s);
}

polar_status_t run_single(polar_plan_s* p, const float* A, int64_t lda, float* U, int64_t ldu, float* H,
                          int64_t ldh, double tol, polar_info_t* info, cudaStream_t s) {
  const int64_t m = p->m, n = p->n;
  if (!(tol > 0)) tol = p->opt.tol;
  StopRule rule = make_rule(p, tol);
  p->launches = 0;
  p->prof_used = 0;
  CK(cudaEventRecord(p->ev_start, s));
  // ||A||_F and X_0 = A / ||A||_F (+ planes of X_0)
  int fb = frob_partials_blocks(m, n);
  CK(launch_frob_partials(A, m, n, lda, p->partials, fb, s));
  CK(launch_norm_finalize(p->partials, fb, p->st, 1.0 / sqrt((double)n),
                          rule.sched == 2 ? 0 : rule.sched == 1 ? 1 : p->P, rule.sched == 2 ? 1 : 0, s));
  if (p->P == 0)
    CK(launch_scale_split(A, lda, m, n, p->st, true, p->X[0], p->ldx, nullptr, 0, 0, 0, s));
  else
    CK(launch_scale_split(A, lda, m, n, p->st, true, nullptr, 0, p->Xp[0], p->ldp, p->xps, kStoredPlanes, s));
  p->launches += 3;

  // Iterations in chunks; two chunks in flight so the device never waits on the host.
  // Kernels enqueued after the stop rule fired return at once (they read the status).
  const int chunk = 4;
  int k = 0;
  int head = 0, queued = 0;
  int status = ST_RUNNING;
  while (true) {
    while (queued < 2 && k <= p->opt.max_iter) {
      for (int c = 0; c < chunk && k <= p->opt.max_iter; ++c, ++k) {
        if (p->P == 0) {
          CK(enqueue_gram_fp32(p, k, rule, s));
          if (k < p->opt.max_iter) CK(enqueue_update_fp32(p, k, s));
        } else {
          CK(enqueue_gram_tc(p, k, rule, s));
          if (k < p->opt.max_iter) CK(enqueue_update_tc(p, k, rule, s));
        }
      }
      CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(p->ev_chunk[(head + queued) & 1], s));
      ++queued;
    }
    if (queued == 0) break;
    CK(cudaEventSynchronize(p->ev_chunk[head]));
    head ^= 1;
    --queued;
    if (p->st_host->status != ST_RUNNING) break;
  }
  CK(cudaStreamSynchronize(s));
  DevState& h = *p->st_host;
  status = h.status;
  if (h.err_flags) status = ST_TIMEOUT;
  if (status == ST_NONFINITE || status == ST_TIMEOUT || status == ST_RUNNING) {
    CK(cudaEventRecord(p->ev_stop, s));
    CK(cudaEventSynchronize(p->ev_stop));
    if (info) {
      memset(info, 0, sizeof(*info));
      info->status = status == ST_NONFINITE ? POLAR_ENONFINITE : status == ST_TIMEOUT ? POLAR_ETIMEOUT : POLAR_ECUDA;
      info->normA_F = h.normA;
      info->prec = p->prec;
      info->iters = h.iters;
      info->hist_len = h.hist_len;
      memcpy(info->res_hist, h.res_hist, sizeof(h.res_hist));
      memcpy(info->planes_hist, h.planes_hist, sizeof(h.planes_hist));
    }
    return status == ST_NONFINITE ? POLAR_ENONFINITE : status == ST_TIMEOUT ? POLAR_ETIMEOUT : POLAR_ECUDA;
  }
  const int it = h.iters;
  // U = X_it ; C = U^T A ; H = sym(C)
  if (p->P == 0) {
    const float* Uk = p->X[it & 1];
    CK(launch_copy2d(Uk, p->ldx, U, ldu, m, n, s));
    SimtArgs c{};
    c.M = n; c.N = n; c.K = m;
    c.A = Uk; c.lda = p->ldx; c.a_kmajor = 0;
    c.B = A; c.ldb = lda; c.b_kmajor = 0;
    c.C = p->G; c.ldc = p->ldg; c.alpha = 1.f; c.beta = 0.f;
    CK(launch_simt_gemm(c, SIMT_EPI_STORE, s));
    p->launches += 2;
  } else {
    CK(launch_planes_to_f32(p->Xp[it & 1], p->ldp, p->xps, m, n, U, ldu, s));
    CK(launch_scale_split(A, lda, m, n, nullptr, false, nullptr, 0, p->Ap, p->ldp, p->xps, p->P, s));
    TcArgs c{};
    c.M = n; c.N = n; c.K = m;
    c.a = op_planes(p->Xp[it & 1], m, n, p->ldp, p->xps, 0);
    c.b = op_planes(p->Ap, m, n, p->ldp, p->xps, 0);
    c.nplanes = p->P;
    c.epi = TC_EPI_STORE;
    c.C = p->G; c.ldc = p->ldg; c.alpha = 1.f; c.beta = 0.f;
    c.st = nullptr;                  // the solve has stopped: the launch must run
    c.err_out = &p->st->err_flags;   // a timeout still reaches this solve's status
    CK(launch_tc_gemm(c, s));
    p->launches += 3;
  }
  int sb = symmetrize_blocks(n);
  CK(launch_symmetrize(p->G, p->ldg, n, H, ldh, p->partials, sb, s));
  CK(launch_sym_finalize(p->partials, sb, p->st, s));
  p->launches += 2;
  CK(cudaEventRecord(p->ev_stop, s));
  CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (p->st_host->err_flags) status = ST_TIMEOUT;
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, p->ev_start, p->ev_stop));
  polar_status_t ret = status == ST_CONVERGED ? POLAR_OK
                       : status == ST_NOT_CONVERGED ? POLAR_NOT_CONVERGED
                       : POLAR_ETIMEOUT;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = ret;
    info->iters = it;
    info->prec = p->prec;
    info->hist_len = h.hist_len;
    info->residual = (it < POLAR_HIST && it < h.hist_len) ? h.res_hist[it] : h.ring[it & 3];
    info->normA_F = h.normA;
    info->sym_err = h.sym_err;
    info->ms_total = ms;
    info->launches = p->launches;
    info->n_precond = std::min(rule.n_pre, it);
    for (size_t i = 0; i < p->prof_used; ++i) {
      const auto& pr = p->prof[i];
      if ((pr.kind == 0 && pr.k > it) || (pr.kind == 1 && pr.k >= it)) continue;  // launches after the stop
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, pr.a, pr.b));
      if (pr.kind == 0) { info->ms_gram += t; info->n_gram++; }
      else { info->ms_update += t; info->n_update++; }
    }
    memcpy(info->res_hist, h.res_hist, sizeof(h.res_hist));
    memcpy(info->planes_hist, h.planes_hist, sizeof(h.planes_hist));
  }
  return ret;
}

}  // namespace

extern "C" {

polar_status_t polar_plan_create(polar_plan_t* plan, int64_t m, int64_t n, const polar_options_t* o) {
  if (!plan) return POLAR_EINVAL;
  *plan = nullptr;
  if (n < 1 || m < n) return POLAR_EINVAL;
  polar_options_t opt;
  if (o) opt = *o; else polar_default_options(&opt);
  normalize_options(opt);
  int prec = resolve_prec(opt.prec, n);
  if (prec == POLAR_TF32X3) return POLAR_ENOTSUP;
  if (prec < 0 || prec > POLAR_BF16) return POLAR_EINVAL;
  int sms = 0;
  if (!device_ok(&sms)) { cudaGetLastError(); return POLAR_ECUDA; }
  if (planes_of(prec) > 0 && !tc_available()) return POLAR_ENOTSUP;
  polar_plan_s* p = new (std::nothrow) polar_plan_s();
  if (!p) return POLAR_ENOMEM;
  p->m = m; p->n = n; p->opt = opt; p->prec = prec; p->sms = sms;
  polar_status_t r = plan_setup(p);
  if (r != POLAR_OK) {
    plan_free(p);
    delete p;
    cudaGetLastError();
    return r;
  }
  *plan = p;
  return POLAR_OK;
}

size_t polar_plan_workspace_bytes(polar_plan_t plan) {
  if (!plan) return 0;
  size_t b = plan->ws_bytes + batched_workspace_bytes(plan->bp);
  for (auto sp : plan->subplans) b += sp->ws_bytes;
  return b;
}

void polar_plan_destroy(polar_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  plan_free(plan);
  delete plan;
}

polar_status_t polar_run(polar_plan_t plan, const float* A, int64_t lda, float* U, int64_t ldu, float* H,
                         int64_t ldh, double tol, polar_info_t* info, polar_stream_t stream) {
  if (!plan || plan->batched || !A || !U || !H) return POLAR_EINVAL;
  const int64_t m = plan->m, n = plan->n;
  if (lda < n || ldu < n || ldh < n) return POLAR_EINVAL;
  size_t na = (size_t)((m - 1) * lda + n) * 4, nu = (size_t)((m - 1) * ldu + n) * 4,
         nh = (size_t)((n - 1) * ldh + n) * 4;
  if (overlaps(A, na, U, nu) || overlaps(A, na, H, nh) || overlaps(U, nu, H, nh)) return POLAR_EINVAL;
  polar_status_t r = run_single(plan, A, lda, U, ldu, H, ldh, tol, info, (cudaStream_t)stream);
  if (r == POLAR_ECUDA) cudaGetLastError();
  return r;
}

polar_status_t polar_run_host(polar_plan_t plan, const float* A, int64_t lda, float* U, int64_t ldu, float* H,
                              int64_t ldh, double tol, polar_info_t* info, polar_stream_t stream) {
  if (!plan || plan->batched || !A || !U || !H) return POLAR_EINVAL;
  const int64_t m = plan->m, n = plan->n;
  if (lda < n || ldu < n || ldh < n) return POLAR_EINVAL;
  size_t na = (size_t)((m - 1) * lda + n) * 4, nu = (size_t)((m - 1) * ldu + n) * 4,
         nh = (size_t)((n - 1) * ldh + n) * 4;
  if (overlaps(A, na, U, nu) || overlaps(A, na, H, nh) || overlaps(U, nu, H, nh)) return POLAR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!plan->hostA) {
    void* v = nullptr;
    polar_status_t r;
    if ((r = plan_alloc(plan, (size_t)m * n * 4, &v)) != POLAR_OK) return r;
    plan->hostA = (float*)v;
    if ((r = plan_alloc(plan, (size_t)m * n * 4, &v)) != POLAR_OK) return r;
    plan->hostU = (float*)v;
    if ((r = plan_alloc(plan, (size_t)n * n * 4, &v)) != POLAR_OK) return r;
    plan->hostH = (float*)v;
  }
  if (cudaMemcpy2DAsync(plan->hostA, (size_t)n * 4, A, (size_t)lda * 4, (size_t)n * 4, (size_t)m,
                        cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return POLAR_ECUDA;
  }
  polar_status_t r = run_single(plan, plan->hostA, n, plan->hostU, n, plan->hostH, n, tol, info, s);
  if (r == POLAR_OK || r == POLAR_NOT_CONVERGED) {
    if (cudaMemcpy2DAsync(U, (size_t)ldu * 4, plan->hostU, (size_t)n * 4, (size_t)n * 4, (size_t)m,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpy2DAsync(H, (size_t)ldh * 4, plan->hostH, (size_t)n * 4, (size_t)n * 4, (size_t)n,
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      r = POLAR_ECUDA;
  }
  if (r == POLAR_ECUDA) cudaGetLastError();
  return r;
}

polar_status_t polar_async_status(polar_stream_t stream) {
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  unsigned int v = 0;
  if (tc_take_error((cudaStream_t)stream, &v) != cudaSuccess) { cudaGetLastError(); return POLAR_ECUDA; }
  return v ? POLAR_ETIMEOUT : POLAR_OK;
}

polar_status_t polar_batched_plan_create(polar_plan_t* plan, int count, const int64_t* m, const int64_t* n,
                                         const polar_options_t* o) {
  if (!plan) return POLAR_EINVAL;
  *plan = nullptr;
  if (count < 1 || !m || !n) return POLAR_EINVAL;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || m[i] < n[i]) return POLAR_EINVAL;
  polar_options_t opt;
  if (o) opt = *o; else polar_default_options(&opt);
  normalize_options(opt);
  int prec = opt.prec == POLAR_AUTO ? POLAR_BF16X6 : opt.prec;
  if (prec < 0 || prec > POLAR_BF16) return POLAR_EINVAL;
  // batched problems run on the tensor-core path with a fixed plane count
  if (prec != POLAR_BF16X6 && prec != POLAR_BF16X3 && prec != POLAR_BF16) return POLAR_ENOTSUP;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  if (!tc_available()) return POLAR_ENOTSUP;
  polar_plan_s* p = new (std::nothrow) polar_plan_s();
  if (!p) return POLAR_ENOMEM;
  p->batched = true;
  p->count = count;
  p->opt = opt;
  p->prec = prec;
  polar_status_t r = batched_create(&p->bp, count, m, n, opt, prec);
  if (r != POLAR_OK) {
    delete p;
    cudaGetLastError();
    return r;
  }
  *plan = p;
  return POLAR_OK;
}

polar_status_t polar_batched_run(polar_plan_t plan, const float* const* A, float* const* U, float* const* H,
                                 double tol, int32_t* iters_dev, double* resid_dev, polar_stream_t stream) {
  if (!plan || !plan->batched || !plan->bp || !A || !U || !H) return POLAR_EINVAL;
  for (int i = 0; i < plan->count; ++i)
    if (!A[i] || !U[i] || !H[i]) return POLAR_EINVAL;
  polar_status_t r = batched_run(plan->bp, A, U, H, tol, iters_dev, resid_dev, (cudaStream_t)stream);
  if (r == POLAR_ECUDA) cudaGetLastError();
  return r;
}

polar_status_t polar_split_bf16(const float* X, int64_t count, int planes, uint16_t* out, polar_stream_t stream) {
  if (count < 0 || planes < 1 || planes > 3) return POLAR_EINVAL;
  if (count == 0) return POLAR_OK;
  if (!X || !out) return POLAR_EINVAL;
  if (overlaps(X, (size_t)count * 4, out, (size_t)count * 2 * planes)) return POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  if (launch_split_flat(X, count, planes, out, (cudaStream_t)stream) != cudaSuccess) return POLAR_ECUDA;
  return POLAR_OK;
}

polar_status_t polar_gemm(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                          int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc, int prec,
                          polar_stream_t stream) {
  if (M < 0 || N < 0 || K < 0) return POLAR_EINVAL;
  if (M == 0 || N == 0) return POLAR_OK;
  if (!C || ldc < N) return POLAR_EINVAL;
  if (K > 0 && (!A || !B)) return POLAR_EINVAL;
  // stored shapes
  const int64_t a_rows = transA ? K : M, a_cols = transA ? M : K;
  const int64_t b_rows = transB ? N : K, b_cols = transB ? K : N;
  if (K > 0 && (lda < a_cols || ldb < b_cols)) return POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  cudaStream_t s = (cudaStream_t)stream;
  prec = resolve_prec(prec, std::min(M, N));
  if (K == 0) {
    // C = beta C
    SimtArgs g{};
    g.M = M; g.N = N; g.K = 0; g.A = C; g.lda = ldc; g.a_kmajor = 1; g.B = C; g.ldb = ldc; g.b_kmajor = 1;
    g.C = C; g.ldc = ldc; g.alpha = 0.f; g.beta = beta;
    return launch_simt_gemm(g, SIMT_EPI_STORE, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
  }
  if (prec == POLAR_FP32) {
    SimtArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.a_kmajor = transA ? 0 : 1;
    g.B = B; g.ldb = ldb; g.b_kmajor = transB ? 1 : 0;
    g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta;
    return launch_simt_gemm(g, SIMT_EPI_STORE, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
  }
  const int P = product_planes(prec);
  if (P == 0) return prec == POLAR_TF32X3 ? POLAR_ENOTSUP : POLAR_EINVAL;
  if (!tc_available()) return POLAR_ENOTSUP;
  const int64_t lpa = round_up(a_cols, 64), lpb = round_up(b_cols, 64);
  const int64_t sa = round_up(a_rows * lpa, 64), sb = round_up(b_rows * lpb, 64);
  void* scr = nullptr;
  polar_status_t r = scratch_get((size_t)P * (sa + sb) * 2, &scr);
  if (r != POLAR_OK) return r;
  uint16_t* pa = (uint16_t*)scr;
  uint16_t* pb = pa + P * sa;
  CK(cudaMemsetAsync(scr, 0, (size_t)P * (sa + sb) * 2, s));
  CK(launch_scale_split(A, lda, a_rows, a_cols, nullptr, false, nullptr, 0, pa, lpa, sa, P, s));
  CK(launch_scale_split(B, ldb, b_rows, b_cols, nullptr, false, nullptr, 0, pb, lpb, sb, P, s));
  TcArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.a = op_planes(pa, a_rows, a_cols, lpa, sa, transA ? 0 : 1);
  g.b = op_planes(pb, b_rows, b_cols, lpb, sb, transB ? 1 : 0);
  g.nplanes = P;
  g.epi = TC_EPI_STORE;
  g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta;
  return launch_tc_gemm(g, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

polar_status_t polar_gemm_fp8(int transA, int transB, int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                              int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                              polar_stream_t stream) {
  if (M < 0 || N < 0 || K < 0) return POLAR_EINVAL;
  if (M == 0 || N == 0) return POLAR_OK;
  if (!C || ldc < N) return POLAR_EINVAL;
  if (K > 0 && (!A || !B)) return POLAR_EINVAL;
  const int64_t a_rows = transA ? K : M, a_cols = transA ? M : K;
  const int64_t b_rows = transB ? N : K, b_cols = transB ? K : N;
  if (K > 0 && (lda < a_cols || ldb < b_cols)) return POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0) {
    SimtArgs g{};
    g.M = M; g.N = N; g.K = 0; g.A = C; g.lda = ldc; g.a_kmajor = 1; g.B = C; g.ldb = ldc; g.b_kmajor = 1;
    g.C = C; g.ldc = ldc; g.alpha = 0.f; g.beta = beta;
    return launch_simt_gemm(g, SIMT_EPI_STORE, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
  }
  if (!tc_available()) return POLAR_ENOTSUP;
  // K-major codes of op(A) (M x K) and op(B)^T (N x K), rows padded to 16 bytes, and the tiles' exponents
  const int64_t kp = round_up(K, 16), kb = (K + 127) / 128;
  const int64_t mb = (M + 127) / 128, nb = (N + 127) / 128;
  const size_t oa = 0, ob = round_up(M * kp, 256), oea = ob + round_up(N * kp, 256), oeb = oea + round_up(mb * kb, 256);
  const size_t oua = oeb + round_up(nb * kb, 256), oub = oua + round_up(mb, 256);
  const size_t bytes = oub + round_up(nb, 256);
  void* scr = nullptr;
  polar_status_t r = scratch_get(bytes, &scr);
  if (r != POLAR_OK) return r;
  uint8_t* w = (uint8_t*)scr;
  uint8_t* ca = w + oa;
  uint8_t* cb = w + ob;
  int8_t* ea = (int8_t*)(w + oea);
  int8_t* eb = (int8_t*)(w + oeb);
  uint8_t* ua = w + oua;
  uint8_t* ub = w + oub;
  // op(A) = A (stored M x K) or A^T (stored K x M: transposed into M x K); op(B)^T = B^T (B stored K x N:
  // transposed into N x K) or B (stored N x K)
  CK(launch_quantize_codes(A, false, lda, 0, a_rows, a_cols, ca, kp, ea, kb, transA != 0, ua, nullptr, s));
  CK(launch_quantize_codes(B, false, ldb, 0, b_rows, b_cols, cb, kp, eb, kb, transB == 0, ub, nullptr, s));
  TcArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.a = op_planes((const uint16_t*)ca, M, K, kp, 0, 1);
  g.b = op_planes((const uint16_t*)cb, N, K, kp, 0, 1);
  g.nplanes = 1;
  g.epi = TC_EPI_STORE;
  g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta;
  g.a_exp = ea; g.lde_a = kb;
  g.b_exp = eb; g.lde_b = kb;
  g.a_uni = ua; g.b_uni = ub;
  return launch_tc_gemm_fp8(g, s) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

polar_status_t polar_syrk(int64_t n, int64_t k, float alpha, const float* A, int64_t lda, float beta, float* C,
                          int64_t ldc, int prec, polar_stream_t stream) {
  if (n < 0 || k < 0) return POLAR_EINVAL;
  if (n == 0) return POLAR_OK;
  if (!C || ldc < n) return POLAR_EINVAL;
  if (k > 0 && (!A || lda < n)) return POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  cudaStream_t s = (cudaStream_t)stream;
  prec = resolve_prec(prec, n);
  if (k == 0 || prec == POLAR_FP32) {
    SimtArgs g{};
    g.M = n; g.N = n; g.K = k;
    g.A = k ? A : C; g.lda = k ? lda : ldc; g.a_kmajor = 0;
    g.B = g.A; g.ldb = g.lda; g.b_kmajor = 0;
    g.C = C; g.ldc = ldc; g.alpha = k ? alpha : 0.f; g.beta = beta; g.triangular = 1;
    CK(launch_simt_gemm(g, SIMT_EPI_STORE, s));
    CK(launch_mirror_f32(C, ldc, n, nullptr, s));
    return POLAR_OK;
  }
  const int P = product_planes(prec);
  if (P == 0) return prec == POLAR_TF32X3 ? POLAR_ENOTSUP : POLAR_EINVAL;
  if (!tc_available()) return POLAR_ENOTSUP;
  const int64_t lp = round_up(n, 64);
  const int64_t sa = round_up(k * lp, 64);
  void* scr = nullptr;
  polar_status_t r = scratch_get((size_t)P * sa * 2, &scr);
  if (r != POLAR_OK) return r;
  uint16_t* pa = (uint16_t*)scr;
  CK(cudaMemsetAsync(scr, 0, (size_t)P * sa * 2, s));
  CK(launch_scale_split(A, lda, k, n, nullptr, false, nullptr, 0, pa, lp, sa, P, s));
  TcArgs g{};
  g.M = n; g.N = n; g.K = k;
  g.a = op_planes(pa, k, n, lp, sa, 0);
  g.b = g.a;
  g.nplanes = P;
  g.epi = TC_EPI_STORE; g.triangular = 1;
  g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta;
  CK(launch_tc_gemm(g, s));
  CK(launch_mirror_f32(C, ldc, n, nullptr, s));
  return POLAR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- Newton-Schulz inverse (Algorithm 2)

extern "C" polar_status_t polar_ns_inverse(const float* A, int64_t rows, int64_t cols, int64_t lda, float* X,
                                           int64_t ldx, int prec, int max_iter, int32_t* iters, double* delta,
                                           polar_stream_t stream) {
  if (!A || !X || cols < 1 || rows < cols || lda < cols || ldx < rows) return POLAR_EINVAL;
  if (overlaps(A, (size_t)((rows - 1) * lda + cols) * 4, X, (size_t)((cols - 1) * ldx + rows) * 4))
    return POLAR_EINVAL;
  if (max_iter <= 0) max_iter = 100;
  if (prec == POLAR_AUTO) prec = POLAR_BF16X6;
  const int P = planes_of(prec);
  if (prec == POLAR_SCHED_BF16_THEN_X3 || P == 0) return prec == POLAR_FP32 ? POLAR_ENOTSUP : POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  if (!tc_available()) return POLAR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = rows, M = cols;
  // workspace: A planes (N x M), X planes x2 (M x N, three planes), P = A X planes (N x N, three planes),
  // C = A^T A (M x M), partials, state
  const int64_t lpa = round_up(M, 64), lpx = round_up(N, 64);
  const int64_t sa = round_up(N * lpa, 64), sx = round_up(M * lpx, 64), sp = round_up(N * lpx, 64);
  const int64_t ldc = round_up(M, 4);
  const int64_t tiles_ns = ((M + 127) / 128) * ((N + 255) / 256);
  const int64_t npairs = tiles_ns * 8;
  const int fb = frob_partials_blocks(M, M);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_a = take((size_t)P * sa * 2), o_x0 = take((size_t)3 * sx * 2), o_x1 = take((size_t)3 * sx * 2),
               o_p = take((size_t)3 * sp * 2), o_c = take((size_t)M * ldc * 4),
               o_part = take((size_t)std::max<int64_t>(2 * npairs, fb) * 8), o_st = take(sizeof(DevState));
  void* ws = nullptr;
  if (cudaMalloc(&ws, off) != cudaSuccess) { cudaGetLastError(); return POLAR_ENOMEM; }
  int* status_host = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaMallocHost(&status_host, 2 * sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    for (auto e : ev) if (e) cudaEventDestroy(e);
    if (status_host) cudaFreeHost(status_host);
    cudaFree(ws);
    return POLAR_ENOMEM;
  }
  uint8_t* w = (uint8_t*)ws;
  uint16_t* ap = (uint16_t*)(w + o_a);
  uint16_t* xp[2] = {(uint16_t*)(w + o_x0), (uint16_t*)(w + o_x1)};
  uint16_t* pp = (uint16_t*)(w + o_p);
  float* C = (float*)(w + o_c);
  double* part = (double*)(w + o_part);
  DevState* st = (DevState*)(w + o_st);
  polar_status_t ret = POLAR_ECUDA;
  DevState h;
  do {
    if (cudaMemsetAsync(ws, 0, off, s) != cudaSuccess) break;
    // a = ||A A^T||_F = ||A^T A||_F: the Gram of A's columns on the tensor cores, mirrored, its norm
    if (launch_scale_split(A, lda, N, M, nullptr, false, nullptr, 0, ap, lpa, sa, P, s) != cudaSuccess) break;
    TcArgs g{};
    g.M = M; g.N = M; g.K = N;
    g.a = op_planes(ap, N, M, lpa, sa, 0);
    g.b = g.a;
    g.nplanes = P;
    g.epi = TC_EPI_STORE; g.triangular = 1;
    g.C = C; g.ldc = ldc; g.alpha = 1.f; g.beta = 0.f;
    g.err_out = &st->err_flags;   // no skip test (st is not RUNNING yet), but a timeout is reported
    if (launch_tc_gemm(g, s) != cudaSuccess) break;
    if (launch_mirror_f32(C, ldc, M, nullptr, s) != cudaSuccess) break;
    if (launch_frob_partials(C, M, M, ldc, part, fb, s) != cudaSuccess) break;
    if (launch_norm_finalize(part, fb, st, 1.0, P, 0, s) != cudaSuccess) break;
    // X_0 = A^T / a; the update X' = 2 X - X (A X)
    if (launch_transpose_scale_split(A, lda, N, M, st, xp[0], lpx, sx, s) != cudaSuccess) break;
    if (launch_inverse_init(st, s) != cudaSuccess) break;
    // Iterations in chunks of four, two chunks in flight; the host reads the status word
    // after each chunk and stops enqueueing once the stop rule has fired (kernels enqueued
    // after that return at once).
    auto enqueue_iter = [&](int k) {
      TcArgs pa{};  // P = A X_k (N x N, K = M)
      pa.M = N; pa.N = N; pa.K = M;
      pa.a = op_planes(ap, N, M, lpa, sa, 1);
      pa.b = op_planes(xp[k & 1], M, N, lpx, sx, 0);
      pa.nplanes = P;
      pa.epi = TC_EPI_PLANES;
      pa.out_planes = pp; pa.ldo = lpx; pa.out_plane_stride = sp; pa.out_nplanes = 3;
      pa.st = st;
      TcArgs u{};   // X_{k+1} = 2 X_k - X_k P (M x N, K = N), with the pairs for delta
      u.M = M; u.N = N; u.K = N;
      u.a = op_planes(xp[k & 1], M, N, lpx, sx, 1);
      u.b = op_planes(pp, N, N, lpx, sp, 0);
      u.nplanes = P;
      u.epi = TC_EPI_NS_STEP;
      u.x_planes = xp[k & 1]; u.ldxp = lpx; u.x_plane_stride = sx;
      u.out_planes = xp[(k + 1) & 1]; u.ldo = lpx; u.out_plane_stride = sx; u.out_nplanes = 3;
      u.partials = part;
      u.st = st;
      return launch_tc_gemm(pa, s) == cudaSuccess && launch_tc_gemm(u, s) == cudaSuccess &&
             launch_inverse_finalize(part, (int)npairs, st, k, max_iter, s) == cudaSuccess;
    };
    const int chunk = 4;
    bool ok = true;
    int k = 0, head = 0, queued = 0;
    while (ok) {
      while (ok && queued < 2 && k < max_iter) {
        for (int c = 0; c < chunk && k < max_iter && ok; ++c, ++k) ok = enqueue_iter(k);
        const int slot = (head + queued) & 1;
        ok = ok && cudaMemcpyAsync(&status_host[slot], &st->status, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaEventRecord(ev[slot], s) == cudaSuccess;
        ++queued;
      }
      if (!ok || queued == 0) break;
      ok = cudaEventSynchronize(ev[head]) == cudaSuccess;
      const int st_now = status_host[head];
      head ^= 1;
      --queued;
      if (st_now != ST_RUNNING) break;
    }
    if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
    if (h.err_flags || h.status == ST_TIMEOUT) { ret = POLAR_ETIMEOUT; break; }
    if (h.status == ST_NONFINITE) { ret = POLAR_ENONFINITE; break; }
    if (launch_planes_to_f32(xp[h.iters & 1], lpx, sx, M, N, X, ldx, s) != cudaSuccess) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
    if (iters) *iters = h.iters;
    if (delta) *delta = h.ring[(h.iters - 1) & 3];
    ret = h.status == ST_CONVERGED ? POLAR_OK : POLAR_NOT_CONVERGED;
  } while (0);
  cudaStreamSynchronize(s);
  for (auto e : ev) cudaEventDestroy(e);
  cudaFreeHost(status_host);
  cudaFree(ws);
  if (ret == POLAR_ECUDA) cudaGetLastError();
  return ret;
}

extern "C" polar_status_t polar_chebyshev_nodes(double a, double b, int degree, double* x) {
  if (!x || degree < 0 || !std::isfinite(a) || !std::isfinite(b) || !(b > a)) return POLAR_EINVAL;
  const double pi = 3.14159265358979323846;
  for (int j = 0; j <= degree; ++j) x[j] = 0.5 * (a + b) + 0.5 * (b - a) * std::cos(pi * (j + 0.5) / (degree + 1));
  return POLAR_OK;
}

extern "C" polar_status_t polar_chebyshev_fit(const double* g, int degree, double* coef) {
  if (!g || !coef || degree < 0) return POLAR_EINVAL;
  const double pi = 3.14159265358979323846;
  for (int j = 0; j <= degree; ++j)
    if (!std::isfinite(g[j])) return POLAR_ENONFINITE;
  for (int k = 0; k <= degree; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= degree; ++j) acc += g[j] * std::cos(k * pi * (j + 0.5) / (degree + 1));
    coef[k] = 2.0 * acc / (degree + 1);
  }
  coef[0] *= 0.5;
  return POLAR_OK;
}

extern "C" polar_status_t polar_chebyshev(const float* A, int64_t n, int64_t lda, double a, double b,
                                          const double* coef, int degree, float* F, int64_t ldf, int prec,
                                          polar_stream_t stream) {
  if (!A || !F || !coef || n < 1 || lda < n || ldf < n || degree < 0) return POLAR_EINVAL;
  if (!std::isfinite(a) || !std::isfinite(b) || !(b > a)) return POLAR_EINVAL;
  for (int k = 0; k <= degree; ++k)
    if (!std::isfinite(coef[k])) return POLAR_EINVAL;
  if (overlaps(A, (size_t)((n - 1) * lda + n) * 4, F, (size_t)((n - 1) * ldf + n) * 4)) return POLAR_EINVAL;
  if (prec == POLAR_AUTO) prec = POLAR_BF16X6;
  const int P = planes_of(prec);
  if (prec == POLAR_SCHED_BF16_THEN_X3 || P == 0) return prec == POLAR_FP32 ? POLAR_ENOTSUP : POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  if (!tc_available()) return POLAR_ENOTSUP;
  cudaStream_t s = (cudaStream_t)stream;
  const double am = 2.0 / (b - a), bm = -(a + b) / (b - a);   // T = am A + bm I
  // workspace: T planes (P), three rotating B_k buffers (three planes each: they are also read
  // as Z = B_{k+2} by the epilogue), device state
  const int64_t ldp = round_up(n, 64), sp = round_up(n * ldp, 64);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t o_t = take((size_t)P * sp * 2), o_b0 = take((size_t)3 * sp * 2), o_b1 = take((size_t)3 * sp * 2),
               o_b2 = take((size_t)3 * sp * 2), o_st = take(sizeof(DevState));
  void* ws = nullptr;
  if (cudaMalloc(&ws, off) != cudaSuccess) { cudaGetLastError(); return POLAR_ENOMEM; }
  uint8_t* w = (uint8_t*)ws;
  uint16_t* tp = (uint16_t*)(w + o_t);
  uint16_t* bk[3] = {(uint16_t*)(w + o_b0), (uint16_t*)(w + o_b1), (uint16_t*)(w + o_b2)};
  DevState* st = (DevState*)(w + o_st);
  polar_status_t ret = POLAR_ECUDA;
  do {
    if (cudaMemsetAsync(ws, 0, off, s) != cudaSuccess) break;   // also status = RUNNING
    bool ok = true;
    if (degree <= 1) {
      // F = c_0 I + c_1 T: no product
      ok = launch_cheb_affine_split(A, lda, n, am, bm, degree == 1 ? coef[1] : 0.0, coef[0], bk[0], ldp, sp, 3, s) ==
           cudaSuccess;
    } else {
      const int d = degree;
      ok = launch_cheb_affine_split(A, lda, n, am, bm, 1.0, 0.0, tp, ldp, sp, P, s) == cudaSuccess &&
           // B_d = c_d I and B_{d-1} = c_{d-1} I + 2 c_d T need no product
           launch_cheb_affine_split(A, lda, n, am, bm, 0.0, coef[d], bk[d % 3], ldp, sp, 3, s) == cudaSuccess &&
           launch_cheb_affine_split(A, lda, n, am, bm, 2.0 * coef[d], coef[d - 1], bk[(d - 1) % 3], ldp, sp, 3, s) ==
               cudaSuccess;
      // B_k = 2 T B_{k+1} - B_{k+2} + c_k I for k = d-2..1, then F = T B_1 - B_2 + c_0 I (into B_0's slot)
      for (int k = d - 2; k >= 0 && ok; --k) {
        TcArgs g{};
        g.M = n; g.N = n; g.K = n;
        g.a = op_planes(tp, n, n, ldp, sp, 0);               // T is symmetric: its K x M view is itself
        g.b = op_planes(bk[(k + 1) % 3], n, n, ldp, sp, 0);
        g.nplanes = P;
        g.epi = TC_EPI_CLENSHAW; g.triangular = 1;
        g.alpha = k > 0 ? 2.0f : 1.0f; g.beta = -1.0f; g.diag = (float)coef[k];
        g.x_planes = bk[(k + 2) % 3]; g.ldxp = ldp; g.x_plane_stride = sp;
        g.out_planes = bk[k % 3]; g.ldo = ldp; g.out_plane_stride = sp; g.out_nplanes = 3;
        g.st = st;
        ok = launch_tc_gemm(g, s) == cudaSuccess;
      }
    }
    if (!ok) break;
    if (launch_planes_to_f32(bk[0], ldp, sp, n, n, F, ldf, s) != cudaSuccess) break;
    DevState h;
    if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
    ret = (h.err_flags || h.status == ST_TIMEOUT) ? POLAR_ETIMEOUT : POLAR_OK;
  } while (0);
  cudaStreamSynchronize(s);
  cudaFree(ws);
  if (ret == POLAR_ECUDA) cudaGetLastError();
  return ret;
}

extern "C" polar_status_t polar_quantize_e4m3(const float* X, int64_t rows, int64_t cols, int64_t ldx, float* Y,
                                             int64_t ldy, polar_stream_t stream) {
  if (rows < 0 || cols < 0) return POLAR_EINVAL;
  if (rows == 0 || cols == 0) return POLAR_OK;
  if (!X || !Y || ldx < cols || ldy < cols) return POLAR_EINVAL;
  if (!device_ok()) { cudaGetLastError(); return POLAR_ECUDA; }
  return launch_quantize_e4m3_f32(X, ldx, rows, cols, Y, ldy, (cudaStream_t)stream) == cudaSuccess ? POLAR_OK
                                                                                                  : POLAR_ECUDA;
}
