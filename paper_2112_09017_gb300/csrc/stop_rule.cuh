// The stop rule of one step of a batched problem, shared by the batched finalize
// kernel and the on-chip small-problem kernel.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace polar {

// Records the residual r = ||X_k^T X_k - I||_F / sqrt(n) of step k in s and applies the
// rule: converged when r <= tol; not converged on stagnation (r > stagnation * r2, r2 the
// residual of step k - 2, while r < stag_floor) or at max_iter; no test during
// Algorithm 1's preconditioning steps. Returns true while the problem keeps running,
// having set the coefficients c1, c3 of update k (a, -(4/27) a^3 while preconditioning,
// then 1.5, -0.5: Eqs. RogueMatrix and NewtonSchulz), also into s.
__device__ __forceinline__ bool batched_step_rule(DevState& s, const StopRule& rule, double tol, double r, double r2,
                                                  int k, int planes, float& c1, float& c3) {
  if (k < POLAR_HIST) {
    s.res_hist[k] = r;
    s.planes_hist[k] = (unsigned char)planes;
    s.hist_len = k + 1;
  }
  s.ring[k & 3] = r;
  s.iters = k;
  const bool testing = k >= rule.n_pre;
  if (!isfinite(r)) s.status = ST_NONFINITE;
  else if (testing && r <= tol) s.status = ST_CONVERGED;
  else if (testing && k >= rule.n_pre + 2 && r > rule.stagnation * r2 && r < rule.stag_floor)
    s.status = ST_NOT_CONVERGED;
  else if (k >= rule.max_iter) s.status = ST_NOT_CONVERGED;
  else {
    update_coeffs(rule, k, c1, c3);
    s.upd_c1 = c1;
    s.upd_c3 = c3;
    return true;
  }
  return false;
}

}  // namespace polar
