"""CPU oracle for the Newton-Schulz polar factorisation (arXiv 2112.09017, Sec. III.D).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check in
``__graft_entry__.smoke`` and the CPU-baseline leg of ``bench.py`` may import
anything from here. The CUDA library never does, and shares no code with it.

Modules:
  ns_polar    float64 Newton-Schulz polar factorisation, Frobenius scaling,
              residual stop rule, H = sym(U^T A), and the error metrics
  scalar      the scalar recurrences (Eqs. NS_scalar, a_def, RogueScalar) and
              the exact-arithmetic residual trajectory predicted from a spectrum
  jacobi_svd  one-sided Jacobi SVD, the independent checker on small inputs
  precision   bit-level BF16 plane split, an emulator of split products, FP8 E4M3
              rounding with per-tile power-of-two scales, and the whole solve under
              each precision schedule (the precision model)
  ns_inverse  the Newton-Schulz matrix inverse of Algorithm 2 and its trajectory
              predicted from a spectrum
  chebyshev   Chebyshev interpolation and Clenshaw summation of a matrix function
              of a symmetric matrix (Eqs. MatFuncEig, EigenvaluePolynomial)
"""
from . import chebyshev, jacobi_svd, ns_inverse, ns_polar, precision, scalar  # noqa: F401
