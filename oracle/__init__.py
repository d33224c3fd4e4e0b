"""FP64 CPU oracle for the Levenberg-Marquardt graph optimiser (test infrastructure).

This package is a plain, slow, obviously correct restatement of what the GPU path
computes, written from the paper's equations:

* Eq. 1-2   total cost 1/2 sum r^T Sigma^-1 r over the constraints;
* Eq. 3-6   LM linearisation, damped step minimiser and normal equations
            (J^T S^-1 J + lambda D^T D) dx = -J^T S^-1 r;
* Eq. 7     Huber robust kernel on the reprojection terms;
* Eq. 8     visual-inertial terms (inertial and bias residuals);
* Sec. IV-E Hessian-diagonal clamping of the damping matrix.

The reduced camera system is formed densely and solved with a dense Cholesky
factorisation; the eliminated points are recovered by back-substitution.  All
arithmetic is float64 numpy / scipy.

It is test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the library and its Python binding never do, and
the oracle never imports them.  It shares no code with the CUDA path.
"""
from . import so3, robust, ba, lm, generic  # noqa: F401
