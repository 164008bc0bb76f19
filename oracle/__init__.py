"""CPU oracle for the layered 3D-IC thermal solve (test infrastructure).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct FP64
implementation of what the GPU solver computes, written from the paper's
equations and algorithms:

* ``discretisation`` - the 7-point finite-volume rows of Eq. (steady-state) and
  Eq. (transient) (Sec. 3.2), assembled into a CSR matrix row by row.
* ``krylov``         - PCG (Algorithm 1), the Jacobi and identity preconditioners
  (Sec. 5.7), the Chebyshev polynomial preconditioner (Algorithm "Chebyshev
  Polynomial Preconditioning", Sec. 4.3) and the Lanczos spectral estimate
  (Sec. 4.3, last paragraph).
* ``solve``          - exact steady and backward-Euler solutions (the definition
  of the method's result), relative residuals, the error metric of Sec. 5.1.
* ``adjoint``        - the log-sum-exp hotspot objective and its adjoint gradient
  with respect to the power map and the per-layer conductivities.
* ``precision``      - the reduced-precision pieces of the paper's adaptive scheme
  (Sec. 4.4): Quad-Diag storage (Sec. 4.2), the FP32/16 product of Algorithm 3 and
  the early-to-late stage switch, Eqs. (switch_a-c).
* ``multigrid``      - the geometric multigrid V-cycle (not in the paper: the
  alternative preconditioner), aggregation, Galerkin coarse operators, damped
  z-line Jacobi smoothing and an exact coarsest solve.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import it.  The GPU library never imports, links or runs
anything here, and this package imports nothing from the GPU library; both take
their inputs from ``thermal_inputs``, which holds no solver arithmetic.

Parity status: every function here is pinned by a test in
``tests/test_oracle_pins.py`` except the iteration counts and mixed-precision
drift magnitudes the paper prints for its (unavailable) benchmark matrices, which
are "parity unpinned".
"""
from . import discretisation, krylov, solve, adjoint  # noqa: F401
