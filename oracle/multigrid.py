"""Geometric multigrid preconditioner (oracle).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` use this module.

Not in the paper: the robust alternative to the Chebyshev preconditioner for stacks
whose layers are in-plane dominated (Si, Cu) or vertically dominated (BEOL, TIM,
bonds) at once.  One V-cycle is M^{-1} r:

* Hierarchy: semi-coarsening in x and y only (all layers kept).  A coarse cell
  aggregates the 2 x 2 fine columns (2X, 2X+1) x (2Y, 2Y+1) of its layer (one or two
  on an odd edge); prolongation P is piecewise constant over the aggregate,
  restriction R = P^T, and the coarse operator is the Galerkin product P^T A P.
  Levels are added while max(nx, ny) > 8.
* Smoother: damped z-line Jacobi, x <- x + omega T^{-1} (b - A x), T = the
  tridiagonal block of A over each (x, y) column (diagonal and vertical couplings),
  omega = 0.8, nu sweeps before and nu after the coarse correction.
* Coarsest level: exact solve (dense Cholesky).
The cycle starts from x = 0 on every level; the smoother is symmetric and
pre/post sweeps match, so M^{-1} is symmetric (required by PCG).

parity pinned by: Galerkin coarse operators equal to the summed-face 7-point
operators, the symmetry of M^{-1}, the one-column case (z-line sweep with omega = 1
is the exact solve) and the two-grid error reduction (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import krylov

OMEGA = 0.8
COARSEST = 8


def coarse_dims(nx, ny):
    return (nx + 1) // 2, (ny + 1) // 2


def prolongation(nx, ny, L):
    """Piecewise-constant P (fine x coarse) of the 2 x 2-column aggregation."""
    nxc, nyc = coarse_dims(nx, ny)
    n = nx * ny * L
    i = np.arange(n)
    x = i % nx
    y = (i // nx) % ny
    z = i // (nx * ny)
    ic = x // 2 + nxc * (y // 2 + nyc * z)
    return sp.csr_matrix((np.ones(n), (i, ic)), shape=(n, nxc * nyc * L))


def hierarchy(A, nx, ny, L):
    """[(A_l, nx_l, ny_l, P_l)] from the finest level down; P_l maps level l+1 to l
    (None on the coarsest)."""
    levels = []
    A = A.tocsr()
    while max(nx, ny) > COARSEST:
        P = prolongation(nx, ny, L)
        levels.append((A, nx, ny, P))
        A = (P.T @ A @ P).tocsr()
        nx, ny = coarse_dims(nx, ny)
    levels.append((A, nx, ny, None))
    return levels


def vcycle(levels, L, b, nu=1, omega=OMEGA):
    """One V-cycle from x = 0: an approximation of A^{-1} b."""
    smoothers = [krylov.zline(A, nx, ny, L) for (A, nx, ny, _) in levels[:-1]]
    Ac = levels[-1][0].toarray()
    coarse = np.linalg.cholesky(Ac)

    def cycle(l, rhs):
        if l == len(levels) - 1:
            y = np.linalg.solve(coarse, rhs)
            return np.linalg.solve(coarse.T, y)
        A, nx, ny, P = levels[l]
        Tinv = smoothers[l]
        x = np.zeros_like(rhs)
        for _ in range(nu):
            x = x + omega * Tinv(rhs - A @ x)
        xc = cycle(l + 1, P.T @ (rhs - A @ x))
        x = x + P @ xc
        for _ in range(nu):
            x = x + omega * Tinv(rhs - A @ x)
        return x

    return cycle(0, np.asarray(b, dtype=np.float64))


def preconditioner(A, nx, ny, L, nu=1, omega=OMEGA):
    """M^{-1} as a callable for ``krylov.pcg``."""
    levels = hierarchy(A, nx, ny, L)
    return lambda r: vcycle(levels, L, r, nu, omega)
