"""Exact steady and backward-Euler solutions (oracle).

The method's result is, up to its stopping tolerance, the solution of the linear
system of Eq. (steady-state) or Eq. (transient).  The oracle therefore computes
that solution directly:

* N <= 4096: dense Cholesky of A (textbook, via numpy's factorisation routine);
* otherwise: sparse LU (SuperLU through scipy) when N <= ``DIRECT_MAX``;
* larger: Algorithm 1 with the Jacobi preconditioner to ||r||/||b|| <= 1e-13 with
  the true residual recomputed at the end.

Temperatures are returned in deg C.  ``rel_residual`` measures
||b - A T|| / ||b_theta|| where b_theta = b - A (T_amb * 1) is the right-hand side of
the same system written for the temperature rise theta = T - T_amb (the residual
vectors of the two forms are equal because every row of the conduction part sums
to zero).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import discretisation as disc
from . import krylov

DIRECT_MAX = 400_000


def cholesky_solve(A, b):
    Ad = A.toarray()
    Lc = np.linalg.cholesky(Ad)
    y = np.linalg.solve(Lc, b)          # forward substitution (dense)
    return np.linalg.solve(Lc.T, y)     # backward substitution


def solve_exact(A, b, tol_rel=1e-13, x0=None):
    n = A.shape[0]
    if n <= 4096:
        return cholesky_solve(A, b)
    if n <= DIRECT_MAX:
        return spla.splu(A.tocsc()).solve(b)
    op = krylov.CountingOp(A)
    x, _, _, _ = krylov.pcg(op, b, krylov.jacobi(A), x0=x0, tol_rel=tol_rel, maxit=200000)
    return x


class Factorised:
    """A reusable exact solver for one matrix (used across backward-Euler steps)."""

    def __init__(self, A, tol_rel=1e-13):
        self.A = A
        self.tol_rel = tol_rel
        n = A.shape[0]
        self.lu = spla.splu(A.tocsc()) if n <= DIRECT_MAX else None

    def __call__(self, b, x0=None):
        if self.lu is not None:
            return self.lu.solve(b)
        op = krylov.CountingOp(self.A)
        x, _, _, _ = krylov.pcg(op, b, krylov.jacobi(self.A), x0=x0, tol_rel=self.tol_rel,
                                maxit=200000)
        return x


def steady(nx, ny, stack, power, half_cell_top=False, k_cell=None):
    """Temperatures (deg C) of Eq. (steady-state) for a power map in W per cell."""
    A = disc.assemble(nx, ny, stack, half_cell_top=half_cell_top, k_cell=k_cell)
    b = disc.rhs_steady(nx, ny, stack, power, half_cell_top)
    return solve_exact(A, b)


def transient(nx, ny, stack, power_schedule, dt, T0, half_cell_top=False, tol_rel=1e-13):
    """Backward-Euler trajectory of Eq. (transient).

    ``power_schedule`` is a list with the power map p_{n+1} of every step.  Returns
    the list of T_{n+1} (deg C) after each step, starting from T0.
    """
    A = disc.assemble(nx, ny, stack, dt=dt, half_cell_top=half_cell_top)
    solver = Factorised(A, tol_rel)
    T = np.asarray(T0, dtype=np.float64)
    out = []
    for p in power_schedule:
        b = disc.rhs_transient(nx, ny, stack, p, T, dt, half_cell_top)
        T = solver(b, x0=T)
        out.append(T)
    return out


def rel_residual(A, T, b, t_amb):
    """||b - A T||_2 / ||b - A t_amb 1||_2 in FP64 (relative residual of the theta system)."""
    r = b - A @ T
    b_theta = b - A @ np.full_like(T, t_amb)
    return float(np.linalg.norm(r) / np.linalg.norm(b_theta))


def rise_relative_error(T, T_ref, t_amb):
    """max_i |T_i - T_ref,i| / max_i |T_ref,i - T_amb| (error relative to the temperature rise)."""
    return float(np.max(np.abs(np.asarray(T) - T_ref)) / np.max(np.abs(T_ref - t_amb)))


def inf_error(T, T_ref):
    """||e||_inf = max_i |x_exact - x_evaluated| (Sec. 5.1), in K."""
    return float(np.max(np.abs(np.asarray(T) - T_ref)))
