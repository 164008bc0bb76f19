"""Hotspot objective and its adjoint gradient (oracle, FP64).

Objective: the log-sum-exp smooth maximum of the temperatures of the selected
(silicon) cells, J = (1/beta) log sum_{i in S} exp(beta T_i), computed with the
maximum subtracted for stability.  Its gradient w.r.t. T is w = softmax(beta T)
on S and 0 elsewhere.

Because A T = b with A symmetric positive definite (Sec. 3.2: A is SPD), the
gradient of J w.r.t. any parameter q of the system is lambda^T (db/dq - dA/dq T)
with the adjoint state A lambda = w.  Hence:

* dJ/dP_i  = lambda_i               (b = P + h S T_amb, P in W per cell);
* dJ/dk_l  = -lambda^T (dA/dk_l) T  (b does not depend on k);
* dJ/dh    = -sum_{top} lambda_i S (T_i - T_amb)  (convective face h S on the top layer).
"""
from __future__ import annotations

import numpy as np

from . import discretisation as disc
from . import solve


def silicon_mask(nx, ny, stack, layers):
    m = np.zeros((stack.L, ny, nx), dtype=bool)
    for l in layers:
        m[l] = True
    return m.reshape(-1)


def lse(T, mask, beta):
    """(J, w): smooth maximum of T over mask and its gradient dJ/dT."""
    t = np.asarray(T, dtype=np.float64)[mask]
    m = t.max()
    e = np.exp(beta * (t - m))
    s = e.sum()
    J = m + np.log(s) / beta
    w = np.zeros(np.asarray(T).size)
    w[mask] = e / s
    return float(J), w


def objective(nx, ny, stack, power, mask, beta):
    """J for a power map (solves the steady system exactly)."""
    T = solve.steady(nx, ny, stack, power)
    return lse(T, mask, beta)[0]


def gradient(nx, ny, stack, power, mask, beta, T=None):
    """(J, dJ/dP [W^-1 per cell], dJ/dk [per layer], dJ/dh, lambda) via one adjoint solve."""
    A = disc.assemble(nx, ny, stack)
    if T is None:
        T = solve.solve_exact(A, disc.rhs_steady(nx, ny, stack, power))
    J, w = lse(T, mask, beta)
    lam = solve.solve_exact(A, w)           # A^T = A
    dJdk = np.array([-(lam @ (disc.d_matrix_d_layer_k(nx, ny, stack, l) @ T))
                     for l in range(stack.L)])
    S = stack.dx * stack.dy
    top = slice((stack.L - 1) * nx * ny, stack.L * nx * ny)
    dJdh = -float(np.sum(lam[top] * S * (T[top] - stack.t_amb)))
    return J, lam.copy(), dJdk, dJdh, lam
