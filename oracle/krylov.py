"""Krylov building blocks of the oracle: PCG, preconditioners, Lanczos.

* ``pcg``        - Algorithm 1 (Preconditioned Conjugate Gradient), Sec. 3.3.
* ``identity`` / ``jacobi`` - the two baseline preconditioners of Sec. 5.7.
* ``chebyshev``  - Algorithm "Chebyshev Polynomial Preconditioning" (Sec. 4.3):
  k steps of the recurrence with sigma_1 = theta/delta, rho_0 = 1/sigma_1,
  d_0 = r/theta, theta = (lmax+lmin)/2, delta = (lmax-lmin)/2.
* ``lanczos``    - the Lanczos reduction to a tridiagonal T whose extreme
  eigenvalues estimate the spectral interval (Sec. 4.3, last paragraph).
* ``splitmix64_uniform`` - the counter-based generator (SplitMix64, Steele, Lea and
  Flood, OOPSLA 2014) both sides use for the Lanczos start vector.

Every function works in FP64 on numpy arrays; operators are plain callables.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class CountingOp:
    """y = A x for a scipy sparse A (or any callable), counting applications (N_SpMV)."""

    def __init__(self, A):
        self.A = A
        self.count = 0

    def __call__(self, x):
        self.count += 1
        if callable(self.A):
            return self.A(x)
        return self.A @ x


def identity():
    """M^{-1} = I (plain CG, Sec. 5.7)."""
    return lambda r: r.copy()


def jacobi(A):
    """M^{-1} = diag(A)^{-1} (Jacobi, Sec. 5.7)."""
    inv = 1.0 / A.diagonal()
    return lambda r: inv * r


def chebyshev(op, r_cg, lam_min, lam_max, k):
    """Algorithm "Chebyshev Polynomial Preconditioning": z_cg ~ A^{-1} r_cg.

    ``op`` applies A.  The loop runs k times; each pass adds d to z, applies A to
    d once, updates the Chebyshev residual and forms the next d.  z starts at 0.
    """
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    r = np.array(r_cg, dtype=np.float64, copy=True)
    sigma1 = theta / delta
    rho = 1.0 / sigma1
    d = r / theta
    z = np.zeros_like(r)
    for _ in range(k):
        z = z + d
        Ad = op(d)
        r = r - Ad
        rho_next = 1.0 / (2.0 * sigma1 - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * r
        rho = rho_next
    return z


def chebyshev_residual_poly(lam, lam_min, lam_max, k):
    """P_k(lambda) = C_k((theta - lambda)/delta) / C_k(theta/delta) (Sec. 4.3, minimax).

    C_k is evaluated by its three-term recurrence C_k = 2x C_{k-1} - C_{k-2}.
    """
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)

    def C(x):
        x = np.asarray(x, dtype=np.float64)
        c0, c1 = np.ones_like(x), x.copy()
        if k == 0:
            return c0
        for _ in range(k - 1):
            c0, c1 = c1, 2.0 * x * c1 - c0
        return c1

    return C((theta - np.asarray(lam)) / delta) / C(theta / delta)


def pcg(op, b, precond, x0=None, eps_abs=None, tol_rel=None, maxit=100000):
    """Algorithm 1 (PCG).  Stops when ||r_k||_2 <= eps (absolute, as in Sec. 5.1) or
    when ||r_k||_2 <= tol_rel * ||b||_2.

    ``op`` is a CountingOp (its count gives N_SpMV: one for r_0, one per iteration,
    plus whatever the preconditioner applies).  After the loop the true residual
    ||b - A x|| is recomputed once, which is counted as one more application.
    Returns (x, n_iter, history of ||r_k||, true residual norm).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bn = np.linalg.norm(b)
    eps = eps_abs if eps_abs is not None else tol_rel * bn
    r = b - op(x)
    z = precond(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r)]
    k = 0
    while hist[-1] > eps and k < maxit:
        mu = op(p)
        pmu = p @ mu
        alpha = rz / pmu
        x = x + alpha * p
        r = r - alpha * mu
        z = precond(r)
        rz_next = r @ z
        beta = rz_next / rz
        p = z + beta * p
        rz = rz_next
        k += 1
        hist.append(np.linalg.norm(r))
    true_res = np.linalg.norm(b - op(x))
    return x, k, hist, true_res


def splitmix64_uniform(n, seed):
    """Counter-based uniform numbers in [-1, 1): element i is SplitMix64 of
    state seed + (i+1)*0x9E3779B97F4A7C15, top 53 bits scaled to [0,1), mapped to [-1,1).
    """
    M = np.uint64(0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        s = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
        z = s & M
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def lanczos(op, v0, m):
    """m steps of Lanczos (no reorthogonalisation) from v0.

    Returns the diagonal alpha[0..m-1] and off-diagonal beta[0..m-2] of T.  Stops
    early if an invariant subspace is found (beta == 0).
    """
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    beta_prev = 0.0
    alphas, betas = [], []
    for j in range(m):
        w = op(v) - beta_prev * v_prev
        a = w @ v
        w = w - a * v
        alphas.append(a)
        bnorm = np.linalg.norm(w)
        if j == m - 1 or bnorm == 0.0:
            break
        betas.append(bnorm)
        v_prev, v = v, w / bnorm
        beta_prev = bnorm
    return np.array(alphas), np.array(betas)


def ritz_extremes(alpha, beta):
    """Smallest and largest eigenvalue of the symmetric tridiagonal T (FP64, host)."""
    ev = sla.eigh_tridiagonal(alpha, beta, eigvals_only=True)
    return float(ev[0]), float(ev[-1])


def chebyshev_bounds(theta_min, theta_max, inflate=1.05, min_ratio=1e-7):
    """Interval used by the preconditioner from Lanczos Ritz values.

    The paper does not state the margins.  Reading: lmax = 1.05 * theta_max (Ritz
    values approach lmax from below, and an over-estimate keeps M^{-1} SPD);
    lmin = max(theta_min, lmax * 1e-7).
    """
    lmax = inflate * theta_max
    lmin = max(theta_min, lmax * min_ratio)
    return lmin, lmax


def jacobi_scaled(A):
    """The operator D^{-1/2} A D^{-1/2} (symmetric Jacobi scaling) and D^{-1/2}."""
    s = 1.0 / np.sqrt(A.diagonal())
    return (lambda x: s * (A @ (s * x))), s


def zline(A, nx, ny, L):
    """Block Jacobi with one block per (x, y) column: the L x L submatrix of A over the
    column's cells (main diagonal and the vertical couplings), solved densely per column.
    (Not in the paper; the z-line alternative the GPU path offers.)
    """
    Ad = A.tocsr()
    blocks = []
    for y in range(ny):
        for x in range(nx):
            idx = np.array([x + nx * (y + ny * z) for z in range(L)])
            blocks.append((idx, np.linalg.inv(Ad[idx][:, idx].toarray())))

    def apply(r):
        z = np.zeros_like(r, dtype=np.float64)
        for idx, inv in blocks:
            z[idx] = inv @ r[idx]
        return z
    return apply
