"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form,
an invariant, a textbook/library routine, brute force on a tiny grid, or numbers
the paper prints.  A plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed operand) fails at least one of them.
"""
import numpy as np
import numpy.polynomial.chebyshev as npcheb
import pytest

import thermal_inputs as ti
from oracle import adjoint, discretisation as disc, krylov, solve
from conftest import read_golden


def uniform_power(stack, nx, ny, q_wcm2=20.0):
    dens = [np.full((ny, nx), q_wcm2) for _ in stack.power_layers()]
    return ti.power_cells(stack, nx, ny, dens, np.float64)


# ----------------------------------------------------------------- discretisation

@pytest.mark.parametrize("nx,ny", [(8, 8), (5, 3), (1, 1)])
@pytest.mark.parametrize("half", [False, True])
def test_slab_golden_c1(nx, ny, half):
    """Eq. (steady-state) on a laterally uniform slab equals the hand-derived layer temperatures."""
    rows = read_golden("slab_c1_uniform.txt")
    want = {r[0]: float(r[2] if half else r[1]) for r in rows}
    st = ti.stack_c1()
    T = solve.steady(nx, ny, st, uniform_power(st, nx, ny), half_cell_top=half)
    T = T.reshape(st.L, ny, nx)
    for l, layer in enumerate(st.layers):
        name = {"si": "si", "beol": "beol", "tim": "tim", "cu": "cu"}[layer.name]
        np.testing.assert_allclose(T[l], want[name], rtol=1e-10, atol=0)


def test_slab_series_closed_form_multi_source():
    """Two powered layers (8-layer stack): column temperatures from the series-resistance chain.

    theta_top = Q_total/(h S); crossing the face between layers l and l+1 downwards adds
    (power generated in layers <= l) / g_{l,l+1}.
    """
    st = ti.stack_c2()
    nx, ny = 4, 3
    T = solve.steady(nx, ny, st, uniform_power(st, nx, ny, 37.0)).reshape(st.L, ny, nx)
    S = st.dx * st.dy
    Q = np.zeros(st.L)
    for l in st.power_layers():
        Q[l] = 37.0 * 1e4 * S
    theta = np.zeros(st.L)
    theta[-1] = Q.sum() / (st.h * S)
    for l in range(st.L - 2, -1, -1):
        a, b = st.layers[l], st.layers[l + 1]
        R = a.thickness / (2 * a.k * S) + b.thickness / (2 * b.k * S)
        theta[l] = theta[l + 1] + Q[: l + 1].sum() * R
    for l in range(st.L):
        np.testing.assert_allclose(T[l] - st.t_amb, theta[l], rtol=1e-10)


def _bruteforce_apply(nx, ny, stack, x, dt=None):
    """Face-by-face application of Eq. (steady-state)/(transient) in pure Python loops.

    Enumerates every interior face once and adds g (x_a - x_b) to a and g (x_b - x_a)
    to b, then the convective and capacity terms: a second, loop-based statement of
    the discretisation that shares nothing with the row-wise CSR assembly.
    """
    L = stack.L
    dx, dy = stack.dx, stack.dy
    y = np.zeros(nx * ny * L)
    ks = [l.k for l in stack.layers]
    dzs = [l.thickness for l in stack.layers]

    def at(x_, y_, z_):
        return x_ + nx * (y_ + ny * z_)

    for z in range(L):
        for j in range(ny):
            for i in range(nx):
                a = at(i, j, z)
                if i + 1 < nx:
                    g = ks[z] * dy * dzs[z] / dx
                    b = at(i + 1, j, z)
                    y[a] += g * (x[a] - x[b]); y[b] += g * (x[b] - x[a])
                if j + 1 < ny:
                    g = ks[z] * dx * dzs[z] / dy
                    b = at(i, j + 1, z)
                    y[a] += g * (x[a] - x[b]); y[b] += g * (x[b] - x[a])
                if z + 1 < L:
                    g = dx * dy / (dzs[z] / (2 * ks[z]) + dzs[z + 1] / (2 * ks[z + 1]))
                    b = at(i, j, z + 1)
                    y[a] += g * (x[a] - x[b]); y[b] += g * (x[b] - x[a])
                if z == L - 1:
                    y[a] += stack.h * dx * dy * x[a]
                if dt is not None:
                    y[a] += stack.layers[z].c * dx * dy * dzs[z] / dt * x[a]
    return y



# ----------------------------------------------------------------- error metrics (Sec. 5.1)

def _two_cell_column():
    """A 1 x 1 x 2 column worked by hand: face conductance g = 2 W/K between the cells,
    top sink hS = 3 W/K, T_amb = 45 C, power P = (1, 0.5) W.  The rows of
    Eq. (steady-state) are g(T0 - T1) = P0 and g(T1 - T0) + hS T1 = P1 + hS T_amb,
    whose solution is theta = T - T_amb = (1.0, 0.5) K."""
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[2.0, -2.0], [-2.0, 5.0]]))
    b = np.array([1.0, 0.5 + 3.0 * 45.0])
    return A, b, 45.0


def test_rel_residual_hand_computed():
    """||b - A T|| / ||b_theta||: for T = T_amb + (1.1, 0.5) the residual is (-0.2, 0.2)
    and b_theta = P = (1, 0.5), so the value is 0.2 sqrt(2) / sqrt(1.25) = 0.252982...
    Normalising by ||b|| (which holds hS T_amb = 135) would give 0.00209 instead."""
    A, b, ta = _two_cell_column()
    exact = ta + np.array([1.0, 0.5])
    assert solve.rel_residual(A, exact, b, ta) == 0.0
    T = ta + np.array([1.1, 0.5])
    want = 0.2 * np.sqrt(2.0) / np.sqrt(1.25)
    assert abs(solve.rel_residual(A, T, b, ta) - want) <= 1e-14
    assert abs(np.linalg.norm(b - A @ T) / np.linalg.norm(b) - want) > 0.2   # the other normalisation
    # scale invariance of a relative residual: P and theta scaled together
    T2 = ta + 7.0 * np.array([1.1, 0.5])
    b2 = np.array([7.0, 3.5 + 3.0 * 45.0])
    assert abs(solve.rel_residual(A, T2, b2, ta) - want) <= 1e-13


def test_rise_relative_and_inf_error_hand_computed():
    """max|T - T_ref| / max|T_ref - T_amb| = 0.1 / 1.0 for the column above; relative to
    the absolute temperature (about 46 C) it would be 0.00217.  ||e||_inf = 0.1 K."""
    ta = 45.0
    T_ref = ta + np.array([1.0, 0.5])
    T = ta + np.array([1.1, 0.45])
    assert abs(solve.rise_relative_error(T, T_ref, ta) - 0.1) <= 1e-13
    assert abs(solve.inf_error(T, T_ref) - 0.1) <= 1e-13
    # the metric is symmetric in sign and unchanged by a common shift of T_amb
    assert abs(solve.rise_relative_error(2 * T_ref - T, T_ref, ta) - 0.1) <= 1e-13
    assert abs(solve.rise_relative_error(T + 10, T_ref + 10, ta + 10) - 0.1) <= 1e-12


def test_rel_residual_on_an_assembled_stack_matches_theta_system():
    """On an assembled stack the metric equals ||P - G theta|| / ||P|| computed from the
    theta form directly (G = A, b_theta = P: every conduction row sums to zero)."""
    st = ti.stack_c1()
    nx, ny = 6, 5
    A = disc.assemble(nx, ny, st)
    P = uniform_power(st, nx, ny)
    b = disc.rhs_steady(nx, ny, st, P)
    theta = ti.random_vector(A.shape[0], 4, lo=0.0, hi=30.0)
    want = np.linalg.norm(P - A @ theta) / np.linalg.norm(P)
    got = solve.rel_residual(A, st.t_amb + theta, b, st.t_amb)
    assert abs(got - want) <= 1e-12 * want


@pytest.mark.parametrize("nx,ny,mk", [(3, 2, "c1"), (4, 5, "c2"), (1, 3, "mol")])
@pytest.mark.parametrize("dt", [None, 1e-4])
def test_assembly_matches_bruteforce(nx, ny, mk, dt):
    st = {"c1": ti.stack_c1(), "c2": ti.stack_c2(), "mol": ti.stack_mol()}[mk]
    A = disc.assemble(nx, ny, st, dt=dt)
    x = ti.random_vector(A.shape[0], 7)
    np.testing.assert_allclose(A @ x, _bruteforce_apply(nx, ny, st, x, dt), rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("dt", [None, 2e-4])
def test_matrix_structure(dt):
    """Symmetry, sign pattern, 7 diagonals (Sec. 3.2) and row sums A 1 = h S (+ C V/dt)."""
    st = ti.stack_c2()
    nx, ny = 6, 5
    A = disc.assemble(nx, ny, st, dt=dt)
    assert (abs(A - A.T)).max() == 0.0
    off = A - __import__("scipy.sparse", fromlist=["diags"]).diags(A.diagonal())
    assert off.max() <= 0.0
    # at most 7 distinct diagonals: offsets 0, +-1, +-nx, +-nx*ny
    coo = A.tocoo()
    assert set(np.unique(coo.col - coo.row)) <= {0, 1, -1, nx, -nx, nx * ny, -nx * ny}
    expect = disc.top_sink(nx, ny, st)
    if dt is not None:
        expect = expect + disc.capacity_over_dt(nx, ny, st, dt)
    # rounding floor: a few ulps of the largest conductance in a row
    np.testing.assert_allclose(A @ np.ones(A.shape[0]), expect, rtol=1e-12, atol=1e-15 * abs(A).max())
    np.testing.assert_allclose(A.diagonal(), -np.asarray(off.sum(axis=1)).ravel() + expect, rtol=1e-14)


def test_energy_balance_c1():
    """Sum of injected power equals convective outflow sum_top h S theta (to 1e-9)."""
    inst = ti.c1(dtype=np.float64)
    st = inst.stack
    T = solve.steady(inst.nx, inst.ny, st, inst.power)
    top = T[(st.L - 1) * inst.nx * inst.ny:]
    out = np.sum(st.h * st.dx * st.dy * (top - st.t_amb))
    assert abs(out - inst.power.sum()) / inst.power.sum() < 1e-9


def test_superposition_and_scaling():
    st = ti.stack_c1()
    nx, ny = 12, 9
    p1 = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 3)], np.float64)
    p2 = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, 4)], np.float64)
    th = lambda p: solve.steady(nx, ny, st, p) - st.t_amb
    np.testing.assert_allclose(th(p1 + p2), th(p1) + th(p2), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(th(2.5 * p1), 2.5 * th(p1), rtol=1e-10, atol=1e-12)


def test_direct_paths_agree():
    """Dense Cholesky, sparse LU and Algorithm 1 (Jacobi, 1e-13) give the same solution."""
    st = ti.stack_c1()
    nx, ny = 16, 16
    A = disc.assemble(nx, ny, st)
    b = disc.rhs_steady(nx, ny, st, ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 5)]))
    x_ch = solve.cholesky_solve(A, b)
    x_lu = __import__("scipy.sparse.linalg", fromlist=["spsolve"]).spsolve(A.tocsc(), b)
    x_cg, it, _, _ = krylov.pcg(krylov.CountingOp(A), b, krylov.jacobi(A), tol_rel=1e-14)
    np.testing.assert_allclose(x_lu, x_ch, rtol=1e-12)
    np.testing.assert_allclose(x_cg, x_ch, rtol=1e-11)


# ----------------------------------------------------------------- Algorithm 1

def test_pcg_finite_termination():
    """CG on a matrix with m distinct eigenvalues terminates in m iterations (exact-arithmetic theory)."""
    import scipy.sparse as sp
    vals = np.repeat([1.0, 2.0, 5.0, 11.0, 30.0], 20)
    A = sp.diags(vals).tocsr()
    b = ti.random_vector(vals.size, 11)
    x, it, hist, true_res = krylov.pcg(krylov.CountingOp(A), b, krylov.identity(), tol_rel=1e-12)
    assert it == 5
    np.testing.assert_allclose(x, b / vals, rtol=1e-10)


def test_pcg_residual_history_monotone_energy():
    """PCG error in the A-norm decreases monotonically (a defining property of CG)."""
    st = ti.stack_c1()
    nx, ny = 10, 10
    A = disc.assemble(nx, ny, st)
    b = ti.random_vector(A.shape[0], 3, lo=0.0, hi=1e-4)
    xs = solve.cholesky_solve(A, b)
    errs = []
    for m in range(1, 25):
        x, _, _, _ = krylov.pcg(krylov.CountingOp(A), b, krylov.jacobi(A), tol_rel=0.0, maxit=m)
        e = x - xs
        errs.append(e @ (A @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))


def test_nspmv_convention_golden_and_oracle():
    """The paper's N_SpMV equals (N_ite+1) k + N_ite + 2 for CUTh1-3, and the oracle counts the same way."""
    for bench, n_ite, n_spmv, k in read_golden("nspmv_counts.txt"):
        n_ite, n_spmv, k = int(n_ite), int(n_spmv), int(k)
        assert (n_ite + 1) * k + n_ite + 2 == n_spmv, bench
    st = ti.stack_c1()
    nx, ny = 12, 12
    A = disc.assemble(nx, ny, st)
    b = disc.rhs_steady(nx, ny, st, uniform_power(st, nx, ny))
    ev = np.linalg.eigvalsh(A.toarray())
    op = krylov.CountingOp(A)
    k = 30
    prec = lambda r: krylov.chebyshev(op, r, ev[0], 1.05 * ev[-1], k)
    x, n_ite, _, _ = krylov.pcg(op, b, prec, tol_rel=1e-12)
    assert n_ite > 0
    assert op.count == (n_ite + 1) * k + n_ite + 2


# ----------------------------------------------------------------- Chebyshev

def _cheb_closed(k, x):
    """Textbook first-kind Chebyshev polynomial via numpy's Chebyshev series (coefficient e_k)."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    return npcheb.chebval(x, c)


@pytest.mark.parametrize("k", [1, 2, 5, 30])
def test_chebyshev_spectral_closed_form(k):
    """z = V diag((1 - P_k(l))/l) V^T r with P_k(l) = C_k((theta-l)/delta)/C_k(theta/delta) (Sec. 4.3)."""
    st = ti.stack_c1()
    nx, ny = 5, 4
    A = disc.assemble(nx, ny, st)
    lam, V = np.linalg.eigh(A.toarray())
    lo, hi = lam[0] * 1.5, lam[-1] * 1.02
    r = ti.random_vector(A.shape[0], 13)
    z = krylov.chebyshev(krylov.CountingOp(A), r, lo, hi, k)
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    Pk = _cheb_closed(k, (theta - lam) / delta) / _cheb_closed(k, theta / delta)
    z_ref = V @ (((1.0 - Pk) / lam) * (V.T @ r))
    np.testing.assert_allclose(z, z_ref, rtol=1e-9, atol=1e-12 * np.abs(z_ref).max())
    np.testing.assert_allclose(krylov.chebyshev_residual_poly(lam, lo, hi, k), Pk, rtol=1e-10, atol=1e-300)


def test_chebyshev_minimax_level_and_spd():
    """max_{[a,b]} |P_k| = 1/C_k(theta/delta); M^{-1} is SPD when lmax is over-estimated."""
    a, b, k = 0.01, 2.0, 7
    grid = np.linspace(a, b, 20001)
    Pk = krylov.chebyshev_residual_poly(grid, a, b, k)
    theta, delta = (a + b) / 2, (b - a) / 2
    assert abs(np.abs(Pk).max() - 1.0 / np.cosh(k * np.arccosh(theta / delta))) < 1e-10
    st = ti.stack_c1()
    A = disc.assemble(4, 4, st)
    lam = np.linalg.eigvalsh(A.toarray())
    n = A.shape[0]
    M = np.column_stack([krylov.chebyshev(krylov.CountingOp(A), e, lam[0] * 3, lam[-1] * 1.05, 6)
                         for e in np.eye(n)])
    np.testing.assert_allclose(M, M.T, atol=1e-8 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


# ----------------------------------------------------------------- Lanczos

def test_splitmix64_published_vector():
    """SplitMix64 from state 0 gives 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    outs = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = krylov.splitmix64_uniform(3, 0)
    want = np.array([2.0 * ((o >> 11) / 2.0 ** 53) - 1.0 for o in outs])
    np.testing.assert_array_equal(u, want)


def test_lanczos_extremes_vs_eigvalsh():
    st = ti.stack_c2()
    nx, ny = 6, 6
    A = disc.assemble(nx, ny, st, dt=1e-4)
    lam = np.linalg.eigvalsh(A.toarray())
    a, b = krylov.lanczos(krylov.CountingOp(A), krylov.splitmix64_uniform(A.shape[0], 1), 60)
    lo, hi = krylov.ritz_extremes(a, b)
    assert abs(hi - lam[-1]) / lam[-1] < 0.01
    assert lo >= lam[0] * (1 - 1e-9)         # Ritz values lie inside the spectrum
    # a full-length run (m = N) recovers the smallest eigenvalue as well
    a, b = krylov.lanczos(krylov.CountingOp(A), krylov.splitmix64_uniform(A.shape[0], 1), A.shape[0])
    lo_full, _ = krylov.ritz_extremes(a, b)
    assert abs(lo_full - lam[0]) / lam[0] < 1e-6
    # the Jacobi-scaled operator: its Ritz interval lies inside the spectrum of D^-1/2 A D^-1/2
    opj, s = krylov.jacobi_scaled(A)
    lamj = np.linalg.eigvalsh((s[:, None] * A.toarray()) * s[None, :])
    a, b = krylov.lanczos(opj, krylov.splitmix64_uniform(A.shape[0], 1), 60)
    lo, hi = krylov.ritz_extremes(a, b)
    assert lamj[0] * (1 - 1e-9) <= lo and hi <= lamj[-1] * (1 + 1e-9)
    assert abs(hi - lamj[-1]) / lamj[-1] < 0.01


# ----------------------------------------------------------------- transient

def test_transient_single_cell_closed_form():
    """1x1x1 grid: T_{n+1} = (C V T_n/dt + P + h S T_amb) / (C V/dt + h S) (Eq. transient)."""
    st = ti.Stack((ti.Layer("si", 100e-6, 150.0, 1.63e6, True),), h=1e4)
    p, dt = 3e-4, 1e-3
    sched = [np.array([p])] * 6
    Ts = solve.transient(1, 1, st, sched, dt, np.array([st.t_amb]))
    CV = 1.63e6 * st.dx * st.dy * 100e-6
    hS = st.h * st.dx * st.dy
    T = st.t_amb
    for Tn in Ts:
        T = (CV * T / dt + p + hS * st.t_amb) / (CV / dt + hS)
        assert abs(Tn[0] - T) < 1e-12


def test_transient_energy_balance_and_steady_limit():
    st = ti.stack_c2()
    nx, ny = 8, 6
    dt = 1e-4
    P = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (1, 2)], np.float64)
         for _ in range(3)]
    T0 = np.full(nx * ny * st.L, st.t_amb)
    Ts = solve.transient(nx, ny, st, P, dt, T0)
    cdt = disc.capacity_over_dt(nx, ny, st, dt)
    sink = disc.top_sink(nx, ny, st)
    prev = T0
    for T, p in zip(Ts, P):
        lhs = np.sum(cdt * (T - prev)) + np.sum(sink * (T - st.t_amb))
        assert abs(lhs - p.sum()) / p.sum() < 1e-10
        prev = T
    # dt -> infinity reduces Eq. (transient) to Eq. (steady-state)
    Tinf = solve.transient(nx, ny, st, P[:1], 1e12, T0)[0]
    np.testing.assert_allclose(Tinf, solve.steady(nx, ny, st, P[0]), rtol=1e-9)


# ----------------------------------------------------------------- adjoint

def _small_case():
    st = ti.stack_c1()
    nx, ny = 10, 8
    p = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 9, dx=st.dx, dy=st.dy)], np.float64)
    mask = adjoint.silicon_mask(nx, ny, st, st.power_layers())
    return st, nx, ny, p, mask


def test_adjoint_vs_central_differences():
    st, nx, ny, p, mask = _small_case()
    beta = 2.0
    J, dJdP, dJdk, dJdh, lam = adjoint.gradient(nx, ny, st, p, mask, beta)
    rng = np.random.default_rng(0)
    for i in rng.choice(p.size, 8, replace=False):
        h = 1e-3 * max(abs(p[i]), 1e-4)
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (adjoint.objective(nx, ny, st, pp, mask, beta) - adjoint.objective(nx, ny, st, pm, mask, beta)) / (2 * h)
        assert abs(fd - dJdP[i]) <= 1e-4 * abs(dJdP[i]) + 1e-9
    k = st.k()
    for l in range(st.L):
        h = 1e-3 * k[l]
        kp, km = k.copy(), k.copy()
        kp[l] += h
        km[l] -= h
        fd = (adjoint.objective(nx, ny, st.with_k(kp), p, mask, beta)
              - adjoint.objective(nx, ny, st.with_k(km), p, mask, beta)) / (2 * h)
        assert abs(fd - dJdk[l]) <= 1e-4 * abs(dJdk[l]) + 1e-12, (l, fd, dJdk[l])


def test_adjoint_invariants():
    """sum_top h S lambda = sum w = 1 (since A^T 1 = h S e_top); Euler homogeneity in (k, h)."""
    st, nx, ny, p, mask = _small_case()
    beta = 2.0
    J, dJdP, dJdk, dJdh, lam = adjoint.gradient(nx, ny, st, p, mask, beta)
    sink = disc.top_sink(nx, ny, st)
    assert abs(np.sum(sink * lam) - 1.0) < 1e-10
    T = solve.steady(nx, ny, st, p)
    _, w = adjoint.lse(T, mask, beta)
    # theta(s k, s h) = theta / s  =>  sum_l k_l dJ/dk_l + h dJ/dh = -sum_i w_i theta_i
    lhs = np.sum(st.k() * dJdk) + st.h * dJdh
    rhs = -np.sum(w * (T - st.t_amb))
    assert abs(lhs - rhs) < 1e-9 * abs(rhs)


def test_lse_properties():
    T = np.array([1.0, 3.0, 2.0, 100.0])
    mask = np.array([True, True, True, False])
    J, w = adjoint.lse(T, mask, 2.0)
    assert 3.0 < J < 3.0 + np.log(3) / 2.0
    assert w[3] == 0.0 and abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(J, np.log(np.sum(np.exp(2.0 * T[:3]))) / 2.0, rtol=1e-15)


def _bruteforce_kmap(nx, ny, stack, kc, x):
    """Face loop with per-cell conductivities (series half cells), pure Python."""
    L = stack.L
    dx, dy = stack.dx, stack.dy
    dz = [l.thickness for l in stack.layers]
    y = np.zeros(nx * ny * L)
    at = lambda i, j, z: i + nx * (j + ny * z)
    for z in range(L):
        for j in range(ny):
            for i in range(nx):
                a = at(i, j, z)
                for (b, S, la, lb) in ((at(i + 1, j, z) if i + 1 < nx else None, dy * dz[z], dx, dx),
                                       (at(i, j + 1, z) if j + 1 < ny else None, dx * dz[z], dy, dy),
                                       (at(i, j, z + 1) if z + 1 < L else None, dx * dy, dz[z], dz[z + 1] if z + 1 < L else 0)):
                    if b is None:
                        continue
                    g = S / (la / (2 * kc[a]) + lb / (2 * kc[b]))
                    y[a] += g * (x[a] - x[b]); y[b] += g * (x[b] - x[a])
                if z == L - 1:
                    y[a] += stack.h * dx * dy * x[a]
    return y


def test_kmap_assembly_bruteforce_and_uniform_limit():
    """Per-cell conductivities: face loop brute force; a map equal to the layer values
    reproduces the layer-wise assembly."""
    st = ti.stack_c2()
    nx, ny = 4, 3
    n = nx * ny * st.L
    kc = np.repeat(st.k(), nx * ny) * np.random.default_rng(3).uniform(0.5, 2.0, n)
    A = disc.assemble(nx, ny, st, k_cell=kc)
    x = ti.random_vector(n, 4)
    np.testing.assert_allclose(A @ x, _bruteforce_kmap(nx, ny, st, kc, x), rtol=1e-12, atol=1e-18)
    assert abs(A - A.T).max() == 0.0
    Au = disc.assemble(nx, ny, st, k_cell=np.repeat(st.k(), nx * ny))
    np.testing.assert_allclose((Au - disc.assemble(nx, ny, st)).toarray(), 0.0, atol=1e-15 * abs(Au).max())


# ------------------------------------------------ Sec. 4.4: reduced-precision pieces

def test_quad_diag_round_trip():
    """The four stored diagonals (Sec. 4.2) rebuild the assembled matrix exactly."""
    from oracle import precision as prc
    st = ti.stack_c1()
    nx, ny = 5, 4
    A = disc.assemble(nx, ny, st, dt=1e-4)
    D = prc.quad_diag(A, nx, ny)
    np.testing.assert_array_equal(prc.from_quad_diag(*D, nx, ny), A.toarray())
    assert np.all(D[1] <= 0) and np.all(D[2] <= 0) and np.all(D[3] <= 0)


def test_a3_spmv_exact_on_fp16_representable_values():
    """With small-integer diagonals and inputs every FP16/FP32 step of Algorithm 3 is
    exact, so the product equals the dense matrix-vector product."""
    from oracle import precision as prc
    nx, ny, L = 4, 3, 3
    n = nx * ny * L
    rng = np.random.default_rng(7)
    i = np.arange(n)
    D4 = rng.integers(20, 41, n).astype(np.float64)
    D5 = np.where(i % nx + 1 < nx, -rng.integers(1, 5, n), 0).astype(np.float64)
    D6 = np.where((i // nx) % ny + 1 < ny, -rng.integers(1, 5, n), 0).astype(np.float64)
    D7 = np.where(i // (nx * ny) + 1 < L, -rng.integers(1, 5, n), 0).astype(np.float64)
    x = rng.integers(0, 8, n).astype(np.float32)
    e = prc.a3_scale_exponent(D4)
    assert 16 <= D4.max() * 2.0 ** e < 32
    y = prc.a3_spmv(D4, D5, D6, D7, x, nx, ny, e)
    np.testing.assert_array_equal(y.astype(np.float64), prc.from_quad_diag(D4, D5, D6, D7, nx, ny) @ x)


def test_a3_spmv_fp16_error_bound():
    """On a physical matrix the FP16 roundings (stored values, x, in-plane products;
    unit roundoff 2^-11 each) bound the error: |y - A x| <= 3.2 * 2^-11 sum_j |a_ij x_j|,
    and the product is not exact (the FP16 path is really taken)."""
    from oracle import precision as prc
    st = ti.stack_c2()
    nx, ny = 9, 7
    A = disc.assemble(nx, ny, st, dt=1e-4)
    D = prc.quad_diag(A, nx, ny)
    x = ti.random_vector(A.shape[0], 31, lo=-3.0, hi=5.0).astype(np.float32)
    y = prc.a3_spmv(*D, x, nx, ny, prc.a3_scale_exponent(D[0])).astype(np.float64)
    xd = x.astype(np.float64)
    err = np.abs(y - A @ xd)
    bound = 3.2 * 2.0 ** -11 * (abs(A) @ np.abs(xd))
    assert np.all(err <= bound), np.max(err / bound)
    assert err.max() > 0.0


def test_stage_switch_criteria():
    """Eqs. (switch_a-c), one at a time."""
    from oracle import precision as prc
    eps = 1e-8
    assert prc.stage_switch(0.9e-4, 1.0, None, 0.0, eps)            # (a) ||r_low|| <= sqrt(eps)
    assert not prc.stage_switch(1.1e-4, 1.0, None, 0.0, eps)
    assert prc.stage_switch(1.0, 0.95, 1.0, 0.0, eps)               # (b) stagnation of r_true
    assert not prc.stage_switch(1.0, 0.85, 1.0, 0.0, eps)
    assert prc.stage_switch(1.0, 1.0, None, 0.5, eps)               # (c) drift between r_true and r_low
    assert not prc.stage_switch(1.0, 1.0, None, 0.49, eps)


# ------------------------------------------------ geometric multigrid (oracle)

def test_multigrid_galerkin_is_summed_face_operator():
    """P^T A P of the 2 x 2-column aggregation is the 7-point operator whose faces
    are the sums of the fine faces crossing the aggregate boundary and whose
    per-cell term is the sum of the fine sink/capacity terms (odd sizes included)."""
    from oracle import multigrid as mg
    st = ti.stack_c1()
    for nx, ny in ((6, 4), (7, 5)):
        L = st.L
        A = disc.assemble(nx, ny, st, dt=1e-4).tocsr()
        P = mg.prolongation(nx, ny, L)
        Ac = (P.T @ A @ P).toarray()
        nxc, nyc = mg.coarse_dims(nx, ny)
        s_f = np.asarray(A.sum(axis=1)).ravel()           # row sums = sink + capacity terms
        gx = -np.asarray([A[i, i + 1] if (i % nx) + 1 < nx else 0.0 for i in range(A.shape[0])])
        gy = -np.asarray([A[i, i + nx] if ((i // nx) % ny) + 1 < ny else 0.0 for i in range(A.shape[0])])
        gz = -np.asarray([A[i, i + nx * ny] if i // (nx * ny) + 1 < L else 0.0 for i in range(A.shape[0])])
        nc = nxc * nyc * L
        want = np.zeros((nc, nc))
        cidx = lambda X, Y, z: X + nxc * (Y + nyc * z)
        for z in range(L):
            for y in range(ny):
                for x in range(nx):
                    i = x + nx * (y + ny * z)
                    I = cidx(x // 2, y // 2, z)
                    want[I, I] += s_f[i]
                    for (dx_, dy_, dz_, g) in ((1, 0, 0, gx[i]), (0, 1, 0, gy[i]), (0, 0, 1, gz[i])):
                        if g == 0.0:
                            continue
                        J = cidx((x + dx_) // 2, (y + dy_) // 2, z + dz_)
                        if J != I:
                            want[I, J] -= g; want[J, I] -= g; want[I, I] += g; want[J, J] += g
        np.testing.assert_allclose(Ac, want, rtol=1e-12, atol=1e-15 * np.abs(want).max())


def test_multigrid_vcycle_symmetric_and_exact_on_one_column():
    from oracle import multigrid as mg
    st = ti.stack_c2()
    nx, ny, L = 9, 7, st.L
    A = disc.assemble(nx, ny, st, dt=1e-4)
    M = mg.preconditioner(A, nx, ny, L)
    u, v = ti.random_vector(A.shape[0], 1), ti.random_vector(A.shape[0], 2)
    a, b = u @ M(v), v @ M(u)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert u @ M(u) > 0
    # the V-cycle as a stationary iteration contracts the error in the A-norm
    anorm = lambda e: np.sqrt(e @ (A @ e))
    for seed in (4, 5, 6):
        e = ti.random_vector(A.shape[0], seed)
        e2 = e - M(A @ e)
        assert anorm(e2) < 0.7 * anorm(e)
    # max(nx, ny) <= 4: a single (coarsest) level, solved exactly
    A1 = disc.assemble(3, 2, st)
    assert len(mg.hierarchy(A1, 3, 2, L)) == 1
    b1 = ti.random_vector(A1.shape[0], 3)
    x = mg.vcycle(mg.hierarchy(A1, 3, 2, L), L, b1)
    assert np.all(np.abs(A1 @ x - b1) <= 1e-12 * (abs(A1) @ np.abs(x)))


def test_multigrid_pcg_steady_iterations_and_solution():
    """MG-preconditioned CG reaches the exact solution in far fewer iterations than
    Jacobi on a steady stack (the case Chebyshev needs ~100 iterations for)."""
    from oracle import multigrid as mg
    inst = ti.c1(nx=32, ny=32)
    st = inst.stack
    A = disc.assemble(inst.nx, inst.ny, st)
    b = disc.rhs_steady(inst.nx, inst.ny, st, inst.power.astype(np.float64))
    ref = solve.solve_exact(A, b)
    x_mg, it_mg, _, _ = krylov.pcg(krylov.CountingOp(A), b, mg.preconditioner(A, inst.nx, inst.ny, st.L),
                                   tol_rel=1e-10)
    x_j, it_j, _, _ = krylov.pcg(krylov.CountingOp(A), b, krylov.jacobi(A), tol_rel=1e-10)
    assert solve.rise_relative_error(x_mg, ref, st.t_amb) <= 1e-8
    assert it_mg * 5 < it_j, (it_mg, it_j)
