"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

* TH_ENOCONV: iteration limits reached before the tolerance (Sec. 4.4's safety
  mechanism ends a stalled stage; here the limits end the solve and say so).
* TH_EBREAKDOWN: a host-prepared input that makes the preconditioner indefinite.
  Two Lanczos steps under-estimate lambda_max of the unscaled operator; a Chebyshev
  polynomial of even degree is then negative far above its interval, and a
  checkerboard power map (the highest-frequency mode) puts r there, so r^T z < 0.
  The oracle confirms that on the host before the GPU runs it.
* The fused Chebyshev kernel's bounded mbarrier wait: the test hook makes every CTA
  wait on a barrier phase that nothing completes; the wait gives up after 2 ms,
  the kernel records TH_ECUDA, waits (bounded) for its own tensor copy, and the
  solve returns the error with the context usable.

After each failure the same grid solves a normal case to the oracle's answer.
"""
import numpy as np
import pytest

import thermal_inputs as ti
from oracle import discretisation as disc, krylov, solve as osolve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()


def _grid(nx, ny, st):
    from paper_2606_17850_gb300 import ThermalGrid
    return ThermalGrid.from_stack(nx, ny, st)


def _normal_solve_matches_oracle(g, nx, ny, st, **opts):
    P = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 3) for _ in st.power_layers()],
                       np.float64)
    T, s = g.solve_steady(torch.from_numpy(P).cuda(), tol_rel=1e-10, **opts)
    T_ref = osolve.steady(nx, ny, st, P)
    assert s["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), T_ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("graph", [0, 1])
def test_iteration_limits_give_enoconv(prec, graph):
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c2()
    nx, ny = 36, 21
    g = _grid(nx, ny, st)
    P = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 2) for _ in st.power_layers()],
                       np.float32)
    lim = dict(max_outer=1, max_inner=2) if prec == "mixed" else dict(max_outer=1, max_iter=2)
    with pytest.raises(ThermalError) as e:
        g.solve_steady(torch.from_numpy(P).cuda(), precision=prec, tol_rel=1e-12, cheb_degree=8,
                       use_graph=graph, **lim)
    assert e.value.status == 4
    _normal_solve_matches_oracle(g, nx, ny, st, precision=prec, cheb_degree=8, use_graph=graph)


def _checkerboard(nx, ny, L, amp=1e-3):
    i = np.arange(nx * ny * L)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    return np.where((x + y + z) % 2 == 0, amp, -amp)


@pytest.mark.parametrize("nx", [36, 37])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_indefinite_preconditioner_gives_ebreakdown(nx, prec):
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c2()
    ny, k, m = 29, 20, 2
    A = disc.assemble(nx, ny, st)
    P = _checkerboard(nx, ny, st.L)
    # host check: the oracle's own two-step interval, unscaled polynomial, r = P
    a, b = krylov.lanczos(lambda v: A @ v, krylov.splitmix64_uniform(A.shape[0], 0x5EED), m)
    lmin, lmax = krylov.chebyshev_bounds(*krylov.ritz_extremes(a, b))
    assert lmax < 0.8 * np.linalg.eigvalsh(A.toarray())[-1]
    z = krylov.chebyshev(lambda v: A @ v, P, lmin, lmax, k)
    assert P @ z < -100 * (P @ P)
    g = _grid(nx, ny, st)
    with pytest.raises(ThermalError) as e:
        g.solve_steady(torch.from_numpy(P).cuda(), precision=prec, precond="cheb", cheb_scaled=0,
                       lanczos_steps=m, cheb_degree=k, tol_rel=1e-10)
    assert e.value.status == 5
    _normal_solve_matches_oracle(g, nx, ny, st, precision=prec, cheb_degree=8)


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("kind", ["steady", "run"])
def test_fused_kernel_wait_expiry_reported(graph, kind):
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c2()
    nx, ny, dt = 76, 37, 1e-4       # several tiles with ragged tails; fused chunks (nx % 4 == 0)
    g = _grid(nx, ny, st)
    P = torch.from_numpy(ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 4)
                                                     for _ in st.power_layers()], np.float32)).cuda()
    opts = dict(precision="mixed", precond="cheb", cheb_degree=12, cheb_fuse=4, tol_rel=1e-10, use_graph=graph)
    with pytest.raises(ThermalError) as e:
        if kind == "steady":
            g.solve_steady(P, test_wait_expire=1, **opts)
        else:
            T = torch.full((g.n,), st.t_amb, dtype=torch.float64, device="cuda")
            g.run_transient([P], 2, 4, dt, T, test_wait_expire=1, **opts)
    assert e.value.status == 3
    assert "timed out" in str(e.value)
    torch.cuda.synchronize()   # the context is still usable
    _normal_solve_matches_oracle(g, nx, ny, st, precision="mixed", cheb_degree=12, cheb_fuse=4, use_graph=graph)
