"""The bench workload at full size (1024 x 1024 x 8, 8.4M unknowns), in the launch
configuration bench.py times (mixed FP32/FP64, Chebyshev degree 29 in fused 4-step
chunks, inner tolerance 1e-4, cubic extrapolated guess, CUDA graph).

The oracle solves the first three backward-Euler steps of the workload exactly
(Algorithm 1 with Jacobi to relative residual 1e-13, about a minute on one host
core), and the GPU's steps at the headline tolerance 1e-8 are compared with them
element by element (error relative to the temperature rise, the metric of
Sec. 5.1 scaled by the rise).  Properties that fix the answer at any size are
checked beside it: the FP64 relative residual against the oracle's own CSR matrix,
the discrete energy balance of each step, agreement with the plain FP64 GPU path,
and sampled rows of the stencil product against the oracle matrix.
"""
import numpy as np
import pytest

import thermal_inputs as ti
from oracle import discretisation as disc, solve as osolve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NX = NY = 1024
DT = 1e-4


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid
    inst = ti.c3(NX, NY, dtype=np.float32)
    g = ThermalGrid.from_stack(NX, NY, inst.stack)
    A = disc.assemble(NX, NY, inst.stack, dt=DT).tocsr()
    return inst, g, A


def test_fullsize_first_steps_match_oracle(setup):
    """Steps 1-3 of the 100-step workload in the bench's configuration (tol 1e-8,
    degree 29 in fused chunks, inner tolerance 1e-4, cubic extrapolated guess, CUDA
    graph) against the oracle's exact backward-Euler steps."""
    inst, g, A = setup
    st = inst.stack
    P0 = inst.power.astype(np.float64)
    exact = osolve.Factorised(A, tol_rel=1e-13)
    T_ref, prev = [], np.full(inst.n, st.t_amb)
    for _ in range(3):
        prev = exact(disc.rhs_transient(NX, NY, st, P0, prev, DT), x0=prev)
        T_ref.append(prev)
    maps = [torch.from_numpy(m).cuda() for m in [inst.power] + list(inst.extra_power)]
    report = []
    for n_steps in (1, 2, 3):
        T = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
        _, stats = g.run_transient(maps, 25, n_steps, DT, T, precision="mixed", precond="cheb", cheb_degree=29,
                                   inner_tol=1e-4, tol_rel=1e-8, guess=3, use_graph=1)
        Th = T.cpu().numpy()
        err = osolve.rise_relative_error(Th, T_ref[n_steps - 1], st.t_amb)
        report.append((n_steps, err, osolve.inf_error(Th, T_ref[n_steps - 1])))
        assert stats["status"] == 0 and stats["rel_res"] <= 1e-8
        assert err <= 1e-6, report
    print("full-size steps vs oracle (step, error / rise, ||e||_inf K):", report)


def test_fullsize_steps_residual_and_energy(setup):
    inst, g, A = setup
    st = inst.stack
    maps = [inst.power] + list(inst.extra_power)
    T = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
    cdt = disc.capacity_over_dt(NX, NY, st, DT)
    sink = disc.top_sink(NX, NY, st)
    prev = np.full(inst.n, st.t_amb)
    for s in range(3):
        P = maps[s % 4]
        T, stats = g.run_transient([torch.from_numpy(P).cuda()], 25, 1, DT, T, precision="mixed",
                                   precond="cheb", cheb_degree=29, inner_tol=1e-4, tol_rel=1e-8, use_graph=1)
        Th = T.cpu().numpy()
        b = disc.rhs_transient(NX, NY, st, P.astype(np.float64), prev, DT)
        rel = osolve.rel_residual(A, Th, b, st.t_amb)
        assert stats["status"] == 0 and rel <= 1.05e-8, (s, rel, stats)
        lhs = np.sum(cdt * (Th - prev)) + np.sum(sink * (Th - st.t_amb))
        assert abs(lhs - P.astype(np.float64).sum()) / P.sum() < 1e-6
        prev = Th


def test_fullsize_mixed_matches_fp64_path(setup):
    inst, g, A = setup
    st = inst.stack
    maps = [torch.from_numpy(m).cuda() for m in [inst.power] + list(inst.extra_power)]
    Tm = torch.full((inst.n,), st.t_amb, dtype=torch.float64, device="cuda")
    Td = Tm.clone()
    # the bench's configuration (cubic extrapolation over the 12 steps, maps switching
    # every 4) against the plain FP64 path warm-started from the previous step
    g.run_transient(maps, 4, 12, DT, Tm, precision="mixed", cheb_degree=29, inner_tol=1e-4, guess=3, tol_rel=1e-10,
                    use_graph=1)
    g.run_transient(maps, 4, 12, DT, Td, precision="fp64", cheb_degree=6, guess=0, tol_rel=1e-10, use_graph=1)
    rise = (Td - st.t_amb).abs().max().item()
    assert (Tm - Td).abs().max().item() <= 1e-6 * rise


def test_fullsize_stencil_sampled_rows(setup):
    inst, g, A = setup
    x = ti.random_vector(inst.n, 3)
    y = g.apply(torch.from_numpy(x).cuda(), DT, "fp64").cpu().numpy()
    rows = np.random.default_rng(0).choice(inst.n, 4096, replace=False)
    rows = np.concatenate([rows, [0, NX - 1, NX * NY - 1, inst.n - 1, inst.n - NX]])
    sub = A[rows]
    ref = sub @ x
    bound = abs(sub) @ np.abs(x)
    assert np.all(np.abs(y[rows] - ref) <= 1e-14 * bound)


# ----------------------------------------------------------------- adjoint at 2048 x 2048 x 10

@pytest.fixture(scope="module")
def c5():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid
    inst = ti.c5(dtype=np.float32)
    g = ThermalGrid.from_stack(inst.nx, inst.ny, inst.stack)
    return inst, g


@pytest.mark.parametrize("pc", ["mg", "cheb"])
def test_fullsize_adjoint_c5(c5, pc):
    """41.9M unknowns: log-sum-exp hotspot gradient, with the multigrid preconditioner
    the bench's adjoint section times and with Chebyshev-30.  Checks that hold at any
    size: sum_top h S lambda = sum w = 1; the directional derivative along the power
    of one FEOL layer and along one layer conductivity against central differences
    (1e-4)."""
    inst, g = c5
    st = inst.stack
    opts = dict(precision="mixed", precond=pc, cheb_degree=30, tol_rel=1e-10)
    layers = st.power_layers()
    beta = 2.0
    P = torch.from_numpy(inst.power).cuda()
    T, s = g.solve_steady(P, **opts)
    J, w = g.hotspot_lse(T, layers, beta)
    dJdP, dJdk, _ = g.grad(T, w, dJdP_dtype=torch.float64, **opts)
    S = st.dx * st.dy
    top = slice((st.L - 1) * inst.nx * inst.ny, st.L * inst.nx * inst.ny)
    assert abs(st.h * S * dJdP[top].sum().item() - 1.0) < 1e-6
    # direction: the power of the logic FEOL layer
    dP = torch.zeros_like(P)
    sl = slice(layers[0] * inst.nx * inst.ny, (layers[0] + 1) * inst.nx * inst.ny)
    dP[sl] = P[sl]
    eps = 1e-3
    Jp = g.hotspot_lse(g.solve_steady(P + eps * dP, **opts)[0], layers, beta, want_grad=False)[0]
    Jm = g.hotspot_lse(g.solve_steady(P - eps * dP, **opts)[0], layers, beta, want_grad=False)[0]
    fd = (Jp - Jm) / (2 * eps)
    an = float((dJdP * dP.double()).sum())
    assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)
    # direction: conductivity of the spreader layer
    k = st.k()
    l = 8
    kp, km = k.copy(), k.copy()
    kp[l] *= 1 + eps
    km[l] *= 1 - eps
    g.set_conductivity(kp)
    Jp = g.hotspot_lse(g.solve_steady(P, **opts)[0], layers, beta, want_grad=False)[0]
    g.set_conductivity(km)
    Jm = g.hotspot_lse(g.solve_steady(P, **opts)[0], layers, beta, want_grad=False)[0]
    g.set_conductivity(k)
    fd = (Jp - Jm) / (2 * eps * k[l])
    assert abs(fd - dJdk[l]) <= 1e-4 * abs(dJdk[l]), (fd, dJdk[l])


# ----------------------------------------------------------------- batched: 64 uneven stacks

@pytest.mark.parametrize("pc", ["cheb", "mg"])
def test_fullsize_batched_c4(pc):
    """The 64-instance batch (about 6e7 unknowns) in one persistent launch, with the
    Chebyshev and the multigrid preconditioner; every instance converges and sampled
    instances (one per size class) meet the relative residual against the oracle's
    own CSR matrix."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid, solve_batched
    insts = ti.c4_instances()
    grids = [ThermalGrid.from_stack(i.nx, i.ny, i.stack) for i in insts]
    powers = [torch.from_numpy(i.power).cuda() for i in insts]
    Ts = [torch.empty(i.n, dtype=torch.float64, device="cuda") for i in insts]
    stats = solve_batched(grids, powers, Ts, tol_rel=1e-8, precond=pc, cheb_degree=30)
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-8 for s in stats)
    seen = set()
    for inst, T in zip(insts, Ts):
        key = (inst.nx, inst.stack.L)
        if key in seen:
            continue
        seen.add(key)
        A = disc.assemble(inst.nx, inst.ny, inst.stack).tocsr()
        b = disc.rhs_steady(inst.nx, inst.ny, inst.stack, inst.power.astype(np.float64))
        assert osolve.rel_residual(A, T.cpu().numpy(), b, inst.stack.t_amb) <= 1.05e-8
