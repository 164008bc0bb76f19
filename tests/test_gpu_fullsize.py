"""The bench workload at full size (1024 x 1024 x 8, 8.4M unknowns), in the launch
configuration bench.py times (mixed FP32/FP64, Chebyshev degree 6, CUDA graph).

The oracle cannot solve this system in seconds, so it checks properties that fix the
answer at any size: the FP64 relative residual of the returned temperatures against
the oracle's own CSR matrix, the discrete energy balance of each backward-Euler
step, and agreement with the plain FP64 GPU path; plus sampled rows of the
stencil product against the oracle matrix.
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
                                   precond="cheb", cheb_degree=6, tol_rel=1e-8, use_graph=1)
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
    g.run_transient(maps, 2, 4, DT, Tm, precision="mixed", cheb_degree=6, tol_rel=1e-10, use_graph=1)
    g.run_transient(maps, 2, 4, DT, Td, precision="fp64", cheb_degree=6, tol_rel=1e-10, use_graph=1)
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
