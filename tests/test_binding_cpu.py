"""The Python binding's argument checks, without a GPU.

The library trusts the sizes and dtypes it is given, so the binding rejects a
buffer of the wrong dtype, length, layout or memory space before its pointer
crosses the C ABI.  These tests build a grid object without touching the device
(no library call is reached)."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")

from paper_2606_17850_gb300 import api  # noqa: E402
from paper_2606_17850_gb300.api import ThermalGrid, solve_batched  # noqa: E402


def fake_grid(nx=4, ny=3, L=2):
    g = ThermalGrid.__new__(ThermalGrid)
    g.nx, g.ny, g.L = nx, ny, L
    g.n = nx * ny * L
    g.t_amb = 45.0
    g._h = C.c_void_p()
    return g


def test_check_accepts_a_valid_buffer():
    t = torch.zeros(24, dtype=torch.float64)
    assert api._check(t, 24, api.F64, "T") is t


@pytest.mark.parametrize("bad,exc,msg", [
    (torch.zeros(24, dtype=torch.float32), TypeError, "float64"),
    (torch.zeros(23, dtype=torch.float64), ValueError, "24 elements"),
    (torch.zeros(48, dtype=torch.float64)[::2], ValueError, "contiguous"),
    ([0.0] * 24, TypeError, "torch.Tensor"),
])
def test_steady_rejects_bad_T(bad, exc, msg):
    g = fake_grid()
    P = torch.zeros(24, dtype=torch.float32)
    with pytest.raises(exc, match=msg):
        g.solve_steady(P, T=bad)


def test_power_checks():
    g = fake_grid()
    T = torch.zeros(24, dtype=torch.float64)
    with pytest.raises(TypeError, match="float32 or float64"):
        g.solve_steady(torch.zeros(24, dtype=torch.int32), T=T)
    with pytest.raises(ValueError, match="24 elements"):
        g.step_transient(torch.zeros(12, dtype=torch.float32), 1e-4, T)
    maps = [torch.zeros(24, dtype=torch.float32), torch.zeros(24, dtype=torch.float64)]
    with pytest.raises(TypeError, match="one dtype"):
        g.run_transient(maps, 1, 2, 1e-4, T)
    with pytest.raises(ValueError, match="non-empty"):
        g.run_transient([], 1, 2, 1e-4, T)
    with pytest.raises(ValueError, match="24 elements"):
        g.run_transient([torch.zeros(24), torch.zeros(25)], 1, 2, 1e-4, T)


def test_device_only_calls_reject_host_tensors():
    g = fake_grid()
    T = torch.zeros(24, dtype=torch.float64)
    for call in (lambda: g.hotspot_lse(T, [0], 2.0), lambda: g.grad(T, T),
                 lambda: g.apply(T, 0.0, "fp64"), lambda: g.precond(T.float())):
        with pytest.raises(ValueError, match="CUDA device"):
            call()
    with pytest.raises(TypeError, match="float32"):
        g.apply(T, 0.0, "mixed")


def test_conductivity_length():
    g = fake_grid()
    with pytest.raises(ValueError, match="2 values"):
        g.set_conductivity([1.0, 2.0, 3.0])
    with pytest.raises(ValueError, match="24 elements"):
        g.set_conductivity_map(torch.ones(10, dtype=torch.float64))


def test_batched_checks():
    g1, g2 = fake_grid(), fake_grid(8, 3, 2)
    p1, p2 = torch.zeros(24), torch.zeros(48)
    t1, t2 = torch.zeros(24, dtype=torch.float64), torch.zeros(48, dtype=torch.float64)
    with pytest.raises(ValueError, match="same length"):
        solve_batched([g1, g2], [p1], [t1, t2])
    with pytest.raises(ValueError, match="own grid"):
        solve_batched([g1, g1], [p1, p1], [t1, t1.clone()])
    with pytest.raises(ValueError, match="own output"):
        solve_batched([g1, g2], [p1, p2], [t1, t1])
    with pytest.raises(ValueError, match="CUDA device"):
        solve_batched([g1, g2], [p1, p2], [t1, t2])
