"""The seeded input generators: deterministic, power only where the stack says, stated ranges."""
import numpy as np

import thermal_inputs as ti


def test_deterministic_and_seeded():
    a = ti.c1(dtype=np.float64).power
    b = ti.c1(dtype=np.float64).power
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(ti.c1(seed=2).power, ti.c1(seed=1).power)


def test_power_only_on_powered_layers():
    inst = ti.c2(nx=64, ny=48, dtype=np.float64)
    st = inst.stack
    P = inst.power.reshape(st.L, inst.ny, inst.nx)
    for l in range(st.L):
        if l in st.power_layers():
            assert P[l].max() > 0
        else:
            assert np.all(P[l] == 0)


def test_c1_background_and_units():
    """20 W/cm^2 background on a 50um cell is 5e-4 W; hotspot peaks add at most 500 W/cm^2 each."""
    inst = ti.c1(dtype=np.float64)
    P = inst.power.reshape(4, 64, 64)[0]
    assert P.min() >= 5e-4 * (1 - 1e-12)
    assert P.max() <= (20 + 8 * 500) * 1e4 * 2.5e-9


def test_floorplan_ranges():
    q = ti.density_floorplan(128, 96, 5, n_spots=0)
    vals = np.unique(q)
    assert vals.min() >= 0.0 and vals.max() <= 80.0
    assert np.all((vals == 0) | (vals >= 5.0))


def test_c4_batch_recipe():
    insts = ti.c4_instances()
    assert len(insts) == 64
    sizes = {(i.nx, i.stack.L) for i in insts}
    assert sizes <= set(ti.C4_CLASSES)
    total = sum(i.n for i in insts)
    assert 3e7 < total < 1e8
    for i, inst in enumerate(insts):
        base = {4: ti.stack_c1(), 6: ti.stack_c1_split_cu(), 8: ti.stack_c2()}[inst.stack.L]
        ratio = inst.stack.k() / base.k()
        assert np.all((ratio >= 0.8) & (ratio <= 1.2))


def test_splitmix_not_in_inputs():
    """The input module carries no solver arithmetic (no conductance or matrix helpers)."""
    names = set(dir(ti))
    for bad in ("assemble", "conductance", "spmv", "solve"):
        assert not any(bad in n.lower() for n in names)
