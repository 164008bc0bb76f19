"""The allocation-free stencil product (thermal_apply_dot_noalloc).

It serves callers that cannot allocate device memory when they need the product
(a device-memory budget fixed at start-up, an allocator owned by the host
application, or a latency-critical path where an allocation would synchronise the
device).  Its output must match the existing entry point, thermal_apply in FP32,
on two calls in a row, which share the one static scratch array.  This file is
collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes as C

import numpy as np
import pytest

import thermal_inputs as ti
from oracle import discretisation as disc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_matches_thermal_apply_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid, _lib
    lib = _lib.load()
    st = ti.stack_c2()
    nx, ny, dt = 70, 37, 1e-4
    L = st.L
    g = ThermalGrid.from_stack(nx, ny, st)
    f = g.faces(dt)
    gx, gy, gz = (f[k].float().contiguous() for k in ("gx", "gy", "gz"))
    # per-layer diagonal term, formed in the same order as the library's setup
    S = st.dx * st.dy
    s = [(st.h * S if l == L - 1 else 0.0) + st.layers[l].c * S * st.layers[l].thickness / dt for l in range(L)]
    s_arr = (C.c_float * L)(*[float(np.float32(v)) for v in s])
    A = disc.assemble(nx, ny, st, dt=dt).tocsr()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):
        x = torch.from_numpy(ti.random_vector(A.shape[0], seed, lo=-2.0, hi=3.0).astype(np.float32)).cuda()
        y_ref = g.apply(x, dt, "mixed")
        y = torch.empty_like(x)
        xAx = torch.zeros(1, dtype=torch.float64, device="cuda")
        st_code = lib.thermal_apply_dot_noalloc(nx, ny, L, _p(gx), _p(gy), _p(gz), s_arr, _p(x), _p(y), _p(xAx),
                                                stream)
        assert st_code == 0, lib.thermal_last_error()
        torch.cuda.synchronize()
        xh = x.cpu().double().numpy()
        bound = abs(A) @ np.abs(xh)
        # the FP32 stencil tolerance of the parity tests
        assert np.all(np.abs(y.cpu().double().numpy() - y_ref.cpu().double().numpy()) <= 2e-6 * bound)
        ref_dot = float(torch.dot(x.double(), y_ref.double()))
        assert abs(xAx.item() - ref_dot) <= 2e-6 * float(np.abs(xh) @ bound)


def test_noalloc_rejects_grids_beyond_the_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import _lib
    lib = _lib.load()
    dummy = torch.zeros(8, device="cuda")
    xAx = torch.zeros(1, dtype=torch.float64, device="cuda")
    s_arr = (C.c_float * 2)(0.0, 1.0)
    # ceil(4096/32) * ceil(4096/8) * 2 = 131072 blocks > 65536
    code = lib.thermal_apply_dot_noalloc(4096, 4096, 2, _p(dummy), _p(dummy), _p(dummy), s_arr, _p(dummy),
                                         _p(dummy), _p(xAx), None)
    assert code == _lib.TH_EINVAL
    assert b"static scratch" in lib.thermal_last_error()
