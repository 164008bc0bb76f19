"""The allocation-free stencil product (thermal_apply_dot_noalloc).

Some callers cannot allocate device memory at the moment they need the product: a
service that reserves its whole device-memory budget at start-up, a host
application whose own allocator owns the device and hands out only pre-sized
buffers, or a latency-critical path where cudaMalloc would synchronise the device.
This entry point takes every input and output from the caller and keeps its only
scratch (the reduction partials) in one static device array.

Its product must match the oracle's assembled matrix applied to the same x, and the
existing entry point (thermal_apply in FP32), on two calls in a row that share the
one static scratch array.  This file is collected last, so a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import thermal_inputs as ti
from oracle import discretisation as disc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def _oracle_faces(A, nx, ny, L):
    """FP32 face conductances and per-layer diagonal terms read off the oracle's CSR
    matrix: gx[i] = -A[i, i+1], gy[i] = -A[i, i+nx], gz[i] = -A[i, i+nx*ny] (0 at the
    grid edge) and s_l = A_ii - sum of the cell's faces (the same for every cell of a layer)."""
    n = A.shape[0]
    i = np.arange(n)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)

    def off(mask, j):
        return np.where(mask, -np.asarray(A[i, np.minimum(j, n - 1)]).ravel(), 0.0)

    gx = off(x + 1 < nx, i + 1)
    gy = off(y + 1 < ny, i + nx)
    gz = off(z + 1 < L, i + nx * ny)
    offsum = np.asarray(-(A - sp.diags(A.diagonal())).sum(axis=1)).ravel()
    s = A.diagonal() - offsum
    s_layer = [float(np.median(s[l * nx * ny:(l + 1) * nx * ny])) for l in range(L)]
    return gx, gy, gz, s_layer


def test_noalloc_matches_oracle_and_thermal_apply_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import ThermalGrid, _lib
    lib = _lib.load()
    st = ti.stack_c2()
    nx, ny, dt = 70, 37, 1e-4
    L = st.L
    A = disc.assemble(nx, ny, st, dt=dt).tocsr()
    gx, gy, gz, s_layer = _oracle_faces(A, nx, ny, L)
    gx, gy, gz = (torch.from_numpy(v.astype(np.float32)).cuda() for v in (gx, gy, gz))
    s_arr = (C.c_float * L)(*[float(np.float32(v)) for v in s_layer])
    g = ThermalGrid.from_stack(nx, ny, st)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):
        x = torch.from_numpy(ti.random_vector(A.shape[0], seed, lo=-2.0, hi=3.0).astype(np.float32)).cuda()
        y = torch.empty_like(x)
        xAx = torch.zeros(1, dtype=torch.float64, device="cuda")
        code = lib.thermal_apply_dot_noalloc(nx, ny, L, _p(gx), _p(gy), _p(gz), s_arr, _p(x), _p(y), _p(xAx),
                                             stream)
        assert code == 0, lib.thermal_last_error()
        torch.cuda.synchronize()
        xh = x.cpu().double().numpy()
        yh = y.cpu().double().numpy()
        bound = abs(A) @ np.abs(xh)
        # FP32 coefficients and ~13 FP32 operations per row: the FP32 stencil tolerance
        # of the parity tests, against the oracle's FP64 product of the same x
        assert np.all(np.abs(yh - A @ xh) <= 2e-6 * bound)
        assert abs(xAx.item() - xh @ (A @ xh)) <= 2e-6 * float(np.abs(xh) @ bound)
        # and against the existing entry point
        y_ref = g.apply(x, dt, "mixed").cpu().double().numpy()
        assert np.all(np.abs(yh - y_ref) <= 2e-6 * bound)


def test_noalloc_rejects_oversized_grids_and_overlap():
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
                                         _p(dummy[4:]), _p(xAx), None)
    assert code == _lib.TH_EINVAL
    assert b"static scratch" in lib.thermal_last_error()
    # in place (x == y) and partly overlapping ranges: rejected before any launch
    buf = torch.zeros(64, device="cuda")
    for xo, yo in ((0, 0), (0, 8)):
        code = lib.thermal_apply_dot_noalloc(4, 4, 1, _p(buf), _p(buf), _p(buf), s_arr,
                                             _p(buf[xo:]), _p(buf[yo:]), _p(xAx), None)
        assert code == _lib.TH_EINVAL
        assert b"overlap" in lib.thermal_last_error()
