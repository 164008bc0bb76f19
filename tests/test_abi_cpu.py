"""The C ABI without a GPU: the library builds, loads, exports every declared entry
point, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "thermal.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(thermal_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2606_17850_gb300 import _lib
    return _lib.load()


def test_header_declares_expected_boundary():
    names = declared_functions()
    for must in ("thermal_grid_create", "thermal_solve_steady", "thermal_step_transient", "thermal_grad",
                 "thermal_run_transient", "thermal_solve_batched", "thermal_apply"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_17850_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_default_opts(lib):
    from paper_2606_17850_gb300 import _lib
    o = _lib.default_opts()
    assert o.tol_rel == 1e-8 and o.cheb_degree == 30 and o.precond == _lib.TH_PC_CHEB
    assert o.precision == _lib.TH_PREC_MIXED_IR
    assert lib.thermal_version().decode().endswith("sm_103a")


def _arr(v):
    return (C.c_double * len(v))(*v)


@pytest.mark.parametrize("nx,ny,L,k,c,h", [
    (0, 4, 2, [1.0, 1.0], [1.0, 1.0], 1.0),
    (4, -1, 2, [1.0, 1.0], [1.0, 1.0], 1.0),
    (4, 4, 0, [1.0], [1.0], 1.0),
    (4, 4, 2, [1.0, -2.0], [1.0, 1.0], 1.0),
    (4, 4, 2, [1.0, float("nan")], [1.0, 1.0], 1.0),
    (4, 4, 2, [1.0, 1.0], [0.0, 1.0], 1.0),
    (4, 4, 2, [1.0, 1.0], [1.0, 1.0], -1.0),
    (4, 4, 2, [1.0, 1.0], [1.0, 1.0], float("inf")),
    (4, 4, 40, [1.0] * 40, [1.0] * 40, 1.0),
])
def test_grid_create_rejects_invalid(lib, nx, ny, L, k, c, h):
    from paper_2606_17850_gb300 import _lib
    out = C.c_void_p()
    st = lib.thermal_grid_create(nx, ny, L, _arr(k), _arr(c), h, C.byref(out))
    assert st == _lib.TH_EINVAL
    assert out.value is None
    assert lib.thermal_last_error().decode()


def test_null_arguments_rejected(lib):
    from paper_2606_17850_gb300 import _lib
    assert lib.thermal_grid_create(4, 4, 1, _arr([1.0]), None, 1.0, None) == _lib.TH_EINVAL
    assert lib.thermal_grid_set_geometry(None, 1.0, 1.0, _arr([1.0]), 0.0) == _lib.TH_EINVAL
    o = _lib.default_opts()
    st = _lib.SolveStats()
    assert lib.thermal_solve_steady(None, None, 0, None, C.byref(o), C.byref(st), None) == _lib.TH_EINVAL
    assert lib.thermal_grid_destroy(None) == _lib.TH_OK


def test_status_enum_matches_header():
    from paper_2606_17850_gb300 import _lib
    text = open(HEADER).read()
    for i, name in enumerate(_lib.STATUS_NAMES):
        m = re.search(rf"\b{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == i, name


def test_struct_layouts_match_header(lib):
    """Field order of the option/statistics structs in the binding follows the header."""
    from paper_2606_17850_gb300 import _lib
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for cname, py in (("thermal_solve_opts", _lib.SolveOpts), ("thermal_solve_stats", _lib.SolveStats)):
        body = re.search(r"typedef struct %s \{(.*?)\}" % cname, text, re.S).group(1)
        fields = re.findall(r"\b(\w+)(?:\[\d+\])?;", body)
        assert fields == [f for f, _ in py._fields_], cname


def test_oracle_zline_exact_without_inplane_coupling():
    """On a 1x1 column grid the z-line block is the whole matrix: its inverse is exact."""
    import thermal_inputs as ti
    from oracle import discretisation as disc, krylov
    st = ti.stack_c2()
    A = disc.assemble(1, 1, st)
    r = ti.random_vector(st.L, 3)
    np.testing.assert_allclose(krylov.zline(A, 1, 1, st.L)(r), np.linalg.solve(A.toarray(), r), rtol=1e-12)


def test_empty_and_negative_batches(lib):
    """n = 0 solves nothing and touches no device; n < 0 and bad options are rejected."""
    from paper_2606_17850_gb300 import _lib
    o = _lib.default_opts()
    assert lib.thermal_solve_batched(None, 0, None, _lib.TH_F64, None, C.byref(o), None, None) == _lib.TH_OK
    assert lib.thermal_solve_batched(None, -1, None, _lib.TH_F64, None, C.byref(o), None, None) == _lib.TH_EINVAL
    assert lib.thermal_solve_batched(None, 0, None, 7, None, C.byref(o), None, None) == _lib.TH_EINVAL
    o.cheb_degree = 0
    assert lib.thermal_solve_batched(None, 0, None, _lib.TH_F64, None, C.byref(o), None, None) == _lib.TH_EINVAL


def test_chebyshev_interval_option_validation(lib):
    """A fixed Chebyshev interval must be both 0 (the Lanczos estimate) or 0 < min < max,
    finite; anything else is rejected before any device work."""
    from paper_2606_17850_gb300 import _lib
    for lo, hi, ok in ((0.0, 0.0, True), (1e-3, 2.0, True), (0.0, 2.0, False), (1e-3, 0.0, False),
                       (2.0, 1.0, False), (-1.0, 2.0, False), (1e-3, float("inf"), False),
                       (float("nan"), 2.0, False)):
        o = _lib.default_opts(cheb_lam_min=lo, cheb_lam_max=hi)
        st = lib.thermal_solve_batched(None, 0, None, _lib.TH_F64, None, C.byref(o), None, None)
        assert st == (_lib.TH_OK if ok else _lib.TH_EINVAL), (lo, hi)


def test_noalloc_rejects_before_any_device_work(lib):
    """The allocation-free product checks sizes, NULLs and x/y overlap on the host
    before it looks up its scratch or launches anything (placeholder addresses here
    are never dereferenced)."""
    from paper_2606_17850_gb300 import _lib
    s_arr = (C.c_float * 2)(0.0, 1.0)
    a, b = C.c_void_p(1 << 20), C.c_void_p(1 << 30)   # two placeholder ranges far apart
    xAx = C.c_void_p(1 << 31)
    f = lib.thermal_apply_dot_noalloc
    assert f(0, 4, 1, a, a, a, s_arr, a, b, xAx, None) == _lib.TH_EINVAL
    assert f(4, 4, 1, a, a, a, s_arr, None, b, xAx, None) == _lib.TH_EINVAL
    # ceil(4096/32) * ceil(4096/8) * 2 = 131072 thread blocks > the 65536 partials
    assert f(4096, 4096, 2, a, a, a, s_arr, a, b, xAx, None) == _lib.TH_EINVAL
    assert b"static scratch" in lib.thermal_last_error()
    # x == y, and y starting inside x's 16 floats
    for y in (a, C.c_void_p((1 << 20) + 32)):
        assert f(4, 4, 1, a, a, a, s_arr, a, y, xAx, None) == _lib.TH_EINVAL
        assert b"overlap" in lib.thermal_last_error()
