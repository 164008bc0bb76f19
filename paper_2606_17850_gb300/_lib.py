"""ctypes view of libthermal.so (the C ABI declared in include/thermal.h).

Argument marshalling only: every computation runs inside the library.  Loading
fails loudly when the shared object is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libthermal.so")

TH_OK, TH_EINVAL, TH_ENOMEM, TH_ECUDA, TH_ENOCONV, TH_EBREAKDOWN, TH_ENONFINITE, TH_ESTATE = range(8)
STATUS_NAMES = ["TH_OK", "TH_EINVAL", "TH_ENOMEM", "TH_ECUDA", "TH_ENOCONV", "TH_EBREAKDOWN",
                "TH_ENONFINITE", "TH_ESTATE"]
TH_PREC_FP64, TH_PREC_MIXED_IR, TH_PREC_MIXED_IR_BF16, TH_PREC_ADAPTIVE = 0, 1, 2, 3
TH_PC_NONE, TH_PC_JACOBI, TH_PC_CHEB, TH_PC_ZLINE, TH_PC_MG = 0, 1, 2, 3, 4
TH_F32, TH_F64 = 0, 1


class SolveOpts(C.Structure):
    _fields_ = [
        ("tol_rel", C.c_double),
        ("inner_tol", C.c_double),
        ("max_outer", C.c_int),
        ("max_inner", C.c_int),
        ("max_iter", C.c_int),
        ("precision", C.c_int),
        ("precond", C.c_int),
        ("cheb_degree", C.c_int),
        ("cheb_scaled", C.c_int),
        ("lanczos_steps", C.c_int),
        ("use_guess", C.c_int),
        ("use_graph", C.c_int),
        ("batched_mode", C.c_int),
        ("guess", C.c_int),
        ("cheb_fuse", C.c_int),
        ("ad_check", C.c_int),
        ("test_wait_expire", C.c_int),
        ("reserved", C.c_int * 3),
        ("cheb_lam_min", C.c_double),
        ("cheb_lam_max", C.c_double),
    ]


class SolveStats(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("outer_it", C.c_int),
        ("inner_it", C.c_int64),
        ("n_spmv", C.c_int64),
        ("rel_res", C.c_double),
        ("t_setup_ms", C.c_double),
        ("t_solve_ms", C.c_double),
        ("lam_min", C.c_double),
        ("lam_max", C.c_double),
        ("steps", C.c_int),
        ("stage_switches", C.c_int),
        ("tile_rows", C.c_int),
        ("tile_layers", C.c_int),
        ("reserved", C.c_int * 4),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class ThermalError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)

# name -> (restype, argtypes), one entry per declaration in include/thermal.h
SIGNATURES = {
    "thermal_version": (C.c_char_p, []),
    "thermal_last_error": (C.c_char_p, []),
    "thermal_default_opts": (None, [C.POINTER(SolveOpts)]),
    "thermal_grid_create": (C.c_int, [C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_double, C.POINTER(_vp)]),
    "thermal_grid_set_geometry": (C.c_int, [_vp, C.c_double, C.c_double, _dp, C.c_double]),
    "thermal_grid_set_conductivity": (C.c_int, [_vp, _dp]),
    "thermal_grid_set_conductivity_map": (C.c_int, [_vp, _vp]),
    "thermal_grid_destroy": (C.c_int, [_vp]),
    "thermal_grid_dims": (C.c_int, [_vp, C.POINTER(C.c_int64), _ip, _ip, _ip]),
    "thermal_grid_faces": (C.c_int, [_vp, C.c_double, _vp, _vp, _vp, _vp, _vp]),
    "thermal_apply": (C.c_int, [_vp, C.c_double, C.c_int, _vp, _vp, _vp]),
    "thermal_precond_apply": (C.c_int, [_vp, C.c_double, C.POINTER(SolveOpts), _vp, _vp, _vp]),
    "thermal_spectral_bounds": (C.c_int, [_vp, C.c_double, C.POINTER(SolveOpts), _dp, _dp, _dp, _dp, _vp]),
    "thermal_kernel_time": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _dp, _vp]),
    "thermal_solve_steady": (C.c_int, [_vp, _vp, C.c_int, _vp, C.POINTER(SolveOpts), C.POINTER(SolveStats), _vp]),
    "thermal_step_transient": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp, C.POINTER(SolveOpts),
                                         C.POINTER(SolveStats), _vp]),
    "thermal_run_transient": (C.c_int, [_vp, C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _vp,
                                        C.POINTER(SolveOpts), C.POINTER(SolveStats), _vp]),
    "thermal_hotspot_lse": (C.c_int, [_vp, _vp, _ip, C.c_int, C.c_double, _dp, _vp, _vp]),
    "thermal_grad": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _dp, C.POINTER(SolveOpts), C.POINTER(SolveStats), _vp]),
    "thermal_solve_batched": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.c_int, C.POINTER(_vp),
                                        C.POINTER(SolveOpts), C.POINTER(SolveStats), _vp]),
    "thermal_csr_spmv": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, _vp, _vp, C.c_int, _dp, _vp]),
    "thermal_apply_dot_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, C.POINTER(C.c_float), _vp,
                                            _vp, _vp, _vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libthermal.so and declare every entry point; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libthermal.so not found at {path}: run __graft_entry__.build() "
                          f"(or python -m paper_2606_17850_gb300.build) first")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != TH_OK:
        raise ThermalError(status, load().thermal_last_error().decode(errors="replace"))
    return status


def default_opts(**kw):
    o = SolveOpts()
    load().thermal_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown option {k}")
        setattr(o, k, v)
    return o
