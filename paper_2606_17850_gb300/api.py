"""Python binding of libthermal: thin wrappers that pass torch tensors' pointers.

PyTorch provides device memory and the current CUDA stream; every step of the
solve runs in the library's kernels.  Tensors may live on the GPU or on the host
(host tensors are copied by the library inside the call).
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import torch

from . import _lib as L

PRECISION = {"fp64": L.TH_PREC_FP64, "mixed": L.TH_PREC_MIXED_IR, "mixed_bf16": L.TH_PREC_MIXED_IR_BF16,
             "adaptive": L.TH_PREC_ADAPTIVE}
PRECOND = {"none": L.TH_PC_NONE, "jacobi": L.TH_PC_JACOBI, "cheb": L.TH_PC_CHEB, "zline": L.TH_PC_ZLINE,
           "mg": L.TH_PC_MG}


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to libthermal must be contiguous")
    return C.c_void_p(t.data_ptr())


F32, F64, F32_OR_F64 = (torch.float32,), (torch.float64,), (torch.float32, torch.float64)


def _check(t, n: int, dtypes, name: str, device_only: bool = False) -> torch.Tensor:
    """Validates a buffer before its pointer crosses the C ABI: a tensor of one of
    ``dtypes`` with exactly ``n`` elements, contiguous, on a CUDA device (or on the
    host where the call accepts host memory).  The library trusts sizes and dtypes,
    so a short or mistyped buffer would be read or written past its end."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor, got {type(t).__name__}")
    if t.dtype not in dtypes:
        want = " or ".join(str(d).replace("torch.", "") for d in dtypes)
        raise TypeError(f"{name} must be {want}, got {str(t.dtype).replace('torch.', '')}")
    if t.numel() != n:
        raise ValueError(f"{name} must hold {n} elements (one per cell), got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.type not in ("cuda", "cpu") or (device_only and t.device.type != "cuda"):
        where = "a CUDA device" if device_only else "a CUDA device or the host"
        raise ValueError(f"{name} must live on {where}, got {t.device}")
    return t


def _check_maps(maps, n: int, name: str = "power maps", device_only: bool = False):
    """A non-empty list of power maps of one dtype (float32 or float64) in one memory space."""
    if not isinstance(maps, (list, tuple)) or not maps:
        raise ValueError(f"{name} must be a non-empty list of tensors")
    for i, m in enumerate(maps):
        _check(m, n, F32_OR_F64, f"{name}[{i}]", device_only)
    if len({m.dtype for m in maps}) != 1:
        raise TypeError(f"all {name} must share one dtype")
    if len({m.device.type for m in maps}) != 1:
        raise ValueError(f"all {name} must be in the same memory space")
    return maps


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t: torch.Tensor):
    if t.dtype == torch.float32:
        return L.TH_F32
    if t.dtype == torch.float64:
        return L.TH_F64
    raise TypeError(f"power maps must be float32 or float64, got {t.dtype}")


def make_opts(precision="mixed", precond="cheb", **kw):
    o = L.default_opts(**kw)
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.precond = PRECOND[precond] if isinstance(precond, str) else int(precond)
    return o


def _darr(v):
    a = (C.c_double * len(v))(*[float(x) for x in v])
    return a


class ThermalGrid:
    """A layered grid of nx * ny * layers cells (x fastest, layer 0 at the bottom)."""

    def __init__(self, nx, ny, k, c, h, dx, dy, dz, t_amb):
        lib = L.load()
        self.nx, self.ny, self.L = int(nx), int(ny), len(k)
        self.n = self.nx * self.ny * self.L
        self.t_amb = float(t_amb)
        self._h = C.c_void_p()
        L.check(lib.thermal_grid_create(self.nx, self.ny, self.L, _darr(k), _darr(c) if c is not None else None,
                                        float(h), C.byref(self._h)))
        L.check(lib.thermal_grid_set_geometry(self._h, float(dx), float(dy), _darr(dz), float(t_amb)))

    @classmethod
    def from_stack(cls, nx, ny, stack):
        """Build from any object with k(), c(), dz() arrays and h, dx, dy, t_amb attributes."""
        return cls(nx, ny, list(stack.k()), list(stack.c()), stack.h, stack.dx, stack.dy, list(stack.dz()),
                   stack.t_amb)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            L.load().thermal_grid_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_conductivity(self, k: Sequence[float]):
        if len(k) != self.L:
            raise ValueError(f"set_conductivity needs {self.L} values (one per layer), got {len(k)}")
        L.check(L.load().thermal_grid_set_conductivity(self._h, _darr(k)))

    def set_conductivity_map(self, k_cell: torch.Tensor):
        """Per-cell conductivities (float64, host or device, n values)."""
        k_cell = _check(k_cell.contiguous().to(torch.float64), self.n, F64, "k_cell")
        L.check(L.load().thermal_grid_set_conductivity_map(self._h, _ptr(k_cell)))

    # ------------------------------------------------------------------ kernels

    def faces(self, dt=0.0, device="cuda"):
        out = {k: torch.empty(self.n, dtype=torch.float64, device=device) for k in ("gx", "gy", "gz", "diag")}
        L.check(L.load().thermal_grid_faces(self._h, float(dt), _ptr(out["gx"]), _ptr(out["gy"]), _ptr(out["gz"]),
                                            _ptr(out["diag"]), _stream()))
        return out

    def apply(self, x: torch.Tensor, dt=0.0, precision="fp64"):
        _check(x, self.n, F64 if precision == "fp64" else F32, "x", device_only=True)
        y = torch.empty_like(x)
        L.check(L.load().thermal_apply(self._h, float(dt), PRECISION[precision], _ptr(x), _ptr(y), _stream()))
        return y

    def precond(self, r: torch.Tensor, dt=0.0, **opts):
        _check(r, self.n, F32, "r", device_only=True)
        z = torch.empty_like(r)
        o = make_opts(**opts)
        L.check(L.load().thermal_precond_apply(self._h, float(dt), C.byref(o), _ptr(r), _ptr(z), _stream()))
        return z

    def spectral_bounds(self, dt=0.0, **opts):
        o = make_opts(**opts)
        v = [C.c_double() for _ in range(4)]
        L.check(L.load().thermal_spectral_bounds(self._h, float(dt), C.byref(o), *[C.byref(x) for x in v],
                                                 _stream()))
        return tuple(x.value for x in v)

    KERNELS = {"stencil_f32": 0, "cheb_f32": 1, "cheb_bf16": 2, "spmv_dot_f32": 3, "update_f32": 4,
               "residual_f64": 5, "stencil_f64": 6, "cheb_f64": 7, "residual_df": 8,
               "cheb_f32_faces": 9, "spmv_dot_f32_faces": 10, "residual_df_faces": 11, "stencil_f32_faces": 12,
               "cheb_tb4": 13, "cheb_tb2": 14, "cheb_tb3": 15,
               "ad_cheb_a3": 16, "ad_spmv_early": 17, "ad_spmv_late": 18,
               "mg_vcycle": 19, "cheb_tbf4": 20, "cheb_tbf2": 21, "cheb_tbf3": 22}

    def kernel_time(self, kernel, reps=50, dt=0.0):
        """Average duration (ms) of one launch of a hot kernel on this grid (CUDA events)."""
        ms = C.c_double()
        kid = self.KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        L.check(L.load().thermal_kernel_time(self._h, kid, int(reps), float(dt), C.byref(ms), _stream()))
        return ms.value

    def csr_spmv(self, x: torch.Tensor, dt: float = 0.0, variant: str = "scalar", reps: int = 0):
        """y = A x through a CSR copy of the matrix (Sec. 5.5 comparison).  x float32 or
        float64 on the device.  Returns (y, ms): ms is the mean launch time over reps
        timed launches, or None when reps == 0."""
        _check(x, self.n, F32_OR_F64, "x", device_only=True)
        prec = "fp64" if x.dtype == torch.float64 else "mixed"
        y = torch.empty_like(x)
        ms = C.c_double()
        L.check(L.load().thermal_csr_spmv(self._h, {"scalar": 0, "vector": 1}[variant], PRECISION[prec], float(dt),
                                          _ptr(x), _ptr(y), max(int(reps), 1),
                                          C.byref(ms) if reps > 0 else None, _stream()))
        return y, (ms.value if reps > 0 else None)

    # ------------------------------------------------------------------ solves

    def solve_steady(self, power: torch.Tensor, T: Optional[torch.Tensor] = None, **opts):
        """Returns (T, stats).  T (float64, deg C) is allocated on power's device when not given."""
        _check(power, self.n, F32_OR_F64, "power")
        if T is None:
            T = torch.empty(self.n, dtype=torch.float64, device=power.device)
        _check(T, self.n, F64, "T")
        o = make_opts(**opts)
        st = L.SolveStats()
        L.check(L.load().thermal_solve_steady(self._h, _ptr(power), _dtype_code(power), _ptr(T), C.byref(o),
                                              C.byref(st), _stream()))
        return T, st.as_dict()

    def step_transient(self, power: torch.Tensor, dt: float, T: torch.Tensor, **opts):
        """One backward-Euler step in place on T (T_n -> T_{n+1})."""
        _check(power, self.n, F32_OR_F64, "power")
        _check(T, self.n, F64, "T")
        o = make_opts(**opts)
        st = L.SolveStats()
        L.check(L.load().thermal_step_transient(self._h, _ptr(power), _dtype_code(power), float(dt), _ptr(T),
                                                C.byref(o), C.byref(st), _stream()))
        return T, st.as_dict()

    def run_transient(self, maps: List[torch.Tensor], steps_per_map: int, n_steps: int, dt: float,
                      T: torch.Tensor, **opts):
        """n_steps backward-Euler steps in place on T; step s uses maps[(s // steps_per_map) % len(maps)]."""
        _check_maps(maps, self.n)
        _check(T, self.n, F64, "T")
        o = make_opts(**opts)
        st = L.SolveStats()
        arr = (C.c_void_p * len(maps))(*[m.data_ptr() for m in maps])
        L.check(L.load().thermal_run_transient(self._h, arr, len(maps), _dtype_code(maps[0]), int(steps_per_map),
                                               int(n_steps), float(dt), _ptr(T), C.byref(o), C.byref(st),
                                               _stream()))
        return T, st.as_dict()

    # ------------------------------------------------------------------ adjoint

    def hotspot_lse(self, T: torch.Tensor, layers: Sequence[int], beta: float, want_grad=True):
        _check(T, self.n, F64, "T", device_only=True)
        if not layers or any(not 0 <= int(l) < self.L for l in layers):
            raise ValueError(f"layers must be a non-empty list of indices in [0, {self.L})")
        ids = (C.c_int * len(layers))(*[int(l) for l in layers])
        J = C.c_double()
        g = torch.empty_like(T) if want_grad else None
        L.check(L.load().thermal_hotspot_lse(self._h, _ptr(T), ids, len(layers), float(beta), C.byref(J), _ptr(g),
                                             _stream()))
        return J.value, g

    def grad(self, T: torch.Tensor, dJdT: torch.Tensor, dJdP_dtype=torch.float32, want_k=True, **opts):
        """Adjoint gradient: (dJ/dP on the device, dJ/dk per layer as a list)."""
        _check(T, self.n, F64, "T", device_only=True)
        _check(dJdT, self.n, F64, "dJdT", device_only=True)
        if dJdP_dtype not in F32_OR_F64:
            raise TypeError("dJdP_dtype must be torch.float32 or torch.float64")
        dJdP = torch.empty(self.n, dtype=dJdP_dtype, device=T.device)
        dk = (C.c_double * self.L)() if want_k else None
        o = make_opts(**opts)
        st = L.SolveStats()
        L.check(L.load().thermal_grad(self._h, _ptr(T), _ptr(dJdT), _ptr(dJdP), _dtype_code(dJdP),
                                      dk, C.byref(o), C.byref(st), _stream()))
        return dJdP, (list(dk) if want_k else None), st.as_dict()


def solve_batched(grids: List[ThermalGrid], powers: List[torch.Tensor], Ts: List[torch.Tensor], **opts):
    n = len(grids)
    if not (len(powers) == len(Ts) == n):
        raise ValueError("grids, powers and Ts must have the same length")
    if len({id(g) for g in grids}) != n:
        raise ValueError("each instance needs its own grid (the same grid appears twice)")
    if len({id(t) for t in Ts}) != n:
        raise ValueError("each instance needs its own output T (the same tensor appears twice)")
    for i, (g, p, t) in enumerate(zip(grids, powers, Ts)):
        _check(p, g.n, F32_OR_F64, f"powers[{i}]", device_only=True)
        _check(t, g.n, F64, f"Ts[{i}]", device_only=True)
    if n and len({p.dtype for p in powers}) != 1:
        raise TypeError("all power maps of a batch must share one dtype")
    o = make_opts(**opts)
    stats = (L.SolveStats * n)()
    gh = (C.c_void_p * n)(*[g.handle.value for g in grids])
    ph = (C.c_void_p * n)(*[p.data_ptr() for p in powers])
    th = (C.c_void_p * n)(*[t.data_ptr() for t in Ts])
    pdt = _dtype_code(powers[0]) if n else L.TH_F64
    L.check(L.load().thermal_solve_batched(gh, n, ph, pdt, th, C.byref(o), stats, _stream()))
    return [s.as_dict() for s in stats]


class SteadyAdjoint(torch.autograd.Function):
    """T = solve(P, k): forward is a steady solve, backward one adjoint solve.

    forward(grid, power [n], k [L] float64 (CPU), opts dict) -> T [n] float64 (deg C).
    backward returns dJ/dP (power's dtype) and dJ/dk (float64, CPU).
    """

    @staticmethod
    def forward(ctx, grid: ThermalGrid, power: torch.Tensor, k: torch.Tensor, opts: dict):
        grid.set_conductivity(k.detach().cpu().double().tolist())
        T, _ = grid.solve_steady(power.detach(), **opts)
        ctx.grid, ctx.opts, ctx.pdtype = grid, opts, power.dtype
        ctx.save_for_backward(T)
        return T

    @staticmethod
    def backward(ctx, grad_T):
        (T,) = ctx.saved_tensors
        dJdP, dJdk, _ = ctx.grid.grad(T, grad_T.contiguous().double(), dJdP_dtype=ctx.pdtype, **ctx.opts)
        return None, dJdP, torch.tensor(dJdk, dtype=torch.float64), None


class HotspotLSE(torch.autograd.Function):
    """J = (1/beta) log sum exp(beta T_i) over the given layers (library kernel)."""

    @staticmethod
    def forward(ctx, grid: ThermalGrid, T: torch.Tensor, layers, beta: float):
        J, g = grid.hotspot_lse(T.detach().contiguous(), layers, beta)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=T.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return None, g * gJ, None, None
