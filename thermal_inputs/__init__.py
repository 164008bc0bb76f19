"""Seeded synthetic inputs for the layered 3D-IC thermal workloads.

This module is shared by the CPU oracle and by the CUDA path, and holds only
input data: layer stacks (thickness, conductivity, heat capacity), boundary
constants and seeded power maps in watts per cell.  It contains none of the
solver's arithmetic (no conductances, no matrix, no solve).

Cell ordering used for every flat array: i = x + nx * (y + ny * z), x fastest,
z = layer index with z = 0 the bottom (adiabatic) layer and z = L-1 the top
layer whose upper face is convective.

Stacks follow the workloads of the paper's experiments (Sec. 5.1, the 10-layer
memory-on-logic stack) and the synthetic configurations this project measures:

* ``c1``   64x64x4  single die: Si 100um, BEOL/bond 10um, TIM 25um, Cu 1mm.
* ``c2``   512x512x8: two Si dies (100um Si + 10um bond each), TIM, Cu spreader
           split into three 333.3um sublayers.
* ``c3``   1024x1024x8: the ``c2`` stack, transient, four floorplans.
* ``c4``   64 independent stacks of uneven size with perturbed conductivities.
* ``c5``   2048x2048x10: the paper's memory-on-logic stack (Sec. 5.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Sequence

import numpy as np

UM = 1e-6
W_PER_CM2 = 1e4  # W/cm^2 -> W/m^2


@dataclass(frozen=True)
class Layer:
    name: str
    thickness: float      # m
    k: float              # W/(m K)
    c: float              # J/(m^3 K), volumetric heat capacity
    powered: bool = False  # carries a power map


@dataclass(frozen=True)
class Stack:
    layers: tuple          # bottom -> top
    h: float = 1e4         # W/(m^2 K), convective top face
    t_amb: float = 45.0    # deg C
    dx: float = 50 * UM
    dy: float = 50 * UM

    @property
    def L(self) -> int:
        return len(self.layers)

    def k(self) -> np.ndarray:
        return np.array([l.k for l in self.layers], dtype=np.float64)

    def c(self) -> np.ndarray:
        return np.array([l.c for l in self.layers], dtype=np.float64)

    def dz(self) -> np.ndarray:
        return np.array([l.thickness for l in self.layers], dtype=np.float64)

    def power_layers(self) -> List[int]:
        return [i for i, l in enumerate(self.layers) if l.powered]

    def with_k(self, k: Sequence[float]) -> "Stack":
        return replace(self, layers=tuple(replace(l, k=float(kk)) for l, kk in zip(self.layers, k)))


# Volumetric heat capacities (J/m^3 K) of the transient configuration.
C_SI, C_CU, C_TIM, C_BOND = 1.63e6, 3.45e6, 2.0e6, 1.5e6


def si(th_um=100.0, powered=True, name="si"):
    return Layer(name, th_um * UM, 150.0, C_SI, powered)


def bond(th_um=10.0, name="bond"):
    return Layer(name, th_um * UM, 2.5, C_BOND)


def tim(th_um=25.0):
    return Layer("tim", th_um * UM, 4.0, C_TIM)


def cu(th_um=1000.0, name="cu"):
    return Layer(name, th_um * UM, 400.0, C_CU)


def stack_c1(h=1e4) -> Stack:
    """Si die 100um (powered) / BEOL-bond 10um / TIM 25um / Cu spreader 1mm."""
    return Stack((si(), bond(name="beol"), tim(), cu()), h=h)


def stack_c1_split_cu(h=1e4) -> Stack:
    """The single-die stack with the 1mm Cu spreader split into 3 sublayers (6 layers)."""
    t = 1000.0 / 3.0
    return Stack((si(), bond(name="beol"), tim(), cu(t, "cu0"), cu(t, "cu1"), cu(t, "cu2")), h=h)


def stack_c2(h=1e4) -> Stack:
    """Two stacked dies (100um Si + 10um bond each), TIM 25um, Cu 1mm as 3 sublayers."""
    t = 1000.0 / 3.0
    return Stack((si(name="si0"), bond(name="bond0"), si(name="si1"), bond(name="bond1"), tim(),
                  cu(t, "cu0"), cu(t, "cu1"), cu(t, "cu2")), h=h)


def stack_mol(h=1e4) -> Stack:
    """The paper's 10-layer memory-on-logic F2F stack (Sec. 5.1, bottom to top).

    Conductivities are not given in the paper; bulk/FEOL Si 150, BEOL and hybrid
    bond 2.5, TIM 4, spreader and sink Cu 400 W/mK.  Power on the two FEOL layers.
    """
    return Stack((
        Layer("logic_bulk", 10 * UM, 150.0, C_SI),
        Layer("logic_feol", 2 * UM, 150.0, C_SI, True),
        Layer("logic_beol", 10 * UM, 2.5, C_BOND),
        Layer("hybrid_bond", 2 * UM, 2.5, C_BOND),
        Layer("mem_beol", 10 * UM, 2.5, C_BOND),
        Layer("mem_feol", 2 * UM, 150.0, C_SI, True),
        Layer("mem_bulk", 200 * UM, 150.0, C_SI),
        Layer("tim", 100 * UM, 4.0, C_TIM),
        Layer("spreader", 400 * UM, 400.0, C_CU),
        Layer("sink", 1000 * UM, 400.0, C_CU),
    ), h=h)


# ---------------------------------------------------------------- power maps

def _gauss_1d(n, d, centre, sigma):
    x = (np.arange(n, dtype=np.float64) + 0.5) * d
    return np.exp(-((x - centre) ** 2) / (2.0 * sigma * sigma))


def add_gaussian_hotspots(q, rng, n_spots, dx, dy):
    """Add ``n_spots`` Gaussian hotspots (W/cm^2) to the 2D density map ``q`` in place.

    Each spot: peak U[200,500] W/cm^2, sigma U[100,300] um, centre uniform over the
    die; the value at a cell centre is peak * exp(-r^2 / (2 sigma^2)).
    """
    ny, nx = q.shape
    for _ in range(n_spots):
        cx = rng.uniform(0.0, nx * dx)
        cy = rng.uniform(0.0, ny * dy)
        sigma = rng.uniform(100.0, 300.0) * UM
        peak = rng.uniform(200.0, 500.0)
        q += peak * np.outer(_gauss_1d(ny, dy, cy, sigma), _gauss_1d(nx, dx, cx, sigma))
    return q


def density_uniform_hotspots(nx, ny, seed, background=20.0, n_spots=8, dx=50 * UM, dy=50 * UM):
    """Uniform background (W/cm^2) plus Gaussian hotspots: the single-die workload."""
    rng = np.random.default_rng(seed)
    q = np.full((ny, nx), background, dtype=np.float64)
    return add_gaussian_hotspots(q, rng, n_spots, dx, dy)


def density_floorplan(nx, ny, seed, n_rects=64, n_spots=16, dx=50 * UM, dy=50 * UM):
    """Random block floorplan (W/cm^2): ``n_rects`` rectangles painted in order.

    Rectangle sides are uniform integers in [n/32, n/4] cells (at least 1), the
    position is uniform among placements that fit, the density is U[5,80] W/cm^2 and
    a later rectangle overrides an earlier one; cells no rectangle covers are 0.
    Then ``n_spots`` additive Gaussian hotspots.
    """
    rng = np.random.default_rng(seed)
    q = np.zeros((ny, nx), dtype=np.float64)
    lo_x, hi_x = max(1, nx // 32), max(1, nx // 4)
    lo_y, hi_y = max(1, ny // 32), max(1, ny // 4)
    for _ in range(n_rects):
        w = int(rng.integers(lo_x, hi_x + 1))
        h = int(rng.integers(lo_y, hi_y + 1))
        x0 = int(rng.integers(0, nx - w + 1))
        y0 = int(rng.integers(0, ny - h + 1))
        q[y0:y0 + h, x0:x0 + w] = rng.uniform(5.0, 80.0)
    return add_gaussian_hotspots(q, rng, n_spots, dx, dy)


def power_cells(stack: Stack, nx, ny, densities, dtype=np.float64) -> np.ndarray:
    """Place per-layer 2D densities (W/cm^2) on the powered layers; return W per cell.

    ``densities`` is a list with one (ny, nx) map per powered layer.  The value of a
    cell is q [W/cm^2] * 1e4 * dx * dy (the power of the cell's footprint), on the
    powered layers only.  Flat, x fastest, length nx*ny*L.
    """
    L = stack.L
    out = np.zeros((L, ny, nx), dtype=np.float64)
    area = stack.dx * stack.dy
    for layer, q in zip(stack.power_layers(), densities):
        out[layer] = q * W_PER_CM2 * area
    return out.reshape(-1).astype(dtype)


# ---------------------------------------------------------------- workloads

@dataclass
class Instance:
    name: str
    nx: int
    ny: int
    stack: Stack
    power: np.ndarray                       # W per cell, flat (primary map)
    extra_power: List[np.ndarray] = field(default_factory=list)  # further maps (transient)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.stack.L


def c1(nx=64, ny=64, seed=1, dtype=np.float32) -> Instance:
    st = stack_c1()
    q = density_uniform_hotspots(nx, ny, seed, dx=st.dx, dy=st.dy)
    return Instance("c1", nx, ny, st, power_cells(st, nx, ny, [q], dtype))


def _floorplans(st, nx, ny, seed):
    # one independent floorplan per powered layer, seeds derived from the workload seed
    return [density_floorplan(nx, ny, seed * 1000 + j, dx=st.dx, dy=st.dy)
            for j in range(len(st.power_layers()))]


def c2(nx=512, ny=512, seed=2, dtype=np.float32) -> Instance:
    st = stack_c2()
    return Instance("c2", nx, ny, st, power_cells(st, nx, ny, _floorplans(st, nx, ny, seed), dtype))


C3_DT = 1e-4
C3_STEPS = 100
C3_STEPS_PER_MAP = 25


def c3(nx=1024, ny=1024, seeds=(30, 31, 32, 33), dtype=np.float32) -> Instance:
    """Transient workload: four floorplans, switched every 25 backward-Euler steps."""
    st = stack_c2()
    maps = [power_cells(st, nx, ny, _floorplans(st, nx, ny, s), dtype) for s in seeds]
    return Instance("c3", nx, ny, st, maps[0], maps[1:])


C4_CLASSES = ((128, 4), (256, 6), (384, 8), (512, 8))


def c4_instances(n=64, class_seed=4, scale=1, dtype=np.float32) -> List[Instance]:
    """64 independent stacks of uneven size; per-layer k perturbed by U[0.8, 1.2].

    The size class of each instance is drawn uniformly from C4_CLASSES with
    ``class_seed``; instance i uses seed 400 + i for its k perturbation and power map.
    ``scale`` divides the in-plane size (test-size batches keep the same recipe).
    """
    rng = np.random.default_rng(class_seed)
    classes = rng.integers(0, len(C4_CLASSES), size=n)
    out = []
    for i, ci in enumerate(classes):
        side, L = C4_CLASSES[int(ci)]
        side = max(4, side // scale)
        base = {4: stack_c1(), 6: stack_c1_split_cu(), 8: stack_c2()}[L]
        r = np.random.default_rng(400 + i)
        k = base.k() * r.uniform(0.8, 1.2, size=L)
        st = base.with_k(k)
        maps = [density_floorplan(side, side, 400 + i + 7919 * j, dx=st.dx, dy=st.dy)
                for j in range(len(st.power_layers()))]
        out.append(Instance(f"c4_{i}", side, side, st, power_cells(st, side, side, maps, dtype)))
    return out


def c5(nx=2048, ny=2048, seed=50, dtype=np.float32) -> Instance:
    """Adjoint workload: the memory-on-logic stack, floorplans on the two FEOL layers."""
    st = stack_mol()
    dens = [density_floorplan(nx, ny, seed + j, dx=st.dx, dy=st.dy) for j in range(2)]
    return Instance("c5", nx, ny, st, power_cells(st, nx, ny, dens, dtype))


def random_vector(n, seed, dtype=np.float64, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=n).astype(dtype)
