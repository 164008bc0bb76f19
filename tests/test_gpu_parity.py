"""GPU path vs the CPU oracle, through the C ABI (libthermal.so).

Grids span several 32x8 thread tiles with ragged tails (nx, ny not multiples of
the tile) and the stacks of the measured workloads.  Tolerances follow from the
arithmetic:

* FP64 stencil: componentwise |dy_i| <= 1e-14 * sum_j |a_ij x_j| (a handful of
  roundings of size 2^-53 per term).
* FP32 stencil: coefficients rounded to FP32 (2^-24) and ~13 FP32 operations:
  |dy_i| <= 2e-6 * sum_j |a_ij x_j|.  BF16 coefficients (2^-9): 1e-2.
* Solves: max|T - T_ref| / max|T_ref - T_amb| <= 1e-6 at tol_rel 1e-10 (FP64 and
  mixed paths), the target accuracy of the method on this hardware.
"""
import numpy as np
import pytest

import thermal_inputs as ti
from oracle import adjoint as oadj, discretisation as disc, krylov, solve as osolve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as ge
    ge.build()


def grid_of(nx, ny, st):
    from paper_2606_17850_gb300 import ThermalGrid
    return ThermalGrid.from_stack(nx, ny, st)


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# nx % 4 != 0 runs the scalar kernels, nx % 4 == 0 the vectorised z-walk kernels
SHAPES = [(70, 19, "c1"), (37, 45, "c2"), (33, 9, "mol"), (5, 3, "c2"),
          (72, 19, "c1"), (36, 45, "c2"), (132, 9, "mol"), (4, 3, "c2")]
STACKS = {"c1": ti.stack_c1, "c2": ti.stack_c2, "mol": ti.stack_mol,
          # 5, 6 and 7 layers: the fused kernels pair layer k with layer k + 4, so these
          # put real and zero-padded layers in the same pair
          "l5": lambda: ti.Stack((ti.si(), ti.bond(), ti.si(name="si1"), ti.tim(), ti.cu()), h=1e4),
          "l6": ti.stack_c1_split_cu,
          "l7": lambda: ti.Stack((ti.si(name="si0"), ti.bond(name="b0"), ti.si(name="si1"), ti.bond(name="b1"),
                                  ti.tim(), ti.cu(500.0, "cu0"), ti.cu(500.0, "cu1")), h=1e4)}


# ----------------------------------------------------------------- A1: setup

@pytest.mark.parametrize("nx,ny,mk", SHAPES)
@pytest.mark.parametrize("dt", [0.0, 1e-4])
def test_faces_and_diagonal(nx, ny, mk, dt):
    st = STACKS[mk]()
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None).tocsr()
    g = grid_of(nx, ny, st)
    f = {k: v.cpu().numpy() for k, v in g.faces(dt).items()}
    n = nx * ny * st.L
    i = np.arange(n)
    x = i % nx
    y = (i // nx) % ny
    z = i // (nx * ny)
    want_gx = np.where(x + 1 < nx, -np.asarray(A[i, np.minimum(i + 1, n - 1)]).ravel(), 0.0)
    want_gy = np.where(y + 1 < ny, -np.asarray(A[i, np.minimum(i + nx, n - 1)]).ravel(), 0.0)
    want_gz = np.where(z + 1 < st.L, -np.asarray(A[i, np.minimum(i + nx * ny, n - 1)]).ravel(), 0.0)
    np.testing.assert_allclose(f["gx"], want_gx, rtol=1e-15, atol=0)
    np.testing.assert_allclose(f["gy"], want_gy, rtol=1e-15, atol=0)
    np.testing.assert_allclose(f["gz"], want_gz, rtol=1e-15, atol=0)
    np.testing.assert_allclose(f["diag"], A.diagonal(), rtol=1e-14, atol=0)


# ----------------------------------------------------------------- A2: stencil

@pytest.mark.parametrize("nx,ny,mk", SHAPES)
@pytest.mark.parametrize("dt", [0.0, 1e-4])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-14), ("mixed", 2e-6), ("mixed_bf16", 1e-2)])
def test_stencil_product(nx, ny, mk, dt, prec, rtol):
    st = STACKS[mk]()
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None).tocsr()
    g = grid_of(nx, ny, st)
    xh = ti.random_vector(A.shape[0], 21, lo=-3.0, hi=5.0)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xd = cuda(xh, dtype)
    y = g.apply(xd, dt, prec).cpu().double().numpy()
    x_used = xd.cpu().double().numpy()          # the rounded input both sides see
    y_ref = A @ x_used
    bound = abs(A) @ np.abs(x_used)
    assert np.all(np.abs(y - y_ref) <= rtol * bound), np.max(np.abs(y - y_ref) / bound)


def test_stencil_misaligned_view_fp32():
    """A tensor view that is not 16-byte aligned takes the scalar kernel: same result."""
    st = ti.stack_c2()
    nx, ny = 36, 10
    A = disc.assemble(nx, ny, st).tocsr()
    g = grid_of(nx, ny, st)
    buf = cuda(ti.random_vector(A.shape[0] + 1, 9).astype(np.float32))
    x = buf[1:]
    y = g.apply(x, 0.0, "mixed").cpu().double().numpy()
    xh = x.cpu().double().numpy()
    assert np.all(np.abs(y - A @ xh) <= 2e-6 * (abs(A) @ np.abs(xh)))


def test_stencil_symmetry_fp64():
    st = ti.stack_c2()
    g = grid_of(41, 23, st)
    n = 41 * 23 * st.L
    x = cuda(ti.random_vector(n, 1))
    yv = cuda(ti.random_vector(n, 2))
    a = torch.dot(g.apply(x, 0.0, "fp64"), yv).item()
    b = torch.dot(x, g.apply(yv, 0.0, "fp64")).item()
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


# ------------------------------------------------- Sec. 5.5: CSR copy of the matrix

@pytest.mark.parametrize("variant", ["scalar", "vector"])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-14), ("mixed", 2e-6)])
@pytest.mark.parametrize("nx,ny,mk,dt", [(37, 21, "c2", 1e-4), (5, 3, "c1", 0.0), (1, 1, "c1", 0.0)])
def test_csr_spmv_matches_oracle(variant, prec, rtol, nx, ny, mk, dt):
    """The CSR product (device-assembled, closed-form row offsets) equals the oracle's
    row-wise CSR product, including 1-cell-wide grids and the transient diagonal."""
    st = STACKS[mk]()
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None).tocsr()
    g = grid_of(nx, ny, st)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    xd = cuda(ti.random_vector(A.shape[0], 23, lo=-2.0, hi=3.0), dtype)
    y, ms = g.csr_spmv(xd, dt=dt, variant=variant, reps=2)
    assert ms is not None and ms > 0
    xh = xd.cpu().double().numpy()
    err = np.abs(y.cpu().double().numpy() - A @ xh)
    assert np.all(err <= rtol * (abs(A) @ np.abs(xh))), np.max(err / (abs(A) @ np.abs(xh)))


def test_csr_spmv_rejects_bad_arguments():
    st = ti.stack_c1()
    g = grid_of(8, 8, st)
    x = cuda(np.ones(8 * 8 * st.L), torch.float64)
    with pytest.raises(Exception):
        g.csr_spmv(x, variant="diagonal")
    import ctypes as C
    from paper_2606_17850_gb300 import _lib as L
    assert L.load().thermal_csr_spmv(g._h, 0, 0, 0.0, C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 1,
                                     None, None) == L.TH_EINVAL


def _kmap(st, nx, ny, seed=5):
    return np.repeat(st.k(), nx * ny) * np.random.default_rng(seed).uniform(0.5, 2.0, nx * ny * st.L)


@pytest.mark.parametrize("nx", [36, 37])
@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-14), ("mixed", 2e-6)])
def test_conductivity_map_faces_and_stencil(nx, prec, rtol):
    """Per-cell conductivities: faces against the oracle's half-cell series and the
    stencil product through the per-face kernels (scalar and vectorised)."""
    st = ti.stack_c2()
    ny, dt = 23, 1e-4
    kc = _kmap(st, nx, ny)
    A = disc.assemble(nx, ny, st, dt=dt, k_cell=kc).tocsr()
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(torch.from_numpy(kc))
    f = {k: v.cpu().numpy() for k, v in g.faces(dt).items()}
    np.testing.assert_allclose(f["diag"], A.diagonal(), rtol=1e-14, atol=0)
    xd = cuda(ti.random_vector(A.shape[0], 2), torch.float64 if prec == "fp64" else torch.float32)
    y = g.apply(xd, dt, prec).cpu().double().numpy()
    x_used = xd.cpu().double().numpy()
    assert np.all(np.abs(y - A @ x_used) <= rtol * (abs(A) @ np.abs(x_used)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_conductivity_map_solve(prec):
    st = ti.stack_c2()
    nx, ny = 40, 29
    kc = _kmap(st, nx, ny, 8)
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (3, 4)], np.float64)
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(cuda(kc))
    T, stats = g.solve_steady(cuda(P), precision=prec, cheb_degree=12, tol_rel=1e-10)
    ref = osolve.steady(nx, ny, st, P, k_cell=kc)
    assert stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


def test_uniform_map_equals_layer_table():
    """A map holding the layer values gives the same faces as the per-layer setup, and
    the per-face kernels then agree with the layer-table kernels."""
    st = ti.stack_c2()
    nx, ny, dt = 44, 21, 1e-4
    P = cuda(ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (5, 6)], np.float32))
    a, b = grid_of(nx, ny, st), grid_of(nx, ny, st)
    b.set_conductivity_map(cuda(np.repeat(st.k(), nx * ny)))
    fa, fb = a.faces(dt), b.faces(dt)
    for k in ("gx", "gy", "gz", "diag"):
        assert torch.equal(fa[k], fb[k]), k
    Ta, _ = a.solve_steady(P, tol_rel=1e-10)
    Tb, _ = b.solve_steady(P, tol_rel=1e-10)
    assert (Ta - Tb).abs().max().item() <= 1e-7 * (Ta - st.t_amb).abs().max().item()


def test_grad_k_undefined_with_map():
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c1()
    g = grid_of(16, 12, st)
    g.set_conductivity_map(cuda(_kmap(st, 16, 12)))
    P = cuda(ti.power_cells(st, 16, 12, [ti.density_uniform_hotspots(16, 12, 1)], np.float64))
    T, _ = g.solve_steady(P, tol_rel=1e-10)
    J, w = g.hotspot_lse(T, st.power_layers(), 2.0)
    with pytest.raises(ThermalError) as e:
        g.grad(T, w)
    assert e.value.status == 7
    dJdP, _, _ = g.grad(T, w, want_k=False, tol_rel=1e-10)
    assert torch.isfinite(dJdP).all()


# ----------------------------------------------------------------- A3/A4: preconditioners

@pytest.mark.parametrize("dt", [0.0, 1e-4])
def test_lanczos_matches_oracle(dt):
    st = ti.stack_c2()
    nx, ny = 45, 38
    g = grid_of(nx, ny, st)
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None)
    op, _ = krylov.jacobi_scaled(A)
    a, b = krylov.lanczos(op, krylov.splitmix64_uniform(A.shape[0], 0x5EED), 50)
    lo, hi = krylov.ritz_extremes(a, b)
    rmin, rmax, lmin, lmax = g.spectral_bounds(dt, lanczos_steps=50, cheb_scaled=1)
    assert abs(rmax - hi) <= 1e-3 * hi
    assert abs(rmin - lo) <= 2e-2 * lo
    assert abs(lmax - 1.05 * rmax) <= 1e-12 * lmax


# the Jacobi scaling option applies to the Chebyshev preconditioner only
@pytest.mark.parametrize("nx", [37, 36])
@pytest.mark.parametrize("pc,scaled", [("none", 1), ("jacobi", 1), ("zline", 1), ("cheb", 1), ("cheb", 0)])
def test_preconditioner_apply(pc, scaled, nx):
    st = ti.stack_c2()
    ny, dt = 29, 1e-4
    g = grid_of(nx, ny, st)
    A = disc.assemble(nx, ny, st, dt=dt)
    r = ti.random_vector(A.shape[0], 5).astype(np.float32)
    k = 12
    z = g.precond(cuda(r), dt, precond=pc, cheb_degree=k, cheb_scaled=scaled).cpu().double().numpy()
    r64 = r.astype(np.float64)
    if pc == "none":
        ref = r64
    elif pc == "jacobi":
        ref = r64 / A.diagonal()
    elif pc == "zline":
        ref = krylov.zline(A, nx, ny, st.L)(r64)
    else:
        _, _, lmin, lmax = g.spectral_bounds(dt, cheb_scaled=scaled)
        D = A.diagonal()
        op = (lambda v: (A @ v) / D) if scaled else (lambda v: A @ v)
        ref = krylov.chebyshev(op, r64 / D if scaled else r64, lmin, lmax, k)
    np.testing.assert_allclose(z, ref, rtol=0, atol=2e-4 * np.abs(ref).max())


# the whole chain on each side: the oracle's own FP64 Lanczos interval feeds the
# oracle's polynomial, the GPU's FP32 Lanczos feeds the GPU's.  Transient systems
# with m close to N Lanczos steps, where FP64 Ritz values equal the extreme
# eigenvalues (numpy eigvalsh) and FP32 ones agree with them to < 3e-6.
@pytest.mark.parametrize("nx,ny,mk,m,scaled", [(36, 29, "c2", 300, 1), (37, 29, "c2", 300, 1),
                                               (6, 5, "c2", 240, 1), (6, 5, "c2", 240, 0),
                                               (12, 10, "c1", 480, 1)])
def test_chebyshev_chain_from_oracle_lanczos(nx, ny, mk, m, scaled):
    st = STACKS[mk]()
    dt, k = 1e-4, 12
    A = disc.assemble(nx, ny, st, dt=dt)
    D = A.diagonal()
    op_l = krylov.jacobi_scaled(A)[0] if scaled else (lambda v: A @ v)
    a, b = krylov.lanczos(op_l, krylov.splitmix64_uniform(A.shape[0], 0x5EED), m)
    lmin, lmax = krylov.chebyshev_bounds(*krylov.ritz_extremes(a, b))
    M = (A.toarray() / np.sqrt(D)[:, None] / np.sqrt(D)[None, :]) if scaled else A.toarray()
    ev = np.linalg.eigvalsh(M)
    ex_min, ex_max = krylov.chebyshev_bounds(ev[0], ev[-1])
    assert abs(lmax / ex_max - 1) <= 1e-10 and abs(lmin / ex_min - 1) <= 1e-6   # the oracle's interval
    g = grid_of(nx, ny, st)
    _, _, glmin, glmax = g.spectral_bounds(dt, lanczos_steps=m, cheb_scaled=scaled)
    assert abs(glmax / lmax - 1) <= 1e-5 and abs(glmin / lmin - 1) <= 1e-4
    r = ti.random_vector(A.shape[0], 6).astype(np.float32)
    z = g.precond(cuda(r), dt, precond="cheb", cheb_degree=k, cheb_scaled=scaled,
                  lanczos_steps=m).cpu().double().numpy()
    r64 = r.astype(np.float64)
    op = (lambda v: (A @ v) / D) if scaled else (lambda v: A @ v)
    ref = krylov.chebyshev(op, r64 / D if scaled else r64, lmin, lmax, k)
    np.testing.assert_allclose(z, ref, rtol=0, atol=2e-4 * np.abs(ref).max())


@pytest.mark.parametrize("k", [2, 5, 8, 12])
@pytest.mark.parametrize("dt", [0.0, 1e-4])
@pytest.mark.parametrize("mk", ["c2", "c1", "mol", "l5", "l6", "l7"])
def test_fused_chebyshev_equals_stepwise(k, dt, mk):
    """Temporal blocking (1..4 steps per launch, TMA-staged tiles) computes the same
    polynomial as one launch per step: tiles with ragged x/y tails, 1..3 chunks,
    8 layers, 4 to 7 layers (zero-padded to 8) and 10 layers (the 12-layer variant)."""
    st = STACKS[mk]()
    nx, ny = 76, 37           # nx % 32 != 0 and ny % 16 != 0: partial tiles on both axes
    g = grid_of(nx, ny, st)
    r = cuda(ti.random_vector(nx * ny * st.L, 5).astype(np.float32))
    z1 = g.precond(r, dt, precond="cheb", cheb_degree=k, cheb_fuse=1)
    scale = z1.abs().max().item()
    # The fused chunks take the product in expanded form, d v - sum_f g_f v_f, the
    # one-step kernel in difference form, sum_f g_f (v - v_f); in steady state d is
    # the sum of the faces, so the expanded form rounds at the level of d |v|: a few
    # FP32 ulps of max|z| per step (the Jacobi-scaled terms are at most |v|), summed
    # over the k - 1 steps.  Measured up to 1.2e-6 of max|z| (5 layers, steady, k 8).
    tol = max(1e-6, 2.5e-7 * k)
    for fuse in (0, 2, 3, 4):
        zf = g.precond(r, dt, precond="cheb", cheb_degree=k, cheb_fuse=fuse)
        assert (zf - z1).abs().max().item() <= tol * scale, fuse


@pytest.mark.parametrize("k", [2, 5, 8, 12])
@pytest.mark.parametrize("dt", [0.0, 1e-4])
@pytest.mark.parametrize("mk", ["c2", "c1", "l5", "l7"])
def test_fused_chebyshev_per_face_equals_stepwise(k, dt, mk):
    """Fused chunks on per-face arrays (a per-cell conductivity map; 32 x 24 tiles with
    the faces staged beside the vectors) compute the same polynomial as one launch per
    step: ragged tiles on both axes, 8 layers and 4, 5 and 7 layers (zero-padded)."""
    st = STACKS[mk]()
    nx, ny = 76, 37
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(cuda(_kmap(st, nx, ny, 21)))
    r = cuda(ti.random_vector(nx * ny * st.L, 5).astype(np.float32))
    z1 = g.precond(r, dt, precond="cheb", cheb_degree=k, cheb_fuse=1)
    scale = z1.abs().max().item()
    for fuse in (0, 2, 3, 4):
        zf = g.precond(r, dt, precond="cheb", cheb_degree=k, cheb_fuse=fuse)
        assert (zf - z1).abs().max().item() <= 1e-6 * scale, fuse


@pytest.mark.parametrize("k", [5, 9])
def test_fused_chebyshev_on_slabs_with_halo(k):
    """The one-grid multi-GPU partition on one GPU: each y-slab of a grid with a halo,
    run as a grid of its own through the fused chunks (k - 1 steps: one chunk at
    k = 5, two at k = 9) with the whole grid's spectral interval, gives the whole
    grid's preconditioned vector on the slab's rows bit for bit.  The halo rows absorb
    the sub-grid's artificial edge: k - 1 rows for the steps' reach, plus one because
    the edge row takes a boundary cell's diagonal in z_1 = D^-1 r / theta (a slab
    kernel given the whole grid's diagonal needs only the k - 1)."""
    from paper_2606_17850_gb300.dist import slab_cells, slab_halo, slab_rows
    st = ti.stack_c2()
    nx, ny, dt, world = 64, 50, 1e-4, 3
    g = grid_of(nx, ny, st)
    _, _, lmin, lmax = g.spectral_bounds(dt)
    r = ti.random_vector(nx * ny * st.L, 12).astype(np.float32)
    opts = dict(precond="cheb", cheb_degree=k, cheb_lam_min=lmin, cheb_lam_max=lmax)
    z = g.precond(cuda(r), dt, **opts).cpu().numpy()
    # the fixed interval equal to the estimate gives the default result; the estimate
    # call itself ignores a fixed interval
    z0 = g.precond(cuda(r), dt, precond="cheb", cheb_degree=k).cpu().numpy()
    assert np.array_equal(z, z0)
    assert g.spectral_bounds(dt, cheb_lam_min=1.0, cheb_lam_max=2.0)[2:] == (lmin, lmax)
    for q in range(world):
        y0, y1 = slab_rows(ny, q, world)
        h0, h1 = slab_halo(ny, q, world, k)
        ext = slab_cells(nx, ny, st.L, h0, h1)
        own = slab_cells(nx, ny, st.L, y0, y1)
        gs = grid_of(nx, h1 - h0, st)
        zs = gs.precond(cuda(r[ext]), dt, **opts).cpu().numpy()
        assert np.array_equal(zs[np.searchsorted(ext, own)], z[own]), q
        gs.close()


def test_slab_pcg_with_library_kernels_matches_whole_grid():
    """PCG on three y-slabs of one grid with the library's kernels per slab (FP64
    product with a 1-row halo, the fused Chebyshev preconditioner with a k-row halo
    and the whole grid's interval), the halos rebuilt from the neighbours' rows before
    each product or preconditioner, and two reductions per iteration: it reaches the
    same solution as the same iteration on the whole grid.  The CG vector updates and
    dot products are this test's (torch); no kernel waits on another."""
    from paper_2606_17850_gb300.dist import slab_cells, slab_halo, slab_rows
    st = ti.stack_c2()
    nx, ny, dt, k = 64, 50, 1e-4, 9
    g = grid_of(nx, ny, st)
    _, _, lmin, lmax = g.spectral_bounds(dt)
    popt = dict(precond="cheb", cheb_degree=k, cheb_lam_min=lmin, cheb_lam_max=lmax)
    b = cuda(ti.random_vector(g.n, 21))

    def solve(world):
        own = [torch.from_numpy(slab_cells(nx, ny, st.L, *slab_rows(ny, q, world))).cuda() for q in range(world)]
        sub = []
        for q in range(world):
            for width in (1, k):
                h0, h1 = slab_halo(ny, q, world, width)
                ext = torch.from_numpy(slab_cells(nx, ny, st.L, h0, h1)).cuda()
                gs = g if world == 1 else grid_of(nx, h1 - h0, st)
                sub.append((gs, ext, torch.searchsorted(ext, own[q])))
        n_reduce = [0]

        def gather(parts):                       # the halo exchange: owned rows to every slab
            v = torch.empty(g.n, dtype=parts[0].dtype, device="cuda")
            for q in range(world):
                v[own[q]] = parts[q]
            return v

        def op(parts):                           # y = A x, 1-row halos
            v = gather(parts)
            out = []
            for q in range(world):
                gs, ext, pos = sub[2 * q]
                out.append(gs.apply(v[ext].contiguous(), dt, "fp64")[pos])
            return out

        def prec(parts):                         # z = M r, k-row halos
            v = gather(parts).float()
            out = []
            for q in range(world):
                gs, ext, pos = sub[2 * q + 1]
                out.append(gs.precond(v[ext].contiguous(), dt, **popt)[pos].double())
            return out

        def dots(*pairs):                        # one reduction of several scalars
            n_reduce[0] += 1
            return [sum(float((a[q] * c[q]).sum()) for q in range(world)) for a, c in pairs]

        bp = [b[o] for o in own]
        x = [torch.zeros_like(v) for v in bp]
        r = [v.clone() for v in bp]
        z = prec(r)
        rz, bb = dots((r, z), (bp, bp))
        p_ = [v.clone() for v in z]
        per_it = set()
        for it in range(300):
            before = n_reduce[0]
            q_ = op(p_)
            (pq,) = dots((p_, q_))
            alpha = rz / pq
            x = [xi + alpha * pi for xi, pi in zip(x, p_)]
            r = [ri - alpha * qi for ri, qi in zip(r, q_)]
            z = prec(r)
            rz_new, rr = dots((r, z), (r, r))
            per_it.add(n_reduce[0] - before)
            if rr <= 1e-18 * bb:
                break
            p_ = [zi + (rz_new / rz) * pi for zi, pi in zip(z, p_)]
            rz = rz_new
        for gs, _, _ in sub:
            if gs is not g:
                gs.close()
        return gather(x), it, per_it

    xw, itw, _ = solve(1)
    xs, its, per_it = solve(3)
    assert itw < 300 and its < 300 and per_it == {2}
    assert abs(its - itw) <= 1
    assert (xs - xw).abs().max().item() <= 1e-9 * xw.abs().max().item()


def test_fused_chebyshev_per_face_matches_oracle():
    """The per-face fused preconditioner against the oracle's Chebyshev algorithm on
    the assembled per-cell-conductivity matrix (same spectral interval)."""
    st = ti.stack_c2()
    nx, ny, dt, k = 44, 29, 1e-4, 12
    kc = _kmap(st, nx, ny, 22)
    A = disc.assemble(nx, ny, st, dt=dt, k_cell=kc)
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(cuda(kc))
    r = ti.random_vector(A.shape[0], 9).astype(np.float32)
    z = g.precond(cuda(r), dt, precond="cheb", cheb_degree=k).cpu().double().numpy()
    _, _, lmin, lmax = g.spectral_bounds(dt)
    D = A.diagonal()
    ref = krylov.chebyshev(lambda v: (A @ v) / D, r.astype(np.float64) / D, lmin, lmax, k)
    np.testing.assert_allclose(z, ref, rtol=0, atol=2e-4 * np.abs(ref).max())


# ----------------------------------------------------------------- A5/A6: steady solves

@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
@pytest.mark.parametrize("pc", ["cheb", "jacobi", "none", "zline"])
def test_steady_solve_c1(prec, pc):
    inst = ti.c1(dtype=np.float32)
    st = inst.stack
    g = grid_of(inst.nx, inst.ny, st)
    T, stats = g.solve_steady(cuda(inst.power), precision=prec, precond=pc, cheb_degree=10, tol_rel=1e-10)
    T_ref = osolve.steady(inst.nx, inst.ny, st, inst.power.astype(np.float64))
    err = osolve.rise_relative_error(T.cpu().numpy(), T_ref, st.t_amb)
    assert stats["status"] == 0 and stats["rel_res"] <= 1e-10
    assert err <= 1e-6, err
    A = disc.assemble(inst.nx, inst.ny, st)
    b = disc.rhs_steady(inst.nx, inst.ny, st, inst.power.astype(np.float64))
    assert osolve.rel_residual(A, T.cpu().numpy(), b, st.t_amb) <= 2e-10


@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_steady_ragged_graph(graph, prec):
    st = ti.stack_c2()
    nx, ny = 45, 27
    dens = [ti.density_floorplan(nx, ny, s) for s in (8, 9)]
    P = ti.power_cells(st, nx, ny, dens, np.float64)
    g = grid_of(nx, ny, st)
    T, stats = g.solve_steady(cuda(P), precision=prec, precond="cheb", cheb_degree=16, tol_rel=1e-10,
                              use_graph=graph)
    T_ref = osolve.steady(nx, ny, st, P)
    assert stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), T_ref, st.t_amb) <= 1e-6
    # a second call reuses the cached graph and must give the same answer
    T2, _ = g.solve_steady(cuda(P), precision=prec, precond="cheb", cheb_degree=16, tol_rel=1e-10,
                           use_graph=graph)
    np.testing.assert_array_equal(T.cpu().numpy(), T2.cpu().numpy())


def test_steady_host_buffers_and_guess():
    inst = ti.c1(nx=40, ny=33, dtype=np.float32)
    st = inst.stack
    g = grid_of(inst.nx, inst.ny, st)
    P = torch.from_numpy(inst.power)                   # host memory
    T = torch.full((inst.n,), 60.0, dtype=torch.float64)  # host initial guess
    T, stats = g.solve_steady(P, T=T, tol_rel=1e-10, use_guess=1)
    T_ref = osolve.steady(inst.nx, inst.ny, st, inst.power.astype(np.float64))
    assert osolve.rise_relative_error(T.numpy(), T_ref, st.t_amb) <= 1e-6


def test_energy_balance_gpu():
    inst = ti.c1(dtype=np.float32)
    st = inst.stack
    g = grid_of(inst.nx, inst.ny, st)
    T, _ = g.solve_steady(cuda(inst.power), tol_rel=1e-10)
    top = T.cpu().numpy()[(st.L - 1) * inst.nx * inst.ny:]
    out = np.sum(st.h * st.dx * st.dy * (top - st.t_amb))
    assert abs(out - inst.power.astype(np.float64).sum()) / inst.power.sum() < 1e-9


# ----------------------------------------------------------------- A7/A8: transient

@pytest.mark.parametrize("nx", [50, 52])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
def test_transient_step(prec, nx):
    st = ti.stack_c2()
    ny, dt = 35, 1e-4
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (30, 31)], np.float32)
    g = grid_of(nx, ny, st)
    T0 = np.full(nx * ny * st.L, st.t_amb)
    T0[::7] += 3.0
    T = cuda(T0.copy())
    T, stats = g.step_transient(cuda(P), dt, T, precision=prec, tol_rel=1e-10, cheb_degree=6)
    ref = osolve.transient(nx, ny, st, [P.astype(np.float64)], dt, T0)[0]
    assert stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("guess", [0, 1, 2, 3])
@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_transient_schedule(graph, prec, guess):
    st = ti.stack_c2()
    nx, ny, dt = 40, 26, 1e-4
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float32)
            for s in (30, 32)]
    n_steps, spm = 7, 3
    g = grid_of(nx, ny, st)
    T = cuda(np.full(nx * ny * st.L, st.t_amb))
    T, stats = g.run_transient([cuda(m) for m in maps], spm, n_steps, dt, T, precision=prec, tol_rel=1e-10,
                               cheb_degree=6, use_graph=graph, guess=guess)
    sched = [maps[(s // spm) % 2].astype(np.float64) for s in range(n_steps)]
    ref = osolve.transient(nx, ny, st, sched, dt, np.full(nx * ny * st.L, st.t_amb))[-1]
    assert stats["steps"] == n_steps and stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("guess", [2, 3])
@pytest.mark.parametrize("graph", [0, 1])
def test_run_transient_high_order_guess_across_switches(graph, guess):
    """Quadratic and cubic extrapolated guesses on a schedule long enough to reach the
    full order before and after a power-map switch (steps 3-4 and 8-10 run cubic; the
    order drops to 0 at the switch and rebuilds), against the oracle's trajectory."""
    st = ti.stack_c2()
    nx, ny, dt = 44, 26, 1e-4
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float32)
            for s in (40, 42)]
    n_steps, spm = 11, 5
    g = grid_of(nx, ny, st)
    T = cuda(np.full(nx * ny * st.L, st.t_amb))
    T, stats = g.run_transient([cuda(m) for m in maps], spm, n_steps, dt, T, tol_rel=1e-10, cheb_degree=8,
                               use_graph=graph, guess=guess)
    sched = [maps[(s // spm) % 2].astype(np.float64) for s in range(n_steps)]
    ref = osolve.transient(nx, ny, st, sched, dt, np.full(nx * ny * st.L, st.t_amb))[-1]
    assert stats["steps"] == n_steps and stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_run_transient_long_schedule(prec):
    """Many more refinement steps in total than max_outer: the limit applies per step."""
    st = ti.stack_c2()
    nx, ny, dt = 24, 17, 1e-4
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float32)
            for s in (40, 42, 44)]
    n_steps, spm = 40, 5
    g = grid_of(nx, ny, st)
    T = cuda(np.full(nx * ny * st.L, st.t_amb))
    T, stats = g.run_transient([cuda(m) for m in maps], spm, n_steps, dt, T, precision=prec, tol_rel=1e-10,
                               cheb_degree=4, use_graph=1, max_outer=5)
    assert stats["steps"] == n_steps and stats["status"] == 0
    assert stats["outer_it"] > 5
    sched = [maps[(s // spm) % 3].astype(np.float64) for s in range(n_steps)]
    ref = osolve.transient(nx, ny, st, sched, dt, np.full(nx * ny * st.L, st.t_amb))[-1]
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


# ----------------------------------------------------- geometric multigrid (not in the paper)

@pytest.mark.parametrize("nx,ny,mk,dt", [(37, 21, "c2", 1e-4), (37, 21, "c2", 0.0), (9, 30, "mol", 0.0),
                                         (3, 2, "c1", 0.0), (64, 64, "c1", 1e-4), (36, 30, "mol", 0.0),
                                         (68, 22, "mol", 1e-4), (128, 64, "c2", 0.0), (64, 32, "mol", 1e-4),
                                         (72, 40, "c2", 0.0)])
def test_mg_vcycle_matches_oracle(nx, ny, mk, dt):
    """One V-cycle (aggregation semi-coarsening, damped z-line Jacobi, exact coarsest
    solve) in FP32 on the GPU against the oracle's FP64 V-cycle, on odd sizes, a
    single-level grid, grids whose levels are layer-uniform down to the coarsest
    (coefficient tables, 4-column kernels on every level with nx % 4 == 0) and one
    that turns to per-cell arrays part-way (72 -> 36 -> 18 columns)."""
    from oracle import multigrid as mg
    st = STACKS[mk]()
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None).tocsr()
    g = grid_of(nx, ny, st)
    r = ti.random_vector(A.shape[0], 17).astype(np.float32)
    z = g.precond(cuda(r), dt, precond="mg").cpu().double().numpy()
    z_ref = mg.vcycle(mg.hierarchy(A, nx, ny, st.L), st.L, r.astype(np.float64))
    assert np.max(np.abs(z - z_ref)) <= 2e-5 * np.max(np.abs(z_ref))


def test_mg_vcycle_conductivity_map_matches_oracle():
    """The finest level reads per-face arrays when the grid has a per-cell map."""
    from oracle import multigrid as mg
    st = ti.stack_c2()
    nx, ny, dt = 40, 22, 1e-4
    kc = _kmap(st, nx, ny, 21)
    A = disc.assemble(nx, ny, st, dt=dt, k_cell=kc).tocsr()
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(cuda(kc))
    r = ti.random_vector(A.shape[0], 18).astype(np.float32)
    z = g.precond(cuda(r), dt, precond="mg").cpu().double().numpy()
    z_ref = mg.vcycle(mg.hierarchy(A, nx, ny, st.L), st.L, r.astype(np.float64))
    assert np.max(np.abs(z - z_ref)) <= 2e-5 * np.max(np.abs(z_ref))


@pytest.mark.parametrize("graph", [0, 1])
def test_mg_steady_solve(graph):
    st = ti.stack_c2()
    nx, ny = 70, 45
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (14, 15)], np.float64)
    g = grid_of(nx, ny, st)
    T, stats = g.solve_steady(cuda(P), precond="mg", tol_rel=1e-10, use_graph=graph)
    _, sj = g.solve_steady(cuda(P), precond="jacobi", tol_rel=1e-10, use_graph=graph)
    ref = osolve.steady(nx, ny, st, P)
    assert stats["status"] == 0 and stats["rel_res"] <= 1e-10
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6
    assert stats["inner_it"] * 5 < sj["inner_it"], (stats["inner_it"], sj["inner_it"])


def test_mg_transient_schedule_and_invalid_precision():
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c2()
    nx, ny, dt = 40, 26, 1e-4
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float32)
            for s in (60, 62)]
    g = grid_of(nx, ny, st)
    T = cuda(np.full(nx * ny * st.L, st.t_amb))
    T, stats = g.run_transient([cuda(m) for m in maps], 2, 5, dt, T, precond="mg", tol_rel=1e-10)
    sched = [maps[(s // 2) % 2].astype(np.float64) for s in range(5)]
    ref = osolve.transient(nx, ny, st, sched, dt, np.full(nx * ny * st.L, st.t_amb))[-1]
    assert stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6
    with pytest.raises(ThermalError) as e:
        g.solve_steady(cuda(maps[0]), precision="fp64", precond="mg")
    assert e.value.status == 1


# ------------------------------------- Sec. 4.4: the paper's adaptive mixed precision

@pytest.mark.parametrize("nx,ny,mk,dt", [(37, 21, "c2", 1e-4), (36, 17, "mol", 0.0), (5, 3, "c1", 0.0)])
def test_a3_product_matches_oracle(nx, ny, mk, dt):
    """Algorithm 3 (FP16 A3, in-plane FP16 products, out-of-plane FP32) on the GPU
    equals the oracle's step-by-step emulation; the two can differ only where the FP64
    diagonal sums round to FP16 on opposite sides of a tie."""
    from oracle import precision as prc
    st = STACKS[mk]()
    A = disc.assemble(nx, ny, st, dt=dt if dt > 0 else None).tocsr()
    g = grid_of(nx, ny, st)
    x = cuda(ti.random_vector(A.shape[0], 41, lo=-3.0, hi=5.0).astype(np.float32))
    y = g.apply(x, dt, "adaptive").cpu().double().numpy()
    D = prc.quad_diag(A, nx, ny)
    xh = x.cpu().numpy()
    y_ref = prc.a3_spmv(*D, xh, nx, ny, prc.a3_scale_exponent(D[0])).astype(np.float64)
    err = np.abs(y - y_ref)
    assert np.mean(err == 0.0) >= 0.99
    assert np.all(err <= 2.0 ** -10 * (abs(A) @ np.abs(xh.astype(np.float64))))


@pytest.mark.parametrize("pc,scaled", [("cheb", 1), ("cheb", 0), ("jacobi", 1), ("none", 1)])
@pytest.mark.parametrize("graph", [0, 1])
def test_adaptive_steady_matches_oracle(pc, scaled, graph):
    """FP64 PCG with the early FP64/32 SpMV, the FP32/16 Chebyshev preconditioner,
    the stage switch and the hot restart reaches the exact solution."""
    st = ti.stack_c2()
    nx, ny = 30, 22
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (12, 13)], np.float64)
    g = grid_of(nx, ny, st)
    T, stats = g.solve_steady(cuda(P), precision="adaptive", precond=pc, cheb_degree=10, cheb_scaled=scaled,
                              tol_rel=1e-10, use_graph=graph)
    ref = osolve.steady(nx, ny, st, P)
    assert stats["status"] == 0 and stats["rel_res"] <= 1e-10
    assert stats["stage_switches"] == 1
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("graph", [0, 1])
def test_adaptive_run_transient(graph):
    st = ti.stack_c2()
    nx, ny, dt = 36, 26, 1e-4
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float32)
            for s in (50, 52)]
    n_steps, spm = 6, 2
    g = grid_of(nx, ny, st)
    T = cuda(np.full(nx * ny * st.L, st.t_amb))
    T, stats = g.run_transient([cuda(m) for m in maps], spm, n_steps, dt, T, precision="adaptive", tol_rel=1e-10,
                               cheb_degree=6, use_graph=graph)
    sched = [maps[(s // spm) % 2].astype(np.float64) for s in range(n_steps)]
    ref = osolve.transient(nx, ny, st, sched, dt, np.full(nx * ny * st.L, st.t_amb))[-1]
    assert stats["steps"] == n_steps and stats["status"] == 0
    assert 1 <= stats["stage_switches"] <= n_steps
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


def test_adaptive_rejects_zline():
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c1()
    g = grid_of(8, 8, st)
    with pytest.raises(ThermalError) as e:
        g.solve_steady(cuda(np.ones(8 * 8 * st.L)), precision="adaptive", precond="zline")
    assert e.value.status == 1


# ----------------------------------------------------------------- A10: adjoint

def test_lse_and_adjoint_gradient():
    st = ti.stack_c1()
    nx, ny = 34, 30
    P = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 9)], np.float64)
    mask = oadj.silicon_mask(nx, ny, st, st.power_layers())
    g = grid_of(nx, ny, st)
    T, _ = g.solve_steady(cuda(P), tol_rel=1e-10, precision="fp64")
    J, w = g.hotspot_lse(T, st.power_layers(), 2.0)
    J_ref, dJdP_ref, dJdk_ref, _, _ = oadj.gradient(nx, ny, st, P, mask, 2.0)
    assert abs(J - J_ref) <= 1e-9 * abs(J_ref)
    dJdP, dJdk, _ = g.grad(T, w, dJdP_dtype=torch.float64, tol_rel=1e-10, precision="mixed")
    np.testing.assert_allclose(dJdP.cpu().numpy(), dJdP_ref, rtol=1e-6, atol=1e-6 * np.abs(dJdP_ref).max())
    np.testing.assert_allclose(dJdk, dJdk_ref, rtol=1e-6, atol=1e-9 * np.abs(dJdk_ref).max())


def test_autograd_function():
    from paper_2606_17850_gb300 import HotspotLSE, SteadyAdjoint
    st = ti.stack_c1()
    nx, ny = 20, 18
    P = ti.power_cells(st, nx, ny, [ti.density_uniform_hotspots(nx, ny, 4)], np.float32)
    g = grid_of(nx, ny, st)
    Pt = cuda(P).requires_grad_(True)
    kt = torch.tensor(st.k(), dtype=torch.float64, requires_grad=True)
    opts = dict(tol_rel=1e-10, precision="mixed")
    T = SteadyAdjoint.apply(g, Pt, kt, opts)
    J = HotspotLSE.apply(g, T, st.power_layers(), 2.0)
    J.backward()
    mask = oadj.silicon_mask(nx, ny, st, st.power_layers())
    _, dJdP_ref, dJdk_ref, _, _ = oadj.gradient(nx, ny, st, P.astype(np.float64), mask, 2.0)
    np.testing.assert_allclose(Pt.grad.cpu().double().numpy(), dJdP_ref, rtol=1e-5, atol=1e-6 * np.abs(dJdP_ref).max())
    np.testing.assert_allclose(kt.grad.numpy(), dJdk_ref, rtol=1e-5)


# ----------------------------------------------------------------- A9: batched

@pytest.mark.parametrize("mode,pc", [(0, "cheb"), (0, "jacobi"), (0, "none"), (1, "cheb")])
def test_batched_matches_oracle(mode, pc):
    """Uneven instances (the 64-stack recipe at 1/16 size) in one persistent launch
    (mode 0) or one after another (mode 1); every instance against the oracle."""
    from paper_2606_17850_gb300 import solve_batched
    insts = ti.c4_instances(n=9, scale=16)
    grids = [grid_of(i.nx, i.ny, i.stack) for i in insts]
    powers = [cuda(i.power) for i in insts]
    Ts = [torch.empty(i.n, dtype=torch.float64, device="cuda") for i in insts]
    stats = solve_batched(grids, powers, Ts, tol_rel=1e-10, precond=pc, cheb_degree=8, batched_mode=mode)
    assert len({(i.nx, i.stack.L) for i in insts}) > 1
    for inst, T, s in zip(insts, Ts, stats):
        ref = osolve.steady(inst.nx, inst.ny, inst.stack, inst.power.astype(np.float64))
        assert s["status"] == 0 and s["rel_res"] <= 1e-10
        assert osolve.rise_relative_error(T.cpu().numpy(), ref, inst.stack.t_amb) <= 1e-6


def test_batched_multigrid_matches_oracle():
    """The multigrid V-cycle inside the persistent batched kernel: uneven instances
    (the 64-stack recipe at 1/8 size: 16^2 x 4 to 64^2 x 8, hierarchies of 3 to 5
    levels in the same phases), one of them with a per-cell conductivity map; every
    instance against the oracle, and the same answers as the instances solved one
    after another through the single-grid multigrid path."""
    from paper_2606_17850_gb300 import solve_batched
    insts = ti.c4_instances(n=9, scale=8)
    grids = [grid_of(i.nx, i.ny, i.stack) for i in insts]
    kmap = _kmap(insts[0].stack, insts[0].nx, insts[0].ny, 31)
    grids[0].set_conductivity_map(cuda(kmap))
    powers = [cuda(i.power) for i in insts]
    Ts = [torch.empty(i.n, dtype=torch.float64, device="cuda") for i in insts]
    stats = solve_batched(grids, powers, Ts, tol_rel=1e-10, precond="mg")
    assert len({(i.nx, i.stack.L) for i in insts}) > 2
    for j, (inst, T, s) in enumerate(zip(insts, Ts, stats)):
        ref = osolve.steady(inst.nx, inst.ny, inst.stack, inst.power.astype(np.float64),
                            k_cell=kmap if j == 0 else None)
        assert s["status"] == 0 and s["rel_res"] <= 1e-10, (j, s)
        assert osolve.rise_relative_error(T.cpu().numpy(), ref, inst.stack.t_amb) <= 1e-6, j
    Ts2 = [torch.empty(i.n, dtype=torch.float64, device="cuda") for i in insts]
    solve_batched(grids, powers, Ts2, tol_rel=1e-10, precond="mg", batched_mode=1)
    for T, T2, inst in zip(Ts, Ts2, insts):
        assert (T - T2).abs().max().item() <= 1e-7 * (T2 - inst.stack.t_amb).abs().max().item()


def test_batched_conductivity_map_and_ragged_tiles():
    """One persistent launch over instances with a per-cell conductivity map (per-face
    kernels), ragged 128 x 8 tiles (nx = 132, ny = 13) and the layer-table kernels;
    an instance with nx % 4 != 0 sends the whole batch through the sequential path."""
    from paper_2606_17850_gb300 import solve_batched
    shapes = [(132, 13, ti.stack_c2()), (20, 36, ti.stack_c1()), (44, 9, ti.stack_mol())]
    for extra in ([], [(21, 10, ti.stack_c1())]):
        cases = shapes + extra
        grids, powers, Ts, refs = [], [], [], []
        for j, (nx, ny, st) in enumerate(cases):
            P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, 60 + j)] * len(st.power_layers()),
                               np.float64)
            g = grid_of(nx, ny, st)
            kc = None
            if j == 0:
                kc = _kmap(st, nx, ny, 11)
                g.set_conductivity_map(cuda(kc))
            grids.append(g)
            powers.append(cuda(P.astype(np.float32)))
            Ts.append(torch.empty(nx * ny * st.L, dtype=torch.float64, device="cuda"))
            refs.append(osolve.steady(nx, ny, st, P.astype(np.float32).astype(np.float64), k_cell=kc))
        stats = solve_batched(grids, powers, Ts, tol_rel=1e-10, precond="cheb", cheb_degree=8)
        for (nx, ny, st), T, s, ref in zip(cases, Ts, stats, refs):
            assert s["status"] == 0 and s["rel_res"] <= 1e-10
            assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


def test_batched_initial_guess_and_repeat():
    from paper_2606_17850_gb300 import solve_batched
    insts = ti.c4_instances(n=4, scale=8)
    grids = [grid_of(i.nx, i.ny, i.stack) for i in insts]
    powers = [cuda(i.power) for i in insts]
    Ts = [torch.full((i.n,), 70.0, dtype=torch.float64, device="cuda") for i in insts]
    solve_batched(grids, powers, Ts, tol_rel=1e-10, use_guess=1)
    first = [T.clone() for T in Ts]
    stats = solve_batched(grids, powers, Ts, tol_rel=1e-10, use_guess=1)   # restart from the solution
    for a, b, s in zip(first, Ts, stats):
        assert s["status"] == 0 and s["outer_it"] <= 1
        assert (a - b).abs().max().item() <= 1e-8 * (a - 45.0).abs().max().item()


def test_batched_rejects_a_repeated_grid_or_output():
    """Through the C ABI directly (the binding rejects this before the call): one grid
    handle twice, or one output buffer twice, is TH_EINVAL and nothing is solved;
    separate grids on one shared power map solve normally."""
    import ctypes as C
    from paper_2606_17850_gb300 import _lib, solve_batched
    lib = _lib.load()
    inst = ti.c4_instances(n=1, scale=8)[0]
    g1, g2 = grid_of(inst.nx, inst.ny, inst.stack), grid_of(inst.nx, inst.ny, inst.stack)
    P = cuda(inst.power)
    T1 = torch.full((inst.n,), -1.0, dtype=torch.float64, device="cuda")
    T2 = T1.clone()
    o = _lib.default_opts(tol_rel=1e-10)
    stats = (_lib.SolveStats * 2)()
    pdt = _lib.TH_F32 if P.dtype == torch.float32 else _lib.TH_F64

    def call(grids, outs):
        gh = (C.c_void_p * 2)(*[g.handle.value for g in grids])
        ph = (C.c_void_p * 2)(P.data_ptr(), P.data_ptr())
        th = (C.c_void_p * 2)(*[t.data_ptr() for t in outs])
        return lib.thermal_solve_batched(gh, 2, ph, pdt, th, C.byref(o), stats, None)

    assert call([g1, g1], [T1, T2]) == _lib.TH_EINVAL
    assert b"same grid" in lib.thermal_last_error()
    assert call([g1, g2], [T1, T1]) == _lib.TH_EINVAL
    torch.cuda.synchronize()
    assert (T1 == -1.0).all() and (T2 == -1.0).all()
    st = solve_batched([g1, g2], [P, P], [T1, T2], tol_rel=1e-10)
    T_ref = osolve.steady(inst.nx, inst.ny, inst.stack, inst.power.astype(np.float64))
    for T, s in zip((T1, T2), st):
        assert s["status"] == 0
        assert osolve.rise_relative_error(T.cpu().numpy(), T_ref, inst.stack.t_amb) <= 1e-6


# ----------------------------------------------------------------- errors

def test_nonfinite_power_reported():
    from paper_2606_17850_gb300 import ThermalError
    inst = ti.c1(nx=16, ny=16)
    g = grid_of(16, 16, inst.stack)
    P = inst.power.copy()
    P[5] = np.nan
    with pytest.raises(ThermalError) as e:
        g.solve_steady(cuda(P))
    assert e.value.status == 6
    T, st = g.solve_steady(cuda(inst.power))   # the grid stays usable
    assert st["status"] == 0


def test_invalid_options_rejected():
    from paper_2606_17850_gb300 import ThermalError
    inst = ti.c1(nx=8, ny=8)
    g = grid_of(8, 8, inst.stack)
    with pytest.raises(ThermalError):
        g.solve_steady(cuda(inst.power), inner_tol=2.0)
    with pytest.raises(ThermalError):
        g.solve_steady(cuda(inst.power), cheb_degree=0)


# ----------------------------------------------------------------- degenerate inputs

def _one_layer(h=1e4):
    return ti.Stack((ti.Layer("si", 100e-6, 150.0, 1.63e6, True),), h=h)


@pytest.mark.parametrize("nx,ny", [(36, 21), (37, 21), (1, 1), (4, 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_layer_steady_and_transient(nx, ny, prec):
    """L = 1: no vertical faces, the top layer is also the bottom one."""
    st = _one_layer()
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, 3)], np.float64)
    g = grid_of(nx, ny, st)
    T, stats = g.solve_steady(cuda(P), precision=prec, tol_rel=1e-10, cheb_degree=8)
    assert stats["status"] == 0
    ref = osolve.steady(nx, ny, st, P)
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6
    dt = 1e-4
    T0 = np.full(nx * ny, st.t_amb)
    T = cuda(T0.copy())
    T, stats = g.run_transient([cuda(P)], 1, 5, dt, T, precision=prec, tol_rel=1e-10, cheb_degree=8, guess=2)
    ref = osolve.transient(nx, ny, st, [P] * 5, dt, T0)[-1]
    assert stats["status"] == 0 and stats["steps"] == 5
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


def test_single_layer_fused_chebyshev():
    st = _one_layer()
    nx, ny, dt = 64, 40, 1e-4
    g = grid_of(nx, ny, st)
    r = cuda(ti.random_vector(nx * ny, 9), torch.float32)
    z1 = g.precond(r, dt, precond="cheb", cheb_degree=12, cheb_fuse=1)
    scale = z1.abs().max().item()
    for fuse in (0, 2, 3, 4):
        zf = g.precond(r, dt, precond="cheb", cheb_degree=12, cheb_fuse=fuse)
        assert (zf - z1).abs().max().item() <= 1e-6 * scale, fuse


def test_adiabatic_grid():
    """h = 0: G 1 = 0, so the steady system is singular and rejected; transient steps
    are well posed and conserve energy, sum_i C_i V_i (T_{n+1} - T_n)_i = dt sum_i p_i."""
    from paper_2606_17850_gb300 import ThermalError
    st = ti.stack_c1(h=0.0)
    nx, ny, dt = 40, 23, 1e-4
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, 7)], np.float64)
    g = grid_of(nx, ny, st)
    with pytest.raises(ThermalError) as e:
        g.solve_steady(cuda(P))
    assert e.value.status == 1
    T0 = np.full(nx * ny * st.L, st.t_amb)
    for prec in ("fp64", "mixed"):
        T = cuda(T0.copy())
        T, stats = g.run_transient([cuda(P)], 1, 6, dt, T, precision=prec, tol_rel=1e-11, cheb_degree=8)
        assert stats["status"] == 0
        ref = osolve.transient(nx, ny, st, [P] * 6, dt, T0)[-1]
        Th = T.cpu().numpy()
        assert osolve.rise_relative_error(Th, ref, st.t_amb) <= 1e-6
        c = disc.capacity_over_dt(nx, ny, st, dt) * dt
        assert abs(c @ (Th - T0) - 6 * dt * P.sum()) <= 1e-7 * 6 * dt * P.sum()
    from paper_2606_17850_gb300 import solve_batched
    with pytest.raises(ThermalError):
        solve_batched([g], [cuda(P)], [cuda(T0.copy())])


def test_empty_runs():
    from paper_2606_17850_gb300 import solve_batched
    inst = ti.c1(nx=8, ny=8)
    g = grid_of(8, 8, inst.stack)
    T0 = cuda(np.full(inst.n, inst.stack.t_amb + 1.0))
    T = T0.clone()
    g.run_transient([cuda(inst.power)], 1, 0, 1e-4, T)
    assert torch.equal(T, T0)
    assert solve_batched([], [], []) == []


@pytest.mark.parametrize("guess", [1, 2, 3])
@pytest.mark.parametrize("graph", [0, 1])
def test_run_transient_conductivity_map(guess, graph):
    """Per-cell conductivities (per-face kernels, no layer table) with the
    extrapolated guess, against backward-Euler steps assembled by the oracle."""
    st = ti.stack_c2()
    nx, ny, dt = 36, 21, 1e-4
    kc = _kmap(st, nx, ny, 12)
    maps = [ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s + j) for j in (0, 1)], np.float64)
            for s in (70, 72)]
    n_steps, spm = 6, 2
    g = grid_of(nx, ny, st)
    g.set_conductivity_map(cuda(kc))
    T0 = np.full(nx * ny * st.L, st.t_amb)
    T = cuda(T0.copy())
    T, stats = g.run_transient([cuda(m) for m in maps], spm, n_steps, dt, T, tol_rel=1e-10, cheb_degree=8,
                               use_graph=graph, guess=guess)
    assert stats["status"] == 0 and stats["steps"] == n_steps
    A = disc.assemble(nx, ny, st, dt=dt, k_cell=kc)
    solve = osolve.Factorised(A)
    ref = T0
    for s in range(n_steps):
        ref = solve(disc.rhs_transient(nx, ny, st, maps[(s // spm) % 2], ref, dt))
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6


@pytest.mark.parametrize("scaled,fuse,k", [(1, 1, 8), (0, 0, 8), (1, 4, 8), (1, 0, 1), (1, 0, 2)])
def test_mixed_solve_chebyshev_variants(scaled, fuse, k):
    """The residual kernel starts each inner solve itself on layer-table grids: with
    the stepwise polynomial (fuse 1), the unscaled one, fused chunks (z_1 formed in
    the first chunk), degree 1 (the start supplies r^T z) and degree 2 (one fused
    chunk that is first and last at once), steady and transient, against the oracle."""
    st = ti.stack_c2()
    nx, ny, dt = 40, 26, 1e-4
    P = ti.power_cells(st, nx, ny, [ti.density_floorplan(nx, ny, s) for s in (80, 81)], np.float64)
    g = grid_of(nx, ny, st)
    o = dict(precision="mixed", precond="cheb", cheb_degree=k, cheb_scaled=scaled, cheb_fuse=fuse, tol_rel=1e-10)
    T, stats = g.solve_steady(cuda(P), **o)
    assert stats["status"] == 0
    assert osolve.rise_relative_error(T.cpu().numpy(), osolve.steady(nx, ny, st, P), st.t_amb) <= 1e-6
    T0 = np.full(nx * ny * st.L, st.t_amb)
    T = cuda(T0.copy())
    T, stats = g.run_transient([cuda(P)], 1, 4, dt, T, guess=2, **o)
    assert stats["status"] == 0
    ref = osolve.transient(nx, ny, st, [P] * 4, dt, T0)[-1]
    assert osolve.rise_relative_error(T.cpu().numpy(), ref, st.t_amb) <= 1e-6
