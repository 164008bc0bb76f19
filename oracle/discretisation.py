"""7-point finite-volume discretisation of the layered stack (oracle).

Follows Sec. 3.2 of the paper:

* Eq. (steady-state): for cell 0,
  sum_i g_{0,i} (T_0 - T_i) + h S_0 T_0 = p_0 V_0 + h S_0 T_amb.
* Eq. (transient), backward Euler:
  C_0 V_0 T_{0,n+1}/dt + sum_i g_{0,i}(T_{0,n+1} - T_{i,n+1}) + h S_0 T_{0,n+1}
  = p_{0,n+1} V_0 + h S_0 T_amb + C_0 V_0 T_{0,n}/dt.

The paper leaves g_{0,i} undefined.  The reading used here: the conductance of a
face is the series combination of the two half cells it joins,
g = S / (l_a / (2 k_a) + l_b / (2 k_b)), where S is the face area and l the cell
extent normal to the face.  Within one layer this is k S / l.  Faces on the
domain's sides and bottom are adiabatic (Eq. Neumann, q = 0: no term), and the
top face of the top layer is convective (Eq. Robin): h S_0 acts on the cell-centre
temperature as written in Eq. (steady-state).  With ``half_cell_top=True`` the
convective conductance is instead 1 / (1/(h S) + dz/(2 k S)).

Cell index i = x + nx*(y + ny*z), x fastest, z = 0 bottom layer.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def layer_constants(stack):
    """Per-layer arrays (k, c, dz) and the footprint of a cell."""
    return stack.k(), stack.c(), stack.dz(), stack.dx, stack.dy


def face_conductance(area, la, ka, lb, kb):
    """Series conductance of two half cells of extents la, lb and conductivities ka, kb."""
    return area / (la / (2.0 * ka) + lb / (2.0 * kb))


def convective_conductance(stack, half_cell_top=False):
    h, dx, dy = stack.h, stack.dx, stack.dy
    S = dx * dy
    if not half_cell_top:
        return h * S
    top = stack.layers[-1]
    return 1.0 / (1.0 / (h * S) + top.thickness / (2.0 * top.k * S))


def assemble(nx, ny, stack, dt=None, half_cell_top=False, k_cell=None):
    """Assemble the system matrix A of Eq. (steady-state) (dt=None) or Eq. (transient).

    Row by row: for every cell, each of its (up to) six neighbours j contributes
    +g to A[i,i] and -g to A[i,j]; a top-layer cell adds h S; with a time step the
    cell adds C V / dt.  ``k_cell`` (optional, N values) gives every cell its own
    conductivity; a face then joins two half cells of different k.  Returns CSR, FP64.
    """
    k, c, dz, dx, dy = layer_constants(stack)
    L = stack.L
    n = nx * ny * L
    idx = np.arange(n).reshape(L, ny, nx)
    zz, yy, xx = np.meshgrid(np.arange(L), np.arange(ny), np.arange(nx), indexing="ij")
    if k_cell is not None:
        return _assemble_kmap(nx, ny, stack, dt, half_cell_top, np.asarray(k_cell, dtype=np.float64).reshape(L, ny, nx))

    rows, cols, vals = [], [], []
    diag = np.zeros(n)

    def couple(mask, shift_idx, g):
        i = idx[mask]
        j = shift_idx[mask]
        gv = np.broadcast_to(g, idx.shape)[mask]
        rows.append(i)
        cols.append(j)
        vals.append(-gv)
        np.add.at(diag, i, gv)

    kz = k[zz]
    dzz = dz[zz]
    # neighbour x+1 and x-1 (same layer): faces of area dy*dz, extents dx
    gx = face_conductance(dy * dzz, dx, kz, dx, kz)
    couple(xx < nx - 1, np.roll(idx, -1, axis=2), gx)
    couple(xx > 0, np.roll(idx, 1, axis=2), gx)
    # neighbour y+1 and y-1: faces of area dx*dz, extents dy
    gy = face_conductance(dx * dzz, dy, kz, dy, kz)
    couple(yy < ny - 1, np.roll(idx, -1, axis=1), gy)
    couple(yy > 0, np.roll(idx, 1, axis=1), gy)
    # neighbour z+1 (layer above) and z-1 (layer below): faces of area dx*dy
    zup = np.minimum(zz + 1, L - 1)
    zdn = np.maximum(zz - 1, 0)
    g_up = face_conductance(dx * dy, dzz, kz, dz[zup], k[zup])
    g_dn = face_conductance(dx * dy, dzz, kz, dz[zdn], k[zdn])
    couple(zz < L - 1, np.roll(idx, -1, axis=0), g_up)
    couple(zz > 0, np.roll(idx, 1, axis=0), g_dn)

    # convective top face (Eq. Robin) on the top layer
    top = idx[L - 1].reshape(-1)
    diag[top] += convective_conductance(stack, half_cell_top)
    # heat capacity term of Eq. (transient)
    if dt is not None:
        diag += (c[zz] * dx * dy * dzz / dt).reshape(-1)

    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def _assemble_kmap(nx, ny, stack, dt, half_cell_top, kc):
    """Row-wise assembly with a per-cell conductivity: each face is the series
    combination of its two half cells, g = S / (l/(2 k_a) + l/(2 k_b))."""
    k, c, dz, dx, dy = layer_constants(stack)
    L = stack.L
    n = nx * ny * L
    idx = np.arange(n).reshape(L, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    dzc = np.broadcast_to(dz[:, None, None], (L, ny, nx))

    def couple(i, j, g):
        rows.append(i.ravel()); cols.append(j.ravel()); vals.append(-g.ravel())
        np.add.at(diag, i.ravel(), g.ravel())

    # x faces between (.., x) and (.., x+1), both directions
    g = face_conductance(dy * dzc[:, :, :-1], dx, kc[:, :, :-1], dx, kc[:, :, 1:])
    couple(idx[:, :, :-1], idx[:, :, 1:], g)
    couple(idx[:, :, 1:], idx[:, :, :-1], g)
    g = face_conductance(dx * dzc[:, :-1, :], dy, kc[:, :-1, :], dy, kc[:, 1:, :])
    couple(idx[:, :-1, :], idx[:, 1:, :], g)
    couple(idx[:, 1:, :], idx[:, :-1, :], g)
    g = face_conductance(dx * dy, dzc[:-1], kc[:-1], dzc[1:], kc[1:])
    couple(idx[:-1], idx[1:], g)
    couple(idx[1:], idx[:-1], g)
    if half_cell_top:
        raise NotImplementedError("half-cell convective term with a conductivity map")
    top = idx[L - 1].reshape(-1)
    diag[top] += convective_conductance(stack)
    if dt is not None:
        diag += np.repeat(c * dx * dy * dz / dt, nx * ny)
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def capacity_over_dt(nx, ny, stack, dt):
    """The diagonal C_0 V_0 / dt of Eq. (transient), per cell."""
    k, c, dz, dx, dy = layer_constants(stack)
    return np.repeat(c * dx * dy * dz / dt, nx * ny)


def top_sink(nx, ny, stack, half_cell_top=False):
    """h S_0 per cell: nonzero on the top layer only (S_0 = 0 elsewhere, Sec. 3.2)."""
    s = np.zeros(nx * ny * stack.L)
    s[(stack.L - 1) * nx * ny:] = convective_conductance(stack, half_cell_top)
    return s


def rhs_steady(nx, ny, stack, power, half_cell_top=False):
    """Right-hand side of Eq. (steady-state): p_0 V_0 + h S_0 T_amb (power in W per cell)."""
    return np.asarray(power, dtype=np.float64) + top_sink(nx, ny, stack, half_cell_top) * stack.t_amb


def rhs_transient(nx, ny, stack, power_next, T_n, dt, half_cell_top=False):
    """Right-hand side of Eq. (transient): p V + h S T_amb + C V T_n / dt."""
    return rhs_steady(nx, ny, stack, power_next, half_cell_top) + \
        capacity_over_dt(nx, ny, stack, dt) * np.asarray(T_n, dtype=np.float64)


def d_matrix_d_layer_k(nx, ny, stack, layer):
    """dA/dk_l, assembled row by row from the analytic derivative of each face conductance.

    In-plane faces of layer l: g = k_l S / l, so dg/dk_l = S / l.
    Vertical face between layers a and b: g = S / (dz_a/(2k_a) + dz_b/(2k_b)), so
    dg/dk_a = g^2 dz_a / (2 k_a^2 S).  The convective face (paper-literal form) and
    the capacity term do not depend on k.
    """
    k, c, dz, dx, dy = layer_constants(stack)
    L = stack.L
    # d(stack with k_l -> k_l + t)/dt at t = 0 equals sum of rank-one face derivatives;
    # assemble it by reusing the assembly with conductance derivatives in place of g.
    n = nx * ny * L
    idx = np.arange(n).reshape(L, ny, nx)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)

    def couple(i, j, dg):
        rows.append(i)
        cols.append(j)
        vals.append(-dg)
        np.add.at(diag, i, dg)

    zl = idx[layer]
    # x faces inside layer l
    dgx = dy * dz[layer] / dx
    a, b = zl[:, :-1].reshape(-1), zl[:, 1:].reshape(-1)
    couple(a, b, np.full(a.size, dgx))
    couple(b, a, np.full(a.size, dgx))
    dgy = dx * dz[layer] / dy
    a, b = zl[:-1, :].reshape(-1), zl[1:, :].reshape(-1)
    couple(a, b, np.full(a.size, dgy))
    couple(b, a, np.full(a.size, dgy))
    S = dx * dy
    for other in (layer - 1, layer + 1):
        if 0 <= other < L:
            g = face_conductance(S, dz[layer], k[layer], dz[other], k[other])
            dg = g * g * dz[layer] / (2.0 * k[layer] ** 2 * S)
            a, b = zl.reshape(-1), idx[other].reshape(-1)
            couple(a, b, np.full(a.size, dg))
            couple(b, a, np.full(a.size, dg))
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    M.sum_duplicates()
    return M
