"""Reduced-precision building blocks of the paper's adaptive mixed-precision PCG (oracle).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` use this module.

* ``quad_diag`` - the Quad-Diag storage of Sec. 4.2: the main diagonal D4 and the
  upper off-diagonals D5 (offset 1), D6 (offset nx) and D7 (offset nx*ny) of the
  symmetric matrix; a row's lower neighbours reuse D5/D6/D7 of the neighbour row.
  Entries for neighbours outside the grid are stored as zeros.
* ``a3_scale_exponent`` - the power of two that maps the diagonals into FP16's
  range (the paper's matrices are stored in FP16 as A3; the conductances here span
  2.5e-5..0.5 W/K, partly below FP16's smallest normal number, so every stored value
  is multiplied by 2^e before rounding and the product by 2^-e after).  Reading:
  e is chosen so that max(D4) * 2^e lies in [16, 32).
* ``a3_spmv`` - Algorithm 3 (Physics-Aware FP32/16 SpMV with Arithmetic Decoupling),
  step by step: x is converted once to FP32 and to FP16; the out-of-plane diagonals
  D4 and D7 are loaded from FP16, promoted to FP32 and multiplied with x in FP32; the
  in-plane diagonals D5 and D6 are multiplied with x in FP16 and each product is
  added to the FP32 result.  Order of the accumulation (the algorithm's loop over
  the diagonals): D4, D5 (x+1, x-1), D6 (y+1, y-1), D7 (z+1, z-1); every FP32 step
  is a separate multiply and add (no fused multiply-add).
* ``stage_switch`` - the early-to-late switching criterion, Eqs. (switch_a-c).

parity pinned by: the exact product on FP16-representable inputs, the FP16 error
bound on the physical matrices, and the Quad-Diag round trip (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np


def quad_diag(A, nx, ny):
    """(D4, D5, D6, D7) of a 7-point CSR matrix in cell order i = x + nx (y + ny z)."""
    A = A.tocsr()
    n = A.shape[0]
    pxy = nx * ny
    i = np.arange(n)
    x = i % nx
    y = (i // nx) % ny
    z = i // pxy
    L = n // pxy

    def upper(off, exists):
        d = np.zeros(n)
        j = i[exists]
        d[exists] = np.asarray(A[j, j + off]).ravel()
        return d

    D4 = A.diagonal().copy()
    D5 = upper(1, x + 1 < nx)
    D6 = upper(nx, y + 1 < ny)
    D7 = upper(pxy, z + 1 < L)
    return D4, D5, D6, D7


def from_quad_diag(D4, D5, D6, D7, nx, ny):
    """Dense symmetric matrix rebuilt from the four stored diagonals."""
    n = D4.size
    M = np.diag(D4).astype(np.float64)
    for off, D in ((1, D5), (nx, D6), (nx * ny, D7)):
        for i in range(n - off):
            if D[i] != 0.0:
                M[i, i + off] = D[i]
                M[i + off, i] = D[i]
    return M


def a3_scale_exponent(D4):
    """e with max(D4) * 2^e in [16, 32)."""
    return 4 - int(math.floor(math.log2(float(np.max(np.abs(D4))))))


def a3_spmv(D4, D5, D6, D7, x, nx, ny, e):
    """Algorithm 3: y (FP32) = A3 x with A3 = 2^e (D4..D7) stored in FP16."""
    n = D4.size
    pxy = nx * ny
    s = 2.0 ** e
    v4, v5, v6, v7 = (np.float16(s * np.asarray(D, dtype=np.float64)) for D in (D4, D5, D6, D7))
    x32 = np.asarray(x).astype(np.float32)       # one-time conversions
    x16 = np.asarray(x).astype(np.float16)
    i = np.arange(n)
    xx = i % nx
    yy = (i // nx) % ny
    zz = i // pxy
    L = n // pxy
    y = np.zeros(n, dtype=np.float32)

    def high(v, xv):        # promoted: FP32 product, then FP32 add
        return (y + (v.astype(np.float32) * xv).astype(np.float32)).astype(np.float32)

    def low(v, xv):         # FP16 product, added back in FP32
        return (y + (v * xv).astype(np.float16).astype(np.float32)).astype(np.float32)

    def shifted(a, off, exists, fill):
        out = np.full(n, fill, dtype=a.dtype)
        j = i[exists]
        out[exists] = a[j + off]
        return out

    y = high(v4, x32)
    # D5: neighbour x+1 (coefficient of row i), x-1 (coefficient of row i-1)
    y = low(v5, shifted(x16, 1, xx + 1 < nx, 0))
    y = low(shifted(v5, -1, xx > 0, 0), shifted(x16, -1, xx > 0, 0))
    y = low(v6, shifted(x16, nx, yy + 1 < ny, 0))
    y = low(shifted(v6, -nx, yy > 0, 0), shifted(x16, -nx, yy > 0, 0))
    y = high(v7, shifted(x32, pxy, zz + 1 < L, 0))
    y = high(shifted(v7, -pxy, zz > 0, 0), shifted(x32, -pxy, zz > 0, 0))
    return (y * np.float32(2.0 ** -e)).astype(np.float32)


def stage_switch(r_low, r_true, r_true_prev, r_diff, eps):
    """Eqs. (switch_a-c): True when the early (low-precision) stage must end.

    r_low = ||r_low||_2 (recursive residual), r_true = ||b - A x||_2, r_true_prev = the
    previous evaluation (None at the first), r_diff = ||r_true - r_low||_2, eps = the
    stopping tolerance on ||r||_2 (switch_a: ||r_low|| <= 10^(log10(eps)/2) = sqrt(eps)).
    """
    a = r_low <= 10.0 ** (math.log10(eps) / 2.0)
    b = r_true_prev is not None and r_true > 0.9 * r_true_prev
    c = r_diff >= 0.5 * r_true
    return bool(a or b or c)
