"""Finite-difference building blocks of the oracle (FP64, test infrastructure only).

The paper solves m u_tt - Lap u = f (Sec. 1.1, Sec. 2) with spectral differences
and a PML; the discretisation adopted here is 2nd order in time, 8th order in
space, with a quadratic absorbing sponge added around the stated (interior)
grid.  These readings are listed with the design notes of the repository.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def second_derivative_weights(radius: int = 4) -> list:
    """Exact weights w_0..w_R of the symmetric central stencil for h^2 f''.

    Solves the Taylor moment conditions
        w_0 + 2 sum_k w_k = 0,  sum_k w_k k^2 = 1,  sum_k w_k k^(2j) = 0 (j=2..R)
    in rational arithmetic.  For R = 4 this gives the 8th-order stencil.
    """
    R = radius
    rows = []
    rhs = []
    for j in range(0, 2 * R + 1, 2):
        if j == 0:
            rows.append([Fraction(1)] + [Fraction(2)] * R)
            rhs.append(Fraction(0))
        else:
            rows.append([Fraction(0)] + [Fraction(k) ** j for k in range(1, R + 1)])
            rhs.append(Fraction(1) if j == 2 else Fraction(0))
    n = R + 1
    A = [r[:] + [b] for r, b in zip(rows, rhs)]
    for c in range(n):                                  # Gauss-Jordan, exact
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [A[i][n] for i in range(n)]


_W = [float(w) for w in second_derivative_weights(4)]


def laplacian(u: np.ndarray, h, weights=None) -> np.ndarray:
    """8th-order Laplacian over the trailing ``len(h)`` axes, zero outside the grid.

    ``u`` may carry leading batch axes.  Zero extension makes the operator a
    symmetric matrix on the padded grid.
    """
    w = _W if weights is None else [float(x) for x in weights]
    R = len(w) - 1
    nd = len(h)
    lead = u.ndim - nd
    out = np.zeros_like(u)
    for a in range(nd):
        ax = lead + a
        pw = [(0, 0)] * u.ndim
        pw[ax] = (R, R)
        up = np.pad(u, pw)
        n = u.shape[ax]
        acc = w[0] * u
        for k in range(1, R + 1):
            plus = np.take(up, np.arange(R + k, R + k + n), axis=ax)
            minus = np.take(up, np.arange(R - k, R - k + n), axis=ax)
            acc = acc + w[k] * (plus + minus)
        out = out + acc / (h[a] ** 2)
    return out


def sponge_eta(interior_shape, pad: int, h, cmax: float, R: float = 1e-3) -> np.ndarray:
    """Damping coefficient eta(x) on the padded grid (zero in the interior).

    eta = sum over axes of eta_max_a (rho_a / pad)^2, rho_a = distance in cells
    into the pad along axis a, eta_max_a = 3 cmax ln(1/R) / (2 pad h_a).
    """
    shape = tuple(n + 2 * pad for n in interior_shape)
    eta = np.zeros(shape)
    if pad == 0:
        return eta
    for a, n in enumerate(interior_shape):
        i = np.arange(n + 2 * pad)
        rho = np.maximum(np.maximum(pad - i, i - (pad + n - 1)), 0).astype(np.float64)
        emax = 3.0 * cmax * np.log(1.0 / R) / (2.0 * pad * h[a])
        prof = emax * (rho / pad) ** 2
        sh = [1] * len(shape)
        sh[a] = shape[a]
        eta = eta + prof.reshape(sh)
    return eta
