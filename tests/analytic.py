"""Closed-form solutions used to pin the oracle (test helper, no method code).

2D homogeneous medium, m = 1/c^2 constant:  m u_tt - Lap u = delta(x) w(t).
With the causal Green's function of the 2D wave equation,

    u(r, t) = (c / 2 pi) int_{r/c}^{t} w(t - tau) / sqrt(c^2 tau^2 - r^2) dtau ,

and the substitution tau = (r/c) cosh(xi) this becomes the smooth integral

    u(r, t) = (1 / 2 pi) int_0^{acosh(c t / r)} w(t - (r/c) cosh xi) dxi .
"""
from __future__ import annotations

import numpy as np


def ricker_fn(f0, t0, deriv=0):
    """Ricker wavelet (and its 2nd derivative) as a function of time, zero for t<0."""
    a2 = (np.pi * f0) ** 2

    def w(t):
        t = np.asarray(t, dtype=np.float64)
        s = t - t0
        e = np.exp(-a2 * s * s)
        if deriv == 0:
            v = (1.0 - 2.0 * a2 * s * s) * e
        elif deriv == 2:
            # d^2/ds^2 of (1 - 2 a s^2) e^{-a s^2} = (-6 a + 24 a^2 s^2 - 8 a^3 s^4) e^{-a s^2}
            v = (-6.0 * a2 + 24.0 * a2 * a2 * s * s - 8.0 * a2 ** 3 * s ** 4) * e
        else:
            raise ValueError(deriv)
        return np.where(t >= 0.0, v, 0.0)

    return w


def green2d_trace(w, r, c, times, nxi=6001):
    """u(r, t) for the 2D point source with signature function w (vectorised)."""
    times = np.asarray(times, dtype=np.float64)
    out = np.zeros_like(times)
    for k, t in enumerate(times):
        if c * t <= r:
            continue
        xmax = np.arccosh(c * t / r)
        xi = np.linspace(0.0, xmax, nxi)
        f = w(t - (r / c) * np.cosh(xi))
        # Simpson's rule (nxi odd)
        hx = xi[1] - xi[0]
        out[k] = hx / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())
    return out / (2.0 * np.pi)


def sampled_fn(times, values):
    """Linear interpolant of a finely sampled causal signal (zero before times[0])."""
    times = np.asarray(times, float)
    values = np.asarray(values, float)

    def g(t):
        t = np.asarray(t, dtype=np.float64)
        return np.interp(t, times, values, left=0.0, right=values[-1])

    return g
