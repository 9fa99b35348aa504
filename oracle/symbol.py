"""Symbol expansion, randomized fit and preconditioner of the oracle (FP64).

Test infrastructure only.  What is computed:

* elementary operators B_i with symbol  alpha_lam(x) A_q1(theta) TL_q2(|k|) |k|^e
  (Eq. compr2 and the B_i definition of Sec. 1.2; e = -1 for the inverse
  Hessian, the order of Eq. type10_b), applied as
      B_i x = alpha_lam * IFFT[ A_q1 TL_q2 |k|^e * FFT(x) ]
  on the interior grid zero-padded by ``fft_pad`` cells per side;
* the randomized least-squares fit of Sec. 1.4: with x_j = H y_j, find c
  minimising sum_j || y_j - sum_i c_i B_i x_j ||^2 (Householder QR of the
  stacked columns; the closed form c = M^{-1} (Bx)^T y with
  M_ik = (B_i x)^T (B_k x) is also provided);
* the preconditioner apply  sum_i c_i B_i img  (end of Sec. 1.5).

Readings (the paper uses complex exponentials and leaves the discretisation
open):  real spatial modes phi_k(i) = 1 | cos(2 pi k i/n) | sin(2 pi |k| i/n)
per axis (k = 0 | k > 0 | k < 0, period = the interior size); 2D angular
functions 1 | cos(q theta) | sin(|q| theta) with theta = atan2(k_z, k_x);
3D angular functions the real l = 0, 2 harmonics
{1, kx ky, ky kz, kx kz, kx^2 - ky^2, 3 kz^2 - 1} of the unit wave vector;
TL_q(|k|) = T_q((|k| - L)/(|k| + L)) (rational Chebyshev functions); every
term maps the k = 0 coefficient to zero, and also the Nyquist bins of
even-length FFT axes (such a bin is its own negative wave vector, where the
odd angular factors cannot be made even, so no real-to-real operator can use
them).  Term index i = (lam*NA + a)*NQ + q.
"""
from __future__ import annotations

import numpy as np


class Basis:
    def __init__(self, shape, h, spatial, angular, nradial, L, order=-1.0, fft_pad=16):
        self.shape = tuple(int(n) for n in shape)
        self.ndim = len(self.shape)
        self.h = tuple(float(x) for x in np.broadcast_to(np.asarray(h, float), (self.ndim,)))
        self.spatial = [tuple(int(v) for v in s) for s in spatial]
        self.angular = [int(a) for a in angular]
        self.nradial = int(nradial)
        self.L = float(L)
        self.order = float(order)
        self.fft_pad = int(fft_pad)
        self.fshape = tuple(n + 2 * self.fft_pad for n in self.shape)

    @property
    def P(self):
        return len(self.spatial) * len(self.angular) * self.nradial

    def index(self, i):
        """Term i -> (spatial index, angular index, radial index)."""
        NA, NQ = len(self.angular), self.nradial
        return i // (NA * NQ), (i // NQ) % NA, i % NQ

    # -- the three factors ---------------------------------------------------
    def spatial_mode(self, lam):
        out = np.ones(self.shape)
        for ax, k in enumerate(self.spatial[lam]):
            n = self.shape[ax]
            i = np.arange(n, dtype=np.float64)
            if k == 0:
                f = np.ones(n)
            elif k > 0:
                f = np.cos(2.0 * np.pi * k * i / n)
            else:
                f = np.sin(2.0 * np.pi * (-k) * i / n)
            sh = [1] * self.ndim
            sh[ax] = n
            out = out * f.reshape(sh)
        return out

    def _kgrid(self):
        """Wave-vector components [rad/m] on the rfft grid of the padded box."""
        ks = []
        for ax, N in enumerate(self.fshape):
            if ax == self.ndim - 1:
                f = np.fft.rfftfreq(N, d=self.h[ax])
            else:
                f = np.fft.fftfreq(N, d=self.h[ax])
            sh = [1] * self.ndim
            sh[ax] = f.size
            ks.append((2.0 * np.pi * f).reshape(sh))
        return np.broadcast_arrays(*ks)

    def angular_fn(self, a, kvec):
        q = self.angular[a]
        knorm = np.sqrt(sum(k ** 2 for k in kvec))
        safe = np.where(knorm > 0, knorm, 1.0)
        if self.ndim == 2:
            kz, kx = kvec
            theta = np.arctan2(kz, kx)
            if q == 0:
                return np.ones_like(theta)
            return np.cos(q * theta) if q > 0 else np.sin(-q * theta)
        kz, ky, kx = (k / safe for k in kvec)
        table = {0: np.ones_like(kx), 1: kx * ky, 2: ky * kz, 3: kx * kz,
                 4: kx ** 2 - ky ** 2, 5: 3.0 * kz ** 2 - 1.0}
        return table[q]

    def _nyquist_mask(self):
        """True on the Nyquist bins of even-length axes (rfft grid)."""
        m = np.zeros(tuple(N if ax < self.ndim - 1 else N // 2 + 1
                           for ax, N in enumerate(self.fshape)), dtype=bool)
        for ax, N in enumerate(self.fshape):
            if N % 2 == 0:
                idx = [slice(None)] * self.ndim
                idx[ax] = N // 2
                m[tuple(idx)] = True
        return m

    def multiplier(self, a, q):
        """beta(k) = A_a(theta) T_q((|k|-L)/(|k|+L)) |k|^e, zero at k = 0 and on Nyquist bins."""
        kvec = self._kgrid()
        knorm = np.sqrt(sum(k ** 2 for k in kvec))
        pos = (knorm > 0) & ~self._nyquist_mask()
        safe = np.where(knorm > 0, knorm, 1.0)
        t = (safe - self.L) / (safe + self.L)
        cheb = np.cos(q * np.arccos(np.clip(t, -1.0, 1.0)))
        beta = self.angular_fn(a, kvec) * cheb * safe ** self.order
        return np.where(pos, beta, 0.0)

    # -- operators -------------------------------------------------------------
    def _pad(self, x):
        p = self.fft_pad
        return np.pad(np.asarray(x, dtype=np.float64), [(p, p)] * self.ndim)

    def _crop(self, X):
        p = self.fft_pad
        return X[tuple(slice(p, p + n) for n in self.shape)]

    def apply_term(self, i, x):
        lam, a, q = self.index(i)
        Xh = np.fft.rfftn(self._pad(x))
        w = np.fft.irfftn(Xh * self.multiplier(a, q), s=self.fshape,
                          axes=tuple(range(self.ndim)))
        return self.spatial_mode(lam) * self._crop(w)

    def apply(self, coeffs, x):
        """sum_i c_i B_i x -- the preconditioner applied to an image."""
        out = np.zeros(self.shape)
        for i, c in enumerate(np.asarray(coeffs, dtype=np.float64)):
            if c != 0.0:
                out += c * self.apply_term(i, x)
        return out

    def columns(self, x):
        """Matrix whose column i is B_i x flattened (n rows, P columns)."""
        return np.stack([self.apply_term(i, x).ravel() for i in range(self.P)], axis=1)


def fit(basis: Basis, y, x):
    """Least-squares coefficients c of sum_i c_i B_i ~ H^{-1} from pairs x_j = H y_j.

    y, x: arrays (p, *shape).  Rows of all p trials are stacked (Rn fit).
    Returns (c, resid_rel, cond_R) using Householder QR in FP64.
    """
    y = np.asarray(y, dtype=np.float64).reshape((-1,) + basis.shape)
    x = np.asarray(x, dtype=np.float64).reshape((-1,) + basis.shape)
    A = np.concatenate([basis.columns(xj) for xj in x], axis=0)
    b = y.reshape(-1)
    Q, R = np.linalg.qr(A, mode="reduced")
    c = np.linalg.solve(R, Q.T @ b) if R.shape[0] == R.shape[1] else None
    res = np.linalg.norm(b - A @ c) / max(np.linalg.norm(b), 1e-300)
    sv = np.linalg.svd(R, compute_uv=False)
    cond = float(sv[0] / sv[-1]) if sv[-1] > 0 else np.inf
    return c, float(res), cond


def fit_normal_equations(basis: Basis, y, x):
    """Closed form of Sec. 1.4: c = M^{-1} (Bx)^T y, M_ik = (B_i x)^T (B_k x)."""
    y = np.asarray(y, dtype=np.float64).reshape((-1,) + basis.shape)
    x = np.asarray(x, dtype=np.float64).reshape((-1,) + basis.shape)
    M = np.zeros((basis.P, basis.P))
    rhs = np.zeros(basis.P)
    for xj, yj in zip(x, y):
        A = basis.columns(xj)
        M += A.T @ A
        rhs += A.T @ yj.ravel()
    return np.linalg.solve(M, rhs), M


def relative_mse(dm_ref, dm):
    """Relative error ||dm_ref - dm||_2 / ||dm_ref||_2 (the paper's "MSE", Sec. 2)."""
    dm_ref = np.asarray(dm_ref, dtype=np.float64)
    return float(np.linalg.norm(dm_ref - np.asarray(dm, np.float64)) / np.linalg.norm(dm_ref))
