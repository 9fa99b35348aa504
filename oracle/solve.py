"""Iterative solution of the linearised least-squares problem (oracle, FP64).

Test infrastructure only.  Sec. 2 judges the fitted preconditioners against the
image that 200 gradient-descent steps on the linearised least-squares
functional J(dm) = 1/2 ||F dm - d||^2 produce, names iterative solvers (GMRES,
LSQR) as the practical refinement, and discusses preconditioned gradient
iterations in which the approximate inverse is applied to the migrated residual
F*(d - F dm_k) rather than to F*d (the end of the Krylov/randomized comparison).
Written from those statements and the textbook algorithms:

* gradient descent on J: the negative gradient is the migrated residual
  r_k = F*d - H dm_k (H = F*F); the step along a search direction p is the
  exact minimiser of J on the line, alpha = p.r / p.Hp (J is quadratic);
  with a preconditioner M the direction is p = M r_k (M r_k = r_k without one);
* conjugate gradients on the normal equations H dm = F*d (H symmetric positive
  semi-definite), the textbook recurrence; it minimises the data misfit
  ||d - F dm|| over the growing Krylov space, so that misfit never increases;
* the Krylov trial functions of the Kn preconditioners: y_1 = F*d and
  y_{j+1} = H y_j (normalised), fitted with the pairs (y_j, H y_j).

Every operator is passed in as a function of an interior model-space array, so
the same code runs with the oracle's H and preconditioner or with small dense
matrices in the pins.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return float(np.vdot(np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()))


def gradient_descent(apply_H, rhs, iters, x0=None, apply_M=None):
    """Steepest descent on 1/2 x.Hx - x.rhs with exact line search.

    rhs = F*d (the migrated image); apply_M, if given, maps the residual to the search
    direction (preconditioned descent).  Returns (x, history) with history[k] the residual
    norm ||rhs - H x_k|| for k = 0..iters.
    """
    x = np.zeros_like(np.asarray(rhs, np.float64)) if x0 is None else np.array(x0, np.float64)
    r = np.asarray(rhs, np.float64) - apply_H(x)
    hist = [np.sqrt(_dot(r, r))]
    for _ in range(iters):
        p = r if apply_M is None else np.asarray(apply_M(r), np.float64)
        Hp = apply_H(p)
        pHp = _dot(p, Hp)
        if pHp <= 0.0:  # direction in the null space of H (or not a descent direction): stop
            break
        alpha = _dot(p, r) / pHp
        x = x + alpha * p
        r = r - alpha * Hp
        hist.append(np.sqrt(_dot(r, r)))
    return x, np.array(hist)


def conjugate_gradients(apply_H, rhs, iters, x0=None):
    """Textbook conjugate gradients for H x = rhs with H symmetric positive semi-definite.

    Returns (x, history) with history[k] = ||rhs - H x_k||.  Stops early when the residual or
    the curvature along the search direction vanishes.
    """
    x = np.zeros_like(np.asarray(rhs, np.float64)) if x0 is None else np.array(x0, np.float64)
    r = np.asarray(rhs, np.float64) - apply_H(x)
    p = r.copy()
    rr = _dot(r, r)
    hist = [np.sqrt(rr)]
    for _ in range(iters):
        if rr == 0.0:
            break
        Hp = apply_H(p)
        pHp = _dot(p, Hp)
        if pHp <= 0.0:
            break
        alpha = rr / pHp
        x = x + alpha * p
        r = r - alpha * Hp
        rr_new = _dot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        hist.append(np.sqrt(rr))
    return x, np.array(hist)


def krylov_trials(apply_H, rhs, n):
    """Trial functions of the Kn preconditioner: y_1 = rhs (= F*d), y_{j+1} = H y_j, each
    normalised to unit 2-norm.  Returns (y, x) with x_j = H y_j, arrays of shape (n, *shape)."""
    ys, xs = [], []
    y = np.asarray(rhs, np.float64)
    for _ in range(n):
        y = y / np.sqrt(_dot(y, y))
        x = np.asarray(apply_H(y), np.float64)
        ys.append(y)
        xs.append(x)
        y = x
    return np.stack(ys), np.stack(xs)
