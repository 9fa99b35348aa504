"""Shared measurements for the oracle's wave-operator pins (CPU only)."""
import functools

import numpy as np

from analytic import ricker_fn
import oracle.wave as ow

C, F0, T0 = 2000.0, 15.0, 1.5 / 15.0
_H, _DT, _NT, _WIN = 10.0, 1e-3, 700, 61


def _window_history(n, problem_cls=ow.Problem, pad=20):
    """Incident field of a centred Ricker source on an n x n homogeneous interior, in the
    central _WIN x _WIN window, for _NT steps: shape (nt, _WIN, _WIN)."""
    ic = n // 2
    w = ricker_fn(F0, T0)(np.arange(_NT) * _DT)
    p = problem_cls(np.full((n, n), 1 / C ** 2), (_H, _H), _DT, _NT, pad, [[ic, ic]], [[ic, ic]], w)
    U = p.incident_history(0)
    c, r = ic + pad, _WIN // 2
    return U[:, c - r:c + r + 1, c - r:c + r + 1]


@functools.lru_cache(maxsize=1)
def _reflection_free():
    # 181 cells: nothing reflected at this grid's own edge reaches the window within _NT steps
    # (centre -> edge -> window edge is > 2 * 90 - 30 cells, the wave covers 140 cells)
    return _window_history(181)


def sponge_reflection(problem_cls=ow.Problem, pad=20):
    """Largest L2 norm, over time, of what the sponge of a 61 x 61 interior sends back into the
    window, relative to the peak norm of the reflection-free field there: the field on the
    small grid minus the same field on a grid large enough that no boundary is met."""
    ref = _reflection_free()
    u = _window_history(_WIN, problem_cls, pad)
    d = np.sqrt(((u - ref) ** 2).sum(axis=(1, 2)))
    return float(d.max() / np.sqrt((ref ** 2).sum(axis=(1, 2))).max())
