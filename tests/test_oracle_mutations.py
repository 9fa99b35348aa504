"""Planted mistakes in the oracle must trip its pins (CPU only).

Each case patches one plausible error into the oracle -- a wrong stencil
weight, a dropped 1/h^d source scaling, a flipped Born-source sign, an
off-by-one time index in the imaging condition, a sponge whose damping sign
is flipped, an adjoint that injects the residual at the wrong receivers, a
flipped rational-Chebyshev map, a wrong sign of the symbol order or of a sine
harmonic, a wrong spatial-mode period, a fit with its pairs swapped -- and
checks that the closed-form or invariant pin that guards that part of the
oracle fails.
"""
import numpy as np
import pytest

import oracle.wave as ow
from analytic import green2d_trace, ricker_fn
from oracle.fd import laplacian
from wave_checks import sponge_reflection
from workloads import mini_config

C, F0, T0 = 2000.0, 15.0, 1.5 / 15.0


def _green_err(prob_cls=ow.Problem):
    n, h, dt = 81, 10.0, 1e-3
    ic, k = n // 2, 10
    nt = 351
    w = ricker_fn(F0, T0)(np.arange(nt) * dt)
    p = prob_cls(np.full((n, n), 1 / C ** 2), (h, h), dt, nt, 20, [[ic, ic]], [[ic, ic + k]], w)
    d = p.forward(0)[:, 0]
    ua = green2d_trace(ricker_fn(F0, T0), h * k, C, np.arange(nt) * dt)
    return np.linalg.norm(d - ua) / np.linalg.norm(ua)


def _dot_mismatch():
    wl = mini_config(2, shape=(20, 22), nt=160, ns=1, pad=6)
    p = ow.problem_from_workload(wl)
    rng = np.random.default_rng(1)
    dm = rng.standard_normal(wl.shape)
    r = rng.standard_normal((p.nt, p.nr))
    a, b = np.vdot(p.born(0, dm), r), np.vdot(dm, p.adjoint(0, r))
    return abs(a - b) / max(abs(a), abs(b))


def test_unmutated_baseline():
    assert _green_err() < 5e-3
    assert _dot_mismatch() < 1e-12


def test_wrong_stencil_weight_is_caught(monkeypatch):
    bad = [-205 / 72, 8 / 5, +1 / 5, 8 / 315, -1 / 560]
    monkeypatch.setattr(ow, "laplacian", lambda u, h: laplacian(u, h, weights=bad))
    assert _green_err() > 5e-2


def test_dropped_source_scaling_is_caught(monkeypatch):
    def src(self, shot, n, rhs):
        idx = tuple(int(c[shot]) for c in self.src_p)
        rhs[idx] += self.w[n]                     # missing 1/(h_1 h_2)
    monkeypatch.setattr(ow.Problem, "_source_rhs", src)
    assert _green_err() > 0.5


def test_flipped_born_sign_is_caught(monkeypatch):
    orig = ow.Problem.born

    def born(self, shot, dm, m_int=None):
        return orig(self, shot, -np.asarray(dm), m_int)
    monkeypatch.setattr(ow.Problem, "born", born)
    # F flips sign while F* does not: the transposition pin breaks
    assert _dot_mismatch() > 1.0


def test_imaging_time_index_shift_is_caught(monkeypatch):
    orig = ow.Problem._dtt_segments

    def shifted(self, shot, m_int, ckpt):
        prev = None
        for n, d in orig(self, shot, m_int, ckpt):
            yield n, (d if prev is None else prev)     # uses Dtt u^{n+1} at step n
            prev = d
    monkeypatch.setattr(ow.Problem, "_dtt_segments", shifted)
    assert _dot_mismatch() > 1e-4


def test_flipped_sponge_damping_is_caught():
    class Flipped(ow.Problem):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            self.am = 1.0 + 0.5 * self.dt * self.eta     # a- = 1 + eta dt / 2: no damping
    assert sponge_reflection(Flipped) > 0.5


def test_misplaced_adjoint_injection_is_caught(monkeypatch):
    orig = ow.Problem._inject_adjoint

    def inject(self, lam, r_n):
        orig(self, lam, np.asarray(r_n)[..., ::-1])      # receiver order reversed
    monkeypatch.setattr(ow.Problem, "_inject_adjoint", inject)
    assert _dot_mismatch() > 1e-3


# -- the symbol expansion and the fit: each planted mistake must make one of the pins in
#    test_oracle_symbol.py fail (they are called here as plain functions).
import oracle.symbol as osym
import test_oracle_symbol as sym_pins


def _mutated_multiplier(t_sign=1.0, exp_sign=1.0):
    def multiplier(self, a, q):
        kvec = self._kgrid()
        knorm = np.sqrt(sum(k ** 2 for k in kvec))
        pos = (knorm > 0) & ~self._nyquist_mask()
        safe = np.where(knorm > 0, knorm, 1.0)
        t = t_sign * (safe - self.L) / (safe + self.L)
        cheb = np.cos(q * np.arccos(np.clip(t, -1.0, 1.0)))
        beta = self.angular_fn(a, kvec) * cheb * safe ** (exp_sign * self.order)
        return np.where(pos, beta, 0.0)
    return multiplier


def test_unmutated_symbol_pins_pass():
    sym_pins.test_plane_wave_eigenvalues_2d(-1.0)
    sym_pins.test_spatial_modes_multiply()
    sym_pins.test_exact_recovery_of_known_expansion()


def test_flipped_chebyshev_map_is_caught(monkeypatch):
    monkeypatch.setattr(osym.Basis, "multiplier", _mutated_multiplier(t_sign=-1.0))
    with pytest.raises(AssertionError):
        sym_pins.test_plane_wave_eigenvalues_2d(-1.0)


def test_wrong_symbol_order_sign_is_caught(monkeypatch):
    monkeypatch.setattr(osym.Basis, "multiplier", _mutated_multiplier(exp_sign=-1.0))
    with pytest.raises(AssertionError):
        sym_pins.test_plane_wave_eigenvalues_2d(-1.0)


def test_wrong_sine_harmonic_sign_is_caught(monkeypatch):
    orig = osym.Basis.angular_fn

    def angular_fn(self, a, kvec):
        f = orig(self, a, kvec)
        return -f if self.ndim == 2 and self.angular[a] < 0 else f    # sin(q theta) for q < 0
    monkeypatch.setattr(osym.Basis, "angular_fn", angular_fn)
    with pytest.raises(AssertionError):
        sym_pins.test_plane_wave_eigenvalues_2d(-1.0)


def test_wrong_spatial_period_is_caught(monkeypatch):
    def spatial_mode(self, lam):
        out = np.ones(self.shape)
        for ax, k in enumerate(self.spatial[lam]):
            n = self.shape[ax]
            i = np.arange(n, dtype=np.float64)
            f = np.ones(n) if k == 0 else (np.cos(2 * np.pi * k * i / (n + 1)) if k > 0
                                           else np.sin(2 * np.pi * (-k) * i / (n + 1)))
            sh = [1] * self.ndim
            sh[ax] = n
            out = out * f.reshape(sh)
        return out
    monkeypatch.setattr(osym.Basis, "spatial_mode", spatial_mode)
    with pytest.raises(AssertionError):
        sym_pins.test_spatial_modes_multiply()


def test_fit_with_swapped_pairs_is_caught(monkeypatch):
    orig = osym.fit
    monkeypatch.setattr(sym_pins, "fit", lambda basis, y, x: orig(basis, x, y))
    with pytest.raises(AssertionError):
        sym_pins.test_exact_recovery_of_known_expansion()
