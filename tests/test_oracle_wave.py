"""Pins of the oracle's wave operators against closed forms and invariants (CPU only).

* 2D homogeneous Green's function (forward map) and its Born point-scatterer
  variant (source term -dm (u0)_tt of the Sec. 2 equations), with the
  2nd-order-in-dt convergence of the leapfrog scheme;
* exact transposition (dot-product test) of F and F* (Sec. 1.1);
* symmetry and positive semi-definiteness of a brute-force dense H = F*F
  (Sec. 1.1, and Sec. 1.3 on the fundamental subspaces of the Hessian);
* Born = Jacobian of the nonlinear map (Sec. 1.1 definition of F), and the
  Taylor test of the gradient formula dJ/dm = -F*(d - calF[m]);
* checkpointed recomputation gives the same migration as the stored history;
* the sponge absorbs: against the same field on a grid too large for any boundary to be met,
  the boundary layer sends back a small fraction of the field (no reflecting edge).
"""
import numpy as np
import pytest

from analytic import green2d_trace, ricker_fn, sampled_fn
from oracle.wave import Problem, problem_from_workload
from wave_checks import sponge_reflection
from workloads import gaussian_bumps, mini_config

C = 2000.0
F0 = 15.0
T0 = 1.5 / F0


def _homog(h, dt, T, n=161, rec=None, src=None):
    nt = int(round(T / dt)) + 1
    m0 = np.full((n, n), 1.0 / C ** 2)
    w = ricker_fn(F0, T0)(np.arange(nt) * dt)
    ic = n // 2
    src = [[ic, ic]] if src is None else src
    return Problem(m0, (h, h), dt, nt, 20, src, rec, w), ic


def _green_error(h, dt):
    n = 161
    ic = n // 2
    k = int(round(100 / h))
    kd = int(round(k / np.sqrt(2)))
    rec = np.array([[ic, ic + k], [ic + kd, ic + kd], [ic, ic + 2 * k]])
    p, _ = _homog(h, dt, 0.35, n=n, rec=rec)
    d = p.forward(0)
    times = np.arange(p.nt) * dt
    errs = []
    for j in range(3):
        r = h * np.sqrt(((rec[j] - ic) ** 2).sum())
        ua = green2d_trace(ricker_fn(F0, T0), r, C, times)
        errs.append(np.linalg.norm(d[:, j] - ua) / np.linalg.norm(ua))
    return np.array(errs)


def test_forward_matches_2d_greens_function_and_converges():
    e1 = _green_error(5.0, 5e-4)
    assert np.all(e1 < 2e-3), e1
    e2 = _green_error(5.0, 2.5e-4)
    assert np.all(e2 < 5e-4), e2
    ratio = e1 / e2
    assert np.all((ratio > 3.6) & (ratio < 4.4)), ratio      # 2nd order in dt


def _born_scatterer_error(h, dt):
    n = 161
    ic = n // 2
    k = int(round(60 / h))
    sp = (ic, ic + k)
    rec = np.array([[ic - k, ic + 2 * k]])
    p, _ = _homog(h, dt, 0.40, n=n, rec=rec)
    dmp = 0.05 / C ** 2
    dm = np.zeros((n, n))
    dm[sp] = dmp
    d = p.born(0, dm)[:, 0]
    T = (p.nt - 1) * dt
    tf = np.linspace(0, T, 4001)
    u0tt = green2d_trace(ricker_fn(F0, T0, 2), h * k, C, tf)
    g = sampled_fn(tf, -dmp * h * h * u0tt)        # equivalent point source of the scatterer
    r2 = h * np.sqrt((rec[0][0] - sp[0]) ** 2 + (rec[0][1] - sp[1]) ** 2)
    ua = green2d_trace(g, r2, C, np.arange(p.nt) * dt)
    return np.linalg.norm(d - ua) / np.linalg.norm(ua)


def test_born_point_scatterer_matches_analytic():
    e1 = _born_scatterer_error(5.0, 5e-4)
    assert e1 < 4e-3, e1
    e2 = _born_scatterer_error(5.0, 2.5e-4)
    assert 3.4 < e1 / e2 < 4.6, (e1, e2)


@pytest.fixture(scope="module")
def small():
    wl = mini_config(2, shape=(24, 28), nt=260, ns=2, pad=8)
    return wl, problem_from_workload(wl)


def test_dot_product_fp64(small):
    wl, p = small
    rng = np.random.default_rng(5)
    dm = rng.standard_normal(wl.shape)
    for shot in range(p.ns):
        r = rng.standard_normal((p.nt, p.nr))
        lhs = np.vdot(p.born(shot, dm), r)
        rhs = np.vdot(dm, p.adjoint(shot, r))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_dense_hessian_symmetric_psd():
    # 12x12 interior, pad 8, 200 steps, 2 shots: H assembled column by column.
    wl = mini_config(1, shape=(12, 12), nt=200, ns=2, pad=8)
    p = problem_from_workload(wl)
    n = 144
    E = np.eye(n).reshape(n, 12, 12)
    Fcols = np.stack([p.born(s, E) for s in range(p.ns)], axis=1)   # (n, ns, nt, nr)
    Fmat = Fcols.reshape(n, -1).T                                      # rows: data, cols: model
    H = p.hessian(E).reshape(n, n).T                                   # column j = H e_j
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    lam = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert lam.min() >= -1e-12 * lam.max()
    # brute force: H equals F^T F assembled from the Born columns
    assert np.abs(H - Fmat.T @ Fmat).max() <= 1e-11 * np.abs(H).max()


def test_checkpointed_adjoint_equals_stored_history(small):
    wl, p = small
    rng = np.random.default_rng(2)
    r = rng.standard_normal((p.nt, p.nr))
    a = p.adjoint(1, r)
    for K in (1, 7, 16, 300):
        b = p.adjoint(1, r, ckpt=K)
        assert np.array_equal(a, b), K


def test_born_is_jacobian_of_forward_map(small):
    wl, p = small
    dm = 0.05 * wl.m0.astype(np.float64) * gaussian_bumps(wl.shape, wl.h, 77, n=6, sigma_m=12.0)
    lin = p.born(0, dm)
    errs = []
    for eps in (1.0, 0.5, 0.25):
        fd = (p.forward(0, p.m0 + eps * dm) - p.forward(0, p.m0 - eps * dm)) / (2 * eps)
        errs.append(np.linalg.norm(fd - lin) / np.linalg.norm(lin))
    errs = np.array(errs)
    assert errs[-1] < 1e-3, errs
    r = errs[:-1] / errs[1:]
    assert np.all((r > 3.5) & (r < 4.5)), errs               # O(eps^2)


def test_gradient_taylor(small):
    wl, p = small
    bump = gaussian_bumps(wl.shape, wl.h, 78, n=5, sigma_m=12.0)
    m_true = p.m0 * (1.0 + 0.05 * bump / np.abs(bump).max())
    d_obs = [p.forward(s, m_true) for s in range(p.ns)]
    m = p.m0
    J0 = p.misfit(m, d_obs)
    g = p.gradient(m, d_obs)
    dmv = 0.02 * p.m0 * gaussian_bumps(wl.shape, wl.h, 79, n=5, sigma_m=12.0)
    res = []
    for eps in (1.0, 0.5, 0.25, 0.125):
        res.append(abs(p.misfit(m + eps * dmv, d_obs) - J0 - eps * np.vdot(g, dmv)))
    res = np.array(res)
    r = res[:-1] / res[1:]
    assert np.all((r > 3.3) & (r < 4.7)), res                 # O(eps^2)


def test_sponge_absorbs_against_larger_grid():
    # a 20-cell quadratic sponge (R = 1e-3) sends back 4.6 % of the peak window norm over 0.7 s;
    # at half strength 11 %, without sponge or with its damping sign flipped about 100 %
    assert sponge_reflection() < 0.07
    assert sponge_reflection(pad=0) > 0.5
