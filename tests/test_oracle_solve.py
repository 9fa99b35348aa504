"""Pins of the oracle's iterative solvers (CPU only).

* conjugate gradients terminates in as many steps as the operator has distinct
  eigenvalues (textbook finite termination), and on the normal equations of the
  oracle's Born operator its data misfit never increases;
* steepest descent with exact line search meets the Kantorovich rate
  (kappa - 1)/(kappa + 1) per step in the energy norm, with equality for the
  classical worst-case start on a 2 x 2 operator;
* with the exact inverse as preconditioner one descent step solves the system;
* the Krylov trials are the normalised powers H^j F*d.
A planted mistake in the CG recurrence (the ratio of residual norms inverted)
trips the termination pin.
"""
import numpy as np

from oracle.solve import conjugate_gradients, gradient_descent, krylov_trials
from oracle.wave import problem_from_workload
from workloads import mini_config


def _spd(eigs, seed=0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(eigs), len(eigs))))
    return (Q * np.asarray(eigs, float)) @ Q.T


def _termination_gap(cg):
    """Relative residual of CG after 4 and after 5 steps on a 40 x 40 operator with five
    distinct eigenvalues (each of multiplicity 8)."""
    A = _spd(np.repeat([1.0, 3.0, 10.0, 30.0, 100.0], 8))
    b = np.random.default_rng(1).standard_normal(40)
    r4 = cg(lambda v: A @ v, b, 4)[1][-1] / np.linalg.norm(b)
    x5, h5 = cg(lambda v: A @ v, b, 5)
    return r4, h5[-1] / np.linalg.norm(b), np.linalg.norm(x5 - np.linalg.solve(A, b)) / np.linalg.norm(np.linalg.solve(A, b))


def test_cg_terminates_after_as_many_steps_as_distinct_eigenvalues():
    r4, r5, e5 = _termination_gap(conjugate_gradients)
    assert r4 > 1e-4
    assert r5 < 1e-10 and e5 < 1e-10


def test_planted_cg_mistake_is_caught():
    def bad_cg(apply_H, rhs, iters):
        x = np.zeros_like(rhs)
        r = rhs.copy()
        p = r.copy()
        rr = r @ r
        hist = [np.sqrt(rr)]
        for _ in range(iters):
            Hp = apply_H(p)
            alpha = rr / (p @ Hp)
            x = x + alpha * p
            r = r - alpha * Hp
            rr_new = r @ r
            p = r + (rr / rr_new) * p          # ratio inverted
            rr = rr_new
            hist.append(np.sqrt(rr))
        return x, np.array(hist)
    _, r5, _ = _termination_gap(bad_cg)
    assert r5 > 1e-6


def test_steepest_descent_kantorovich_rate_and_worst_case_equality():
    A = _spd(np.linspace(1.0, 50.0, 30), seed=2)
    kappa = 50.0
    rate = (kappa - 1) / (kappa + 1)
    xs = np.linalg.solve(A, np.ones(30))
    b = A @ xs
    errs = []
    for k in range(12):
        x, _ = gradient_descent(lambda v: A @ v, b, k)
        e = x - xs
        errs.append(np.sqrt(e @ A @ e))
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.all(ratios <= rate * (1 + 1e-12))
    # 2 x 2 worst case: error components (1/l1, 1/l2) attain the bound at every step
    l1, l2 = 1.0, 9.0
    D = np.diag([l1, l2])
    x0 = -np.array([1 / l1, 1 / l2])        # exact solution 0 (rhs 0): error = x0
    x1, _ = gradient_descent(lambda v: D @ v, np.zeros(2), 1, x0=x0)
    en = lambda v: np.sqrt(v @ D @ v)
    assert abs(en(x1) / en(x0) - (l2 - l1) / (l2 + l1)) < 1e-12


def test_exact_inverse_preconditioner_solves_in_one_step():
    A = _spd(np.linspace(1.0, 1e3, 25), seed=3)
    b = np.random.default_rng(4).standard_normal(25)
    Ainv = np.linalg.inv(A)
    x, hist = gradient_descent(lambda v: A @ v, b, 1, apply_M=lambda r: Ainv @ r)
    assert np.linalg.norm(x - Ainv @ b) / np.linalg.norm(Ainv @ b) < 1e-10
    assert hist[-1] / hist[0] < 1e-10


def test_krylov_trials_are_normalised_powers():
    A = _spd(np.linspace(0.5, 4.0, 12), seed=5)
    b = np.random.default_rng(6).standard_normal(12)
    y, x = krylov_trials(lambda v: A @ v, b, 4)
    for j in range(4):
        v = np.linalg.matrix_power(A, j) @ b
        assert np.allclose(y[j], v / np.linalg.norm(v), rtol=0, atol=1e-13)
        assert np.allclose(x[j], A @ y[j], rtol=0, atol=1e-12)


def test_cg_on_the_born_normal_equations_never_increases_the_data_misfit():
    wl = mini_config(2, shape=(12, 14), nt=120, ns=2, pad=6)
    p = problem_from_workload(wl)
    dm_true = wl.trials[0].astype(np.float64)
    d = [p.born(s, dm_true) for s in range(p.ns)]
    rhs = sum(p.adjoint(s, d[s]) for s in range(p.ns))
    misfit = []
    for k in range(6):
        x, _ = conjugate_gradients(p.hessian, rhs, k)
        misfit.append(np.sqrt(sum(np.sum((p.born(s, x) - d[s]) ** 2) for s in range(p.ns))))
    misfit = np.array(misfit)
    assert np.all(misfit[1:] <= misfit[:-1] * (1 + 1e-12))
    assert misfit[-1] < 0.5 * misfit[0]
