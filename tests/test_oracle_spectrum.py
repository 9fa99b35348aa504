"""Pins of the oracle's dense assembly and epsilon-rank (CPU only).

* eps_rank counts singular values strictly above eps times the largest, on
  matrices with prescribed singular values (including the boundary case);
* dense_operator reproduces the matrix of a known linear map;
* on a brute-force dense H of a tiny problem, the epsilon-rank is monotone in
  epsilon and equals the count from H's eigenvalues (H is symmetric PSD).
"""
import numpy as np

from oracle.spectrum import dense_operator, eps_rank
from oracle.wave import problem_from_workload
from workloads import mini_config


def _with_singular_values(s, seed=0):
    rng = np.random.default_rng(seed)
    n = len(s)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (U * np.asarray(s, float)) @ V.T


def test_eps_rank_counts_prescribed_singular_values():
    A = _with_singular_values([4.0, 2.0, 4e-3, 4e-7, 0.0])
    assert eps_rank(A, [1e-1, 1e-2, 1e-4, 1e-8]) == [2, 2, 3, 4]
    assert eps_rank(np.diag([1.0, 0.5]), [0.5]) == [1]        # strictly above
    assert eps_rank(np.zeros((3, 3)), [1e-3]) == [0]


def test_dense_operator_reproduces_a_known_map():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((12, 12))
    A = dense_operator(lambda x: (M @ x.ravel()).reshape(3, 4), (3, 4))
    assert np.array_equal(A, M)


def test_eps_rank_of_a_dense_hessian():
    wl = mini_config(2, shape=(6, 7), nt=90, ns=1, pad=4)
    p = problem_from_workload(wl)
    H = dense_operator(p.hessian, wl.shape)
    ev = np.sort(np.abs(np.linalg.eigvalsh(0.5 * (H + H.T))))[::-1]
    eps = [1e-1, 1e-2, 1e-4, 1e-8]
    r = eps_rank(H, eps)
    assert r == sorted(r)
    assert r == [int(np.count_nonzero(ev > e * ev[0])) for e in eps]
