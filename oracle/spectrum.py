"""Dense assembly of a model-space operator and its epsilon-rank (oracle, FP64).

Test infrastructure only.  Sec. 2 reports, for its 16,384 x 16,384 Hessian, the
epsilon-rank as a function of epsilon with the top singular value normalised to
one: the number of singular values above epsilon.  Written from that definition:

* dense_operator: the matrix of a linear map of interior model-space arrays,
  column i = the map applied to the i-th unit vector (brute force);
* eps_rank: #{ sigma_j > eps * sigma_max } for each eps.
"""
from __future__ import annotations

import numpy as np


def dense_operator(apply, shape):
    """n x n matrix (n = prod(shape)) whose column i is apply(e_i), row-major flattening."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = np.asarray(apply(e.reshape(shape)), np.float64).ravel()
    return A


def eps_rank(A, eps):
    """Number of singular values of A strictly above eps * (largest singular value), for each
    eps in the sequence ``eps``."""
    s = np.linalg.svd(np.asarray(A, np.float64), compute_uv=False)
    if s.size == 0 or s[0] == 0.0:
        return [0 for _ in eps]
    return [int(np.count_nonzero(s > e * s[0])) for e in eps]
