"""Dense H on the GPU and its epsilon-rank (needs a GB300).

Sec. 2 tabulates the epsilon-rank of its Hessian.  Here H is assembled column
by column as batched probe_apply_H calls on unit vectors (one launch sequence
per batch of columns) on a tiny grid, and compared with the oracle's brute-force
dense H (oracle.spectrum.dense_operator on oracle.wave.Problem.hessian):
entries within 1e-4 (FP32 checkpoints), symmetric to 1e-5, every singular
value within 1e-4 of the largest (Weyl: |s_i(A) - s_i(B)| <= ||A - B||_2), and
the same epsilon-ranks wherever no singular value lies that close to a
threshold.
"""
import numpy as np
import pytest

from oracle.spectrum import dense_operator, eps_rank
from oracle.wave import problem_from_workload
from workloads import mini_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dense_H_gpu(p, shape, batch):
    n = int(np.prod(shape))
    H = torch.empty((n, n), dtype=torch.float32, device="cuda:0")
    for i0 in range(0, n, batch):
        k = min(batch, n - i0)
        e = torch.zeros((k, n), dtype=torch.float32, device="cuda:0")
        e[torch.arange(k), torch.arange(i0, i0 + k)] = 1.0
        H[:, i0:i0 + k] = p.apply_H(e.reshape((k,) + tuple(shape))).reshape(k, n).T
    return H


def test_dense_hessian_and_eps_rank_match_oracle(cuda_device):
    from paper_1101_3615_gb300 import Probe
    wl = mini_config(2, shape=(12, 12), nt=200, ns=2, pad=8)
    p = Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)
    Hg = dense_H_gpu(p, wl.shape, 48).cpu().numpy().astype(np.float64)
    Ho = dense_operator(problem_from_workload(wl).hessian, wl.shape)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) < 1e-4
    assert np.linalg.norm(Hg - Hg.T) / np.linalg.norm(Hg) < 1e-5
    sg = np.linalg.svd(Hg, compute_uv=False)
    so = np.linalg.svd(Ho, compute_uv=False)
    assert np.max(np.abs(sg - so)) < 1e-4 * so[0]
    eps = [1e-1, 3e-2, 1e-2, 3e-3, 1e-3]
    clear = [e for e in eps if np.min(np.abs(so - e * so[0])) > 2e-4 * so[0]]
    assert len(clear) >= 3
    assert eps_rank(Hg, clear) == eps_rank(Ho, clear)
