"""Trial-function variants of the probing fit on the GPU (needs a GB300).

The comparison of Sec. 2 between randomized (Rn) and Krylov (Kn) trial
functions, and the H-applied white-noise trials (y = H n), composed from the
library's calls and checked against the same compositions of the FP64 oracle:

* probe_krylov_trials: y_1 = F*d / ||F*d||, y_{j+1} = H y_j / ||H y_j|| and
  x_j = H y_j against oracle.solve.krylov_trials on the oracle's H;
* H-applied white noise: H n and H (H n) against the oracle's;
* generalisation error of a fitted preconditioner on an independent trial
  (the relative "MSE" of Sec. 2): GPU fit + probe_apply_precond against the
  oracle's fit + apply on the oracle's own pairs, for Rn and Kn trials and
  for growing numbers of symbol parameters.
Tolerances: each H application 1e-4 (FP32 checkpoints, as in the H tests),
compounded over the Krylov recursion (2e-4); generalisation errors within 1 %
of the oracle's (the fits agree to 1e-6 on identical inputs; here each side fits
its own H applications, which differ by ~1e-5, amplified by the fit's
condition number).
"""
import numpy as np
import pytest

from oracle.solve import krylov_trials as okrylov
from oracle.symbol import Basis as OBasis
from oracle.symbol import fit as ofit
from oracle.symbol import relative_mse
from oracle.wave import problem_from_workload
from workloads import gaussian_bumps, mini_config, random_sign_trials, white_noise_trials

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPATIAL5 = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda:0")


@pytest.fixture(scope="module")
def setup():
    from paper_1101_3615_gb300 import Probe
    wl = mini_config(2, shape=(56, 60), nt=400, ns=3, pad=10, p=1)
    prob = problem_from_workload(wl)
    c_mean = float(np.mean(1 / np.sqrt(wl.m0.astype(np.float64))))
    dm_ref = gaussian_bumps(wl.shape, wl.h, 2202, n=12, sigma_m=16.0, amp=0.05 / c_mean ** 2)
    # migrated data F*d of the reference perturbation, from the oracle (the common input)
    mig = sum(prob.adjoint(s, prob.born(s, dm_ref.astype(np.float64))) for s in range(wl.ns)).astype(np.float32)
    p = Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)
    return wl, prob, p, mig, c_mean


def test_krylov_trials_match_oracle(cuda_device, setup):
    wl, prob, p, mig, _ = setup
    n = 4
    y, x = p.krylov_trials(dev(mig), n)
    yo, xo = okrylov(prob.hessian, mig.astype(np.float64), n)
    for j in range(n):
        assert rel(y[j].cpu().numpy(), yo[j]) < 2e-4, j
        assert rel(x[j].cpu().numpy(), xo[j]) < 2e-4, j
    assert abs(float(torch.linalg.vector_norm(y[0].double())) - 1.0) < 1e-6
    # host buffers through the C ABI give the same arrays
    yh, xh = p.krylov_trials(mig, n)
    assert np.array_equal(yh, y.cpu().numpy()) and np.array_equal(xh, x.cpu().numpy())


def test_white_noise_trials_match_oracle(cuda_device, setup):
    wl, prob, p, _, _ = setup
    noise = white_noise_trials(wl.m0, 31, p=2)
    y = p.apply_H(dev(noise))
    x = p.apply_H(y)
    for j in range(2):
        yo = prob.hessian(noise[j].astype(np.float64))
        assert rel(y[j].cpu().numpy(), yo) < 1e-4
        xo = prob.hessian(y[j].cpu().numpy().astype(np.float64))   # the oracle's H of the GPU trial
        assert rel(x[j].cpu().numpy(), xo) < 1e-4


@pytest.mark.parametrize("family", ["rn", "kn"])
@pytest.mark.parametrize("nradial", [1, 2, 3])
def test_generalisation_error_matches_oracle(cuda_device, setup, family, nradial):
    """Fit on two trials of one family, then the preconditioner's relative error on an
    independent random trial y_t: || y_t - M (H y_t) || / || y_t ||, for P = 20, 40, 60 terms."""
    from paper_1101_3615_gb300 import Basis
    wl, prob, p, mig, c_mean = setup
    L = 2 * np.pi * 30.0 / c_mean
    g = Basis(2, SPATIAL5, [0, 2, -2, 4], nradial, L, -1.0, 8)
    o = OBasis(wl.shape, wl.h, SPATIAL5, [0, 2, -2, 4], nradial, L, -1.0, 8)
    if family == "rn":
        ys = random_sign_trials(wl.m0, wl.h, 515, p=2)
        y_g = dev(ys)
        x_g = p.apply_H(y_g)
        y_o = ys.astype(np.float64)
        x_o = np.stack([prob.hessian(t) for t in y_o])
    else:
        y_g, x_g = p.krylov_trials(dev(mig), 2)
        y_o, x_o = okrylov(prob.hessian, mig.astype(np.float64), 2)
    yt = random_sign_trials(wl.m0, wl.h, 999, p=1)[0]
    xt_g = p.apply_H(dev(yt[None]))[0].contiguous()
    xt_o = prob.hessian(yt.astype(np.float64))
    c_g, _ = p.fit(g, y_g, x_g)
    mse_g = relative_mse(yt, p.apply_precond(g, c_g, xt_g).cpu().numpy())
    c_o, _, _ = ofit(o, y_o, x_o)
    mse_o = relative_mse(yt, o.apply(c_o, xt_o))
    assert abs(mse_g - mse_o) < 1e-2 * mse_o, (mse_g, mse_o)
