"""GPU parity of probe_fit / probe_apply_precond with the FP64 oracle (needs a GB300).

Both sides receive the same FP32 arrays.  The GPU solves the least-squares
problem of Sec. 1.4 through a CholeskyQR2 factorisation of the stacked columns
in FP64; the oracle uses Householder QR.  Bars: coefficients within 1e-6
(relative L2) of the oracle's -- also on bases with cond(A) of 1e6 to 1e7,
where the normal equations alone would lose about cond(A)^2 eps = 1e-2 -- and
on the largest basis (P = 1024); preconditioned images within 1e-6; exact
recovery of known coefficients limited only by the FP32 rounding of the inputs
(1e-5).
"""
import numpy as np
import pytest

from oracle.symbol import Basis as OBasis
from oracle.symbol import fit as ofit
from workloads import bandpassed_noise, linear_background, mini_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPATIAL5 = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]
ANG4 = [0, 2, -2, 4]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bases(wl, spatial=SPATIAL5, angular=ANG4, nradial=2, order=-1.0, fft_pad=16, lf=30.0):
    from paper_1101_3615_gb300 import Basis
    c_mean = float(np.mean(1 / np.sqrt(wl.m0.astype(np.float64))))
    L = 2 * np.pi * lf / c_mean
    g = Basis(wl.ndim, spatial, angular, nradial, L, order, fft_pad)
    o = OBasis(wl.shape, wl.h, spatial, angular, nradial, L, order, fft_pad)
    return g, o


def make_probe(wl):
    from paper_1101_3615_gb300 import Probe
    return Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)


def test_precond_matches_oracle(cuda_device):
    wl = mini_config(1, shape=(101, 101), nt=50, ns=1)
    g, o = bases(wl)
    rng = np.random.default_rng(21)
    c = rng.standard_normal(g.P)
    img = bandpassed_noise(wl.m0, wl.h, 77, p=1)[0]
    p = make_probe(wl)
    got_dev = p.apply_precond(g, c, torch.tensor(img, device=cuda_device)).cpu().numpy()
    got_host = p.apply_precond(g, c, img)                       # host buffers through the ABI
    ref = o.apply(c, img.astype(np.float64))
    assert rel(got_dev, ref) < 1e-6
    assert np.array_equal(got_dev, got_host)


@pytest.mark.parametrize("shape,fft_pad", [((64, 72), 16), ((57, 43), 5), ((40, 40), 0)])
def test_fit_exact_recovery(cuda_device, shape, fft_pad):
    wl = mini_config(1, shape=shape, nt=50, ns=1)
    g, o = bases(wl, fft_pad=fft_pad)
    c_true = np.random.default_rng(5).standard_normal(g.P)
    xs = bandpassed_noise(wl.m0, wl.h, 4242, p=2)                # FP32 inputs
    ys = np.stack([o.apply(c_true, xj.astype(np.float64)) for xj in xs]).astype(np.float32)
    p = make_probe(wl)
    c_gpu, res_gpu = p.fit(g, torch.tensor(ys, device=cuda_device), torch.tensor(xs, device=cuda_device))
    c_orc, res_orc, cond = ofit(o, ys, xs)
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert rel(c_gpu, c_true) < 1e-5, cond                      # FP32 rounding of y limits this
    assert abs(res_gpu - res_orc) < 1e-6 and res_gpu < 1e-5


def test_fit_on_hessian_applications_config1(cuda_device):
    """Rn fit (Sec. 2) from two band-passed trials and their H applications."""
    wl = mini_config(1, shape=(101, 101), nt=800, ns=4, p=2)
    g, o = bases(wl)
    p = make_probe(wl)
    y = torch.tensor(wl.trials, device=cuda_device)
    x = p.apply_H(y)
    c_gpu, res_gpu = p.fit(g, y, x)
    c_orc, res_orc, cond = ofit(o, wl.trials, x.cpu().numpy())
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert abs(res_gpu - res_orc) < 1e-6
    # the fitted preconditioner applied to H y reproduces the fit's residual
    pre = p.apply_precond(g, c_gpu, x[0].contiguous()).cpu().numpy()
    assert abs(rel(pre, wl.trials[0]) - rel(o.apply(c_orc, x[0].cpu().numpy().astype(np.float64)),
                                             wl.trials[0])) < 1e-5


def test_fit_errors(cuda_device):
    from paper_1101_3615_gb300 import Basis, ProbeError
    wl = mini_config(1, shape=(40, 44), nt=50, ns=1)
    p = make_probe(wl)
    y = torch.tensor(bandpassed_noise(wl.m0, wl.h, 1, p=1), device=cuda_device)
    too_many = Basis(2, [(0, 0)] * 33, [0, 2, -2, 4], 2, 0.05)  # more than 32 spatial modes
    with pytest.raises(ProbeError) as ei:
        p.fit(too_many, y, y)
    assert ei.value.status == -1
    dup = Basis(2, [(0, 0), (0, 0)], [0], 1, 0.05)               # identical columns: M singular
    with pytest.raises(ProbeError) as ei:
        p.fit(dup, y, y)
    assert ei.value.status == -6


# A small basis (P = 64, Gram in one CTA) and a large one (P = 160, chunked Gram), both with
# cond(A) of about 1e6 - 2e6 on these band-limited trials (eight Chebyshev terms on a narrow band)
@pytest.mark.parametrize("spatial,nradial", [([(0, 0), (0, 1)], 8), (SPATIAL5, 8)])
def test_fit_ill_conditioned_basis_matches_qr(cuda_device, spatial, nradial):
    wl = mini_config(1, shape=(48, 52), nt=50, ns=1)
    g, o = bases(wl, spatial=spatial, nradial=nradial, fft_pad=8, lf=60.0)
    c_true = np.random.default_rng(5).standard_normal(g.P)
    xs = bandpassed_noise(wl.m0, wl.h, 4242, p=2)
    ys = np.stack([o.apply(c_true, xj.astype(np.float64)) for xj in xs]).astype(np.float32)
    c_orc, res_orc, cond = ofit(o, ys, xs)
    assert cond > 1e6                                            # the regime the QR is for
    p = make_probe(wl)
    c_gpu, res_gpu = p.fit(g, torch.tensor(ys, device=cuda_device), torch.tensor(xs, device=cuda_device))
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert abs(res_gpu - res_orc) < 1e-7


def test_fit_largest_basis(cuda_device):
    """P = 32 spatial modes x 8 angular x 4 radial = 1024 terms, four trials: exact recovery."""
    wl = mini_config(1, shape=(96, 100), nt=50, ns=1)
    sp = [(a, b) for a in range(-3, 4) for b in range(-3, 4)][:32]
    g, o = bases(wl, spatial=sp, angular=[0, 2, -2, 4, -4, 6, -6, 8], nradial=4, fft_pad=8)
    assert g.P == 1024
    c_true = np.random.default_rng(5).standard_normal(g.P)
    xs = bandpassed_noise(wl.m0, wl.h, 4242, p=4)
    ys = np.stack([o.apply(c_true, xj.astype(np.float64)) for xj in xs]).astype(np.float32)
    c_orc, res_orc, cond = ofit(o, ys, xs)
    p = make_probe(wl)
    c_gpu, res_gpu = p.fit(g, torch.tensor(ys, device=cuda_device), torch.tensor(xs, device=cuda_device))
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert rel(c_gpu, c_true) < 1e-5, cond
