"""Pins of the oracle's symbol expansion, fit and preconditioner (CPU only).

* plane waves are eigenfunctions of every B_i on a periodic box: the eigenvalue
  is the symbol A(theta) TL_q(|k|) |k|^e evaluated at the plane wave's wave
  vector (definition of a Fourier multiplier, Eq. symbol);
* exact recovery of known coefficients when H^{-1} lies in span{B_i}
  (Sec. 1.4, "generalizability");
* the QR solution equals the closed form c = M^{-1} (Bx)^T y of Sec. 1.4.
"""
import numpy as np
import pytest

from oracle.symbol import Basis, fit, fit_normal_equations, relative_mse
from workloads import bandpassed_noise, linear_background

SPATIAL5 = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]
ANG4 = [0, 2, -2, 4]


def _plane(shape, h, kidx):
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = sum(2 * np.pi * kidx[a] * grids[a] / shape[a] for a in range(len(shape)))
    kvec = [2 * np.pi * kidx[a] / (shape[a] * h[a]) for a in range(len(shape))]
    return np.cos(phase), np.array(kvec)


@pytest.mark.parametrize("order", [-1.0, 1.0, 2.0])
def test_plane_wave_eigenvalues_2d(order):
    shape, h = (32, 40), (8.0, 5.0)
    L = 0.05
    b = Basis(shape, h, [(0, 0)], ANG4, 3, L, order=order, fft_pad=0)
    for kidx in [(3, 5), (-4, 7), (6, 0), (0, 9)]:
        x, (kz, kx) = _plane(shape, h, kidx)
        kn = np.hypot(kz, kx)
        th = np.arctan2(kz, kx)
        ang = {0: 1.0, 2: np.cos(2 * th), -2: np.sin(2 * th), 4: np.cos(4 * th)}
        t = (kn - L) / (kn + L)
        cheb = [1.0, t, 2 * t * t - 1]
        for i in range(b.P):
            _, a, q = b.index(i)
            want = ang[ANG4[a]] * cheb[q] * kn ** order
            got = b.apply_term(i, x)
            assert np.allclose(got, want * x, atol=1e-11 * max(1, abs(want))), (kidx, i)


def test_plane_wave_eigenvalues_3d_harmonics():
    shape, h = (16, 12, 20), (10.0, 10.0, 10.0)
    b = Basis(shape, h, [(0, 0, 0)], [0, 1, 2, 3, 4, 5], 1, 0.1, order=-1.0, fft_pad=0)
    x, k = _plane(shape, h, (2, -3, 4))
    kn = np.linalg.norm(k)
    uz, uy, ux = k / kn
    ylm = [1.0, ux * uy, uy * uz, ux * uz, ux ** 2 - uy ** 2, 3 * uz ** 2 - 1]
    for i in range(b.P):
        got = b.apply_term(i, x)
        assert np.allclose(got, ylm[i] / kn * x, atol=1e-12)


def test_spatial_modes_multiply():
    shape, h = (20, 24), (4.0, 4.0)
    b = Basis(shape, h, SPATIAL5, [0], 1, 0.1, order=-1.0, fft_pad=0)
    x, k = _plane(shape, h, (2, 3))
    base = x / np.linalg.norm(k)
    iz, ix = np.meshgrid(np.arange(20), np.arange(24), indexing="ij")
    modes = [np.ones(shape), np.cos(2 * np.pi * ix / 24), np.sin(2 * np.pi * ix / 24),
             np.cos(2 * np.pi * iz / 20), np.sin(2 * np.pi * iz / 20)]
    for i in range(5):
        assert np.allclose(b.apply_term(i, x), modes[i] * base, atol=1e-12)


def test_dc_is_annihilated():
    b = Basis((10, 14), (1.0, 1.0), SPATIAL5, ANG4, 2, 0.3, order=-1.0, fft_pad=0)
    for i in range(b.P):
        assert np.allclose(b.apply_term(i, np.ones((10, 14))), 0.0, atol=1e-12)


def _cfg3_like_basis(shape, h, m0):
    c_mean = float(np.mean(1 / np.sqrt(m0)))
    L = 2 * np.pi * (30.0 / c_mean)            # centre of the trial band [rad/m]
    return Basis(shape, h, SPATIAL5, ANG4, 2, L, order=-1.0, fft_pad=16)


def test_exact_recovery_of_known_expansion():
    shape, h = (48, 56), (8.0, 8.0)
    m0 = linear_background(shape)
    b = _cfg3_like_basis(shape, h, m0)
    rng = np.random.default_rng(11)
    c_true = rng.standard_normal(b.P)
    xs = bandpassed_noise(m0, h, seed=4242, p=2).astype(np.float64)
    ys = np.stack([b.apply(c_true, xj) for xj in xs])         # y_j = K x_j, K in span{B_i}
    c, res, cond = fit(b, ys, xs)
    assert np.linalg.norm(c - c_true) / np.linalg.norm(c_true) <= 1e-10, cond
    assert res <= 1e-12
    assert relative_mse(ys[0], b.apply(c, xs[0])) <= 1e-12


def test_qr_solution_equals_closed_form():
    shape, h = (24, 20), (8.0, 8.0)
    m0 = linear_background(shape)
    b = Basis(shape, h, SPATIAL5[:3], [0, 2], 2, 0.05, order=-1.0, fft_pad=4)
    rng = np.random.default_rng(3)
    xs = rng.standard_normal((2,) + shape)
    ys = rng.standard_normal((2,) + shape)                    # not in the span: a true LS fit
    c_qr, res, _ = fit(b, ys, xs)
    c_ne, M = fit_normal_equations(b, ys, xs)
    assert np.linalg.norm(c_qr - c_ne) / np.linalg.norm(c_qr) <= 1e-9
    assert np.allclose(M, M.T) and np.linalg.eigvalsh(M).min() > 0      # E M positive definite
    assert 0.0 < res < 1.0


def test_terms_map_real_fields_to_real_fields():
    # A real operator has a symbol even in k (Sec. 3, remark on complex matrices):
    # extending beta evenly from the half (real-FFT) grid to the full grid and
    # applying it with a complex FFT must give a real field equal to the
    # real-FFT evaluation -- also on even-length axes, where the Nyquist bin is
    # its own negative wave vector.
    for shape, pad in (((20, 26), 3), ((9, 14, 12), 2)):
        h = (7.0,) * len(shape)
        ang = [0, 2, -2, 4] if len(shape) == 2 else [0, 1, 2, 3, 4, 5]
        b = Basis(shape, h, [(0,) * len(shape)], ang, 2, 0.08, order=-1.0, fft_pad=pad)
        x = np.random.default_rng(4).standard_normal(shape)
        nl = b.fshape[-1]
        neg = [(-np.arange(N)) % N for N in b.fshape[:-1]]
        for i in range(b.P):
            _, a, q = b.index(i)
            half = b.multiplier(a, q)
            nh = half.shape[-1]
            full = np.empty(b.fshape)
            full[..., :nh] = half
            for j in range(nh, nl):
                full[..., j] = half[np.ix_(*neg, [(nl - j) % nl])][..., 0]
            y = np.fft.ifftn(np.fft.fftn(b._pad(x)) * full)
            assert np.abs(y.imag).max() <= 1e-12 * np.abs(y.real).max()
            got = b.spatial_mode(0) * b._crop(y.real)
            assert np.allclose(got, b.apply_term(i, x), atol=1e-12 * np.abs(got).max())
