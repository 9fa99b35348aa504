"""Pins of the oracle's finite-difference pieces (CPU only)."""
from fractions import Fraction

import numpy as np

from oracle.fd import laplacian, second_derivative_weights, sponge_eta


def test_weights_match_textbook_8th_order():
    # Standard 8th-order central second-derivative coefficients (Fornberg 1988).
    w = second_derivative_weights(4)
    assert w == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                 Fraction(8, 315), Fraction(-1, 560)]
    assert second_derivative_weights(1) == [Fraction(-2), Fraction(1)]


def test_laplacian_exact_on_polynomials():
    # An 8th-order stencil differentiates polynomials up to degree 9 exactly.
    h = (0.7, 1.3)
    z = np.arange(40) * h[0]
    x = np.arange(30) * h[1]
    Z, X = np.meshgrid(z, x, indexing="ij")
    for deg in range(0, 10):
        u = (Z - 11.0) ** deg + 0.5 * (X - 9.0) ** deg
        ref = deg * (deg - 1) * ((Z - 11.0) ** max(deg - 2, 0) + 0.5 * (X - 9.0) ** max(deg - 2, 0)) \
            if deg >= 2 else np.zeros_like(u)
        got = laplacian(u, h)
        inner = (slice(4, -4), slice(4, -4))
        scale = max(1.0, np.abs(ref[inner]).max())
        assert np.abs(got[inner] - ref[inner]).max() / scale < 1e-9, deg


def test_laplacian_symmetric_with_zero_extension():
    rng = np.random.default_rng(0)
    for shape, h in (((17, 23), (1.0, 2.0)), ((9, 8, 11), (1.0, 1.5, 0.5))):
        u = rng.standard_normal(shape)
        v = rng.standard_normal(shape)
        a = np.vdot(laplacian(u, h), v)
        b = np.vdot(u, laplacian(v, h))
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def test_laplacian_plane_wave_symbol():
    # Periodic interior: L exp(i k x) = -(4/h^2) sum_k w_k sin^2(k theta/2) ... i.e. the
    # stencil symbol  (w0 + 2 sum w_k cos(k theta)) / h^2.
    n, h = 64, 3.0
    w = [float(x) for x in second_derivative_weights(4)]
    for kk in (1, 5, 13):
        th = 2 * np.pi * kk / n
        u = np.cos(th * np.arange(n))[None, :] * np.ones((12, 1))
        got = laplacian(u, (1.0, h))[6, 20:40]
        sym = (w[0] + 2 * sum(w[k] * np.cos(k * th) for k in range(1, 5))) / h ** 2
        assert np.allclose(got, sym * u[6, 20:40], rtol=0, atol=1e-12)


def test_sponge_profile():
    eta = sponge_eta((10, 12), 5, (2.0, 4.0), cmax=3000.0, R=1e-3)
    assert eta.shape == (20, 22)
    assert np.all(eta[5:15, 5:17] == 0.0)
    emax_z = 3 * 3000.0 * np.log(1e3) / (2 * 5 * 2.0)
    emax_x = 3 * 3000.0 * np.log(1e3) / (2 * 5 * 4.0)
    assert np.isclose(eta[0, 10], emax_z)
    assert np.isclose(eta[10, 0], emax_x)
    assert np.isclose(eta[0, 0], emax_z + emax_x)
    assert np.isclose(eta[2, 10], emax_z * (3 / 5) ** 2)      # rho = 3
    assert np.isclose(eta[19, 10], emax_z)                     # last row, rho = pad
