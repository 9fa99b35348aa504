"""Seeded synthetic workloads (inputs only; no method arithmetic).

The paper's experiments use the Marmousi model, which is not available here.
These seeded stand-ins follow the shapes, spacings, time axes, source/receiver
layouts and value distributions of the five workload configurations of the
matrix-probing hot path:

1. 2D 101x101, h=10 m, c(z) linear 1500->3000 m/s, dt=1 ms, nt=800, 15 Hz,
   4 shots at z=20 m, receivers at every surface node, one band-passed trial.
2. 2D 501x501, h=8 m, smoothed 12-interface layered medium, dt=0.8 ms,
   nt=2500, 12 Hz, 32 shots, dm = 200 random-sign Gaussian bumps (sigma=16 m).
3. Three layered models 301^2, 501^2, 701^2 (config-2 physics), 64 shots each,
   p=8 random-sign band-limited trials.
4. 2D 1001x1001, h=5 m, layered, dt=0.5 ms, nt=4000, 15 Hz, 16 shots,
   m_true = m0 (1 + 0.05 b) with b 200 random-sign bumps (sigma=20 m).
5. 3D 256^3, h=10 m, layered, dt=0.8 ms, nt=1500, 10 Hz, 16 shots on a 4x4
   surface grid, all 65,536 surface receivers, p=4 trials.

Conventions: all arrays are in C order with the depth axis z first, i.e.
shapes (nz, nx) or (nz, ny, nx); index tuples are (iz, ix) or (iz, iy, ix)
into the *interior* grid (the absorbing pad is added by the method, not here).
Seeds: ``seed = 1000*config + 100*model + purpose`` with purpose
0 = background, 1 = trials, 2 = bumps / perturbation, 3 = data noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CONFIG_NAMES = {
    1: "2d-101x101-nt800-4shots",
    2: "2d-501x501-nt2500-32shots",
    3: "2d-3models-301-501-701-nt2500-64shots-p8",
    4: "2d-1001x1001-nt4000-16shots-autograd",
    5: "3d-256cube-nt1500-16shots-p4",
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """One model and its acquisition, ready to hand to either implementation."""

    name: str
    shape: tuple            # interior shape, C order (nz, nx) / (nz, ny, nx)
    h: tuple                # grid spacing per axis [m], same order
    dt: float               # time step [s]
    nt: int                 # number of time samples
    pad: int                # absorbing-sponge width in cells (added on every side)
    f0: float               # Ricker peak frequency [Hz]
    m0: np.ndarray          # float32 interior background slowness squared 1/c^2
    src: np.ndarray         # int32 [ns, ndim] interior source indices
    rec: np.ndarray         # int32 [nr, ndim] interior receiver indices
    wavelet: np.ndarray     # float32 [nt] source signature w(n dt)
    trials: np.ndarray      # float32 [p, *shape] model-space inputs (dm or y)
    seed_base: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def ns(self) -> int:
        return int(self.src.shape[0])

    @property
    def nr(self) -> int:
        return int(self.rec.shape[0])

    @property
    def padded_shape(self) -> tuple:
        return tuple(n + 2 * self.pad for n in self.shape)

    def cells_padded(self) -> int:
        return int(np.prod(self.padded_shape))

    def cmax(self) -> float:
        return float(1.0 / np.sqrt(self.m0.astype(np.float64).min()))

    def cfl(self) -> float:
        return self.cmax() * self.dt / min(self.h)


# ----------------------------------------------------------------------------
# Source wavelet
# ----------------------------------------------------------------------------

def ricker(nt: int, dt: float, f0: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet (second derivative of a Gaussian, sign so that w(t0)=1).

    w(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), default t0 = 1/f0.
    """
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (np.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


# ----------------------------------------------------------------------------
# Backgrounds
# ----------------------------------------------------------------------------

def linear_background(shape, c_top=1500.0, c_bot=3000.0) -> np.ndarray:
    """m0 = 1/c^2 with c linear in depth over the interior, constant laterally."""
    nz = shape[0]
    c = c_top + (c_bot - c_top) * np.arange(nz, dtype=np.float64) / max(nz - 1, 1)
    c = c.reshape((nz,) + (1,) * (len(shape) - 1))
    return np.broadcast_to(1.0 / c**2, shape).astype(np.float32).copy()


def _gauss_smooth_1d(v: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Gaussian smoothing of a 1D profile with edge replication."""
    if sigma_cells <= 0:
        return v.copy()
    r = int(np.ceil(4 * sigma_cells))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma_cells) ** 2)
    k /= k.sum()
    vp = np.pad(v, r, mode="edge")
    return np.convolve(vp, k, mode="valid")


def layered_background(shape, hz, seed, n_interfaces=12, cmin=1500.0, cmax=4500.0,
                       sigma_m=80.0) -> np.ndarray:
    """Seeded flat-layered medium, Gaussian-smoothed in depth; returns m0 = 1/c^2.

    Interfaces at uniform random depths inside the interior, layer speeds
    U[cmin, cmax], smoothing sigma ``sigma_m`` metres.
    """
    rng = _rng(seed)
    nz = shape[0]
    depths = np.sort(rng.uniform(0, nz, size=n_interfaces))
    speeds = rng.uniform(cmin, cmax, size=n_interfaces + 1)
    z = np.arange(nz) + 0.5
    layer = np.searchsorted(depths, z)
    c = _gauss_smooth_1d(speeds[layer], sigma_m / hz)
    c = c.reshape((nz,) + (1,) * (len(shape) - 1))
    return np.broadcast_to(1.0 / c**2, shape).astype(np.float32).copy()


# ----------------------------------------------------------------------------
# Model-space trial functions and perturbations
# ----------------------------------------------------------------------------

def _edge_taper(shape, width=10) -> np.ndarray:
    """Separable raised-cosine taper that goes to zero over ``width`` edge cells."""
    w = np.ones(shape, dtype=np.float64)
    for ax, n in enumerate(shape):
        t = np.ones(n)
        m = min(width, n // 2)
        ramp = 0.5 - 0.5 * np.cos(np.pi * (np.arange(m) + 0.5) / m)
        t[:m] = ramp
        t[n - m:] = ramp[::-1]
        sh = [1] * len(shape)
        sh[ax] = n
        w *= t.reshape(sh)
    return w


def _radial_bandpass(a: np.ndarray, h, nu_lo, nu_hi) -> np.ndarray:
    """Hard radial band-pass in spatial frequency [cycles/m] on the given grid."""
    A = np.fft.fftn(a)
    nu2 = np.zeros(a.shape)
    for ax, n in enumerate(a.shape):
        f = np.fft.fftfreq(n, d=h[ax])
        sh = [1] * a.ndim
        sh[ax] = n
        nu2 = nu2 + f.reshape(sh) ** 2
    nu = np.sqrt(nu2)
    A *= (nu >= nu_lo) & (nu <= nu_hi)
    return np.real(np.fft.ifftn(A))


def _band(m0, f_lo=5.0, f_hi=25.0):
    """Map the temporal band [f_lo, f_hi] Hz to spatial frequency by nu = 2 f / c_mean."""
    c_mean = float(np.mean(1.0 / np.sqrt(m0.astype(np.float64))))
    return 2.0 * f_lo / c_mean, 2.0 * f_hi / c_mean, c_mean


def _normalise(a, m0, level=0.05):
    """Scale to RMS = level * mean(m0): a 5 % slowness-squared perturbation."""
    rms = np.sqrt(np.mean(a**2))
    return a * (level * float(np.mean(m0.astype(np.float64))) / max(rms, 1e-300))


def bandpassed_noise(m0, h, seed, p=1, f_lo=5.0, f_hi=25.0) -> np.ndarray:
    """p trials of iid N(0,1) band-passed to [2 f_lo, 2 f_hi]/c_mean cycles/m.

    Hard radial mask in the FFT of the interior, then a 10-cell cosine edge taper.
    """
    rng = _rng(seed)
    lo, hi, _ = _band(m0, f_lo, f_hi)
    tap = _edge_taper(m0.shape)
    out = []
    for _ in range(p):
        y = _radial_bandpass(rng.standard_normal(m0.shape), h, lo, hi) * tap
        out.append(_normalise(y, m0))
    return np.stack(out).astype(np.float32)


def random_sign_trials(m0, h, seed, p=8, f_lo=5.0, f_hi=25.0) -> np.ndarray:
    """p trials: sign of band-passed noise, band-passed again, tapered."""
    rng = _rng(seed)
    lo, hi, _ = _band(m0, f_lo, f_hi)
    tap = _edge_taper(m0.shape)
    out = []
    for _ in range(p):
        y = np.sign(_radial_bandpass(rng.standard_normal(m0.shape), h, lo, hi))
        y = _radial_bandpass(y, h, lo, hi) * tap
        out.append(_normalise(y, m0))
    return np.stack(out).astype(np.float32)


def white_noise_trials(m0, seed, p=1) -> np.ndarray:
    """p fields of iid N(0,1) noise on the interior, scaled like the other trials (the input of
    the H-applied white-noise trial functions y = H n)."""
    rng = _rng(seed)
    return np.stack([_normalise(rng.standard_normal(m0.shape), m0) for _ in range(p)]).astype(np.float32)


def gaussian_bumps(shape, h, seed, n=200, sigma_m=16.0, amp=1.0) -> np.ndarray:
    """Sum of n random-sign Gaussian bumps exp(-|x-x_k|^2 / 2 sigma^2) * amp.

    Centres uniform in the interior minus a 5-sigma margin (a quarter of the
    axis on grids too small for that).
    """
    rng = _rng(seed)
    h = np.asarray(h, dtype=np.float64)
    sig = sigma_m / h                       # sigma in cells per axis
    margin = np.minimum(5.0 * sig, 0.25 * (np.asarray(shape) - 1))   # clamp only on tiny grids
    centres = np.stack([rng.uniform(margin[a], shape[a] - 1 - margin[a], size=n)
                        for a in range(len(shape))], axis=1)
    signs = rng.choice([-1.0, 1.0], size=n)
    out = np.zeros(shape, dtype=np.float64)
    r = np.ceil(5.0 * sig).astype(int)
    for k in range(n):
        lo = [max(int(np.floor(centres[k, a])) - r[a], 0) for a in range(len(shape))]
        hi = [min(int(np.ceil(centres[k, a])) + r[a] + 1, shape[a]) for a in range(len(shape))]
        grids = np.meshgrid(*[np.arange(lo[a], hi[a]) for a in range(len(shape))],
                            indexing="ij")
        d2 = sum(((grids[a] - centres[k, a]) / sig[a]) ** 2 for a in range(len(shape)))
        sl = tuple(slice(lo[a], hi[a]) for a in range(len(shape)))
        out[sl] += signs[k] * amp * np.exp(-0.5 * d2)
    return out.astype(np.float32)


# ----------------------------------------------------------------------------
# Acquisition layouts
# ----------------------------------------------------------------------------

def _surface_sources(shape, ns, iz=2):
    nx = shape[-1]
    if len(shape) == 2:
        ix = np.round((np.arange(ns) + 0.5) * (nx - 1) / ns).astype(np.int32)
        return np.stack([np.full(ns, iz, np.int32), ix], axis=1).astype(np.int32)
    g = int(round(np.sqrt(ns)))
    assert g * g == ns, "3D source layouts are square surface grids"
    ny = shape[1]
    iy = np.round((np.arange(g) + 0.5) * (ny - 1) / g).astype(np.int32)
    ix = np.round((np.arange(g) + 0.5) * (nx - 1) / g).astype(np.int32)
    YY, XX = np.meshgrid(iy, ix, indexing="ij")
    return np.stack([np.full(ns, iz, np.int32), YY.ravel(), XX.ravel()],
                    axis=1).astype(np.int32)


def _surface_receivers(shape, iz=0):
    if len(shape) == 2:
        ix = np.arange(shape[1], dtype=np.int32)
        return np.stack([np.full_like(ix, iz), ix], axis=1).astype(np.int32)
    YY, XX = np.meshgrid(np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    return np.stack([np.full(YY.size, iz), YY.ravel(), XX.ravel()],
                    axis=1).astype(np.int32)


# ----------------------------------------------------------------------------
# The five configurations (and scaled-down variants with the same recipe)
# ----------------------------------------------------------------------------

def _cfg_params(k: int):
    if k == 1:
        return dict(shape=(101, 101), h=10.0, dt=1e-3, nt=800, f0=15.0, ns=4, bg="linear")
    if k == 2:
        return dict(shape=(501, 501), h=8.0, dt=8e-4, nt=2500, f0=12.0, ns=32, bg="layered")
    if k == 3:
        return dict(shape=(501, 501), h=8.0, dt=8e-4, nt=2500, f0=12.0, ns=64, bg="layered")
    if k == 4:
        return dict(shape=(1001, 1001), h=5.0, dt=5e-4, nt=4000, f0=15.0, ns=16, bg="layered")
    if k == 5:
        return dict(shape=(256, 256, 256), h=10.0, dt=8e-4, nt=1500, f0=10.0, ns=16,
                    bg="layered")
    raise ValueError(f"unknown config {k}")


def _build(k, model, shape, h, dt, nt, f0, ns, bg, pad=20, p=None):
    base = 1000 * k + 100 * model
    hh = (h,) * len(shape)
    if bg == "linear":
        m0 = linear_background(shape)
    else:
        m0 = layered_background(shape, h, base + 0)
    src = _surface_sources(shape, ns)
    if k == 1:
        src = np.array([[2, ix] for ix in (20, 40, 60, 80)], np.int32)
        if shape != (101, 101):     # scaled variant: keep 4 evenly spaced shots
            src = _surface_sources(shape, ns)
    rec = _surface_receivers(shape)
    w = ricker(nt, dt, f0)
    extra = {}
    if k == 1:
        trials = bandpassed_noise(m0, hh, base + 1, p=p or 1)
    elif k == 2:
        c_mean = float(np.mean(1.0 / np.sqrt(m0.astype(np.float64))))
        trials = gaussian_bumps(shape, hh, base + 2, n=200, sigma_m=16.0,
                                amp=0.05 / c_mean**2)[None]
    elif k == 3:
        trials = random_sign_trials(m0, hh, base + 1, p=p or 8)
    elif k == 4:
        b = gaussian_bumps(shape, hh, base + 2, n=200, sigma_m=20.0)
        b = b / max(float(np.abs(b).max()), 1e-30)
        extra["m_true"] = (m0.astype(np.float64) * (1.0 + 0.05 * b)).astype(np.float32)
        trials = bandpassed_noise(m0, hh, base + 1, p=p or 1)
    else:
        trials = random_sign_trials(m0, hh, base + 1, p=p or 4)
        c_mean = float(np.mean(1.0 / np.sqrt(m0.astype(np.float64))))
        extra["dm_ref"] = gaussian_bumps(shape, hh, base + 2, n=200, sigma_m=40.0,
                                         amp=0.05 / c_mean**2)
    return Workload(name=CONFIG_NAMES[k] if model == 0 else f"{CONFIG_NAMES[k]}-m{model}",
                    shape=tuple(shape), h=hh, dt=dt, nt=nt, pad=pad, f0=f0, m0=m0,
                    src=src, rec=rec, wavelet=w, trials=trials, seed_base=base, extra=extra)


def make_config(k: int, model: int = 0) -> Workload:
    """Full-size workload of configuration k (for config 3, model 0/1/2 = 301/501/701)."""
    prm = _cfg_params(k)
    if k == 3:
        n = (301, 501, 701)[model]
        prm["shape"] = (n, n)
    return _build(k, model, **prm)


def mini_config(k: int, shape=None, nt=None, ns=None, p=None, pad=None, model=0) -> Workload:
    """Scaled-down variant of configuration k with the same recipe and seeds."""
    prm = _cfg_params(k)
    if shape is not None:
        prm["shape"] = tuple(shape)
    if nt is not None:
        prm["nt"] = nt
    if ns is not None:
        prm["ns"] = ns
    kw = {}
    if pad is not None:
        kw["pad"] = pad
    wl = _build(k, model, p=p, **prm, **kw)
    wl.name = f"{wl.name}-mini{'x'.join(map(str, wl.shape))}-nt{wl.nt}-ns{wl.ns}"
    return wl


def data_noise(shape, seed, sigma=1.0) -> np.ndarray:
    """iid N(0, sigma^2) noise in data space (for the dot-product test)."""
    return (sigma * _rng(seed).standard_normal(shape)).astype(np.float32)
