"""Discrete wave operators of the oracle (FP64, test infrastructure only).

What is computed (paper, Sec. 1.1 and Sec. 2):

* forward map   calF[m]: solve m u_tt - Lap u = f_s, f_s = delta(x-s) w(t), and
  sample u at the receivers (Sec. 1.1 definition of the prediction);
* Born map      F dm = dcalF/dm [m0] dm: m0 du_tt - Lap du = -dm (u0)_tt with
  m0 (u0)_tt - Lap u0 = f_s, data = du at the receivers (Sec. 2 equations);
* migration     F* = F^T, the exact transpose of the discrete F (reverse-time
  migration, Sec. 1.1);
* normal op.    H = F* F, stacked over sources (Sec. 1.1 eq. H = F*F; Sec. 2
  "stack on ... sources");
* gradient      dJ/dm = -F*(d - calF[m]) for J = 1/2 ||d - calF[m]||^2 (Sec. 1.1).

Discretisation (readings; the paper's own solver is spectral + PML): on the
padded grid, with s = dt^2/m, a+- = 1 +- eta dt/2 and L the 8th-order Laplacian,

    u^{n+1}  = [2 u^n  - a- u^{n-1}  + s (L u^n + f^n)] / a+        n = 0..nt-2
    du^{n+1} = [2 du^n - a- du^{n-1} + s (L du^n - dm * Dtt u^n)] / a+
    Dtt u^n  = (u^{n+1} - 2 u^n + u^{n-1}) / dt^2
    d^n      = R du^n                                                n = 0..nt-1

with u^{-1} = u^0 = 0, f^n = w(n dt) / (h_1 ... h_d) at the source node, R
point sampling.  The transpose is written out step by step (lambda form):

    lam^n = 2 G lam^{n+1} + L (s G lam^{n+1}) - G' lam^{n+2} + R^T r^n
    img   = - sum_{n=0}^{nt-2} Dtt u^n * (s G lam^{n+1})     (restricted to interior)

G = 1/a+, G' = a-/a+.  The model m equals m0 in the pad (edge extension of the
interior m0 given at set-up), eta is fixed by max(c) of m0; model-space vectors
live on the interior only.
"""
from __future__ import annotations

import numpy as np

from .fd import laplacian, sponge_eta


class Problem:
    """One background model with its acquisition geometry and time axis.

    Parameters
    ----------
    m0 : interior slowness squared, shape (nz, nx) or (nz, ny, nx)
    h  : grid spacing per axis (same order)
    dt, nt : time step and number of samples
    pad : sponge width in cells, added on every side
    src : (ns, ndim) interior source indices; rec : (nr, ndim) receiver indices
    wavelet : (nt,) source signature
    """

    def __init__(self, m0, h, dt, nt, pad, src, rec, wavelet, R=1e-3):
        self.m0 = np.asarray(m0, dtype=np.float64)
        self.shape = self.m0.shape
        self.ndim = self.m0.ndim
        self.h = tuple(float(x) for x in np.broadcast_to(np.asarray(h, float), (self.ndim,)))
        self.dt = float(dt)
        self.nt = int(nt)
        self.pad = int(pad)
        self.src = np.asarray(src, dtype=np.int64).reshape(-1, self.ndim)
        self.rec = np.asarray(rec, dtype=np.int64).reshape(-1, self.ndim)
        self.w = np.asarray(wavelet, dtype=np.float64)
        assert self.w.shape[0] >= self.nt
        self.pshape = tuple(n + 2 * self.pad for n in self.shape)
        self.cmax = float(1.0 / np.sqrt(self.m0.min()))
        self.eta = sponge_eta(self.shape, self.pad, self.h, self.cmax, R)
        self.ap = 1.0 + 0.5 * self.dt * self.eta
        self.am = 1.0 - 0.5 * self.dt * self.eta
        self.inner = tuple(slice(self.pad, self.pad + n) for n in self.shape)
        self.vol_inv = 1.0 / float(np.prod(self.h))
        self.src_p = tuple((self.src + self.pad).T)
        self.rec_p = tuple((self.rec + self.pad).T)
        self.rec_flat = np.ravel_multi_index(self.rec_p, self.pshape)

    @property
    def ns(self):
        return self.src.shape[0]

    @property
    def nr(self):
        return self.rec.shape[0]

    # -- small helpers --------------------------------------------------------
    def padded_model(self, m_int=None):
        """Padded model: m in the interior, edge-extended m0 in the pad."""
        mp = np.pad(self.m0, self.pad, mode="edge")
        if m_int is not None:
            mp[self.inner] = np.asarray(m_int, dtype=np.float64)
        return mp

    def embed(self, a_int):
        """Interior model-space array(s) -> padded grid, zero in the pad."""
        a_int = np.asarray(a_int, dtype=np.float64)
        lead = a_int.shape[:a_int.ndim - self.ndim]
        out = np.zeros(lead + self.pshape)
        out[(Ellipsis,) + self.inner] = a_int
        return out

    def restrict(self, a_pad):
        return a_pad[(Ellipsis,) + self.inner]

    def lap(self, u):
        return laplacian(u, self.h)

    def _sample(self, u):
        """R u: values at receiver nodes, shape (..., nr)."""
        return u[(Ellipsis,) + self.rec_p]

    def _inject_adjoint(self, lam, r_n):
        """lam += R^T r_n (accumulating receivers that share a node)."""
        flat = lam.reshape(-1, int(np.prod(self.pshape)))
        rn = np.asarray(r_n, dtype=np.float64).reshape(-1, self.nr)
        for b in range(flat.shape[0]):
            np.add.at(flat[b], self.rec_flat, rn[b])

    def _source_rhs(self, shot, n, rhs):
        idx = tuple(int(c[shot]) for c in self.src_p)
        rhs[idx] += self.w[n] * self.vol_inv

    # -- forward maps -----------------------------------------------------------
    def incident_history(self, shot, m_int=None):
        """All incident-field snapshots u^0..u^{nt-1} for one shot, shape (nt, *pshape)."""
        s = self.dt ** 2 / self.padded_model(m_int)
        U = np.zeros((self.nt,) + self.pshape)
        u_prev = np.zeros(self.pshape)
        u = np.zeros(self.pshape)
        for n in range(self.nt - 1):
            rhs = self.lap(u)
            self._source_rhs(shot, n, rhs)
            u_next = (2.0 * u - self.am * u_prev + s * rhs) / self.ap
            u_prev, u = u, u_next
            U[n + 1] = u
        return U

    def forward(self, shot, m_int=None):
        """Nonlinear prediction calF[m] for one shot: (nt, nr) receiver traces."""
        s = self.dt ** 2 / self.padded_model(m_int)
        d = np.zeros((self.nt, self.nr))
        u_prev = np.zeros(self.pshape)
        u = np.zeros(self.pshape)
        for n in range(self.nt - 1):
            rhs = self.lap(u)
            self._source_rhs(shot, n, rhs)
            u_next = (2.0 * u - self.am * u_prev + s * rhs) / self.ap
            u_prev, u = u, u_next
            d[n + 1] = self._sample(u)
        return d

    def born(self, shot, dm, m_int=None):
        """Born data F dm for one shot; dm is (..., *shape) -> (..., nt, nr)."""
        mp = self.padded_model(m_int)
        s = self.dt ** 2 / mp
        dmp = self.embed(dm)
        lead = dmp.shape[:dmp.ndim - self.ndim]
        d = np.zeros(lead + (self.nt, self.nr))
        u_prev = np.zeros(self.pshape)
        u = np.zeros(self.pshape)
        du_prev = np.zeros(lead + self.pshape)
        du = np.zeros(lead + self.pshape)
        for n in range(self.nt - 1):
            rhs = self.lap(u)
            self._source_rhs(shot, n, rhs)
            u_next = (2.0 * u - self.am * u_prev + s * rhs) / self.ap
            dtt = (u_next - 2.0 * u + u_prev) / self.dt ** 2
            du_next = (2.0 * du - self.am * du_prev
                       + s * (self.lap(du) - dmp * dtt)) / self.ap
            u_prev, u = u, u_next
            du_prev, du = du, du_next
            d[..., n + 1, :] = self._sample(du)
        return d

    # -- the transpose ---------------------------------------------------------
    def _dtt_segments(self, shot, m_int, ckpt):
        """Yield (n, Dtt u^n) for n = nt-2 down to 0.

        ckpt=None stores the whole history; ckpt=K keeps the states
        (u^{kK}, u^{kK-1}) and recomputes each segment in reverse order.
        """
        nt = self.nt
        if ckpt is None:
            U = self.incident_history(shot, m_int)
            for n in range(nt - 2, -1, -1):
                um1 = U[n - 1] if n >= 1 else 0.0
                yield n, (U[n + 1] - 2.0 * U[n] + um1) / self.dt ** 2
            return
        K = int(ckpt)
        s = self.dt ** 2 / self.padded_model(m_int)
        states = {}
        u_prev = np.zeros(self.pshape)
        u = np.zeros(self.pshape)
        for n in range(nt - 1):
            if n % K == 0:
                states[n] = (u.copy(), u_prev.copy())
            rhs = self.lap(u)
            self._source_rhs(shot, n, rhs)
            u_next = (2.0 * u - self.am * u_prev + s * rhs) / self.ap
            u_prev, u = u, u_next
        for k0 in sorted(states, reverse=True):
            u, u_prev = (a.copy() for a in states[k0])
            k1 = min(k0 + K, nt - 1)
            seg = {}
            for n in range(k0, k1):
                rhs = self.lap(u)
                self._source_rhs(shot, n, rhs)
                u_next = (2.0 * u - self.am * u_prev + s * rhs) / self.ap
                seg[n] = (u_next - 2.0 * u + u_prev) / self.dt ** 2
                u_prev, u = u, u_next
            for n in range(k1 - 1, k0 - 1, -1):
                yield n, seg[n]

    def adjoint(self, shot, r, m_int=None, ckpt=None):
        """Migration F^T r for one shot; r is (..., nt, nr) -> image (..., *shape)."""
        mp = self.padded_model(m_int)
        s = self.dt ** 2 / mp
        G = 1.0 / self.ap
        Gp = self.am / self.ap
        sG = s * G
        r = np.asarray(r, dtype=np.float64)
        lead = r.shape[:-2]
        lam1 = np.zeros(lead + self.pshape)    # lam^{n+1}
        lam2 = np.zeros(lead + self.pshape)    # lam^{n+2}
        img = np.zeros(lead + self.pshape)
        dtt_iter = self._dtt_segments(shot, m_int, ckpt)
        for n in range(self.nt - 1, -1, -1):
            lam = 2.0 * G * lam1 + self.lap(sG * lam1) - Gp * lam2
            self._inject_adjoint(lam, r[..., n, :])
            if n <= self.nt - 2:
                n_chk, dtt = next(dtt_iter)
                assert n_chk == n
                img -= dtt * (sG * lam1)
            lam2, lam1 = lam1, lam
        return self.restrict(img)

    # -- composite operators -----------------------------------------------------
    def hessian(self, dm, shots=None, m_int=None, ckpt=None):
        """H dm = sum over shots of F_s^T F_s dm (interior in, interior out)."""
        shots = range(self.ns) if shots is None else shots
        out = 0.0
        for s_ in shots:
            out = out + self.adjoint(s_, self.born(s_, dm, m_int), m_int, ckpt)
        return out

    def misfit(self, m_int, d_obs, shots=None):
        """J[m] = 1/2 sum over shots ||d - calF[m]||^2 (plain Euclidean sum)."""
        shots = range(self.ns) if shots is None else shots
        return 0.5 * sum(float(np.sum((np.asarray(d_obs[i], float) - self.forward(i, m_int)) ** 2))
                         for i in shots)

    def gradient(self, m_int, d_obs, shots=None, ckpt=None):
        """dJ/dm = -F*[m] (d - calF[m]) summed over shots (Sec. 1.1)."""
        shots = range(self.ns) if shots is None else shots
        g = 0.0
        for i in shots:
            resid = np.asarray(d_obs[i], float) - self.forward(i, m_int)
            g = g - self.adjoint(i, resid, m_int, ckpt)
        return g


def problem_from_workload(wl, R=1e-3) -> Problem:
    """Build a Problem from a ``workloads.Workload`` (inputs cast to FP64 as-is)."""
    return Problem(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet, R=R)


def _hessian_shot_worker(args):
    wl_fields, dm, shot, ckpt = args
    p = Problem(*wl_fields)
    return p.adjoint(shot, p.born(shot, dm), ckpt=ckpt)


def hessian_parallel(prob: Problem, dm, shots=None, workers=1, ckpt=None):
    """H dm with shots distributed over a spawn-started process pool."""
    shots = list(range(prob.ns) if shots is None else shots)
    if workers <= 1 or len(shots) <= 1:
        return prob.hessian(dm, shots=shots, ckpt=ckpt)
    import multiprocessing as mp
    fields = (prob.m0, prob.h, prob.dt, prob.nt, prob.pad, prob.src, prob.rec, prob.w)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, len(shots))) as pool:
        parts = pool.map(_hessian_shot_worker, [(fields, dm, s, ckpt) for s in shots])
    return sum(parts)
