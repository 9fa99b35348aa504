"""Thin ctypes binding of the C ABI declared in ``include/probe.h``.

Argument marshalling only: every arithmetic step runs in the CUDA library.
The low-level functions carry the C names (``probe_create``, ``probe_apply_H``
...) and take raw pointers; :class:`Probe` wraps a handle and accepts torch
tensors (device or host) or NumPy arrays (host).  If the shared library is
missing the import of this module raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libprobe.so")

PROBE_OK = 0
STATUS = {0: "PROBE_OK", -1: "PROBE_ERR_ARG", -2: "PROBE_ERR_CUDA", -3: "PROBE_ERR_OOM",
          -4: "PROBE_ERR_TIMEOUT", -5: "PROBE_ERR_NONFINITE", -6: "PROBE_ERR_STATE"}
SNAP = {"fp32": 0, "bf16": 1, "fp16": 2}
SOLVE = {"gd": 0, "cg": 1}
OPT = {"check_finite": 1, "shot_wave": 2, "shot_group": 3, "use_graph": 4, "timing": 5, "tile_z": 6,
       "pipeline": 7, "dtt_history": 8, "autotune": 9, "pipe_rows": 10, "pipeline_adj": 11, "pipe_rows_adj": 12,
       "cluster3d": 13, "tblock": 14, "planes3d": 15, "overlap3d": 16}


class probe_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3), ("pad", C.c_int),
                ("snapshot_dtype", C.c_int), ("kahan", C.c_int), ("ckpt_stride", C.c_int)]


class probe_basis(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nspatial", C.c_int), ("spatial", C.POINTER(C.c_int)),
                ("nangular", C.c_int), ("angular", C.POINTER(C.c_int)), ("nradial", C.c_int),
                ("L", C.c_double), ("order", C.c_double), ("fft_pad", C.c_int)]


class probe_stats(C.Structure):
    _fields_ = [("ms_forward", C.c_double), ("ms_recompute", C.c_double),
                ("ms_adjoint", C.c_double), ("ms_total", C.c_double),
                ("launches_forward", C.c_longlong), ("launches_recompute", C.c_longlong),
                ("launches_adjoint", C.c_longlong), ("launches_total", C.c_longlong),
                ("cell_updates_forward", C.c_double), ("cell_updates_recompute", C.c_double),
                ("cell_updates_adjoint", C.c_double), ("bytes_forward", C.c_double),
                ("bytes_recompute", C.c_double), ("bytes_adjoint", C.c_double),
                ("shot_wave", C.c_int), ("shot_group", C.c_int), ("tile_z", C.c_int),
                ("ckpt_stride", C.c_int), ("pipeline_forward", C.c_int),
                ("pipeline_adjoint", C.c_int), ("dtt_history", C.c_int), ("pipeline_rows", C.c_int),
                ("pipeline_rows_adjoint", C.c_int), ("time_block", C.c_int), ("planes_3d", C.c_int),
                ("pipeline_incident", C.c_int)]


class ProbeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build() or python -m paper_1101_3615_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    P, VP, I, D = C.c_void_p, C.c_void_p, C.c_int, C.c_double
    sig = {
        "probe_create": (I, [C.POINTER(P), C.POINTER(probe_grid), VP, I, VP, I, VP, VP, I, D]),
        "probe_apply_F": (I, [P, VP, VP, I, VP]),
        "probe_apply_F_noalloc": (I, [P, VP, VP, I, VP]),
        "probe_apply_Fadj": (I, [P, VP, VP, I, VP]),
        "probe_apply_H": (I, [P, VP, VP, I, VP]),
        "probe_apply_H_group": (I, [C.POINTER(P), I, C.POINTER(VP), C.POINTER(VP), C.POINTER(I), VP]),
        "probe_fit": (I, [P, C.POINTER(probe_basis), VP, VP, I, VP, VP, VP]),
        "probe_apply_precond": (I, [P, C.POINTER(probe_basis), VP, VP, VP, VP]),
        "probe_solve": (I, [P, I, I, C.POINTER(probe_basis), VP, VP, VP, VP, VP, VP]),
        "probe_krylov_trials": (I, [P, VP, I, VP, VP, VP]),
        "probe_forward_nonlinear": (I, [P, VP, VP, VP]),
        "probe_gradient": (I, [P, VP, VP, VP, VP]),
        "probe_set_option": (I, [P, I, C.c_longlong]),
        "probe_diag_wait_timeout": (I, [P, I, VP]),
        "probe_get_stats": (I, [P, C.POINTER(probe_stats)]),
        "probe_sizes": (I, [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(I),
                            C.POINTER(I), C.POINTER(I)]),
        "probe_last_error": (C.c_char_p, [P]),
        "probe_destroy": (None, [P]),
        "probe_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# --- low-level functions with the C names -----------------------------------------
probe_create = lib.probe_create
probe_apply_F = lib.probe_apply_F
probe_apply_F_noalloc = lib.probe_apply_F_noalloc
probe_apply_Fadj = lib.probe_apply_Fadj
probe_apply_H = lib.probe_apply_H
probe_apply_H_group = lib.probe_apply_H_group
probe_fit = lib.probe_fit
probe_apply_precond = lib.probe_apply_precond
probe_solve = lib.probe_solve
probe_krylov_trials = lib.probe_krylov_trials
probe_forward_nonlinear = lib.probe_forward_nonlinear
probe_gradient = lib.probe_gradient
probe_set_option = lib.probe_set_option
probe_diag_wait_timeout = lib.probe_diag_wait_timeout
probe_get_stats = lib.probe_get_stats
probe_sizes = lib.probe_sizes
probe_last_error = lib.probe_last_error
probe_destroy = lib.probe_destroy
probe_version = lib.probe_version


def _check(status, handle=None):
    if status != PROBE_OK:
        msg = lib.probe_last_error(handle)
        raise ProbeError(status, msg.decode() if msg else "")


# --- marshalling helpers ------------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.float32):
    """(pointer, keepalive) for a torch tensor or array-like; arrays made contiguous."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return C.c_void_p(a.ctypes.data), a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _empty_like_io(ref, shape, dtype=np.float32):
    """Output buffer on the same side (device tensor / host array) as ``ref``."""
    if _is_torch(ref):
        import torch
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


class Basis:
    """Host description of the elementary operators B_i (mirrors probe_basis)."""

    def __init__(self, ndim, spatial, angular, nradial, L, order=-1.0, fft_pad=16):
        self.ndim = int(ndim)
        self.spatial = np.ascontiguousarray(np.asarray(spatial, dtype=np.int32).reshape(-1, ndim))
        self.angular = np.ascontiguousarray(np.asarray(angular, dtype=np.int32).reshape(-1))
        self.nradial = int(nradial)
        self.L = float(L)
        self.order = float(order)
        self.fft_pad = int(fft_pad)

    @property
    def P(self):
        return len(self.spatial) * len(self.angular) * self.nradial

    def c_struct(self):
        return probe_basis(self.ndim, len(self.spatial),
                           self.spatial.ctypes.data_as(C.POINTER(C.c_int)), len(self.angular),
                           self.angular.ctypes.data_as(C.POINTER(C.c_int)), self.nradial,
                           self.L, self.order, self.fft_pad)


class Probe:
    """A library handle for one background model and acquisition geometry.

    Shapes follow the C ABI: model space ``shape`` (interior, depth first),
    data ``[nb, ns, nt, nr]``.  Inputs may be CUDA tensors (outputs are then
    CUDA tensors) or host arrays (outputs are NumPy arrays; the library copies).
    """

    def __init__(self, m0, h, dt, nt, pad, src, rec, wavelet, snapshot_dtype="fp32", kahan=True,
                 ckpt_stride=0):
        m0 = np.asarray(m0, dtype=np.float32) if not _is_torch(m0) else m0
        self.shape = tuple(m0.shape)
        ndim = len(self.shape)
        g = probe_grid()
        g.ndim = ndim
        for a in range(ndim):
            g.n[a] = int(self.shape[a])
            g.h[a] = float(np.broadcast_to(np.asarray(h, float), (ndim,))[a])
        g.pad = int(pad)
        g.snapshot_dtype = SNAP[snapshot_dtype] if isinstance(snapshot_dtype, str) else int(snapshot_dtype)
        g.kahan = 1 if kahan else 0
        g.ckpt_stride = int(ckpt_stride)
        src = np.ascontiguousarray(np.asarray(src, dtype=np.int32).reshape(-1, ndim))
        rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int32).reshape(-1, ndim))
        w = np.ascontiguousarray(np.asarray(wavelet, dtype=np.float32)[:nt])
        pm, keep = _ptr(m0)
        self.handle = C.c_void_p()
        st = lib.probe_create(C.byref(self.handle), C.byref(g), pm, src.shape[0],
                              C.c_void_p(src.ctypes.data), rec.shape[0], C.c_void_p(rec.ctypes.data),
                              C.c_void_p(w.ctypes.data), int(nt), float(dt))
        _check(st, None)
        self.ns, self.nr, self.nt = src.shape[0], rec.shape[0], int(nt)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and h.value:
            lib.probe_destroy(h)
            self.handle = C.c_void_p()

    close = __del__

    @property
    def n_model(self):
        return int(np.prod(self.shape))

    def set_option(self, name, value):
        _check(lib.probe_set_option(self.handle, OPT[name] if isinstance(name, str) else int(name),
                                    int(value)), self.handle)

    def stats(self):
        s = probe_stats()
        _check(lib.probe_get_stats(self.handle, C.byref(s)), self.handle)
        return {k: getattr(s, k) for k, _ in probe_stats._fields_}

    def _nb(self, x, trailing):
        n = int(np.prod(x.shape)) // int(np.prod(trailing))
        if n * int(np.prod(trailing)) != int(np.prod(x.shape)):
            raise ValueError(f"array of shape {tuple(x.shape)} is not a batch of {trailing}")
        return n

    def apply_F(self, dm, out=None, stream=None):
        nb = self._nb(dm, self.shape)
        out = _empty_like_io(dm, (nb, self.ns, self.nt, self.nr)) if out is None else out
        a, ka = _ptr(dm)
        b, kb = _ptr(out)
        _check(lib.probe_apply_F(self.handle, a, b, nb, _stream(stream)), self.handle)
        return out

    def apply_F_noalloc(self, dm, out, stream=None):
        """probe_apply_F_noalloc: dm and out must be CUDA tensors (the call allocates nothing)."""
        if not (_is_torch(dm) and dm.is_cuda and _is_torch(out) and out.is_cuda):
            raise ValueError("apply_F_noalloc takes CUDA tensors for dm and out")
        nb = self._nb(dm, self.shape)
        a, ka = _ptr(dm)
        b, kb = _ptr(out)
        _check(lib.probe_apply_F_noalloc(self.handle, a, b, nb, _stream(stream)), self.handle)
        return out

    def apply_Fadj(self, d, out=None, stream=None):
        nb = self._nb(d, (self.ns, self.nt, self.nr))
        out = _empty_like_io(d, (nb,) + self.shape) if out is None else out
        a, ka = _ptr(d)
        b, kb = _ptr(out)
        _check(lib.probe_apply_Fadj(self.handle, a, b, nb, _stream(stream)), self.handle)
        return out

    def apply_H(self, dm, out=None, stream=None):
        nb = self._nb(dm, self.shape)
        out = _empty_like_io(dm, (nb,) + self.shape) if out is None else out
        a, ka = _ptr(dm)
        b, kb = _ptr(out)
        _check(lib.probe_apply_H(self.handle, a, b, nb, _stream(stream)), self.handle)
        return out

    def forward_nonlinear(self, m, out=None, stream=None):
        out = _empty_like_io(m, (self.ns, self.nt, self.nr)) if out is None else out
        a, ka = _ptr(m)
        b, kb = _ptr(out)
        _check(lib.probe_forward_nonlinear(self.handle, a, b, _stream(stream)), self.handle)
        return out

    def gradient(self, m, resid, out=None, stream=None):
        out = _empty_like_io(m, self.shape) if out is None else out
        a, ka = _ptr(m)
        r, kr = _ptr(resid)
        b, kb = _ptr(out)
        _check(lib.probe_gradient(self.handle, a, r, b, _stream(stream)), self.handle)
        return out

    def fit(self, basis: Basis, y, Hy, stream=None):
        p = self._nb(y, self.shape)
        coeffs = np.zeros(basis.P, dtype=np.float64)
        resid = np.zeros(1, dtype=np.float64)
        bs = basis.c_struct()
        a, ka = _ptr(y)
        b, kb = _ptr(Hy)
        _check(lib.probe_fit(self.handle, C.byref(bs), a, b, p, C.c_void_p(coeffs.ctypes.data),
                             C.c_void_p(resid.ctypes.data), _stream(stream)), self.handle)
        return coeffs, float(resid[0])

    def apply_precond(self, basis: Basis, coeffs, img, out=None, stream=None):
        out = _empty_like_io(img, self.shape) if out is None else out
        bs = basis.c_struct()
        c, kc = _ptr(coeffs, np.float64)
        a, ka = _ptr(img)
        b, kb = _ptr(out)
        _check(lib.probe_apply_precond(self.handle, C.byref(bs), c, a, b, _stream(stream)), self.handle)
        return out

    def solve(self, rhs, iters, method="cg", x0=None, basis: Basis = None, coeffs=None, stream=None):
        """probe_solve: iterate on H x = rhs (rhs = F*d).  Returns (x, resid, done): the last
        iterate (same side as rhs), the residual norms ||rhs - H x_k|| for k = 0..done, and the
        number of iterations performed."""
        if x0 is None:
            x = _empty_like_io(rhs, self.shape)
            x[...] = 0
        else:
            x = x0.clone() if _is_torch(x0) else np.array(x0, dtype=np.float32)
        resid = np.zeros(int(iters) + 1, dtype=np.float64)
        done = C.c_int(0)
        bs = basis.c_struct() if basis is not None else None
        c, kc = _ptr(coeffs, np.float64) if coeffs is not None else (None, None)
        a, ka = _ptr(rhs)
        b, kb = _ptr(x)
        _check(lib.probe_solve(self.handle, SOLVE[method], int(iters), C.byref(bs) if bs is not None else None,
                               c, a, b, C.c_void_p(resid.ctypes.data), C.byref(done), _stream(stream)),
               self.handle)
        return x, resid[:done.value + 1], done.value


    def krylov_trials(self, rhs, n, stream=None):
        """probe_krylov_trials: the Kn trial functions y_1 = rhs/||rhs||, y_{j+1} = H y_j/||H y_j||
        and their H applications; returns (y, Hy), each [n, *shape] on the side of rhs."""
        y = _empty_like_io(rhs, (int(n),) + self.shape)
        x = _empty_like_io(rhs, (int(n),) + self.shape)
        a, ka = _ptr(rhs)
        b, kb = _ptr(y)
        c, kc = _ptr(x)
        _check(lib.probe_krylov_trials(self.handle, a, int(n), b, c, _stream(stream)), self.handle)
        return y, x


def apply_H_group(probes, dms, outs=None, stream=None):
    """probe_apply_H_group over several handles (one launch sequence for all models)."""
    k = len(probes)
    outs = [(_empty_like_io(d, tuple(d.shape)) if outs is None else outs[i]) for i, d in enumerate(dms)]
    keep = []
    hs = (C.c_void_p * k)(*[p.handle.value for p in probes])
    ins = (C.c_void_p * k)()
    ots = (C.c_void_p * k)()
    nbs = (C.c_int * k)()
    for i, (p, d, o) in enumerate(zip(probes, dms, outs)):
        a, ka = _ptr(d)
        b, kb = _ptr(o)
        keep += [ka, kb]
        ins[i] = a.value
        ots[i] = b.value
        nbs[i] = p._nb(d, p.shape)
    st = lib.probe_apply_H_group(hs, k, ins, ots, nbs, _stream(stream))
    _check(st, probes[0].handle)
    return outs
