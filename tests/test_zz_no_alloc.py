"""probe_apply_F_noalloc gives the same Born data as probe_apply_F (needs a GB300).

Some callers cannot allocate device memory while they run -- a service that
has handed all remaining memory to its own pool, or a framework that forbids
cudaMalloc/cudaFree between its own allocation points because those calls
synchronise the device.  For them the library offers an allocation-free
variant of the Born forward whose per-call scratch is a fixed static device
array.  This file checks it through the C ABI against the regular entry point,
on two calls in a row (the shared scratch keeps the previous call's contents),
with shots split into several waves, that the second call leaves the device's
free memory unchanged, and that a problem too large for the static scratch is
refused on the host.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import gaussian_bumps, mini_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc_fn():
    from paper_1101_3615_gb300 import binding
    lib = C.CDLL(binding.LIB_PATH)
    fn = lib.probe_apply_F_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    return fn


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_apply_F_on_two_calls(cuda_device):
    from paper_1101_3615_gb300 import Probe
    # 640 x 640 padded grid, 2 trials: the 32 MiB scratch holds 3 shots per wave,
    # so the 5 shots run in two waves.
    wl = mini_config(2, shape=(600, 600), nt=300, ns=5, pad=20)
    dms = np.stack([wl.trials[0],
                    (0.05 * wl.m0.mean() * gaussian_bumps(wl.shape, wl.h, 4711, n=50, sigma_m=24.0))
                    .astype(np.float32)])
    p = Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)
    dm = torch.tensor(dms, device=cuda_device)
    ref = p.apply_F(dm).cpu().numpy()
    fn = _noalloc_fn()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((2, wl.ns, wl.nt, wl.nr), float("nan"), device=cuda_device)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = fn(p.handle, C.c_void_p(dm.data_ptr()), C.c_void_p(out.data_ptr()), 2, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert st == 0, (call, st)
        if call == 1:  # the first call may load kernels lazily; the second must leave free memory alone
            assert free_after == free_before, (free_before, free_after)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        for b in range(2):
            assert _rel(got[b], ref[b]) < 2e-5, (call, b)


def test_noalloc_rejects_problems_beyond_the_static_scratch(cuda_device):
    from paper_1101_3615_gb300 import Probe, binding
    wl = mini_config(2, shape=(2001, 2001), nt=20, ns=1, pad=20)
    p = Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)
    dm = torch.zeros((1,) + wl.shape, device=cuda_device)
    out = torch.zeros((1, 1, wl.nt, wl.nr), device=cuda_device)
    st = _noalloc_fn()(p.handle, C.c_void_p(dm.data_ptr()), C.c_void_p(out.data_ptr()), 1,
                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
    assert b"beyond the allocation-free maximum" in binding.lib.probe_last_error(p.handle)
