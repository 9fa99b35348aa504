"""3D parity of the CUDA path with the FP64 oracle (needs a GB300).

Reduced grids of the 3D recipe (layered medium, h = 10 m, dt = 0.8 ms, 10 Hz)
with sizes that are not multiples of the 64 x 16 x 32 kernel tiles, receivers
on the surface and anywhere inside, and several shot waves.  Tolerances as in
2D.  The full 256^3 workload (16 shots, p = 4, BF16 checkpoints) is checked
through properties that hold at any size: the FP32 dot test, <y, H y> > 0,
and exact recovery of a known 60-term expansion by probe_fit.
"""
import numpy as np
import pytest

from oracle.symbol import Basis as OBasis
from oracle.symbol import fit as ofit
from oracle.wave import problem_from_workload
from workloads import data_noise, gaussian_bumps, make_config, mini_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPATIAL5_3D = [(0, 0, 0), (0, 0, 1), (0, 0, -1), (1, 0, 0), (-1, 0, 0)]
ANG6 = [0, 1, 2, 3, 4, 5]


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_probe(wl, **kw):
    from paper_1101_3615_gb300 import Probe
    return Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet, **kw)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda:0")


@pytest.fixture(scope="module")
def small3d():
    wl = mini_config(5, shape=(22, 19, 27), nt=160, ns=4, pad=6, p=2)
    rng = np.random.default_rng(3)
    extra = np.stack([rng.integers(0, n, 30) for n in wl.shape], 1).astype(np.int32)
    wl.rec = np.concatenate([wl.rec, extra, extra[:4]])          # interior receivers, repeats
    prob = problem_from_workload(wl)
    dms = wl.trials.astype(np.float64)
    born = np.stack([prob.born(s, dms) for s in range(wl.ns)], axis=1)     # (p, ns, nt, nr)
    hes = np.stack([sum(prob.adjoint(s, born[b, s]) for s in range(wl.ns)) for b in range(2)])
    return wl, prob, born, hes


def test_born_data_3d(cuda_device, small3d):
    wl, prob, born, hes = small3d
    d = make_probe(wl).apply_F(dev(wl.trials)).cpu().numpy()
    for b in range(2):
        for s in range(wl.ns):
            assert rel(d[b, s], born[b, s]) < 2e-5, (b, s)


def test_forward_kernels_3d_agree(cuda_device, small3d):
    """The pipelined 3D kernels (forward, and the adjoint with its receiver injection from the
    per-segment band buffer), with the ring refilled by a producer warp (2) or by the last compute
    warp out of a slot (3), and the one-barrier-per-plane kernels (0; injection assembled in shared
    memory) run the same per-cell arithmetic: F and H agree bit for bit (no grid cell holds more
    than two receivers here, so the injection sums cannot differ in order)."""
    wl, prob, born, hes = small3d
    y = dev(wl.trials)
    out = []
    for pipe in (0, 2, 3):
        p = make_probe(wl)
        p.set_option("pipeline", pipe)
        out.append((p.apply_F(y), p.apply_H(y)))
        st = p.stats()
        assert st["pipeline_forward"] == pipe
        assert st["pipeline_incident"] == pipe
        assert st["pipeline_adjoint"] == pipe
    for o in out[1:]:
        assert torch.equal(out[0][0], o[0])
        assert torch.equal(out[0][1], o[1])
    for b in range(2):
        assert rel(out[2][1][b].cpu().numpy(), hes[b]) < 1e-4


def test_overlapped_forward_3d_gives_identical_bits(cuda_device, small3d):
    """The Born forward with the incident step n+1 on a second stream beside the Born step n (the
    incident step's Dtt plane double-buffered, events ordering each slot's writer after its last
    reader) gives the same bits as the one-stream forward, for F and for H."""
    wl, prob, born, hes = small3d
    y = dev(wl.trials)
    out = []
    for ov in (0, 1):
        p = make_probe(wl)
        p.set_option("overlap3d", ov)
        out.append((p.apply_F(y), p.apply_H(y)))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])


def test_plane_chunks_3d_give_identical_bits(cuda_device, small3d):
    """The z planes one CTA marches (32, 64, 128, or the autotuner's pick) only change how the
    grid is cut into CTAs: F and H are the same bits for every choice (34 padded planes here, so
    32 cuts the column in two)."""
    wl, prob, born, hes = small3d
    y = dev(wl.trials)
    out = []
    for zc in (32, 64, 128, 0):
        p = make_probe(wl)
        p.set_option("planes3d", zc)
        out.append((p.apply_F(y), p.apply_H(y)))
        got = p.stats()["planes_3d"]
        assert got == zc if zc else got in (32, 64, 128)
    for o in out[1:]:
        assert torch.equal(out[0][0], o[0])
        assert torch.equal(out[0][1], o[1])
    p = make_probe(wl)
    from paper_1101_3615_gb300.binding import ProbeError
    with pytest.raises(ProbeError):
        p.set_option("planes3d", 48)


def test_cluster_kernels_3d(cuda_device, small3d):
    """Thread-block-cluster kernels against the one-field-per-CTA kernels: the fused incident +
    Born step gives the same Born data bit for bit (same per-cell arithmetic, Dtt u0 exchanged in
    shared memory instead of HBM); the shot-cluster adjoint (images of 1, 2 or 4 shots summed in
    shared memory before one Kahan update) matches the oracle like the per-shot images do."""
    wl, prob, born, hes = small3d
    y = dev(wl.trials)
    p0 = make_probe(wl)
    p0.set_option("cluster3d", 0)
    d0, h0 = p0.apply_F(y), p0.apply_H(y)
    for g in (1, 2, 4):
        p1 = make_probe(wl)
        p1.set_option("cluster3d", 3)
        p1.set_option("shot_group", g)
        d1, h1 = p1.apply_F(y), p1.apply_H(y)
        assert torch.equal(d0, d1)
        assert p1.stats()["shot_group"] == g
        for b in range(2):
            assert rel(h1[b].cpu().numpy(), hes[b]) < 1e-4, (g, b)
            assert rel(h1[b].cpu().numpy(), h0[b].cpu().numpy()) < 1e-5, (g, b)


@pytest.mark.parametrize("snap,tol,wave", [("fp32", 1e-4, 0), ("fp32", 1e-4, 3), ("fp16", 2e-3, 0),
                                           ("bf16", 2e-3, 0), ("bf16", 2e-3, 3)])
def test_hessian_3d(cuda_device, small3d, snap, tol, wave):
    wl, prob, born, hes = small3d
    p = make_probe(wl, snapshot_dtype=snap)
    if wave:
        p.set_option("shot_wave", wave)
    hd = p.apply_H(dev(wl.trials)).cpu().numpy()
    for b in range(2):
        assert rel(hd[b], hes[b]) < tol, b


def test_migration_and_dot_3d(cuda_device, small3d):
    wl, prob, born, hes = small3d
    p = make_probe(wl)
    r = born[:1] + 0.2 * np.std(born) * data_noise(born[:1].shape, 5003).astype(np.float64)
    img = p.apply_Fadj(dev(r)).cpu().numpy()[0]
    ref = sum(prob.adjoint(s, r[0, s]) for s in range(wl.ns))
    assert rel(img, ref) < 2e-5
    dm = dev(wl.trials[:1])
    d = p.apply_F(dm)
    rr = dev(r.astype(np.float32))
    a = float(torch.sum(d.double() * rr.double()))
    bimg = p.apply_Fadj(rr)
    c = float(torch.sum(dm.double() * bimg.double()))
    assert abs(a - c) / max(abs(a), abs(c)) < 1e-5


def test_nonlinear_and_gradient_3d(cuda_device):
    wl = mini_config(5, shape=(20, 18, 24), nt=140, ns=4, pad=5, p=1)
    prob = problem_from_workload(wl)
    b = gaussian_bumps(wl.shape, wl.h, 321, n=8, sigma_m=20.0)
    m = (wl.m0 * (1 + 0.04 * b / np.abs(b).max())).astype(np.float32)
    p = make_probe(wl)
    d = p.forward_nonlinear(dev(m)).cpu().numpy()
    d_ref = np.stack([prob.forward(s, m.astype(np.float64)) for s in range(wl.ns)])
    assert rel(d, d_ref) < 2e-5
    resid = (d - d_ref * 0.97).astype(np.float32)
    g = p.gradient(dev(m), dev(resid)).cpu().numpy()
    g_ref = sum(prob.adjoint(s, resid[s].astype(np.float64), m_int=m.astype(np.float64)) for s in range(wl.ns))
    assert rel(g, g_ref) < 1e-4


def test_fit_and_precond_3d(cuda_device):
    """60-term basis (5 spatial x 6 harmonics x 2 radial) on a 3D grid, vs the oracle."""
    from paper_1101_3615_gb300 import Basis
    wl = mini_config(5, shape=(26, 22, 30), nt=20, ns=4, pad=4, p=2)
    c_mean = float(np.mean(1 / np.sqrt(wl.m0.astype(np.float64))))
    L = 2 * np.pi * 30.0 / c_mean
    g = Basis(3, SPATIAL5_3D, ANG6, 2, L, -1.0, 6)
    o = OBasis(wl.shape, wl.h, SPATIAL5_3D, ANG6, 2, L, -1.0, 6)
    assert g.P == 60
    rng = np.random.default_rng(8)
    c_true = rng.standard_normal(60)
    xs = wl.trials
    ys = np.stack([o.apply(c_true, x.astype(np.float64)) for x in xs]).astype(np.float32)
    p = make_probe(wl)
    c_gpu, res = p.fit(g, dev(ys), dev(xs))
    c_orc, res_o, cond = ofit(o, ys, xs)
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert rel(c_gpu, c_true) < 1e-4, cond
    img = xs[0]
    out = p.apply_precond(g, c_gpu, dev(img)).cpu().numpy()
    assert rel(out, o.apply(c_gpu, img.astype(np.float64))) < 1e-6


def test_pipeline_3d_precond_of_migrated_data(cuda_device):
    """Fit on H applications of p = 2 trials, then precondition F* d with d = F dm_ref; the GPU
    pipeline and the oracle pipeline agree on the result."""
    from paper_1101_3615_gb300 import Basis
    wl = mini_config(5, shape=(24, 20, 26), nt=150, ns=4, pad=6, p=2)
    prob = problem_from_workload(wl)
    c_mean = float(np.mean(1 / np.sqrt(wl.m0.astype(np.float64))))
    L = 2 * np.pi * 30.0 / c_mean
    g = Basis(3, SPATIAL5_3D, ANG6, 2, L, -1.0, 6)
    o = OBasis(wl.shape, wl.h, SPATIAL5_3D, ANG6, 2, L, -1.0, 6)
    p = make_probe(wl)
    y = dev(wl.trials)
    x = p.apply_H(y)
    c_gpu, _ = p.fit(g, y, x)
    dm_ref = wl.extra["dm_ref"]
    d = p.apply_F(dev(dm_ref[None]))
    mig = p.apply_Fadj(d)[0].contiguous()
    pre = p.apply_precond(g, c_gpu, mig).cpu().numpy()
    # oracle pipeline on the same trials
    xo = np.stack([prob.hessian(t.astype(np.float64)) for t in wl.trials])
    c_o, _, cond = ofit(o, wl.trials, xo.astype(np.float32))
    mig_o = sum(prob.adjoint(s, prob.born(s, dm_ref.astype(np.float64))) for s in range(wl.ns))
    pre_o = o.apply(c_o, mig_o)
    assert rel(c_gpu, c_o) < 1e-3, cond
    assert rel(pre, pre_o) < 1e-3


def test_config5_full_size_properties(cuda_device):
    """256^3 interior (296^3 padded), 16 shots, p = 4, BF16 checkpoints; FP32 dot test."""
    from paper_1101_3615_gb300 import Basis
    wl = make_config(5)
    p = make_probe(wl, snapshot_dtype="bf16")
    p.set_option("check_finite", 0)
    y = dev(wl.trials)
    x = p.apply_H(y)
    q = torch.sum(x.double() * y.double(), dim=(1, 2, 3))
    assert torch.all(q > 0)
    # 60-term fit from the four H applications is well posed
    c_mean = float(np.mean(1 / np.sqrt(wl.m0.astype(np.float64))))
    g = Basis(3, SPATIAL5_3D, ANG6, 2, 2 * np.pi * 30.0 / c_mean, -1.0, 16)
    coeffs, res = p.fit(g, y, x)
    assert np.all(np.isfinite(coeffs)) and 0.0 < res < 1.0
    del p, x
    # FP32 dot test (FP32 checkpoints: F* is then the transpose of F to round-off)
    p32 = make_probe(wl)
    p32.set_option("check_finite", 0)
    d = p32.apply_F(y[:1].contiguous())
    img = p32.apply_Fadj(d)
    a = float(torch.sum(d.double() ** 2))
    c = float(torch.sum(y[:1].double() * img.double()))
    assert abs(a - c) / a < 1e-5
