"""GPU parity of the CUDA path against the FP64 oracle (needs a GB300).

Every comparison runs the same seeded inputs (from ``workloads``) through the
C ABI and through ``oracle``.  Tolerances (relative L2 on the interior):
Born data and migration 2e-5 on the small grids and 1e-4 on the full 2500-step
workload (FP32 round-off grows with the number of steps), H dm 1e-4 with FP32
checkpoints and 2e-3 with 16-bit checkpoints, FP32 dot-product mismatch 1e-5.
"""
import numpy as np
import pytest

from oracle.wave import problem_from_workload
from workloads import data_noise, gaussian_bumps, make_config, mini_config

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
def cfg1():
    wl = make_config(1)
    prob = problem_from_workload(wl)
    dm = wl.trials[0].astype(np.float64)
    born = np.stack([prob.born(s, dm) for s in range(wl.ns)])              # (ns, nt, nr)
    r = born + 0.1 * np.std(born) * data_noise(born.shape, 1003).astype(np.float64)
    adj = sum(prob.adjoint(s, r[s]) for s in range(wl.ns))
    hes = sum(prob.adjoint(s, born[s]) for s in range(wl.ns))
    return wl, prob, born, r, adj, hes


def test_born_data_config1(cuda_device, cfg1):
    wl, prob, born, r, adj, hes = cfg1
    p = make_probe(wl)
    d = p.apply_F(dev(wl.trials)).cpu().numpy()[0]
    for s in range(wl.ns):
        assert rel(d[s], born[s]) < 2e-5, s


def test_migration_config1(cuda_device, cfg1):
    wl, prob, born, r, adj, hes = cfg1
    p = make_probe(wl)
    img = p.apply_Fadj(dev(r[None])).cpu().numpy()[0]
    assert rel(img, adj) < 2e-5


@pytest.mark.parametrize("snap,tol", [("fp32", 1e-4), ("bf16", 2e-3), ("fp16", 2e-3), ("history", 1e-4)])
def test_hessian_config1(cuda_device, cfg1, snap, tol):
    wl, prob, born, r, adj, hes = cfg1
    p = make_probe(wl, snapshot_dtype="fp32" if snap == "history" else snap)
    if snap == "history":
        p.set_option("dtt_history", 1)          # Dtt u^n of every step kept, no recomputation
    hd = p.apply_H(dev(wl.trials)).cpu().numpy()[0]
    assert rel(hd, hes) < tol


def test_dot_product_fp32_config1(cuda_device, cfg1):
    wl, *_ = cfg1
    p = make_probe(wl)
    dm = dev(wl.trials)
    d = p.apply_F(dm)
    r = dev(d.cpu().numpy() + np.float32(np.std(d.cpu().numpy())) * data_noise(tuple(d.shape), 1013))
    img = p.apply_Fadj(r)
    lhs = float(torch.sum(d.double() * r.double()))
    rhs = float(torch.sum(dm.double() * img.double()))
    assert abs(lhs - rhs) / max(abs(lhs), abs(rhs)) < 1e-5


def _ragged_workload(seed=7):
    """Grid that is not a multiple of the tile, receivers anywhere (with repeats)."""
    rng = np.random.default_rng(seed)
    wl = mini_config(2, shape=(37, 53), nt=150, ns=5, pad=5, p=1)
    rec = np.stack([rng.integers(0, 37, 40), rng.integers(0, 53, 40)], 1).astype(np.int32)
    rec = np.concatenate([rec, rec[:5]])                       # receivers sharing nodes
    wl.rec = rec
    wl.src = np.array([[0, 0], [36, 52], [18, 1], [3, 50], [20, 26]], np.int32)
    dms = np.stack([gaussian_bumps(wl.shape, wl.h, 900 + k, n=12, sigma_m=12.0) for k in range(3)])
    wl.trials = (dms * 0.05 * wl.m0.mean()).astype(np.float32)
    return wl


@pytest.fixture(scope="module")
def ragged():
    wl = _ragged_workload()
    prob = problem_from_workload(wl)
    ref = np.stack([prob.hessian(t.astype(np.float64)) for t in wl.trials])
    return wl, ref


@pytest.mark.parametrize("opts", [
    {},
    {"tile_z": 32},
    {"shot_wave": 2},
    {"shot_group": 1},
    {"shot_group": 3, "tile_z": 32},
    {"shot_wave": 3, "shot_group": 2},
    {"pipeline": 0},
    {"pipeline": 3, "shot_group": 3},
    {"pipeline": 3, "shot_wave": 2, "shot_group": 1},
    {"pipeline": 2, "pipe_rows": 1, "shot_group": 2},
    {"pipeline": 3, "pipe_rows": 2, "shot_wave": 3},
    {"pipe_rows": 2, "shot_wave": 2, "shot_group": 1, "dtt_history": 1},
    {"pipeline": 2, "pipe_rows": 1, "pipe_rows_adj": 2, "shot_group": 3},
    {"pipeline": 3, "pipeline_adj": 0, "pipe_rows": 2, "shot_wave": 4},
    {"dtt_history": 1},
    {"dtt_history": 1, "pipeline": 0, "shot_wave": 2},
    {"use_graph": 1},
    {"use_graph": 1, "shot_wave": 2, "dtt_history": 1},
])
def test_hessian_ragged_grid_and_launch_shapes(cuda_device, ragged, opts):
    wl, ref = ragged
    p = make_probe(wl)
    for k, v in opts.items():
        p.set_option(k, v)
    hd = p.apply_H(dev(wl.trials)).cpu().numpy()
    for b in range(3):
        assert rel(hd[b], ref[b]) < 1e-4, (opts, b)
    again = p.apply_H(dev(wl.trials)).cpu().numpy()      # second call (a replayed graph if captured)
    assert np.array_equal(again, hd)


def test_kernel_variants_give_identical_bits(cuda_device, ragged):
    """Every 2D kernel family and tile shape, the Dtt history, and two time levels per launch
    (an odd number of steps and odd checkpoint segments, so single-level launches finish them)
    evaluate the same operations in the same order: F, F* and H agree bit for bit (same shot
    grouping)."""
    wl, _ = ragged
    y = dev(wl.trials)
    d0 = None
    outs = []
    for opts in [{"pipeline": 0}, {"pipeline": 2, "pipe_rows": 1}, {"pipeline": 3, "pipe_rows": 2},
                 {"pipeline": 2, "pipe_rows": 2, "use_graph": 1}, {"pipeline": 3, "pipe_rows": 1, "dtt_history": 1},
                 {"pipeline": 2, "pipe_rows": 1, "pipe_rows_adj": 2},
                 {"pipeline": 2, "pipeline_adj": 0, "pipe_rows": 2},
                 {"tblock": 2}, {"tblock": 2, "dtt_history": 1},
                 {"tblock": 2, "pipeline": 3, "pipe_rows": 1, "use_graph": 1}]:
        p = make_probe(wl)
        p.set_option("shot_group", 2)
        for k, v in opts.items():
            p.set_option(k, v)
        d = p.apply_F(y)
        if d0 is None:
            d0 = d
        assert torch.equal(d, d0), opts
        outs.append((opts, p.apply_Fadj(d0), p.apply_H(y)))
    for opts, img, hy in outs[1:]:
        assert torch.equal(img, outs[0][1]), opts
        assert torch.equal(hy, outs[0][2]), opts


@pytest.mark.parametrize("snap", ["fp32", "fp16", "bf16"])
def test_time_blocked_checkpoints_give_identical_bits(cuda_device, ragged, snap):
    """Checkpoints taken from the four-level states of the two-level forward and restored for
    the two-level recompute hold the same values as with one level per launch."""
    wl, ref = ragged
    y = dev(wl.trials)
    out = []
    for tb in (1, 2):
        p = make_probe(wl, snapshot_dtype=snap)
        p.set_option("shot_group", 2)
        p.set_option("tblock", tb)
        out.append(p.apply_H(y))
        assert p.stats()["time_block"] == tb
    assert torch.equal(out[0], out[1])
    if snap == "fp32":
        for b in range(3):
            assert rel(out[1][b].cpu().numpy(), ref[b]) < 1e-4


@pytest.mark.parametrize("opts", [{}, {"use_graph": 1}, {"use_graph": 1, "dtt_history": 1}])
def test_sweep_timing_events(cuda_device, ragged, opts):
    """PROBE_OPT_TIMING: per-sweep CUDA-event times (also from inside a replayed graph),
    formed when the statistics are read; the timed call's result is unchanged."""
    wl, ref = ragged
    p = make_probe(wl)
    for k, v in opts.items():
        p.set_option(k, v)
    y = dev(wl.trials)
    h0 = p.apply_H(y)
    p.set_option("timing", 1)
    for _ in range(2):
        h1 = p.apply_H(y)
    s = p.stats()
    assert torch.equal(h0, h1)
    assert s["ms_forward"] > 0 and s["ms_adjoint"] > 0
    if opts.get("dtt_history"):
        assert s["ms_recompute"] == 0 and s["dtt_history"] == 1
    else:
        assert s["ms_recompute"] > 0
    assert abs(s["ms_total"] - (s["ms_forward"] + s["ms_recompute"] + s["ms_adjoint"])) < 1e-6


def test_hessian_without_kahan_and_host_buffers(cuda_device, ragged):
    wl, ref = ragged
    p = make_probe(wl, kahan=False)
    hd_dev = p.apply_H(dev(wl.trials)).cpu().numpy()
    hd_host = p.apply_H(wl.trials)                             # NumPy in -> NumPy out
    assert isinstance(hd_host, np.ndarray)
    assert np.array_equal(hd_dev, hd_host)
    for b in range(3):
        assert rel(hd_host[b], ref[b]) < 1e-4


def test_nonlinear_forward_and_gradient(cuda_device):
    wl = mini_config(4, shape=(48, 60), nt=300, ns=2, pad=8)
    prob = problem_from_workload(wl)
    m = wl.extra["m_true"]
    p = make_probe(wl)
    d_gpu = p.forward_nonlinear(dev(m)).cpu().numpy()
    d_ref = np.stack([prob.forward(s, m.astype(np.float64)) for s in range(wl.ns)])
    assert rel(d_gpu, d_ref) < 2e-5
    # gradient of J at m0 for data d_ref: F*[m0] (calF[m0] - d)
    d0 = np.stack([prob.forward(s) for s in range(wl.ns)])
    resid = (d0 - d_ref).astype(np.float32)
    g_gpu = p.gradient(dev(wl.m0), dev(resid)).cpu().numpy()
    g_ref = prob.gradient(prob.m0, d_ref)
    assert rel(g_gpu, g_ref) < 1e-4


def test_invalid_inputs_report_errors(cuda_device):
    from paper_1101_3615_gb300 import ProbeError
    wl = mini_config(1, shape=(20, 22), nt=40, ns=1, pad=4)
    p = make_probe(wl)
    bad = wl.trials.copy()
    bad[0, 3, 4] = np.inf
    with pytest.raises(ProbeError) as ei:
        p.apply_H(dev(bad))
    assert ei.value.status == -5
    # the handle stays usable
    out = p.apply_H(dev(wl.trials)).cpu().numpy()
    assert np.all(np.isfinite(out))
    empty = p.apply_H(dev(np.zeros((0,) + wl.shape, np.float32)))
    assert tuple(empty.shape) == (0,) + wl.shape


@pytest.fixture(scope="module")
def cfg2():
    return make_config(2)


@pytest.fixture(scope="module")
def cfg2_oracle():
    """Oracle runs for three shots of the full workload, in spawned processes
    that work while the GPU tests run."""
    from oracle.jobs import start_pool
    pool, res = start_pool([(2, "born", 0, None), (2, "born", 31, None), (2, "born+adj", 5, 50)])
    yield res
    pool.terminate()


def test_config2_full_size_sampled_shots(cuda_device, cfg2, cfg2_oracle):
    """Full 541^2 x 2500-step workload, all 32 shots resident in one launch:
    the Born traces of two shots and the migration of one shot's data are
    compared with the oracle run for those shots alone."""
    wl = cfg2
    p = make_probe(wl)
    dm = dev(wl.trials)
    d = p.apply_F(dm).cpu().numpy()[0]
    born0, born31, (born5, img5) = cfg2_oracle.get(timeout=3000)
    # 2500 FP32 steps on the full grid: the FP32 tolerance of H dm applies
    assert rel(d[0], born0) < 1e-4
    assert rel(d[31], born31) < 1e-4
    assert rel(d[5], born5) < 1e-4
    r = np.zeros((1, wl.ns, wl.nt, wl.nr), np.float32)
    r[0, 5] = born5.astype(np.float32)
    img = p.apply_Fadj(dev(r)).cpu().numpy()[0]
    assert rel(img, img5) < 1e-4


@pytest.mark.parametrize("snap", ["fp16", "bf16"])
def test_config2_full_size_16bit_vs_oracle(cuda_device, cfg2, cfg2_oracle, snap):
    """The batched path the bench times (all 32 shots resident, 16-bit checkpoints, autotuned
    kernels, CUDA graphs) at full size against the oracle: F* applied to shot 5's Born traces,
    the other shots' data zero, is that shot's term F_5^T F_5 dm of H dm, which the oracle
    computes alone; within the 16-bit bound."""
    wl = cfg2
    p = make_probe(wl, snapshot_dtype=snap)
    p.set_option("use_graph", 1)
    dm = dev(wl.trials)
    d = p.apply_F(dm)
    r = torch.zeros_like(d)
    r[0, 5] = d[0, 5]
    img = p.apply_Fadj(r).cpu().numpy()[0]
    _, _, (_, img5) = cfg2_oracle.get(timeout=3000)
    assert rel(img, img5) < 2e-3


def test_config2_full_size_dot_and_hessian_consistency(cuda_device, cfg2):
    wl = cfg2
    p = make_probe(wl)
    dm = dev(wl.trials)
    d = p.apply_F(dm)
    img = p.apply_Fadj(d)
    hd = p.apply_H(dm)
    lhs = float(torch.sum(d.double() ** 2))
    rhs = float(torch.sum(dm.double() * img.double()))
    assert abs(lhs - rhs) / lhs < 1e-5
    assert rel(hd.cpu().numpy(), img.cpu().numpy()) < 1e-5
    # the bench's batched path (FP16 checkpoints, autotuned, graphs) at full size: within the
    # 16-bit bound of the FP32-checkpoint H, itself within 1e-4 of the oracle (sampled test above)
    p16 = make_probe(wl, snapshot_dtype="fp16")
    p16.set_option("use_graph", 1)
    h16 = p16.apply_H(dm)
    assert rel(h16.cpu().numpy(), hd.cpu().numpy()) < 2e-3


def test_bounded_wait_reports_timeout_and_context_survives(cuda_device):
    """A device wait that nothing satisfies ends by its time limit and is reported."""
    from paper_1101_3615_gb300 import binding
    wl = mini_config(1, shape=(24, 26), nt=60, ns=1, pad=4)
    p = make_probe(wl)
    st = binding.lib.probe_diag_wait_timeout(p.handle, 200, None)
    assert st == -4                                               # PROBE_ERR_TIMEOUT
    assert b"timed out" in binding.lib.probe_last_error(p.handle)
    out = p.apply_H(dev(wl.trials)).cpu().numpy()                 # the context still works
    ref = problem_from_workload(wl).hessian(wl.trials[0].astype(np.float64))
    assert rel(out[0], ref) < 1e-4
