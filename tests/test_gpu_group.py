"""Several models of uneven grid sizes in one launch sequence (needs a GB300).

probe_apply_H_group advances the sweeps of all models in the same kernel
launches; each model's result must equal its own probe_apply_H (identical
arithmetic) and the FP64 oracle.  The full batched-probing workload (three
layered models 301^2 / 501^2 / 701^2, 64 shots, p = 8 trials) is run as one
group, followed by the 40-term FP64 fit of Sec. 1.4 on the 501^2 model.
"""
import numpy as np
import pytest

from oracle.symbol import Basis as OBasis
from oracle.symbol import fit as ofit
from oracle.wave import problem_from_workload
from workloads import make_config, mini_config

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_probe(wl):
    from paper_1101_3615_gb300 import Probe
    return Probe(wl.m0, wl.h, wl.dt, wl.nt, wl.pad, wl.src, wl.rec, wl.wavelet)


def test_group_matches_individual_and_oracle(cuda_device):
    from paper_1101_3615_gb300 import apply_H_group
    wls = [mini_config(3, shape=(41, 45), nt=220, ns=3, pad=6, p=1, model=0),
           mini_config(3, shape=(57, 61), nt=220, ns=5, pad=6, p=2, model=1),
           mini_config(3, shape=(33, 70), nt=220, ns=2, pad=6, p=3, model=2)]
    probes = [make_probe(w) for w in wls]
    for p in probes:      # fixed variants: the group and the solo runs sum in the same order
        p.set_option("shot_group", 4)
        p.set_option("pipeline", 2)
    dms = [torch.tensor(w.trials, device=cuda_device) for w in wls]
    outs = apply_H_group(probes, dms)
    for w, p, d, o in zip(wls, probes, dms, outs):
        solo = p.apply_H(d)
        assert torch.equal(o, solo)
    prob = problem_from_workload(wls[1])
    refs = [prob.hessian(wls[1].trials[b].astype(np.float64)) for b in range(2)]
    for b in range(2):
        assert rel(outs[1][b].cpu().numpy(), refs[b]) < 1e-4
    # autotuned and graph-captured group (variants chosen by timing): same results up to
    # the order of the image sums, twice in a row from the cached graph
    tuned = [make_probe(w) for w in wls]
    for p in tuned:
        p.set_option("use_graph", 1)
    first = apply_H_group(tuned, dms)
    again = apply_H_group(tuned, dms)
    for o, t, u in zip(outs, first, again):
        assert torch.equal(t, u)
        assert rel(t.cpu().numpy(), o.cpu().numpy()) < 1e-6
    for b in range(2):
        assert rel(first[1][b].cpu().numpy(), refs[b]) < 1e-4


def test_group_rejects_mismatched_time_axes(cuda_device):
    from paper_1101_3615_gb300 import ProbeError, apply_H_group
    a = mini_config(3, shape=(30, 30), nt=120, ns=1, pad=4, p=1)
    b = mini_config(3, shape=(30, 30), nt=140, ns=1, pad=4, p=1)
    pa, pb = make_probe(a), make_probe(b)
    with pytest.raises(ProbeError) as ei:
        apply_H_group([pa, pb], [torch.tensor(a.trials, device=cuda_device),
                                 torch.tensor(b.trials, device=cuda_device)])
    assert ei.value.status == -1


def test_config3_full_group_and_40_term_fit(cuda_device):
    from paper_1101_3615_gb300 import Basis, apply_H_group
    wls = [make_config(3, model=k) for k in range(3)]
    probes = [make_probe(w) for w in wls]
    for p in probes:
        p.set_option("check_finite", 0)
    dms = [torch.tensor(w.trials, device=cuda_device) for w in wls]
    outs = apply_H_group(probes, dms)
    torch.cuda.synchronize()
    # every model: H is symmetric positive semi-definite -> <y, H y> >= 0 per trial
    for o, d in zip(outs, dms):
        q = torch.sum(o.double() * d.double(), dim=(1, 2))
        assert torch.all(q > 0)
    # the 501^2 model alone gives the same H applications
    solo = probes[1].apply_H(dms[1])
    assert torch.equal(solo, outs[1])
    # 40-term fit (5 spatial x 4 angular x 2 radial), FP64, vs the oracle on the same arrays
    w = wls[1]
    c_mean = float(np.mean(1 / np.sqrt(w.m0.astype(np.float64))))
    L = 2 * np.pi * 30.0 / c_mean
    sp = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]
    g = Basis(2, sp, [0, 2, -2, 4], 2, L, -1.0, 16)
    c_gpu, res_gpu = probes[1].fit(g, dms[1], outs[1])
    c_orc, res_orc, cond = ofit(OBasis(w.shape, w.h, sp, [0, 2, -2, 4], 2, L, -1.0, 16),
                                w.trials, outs[1].cpu().numpy())
    assert rel(c_gpu, c_orc) < 1e-6, cond
    assert abs(res_gpu - res_orc) < 1e-6
