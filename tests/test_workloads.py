"""Host-side checks of the seeded synthetic inputs (no method arithmetic here)."""
import numpy as np
import pytest

from workloads import CONFIG_NAMES, data_noise, make_config, mini_config

CFL_LIMIT = {2: 0.5547, 3: 0.4529}     # leapfrog + 8th-order Laplacian stability bound


@pytest.mark.parametrize("k", [1, 2, 4])
def test_configs_deterministic_and_stable(k):
    a = make_config(k)
    b = make_config(k)
    assert a.name == CONFIG_NAMES[k]
    assert np.array_equal(a.m0, b.m0) and np.array_equal(a.trials, b.trials)
    assert a.m0.dtype == np.float32 and a.trials.dtype == np.float32
    assert a.cfl() < CFL_LIMIT[a.ndim]
    assert np.all(a.src >= 0) and np.all(a.src < np.array(a.shape))
    assert np.all(a.rec >= 0) and np.all(a.rec < np.array(a.shape))
    assert a.wavelet.shape == (a.nt,)


def test_config_sizes():
    c1 = make_config(1)
    assert c1.shape == (101, 101) and c1.padded_shape == (141, 141) and c1.ns == 4
    assert c1.nr == 101 and c1.nt == 800 and c1.src.tolist() == [[2, 20], [2, 40], [2, 60], [2, 80]]
    c2 = make_config(2)
    assert c2.padded_shape == (541, 541) and c2.ns == 32 and c2.nr == 501
    assert c2.trials.shape == (1, 501, 501)
    for m, n in enumerate((301, 501, 701)):
        c3 = make_config(3, model=m)
        assert c3.shape == (n, n) and c3.ns == 64 and c3.trials.shape[0] == 8
        assert c3.cfl() < CFL_LIMIT[2]


def test_mini_configs_and_noise():
    w = mini_config(2, shape=(40, 44), nt=100, ns=3)
    assert w.shape == (40, 44) and w.nt == 100 and w.ns == 3
    assert np.array_equal(data_noise((3, 4), 7), data_noise((3, 4), 7))
    t = mini_config(1, shape=(30, 30), nt=50).trials[0]
    assert abs(t[0, 0]) < 1e-3 * np.abs(t).max()          # edge taper
