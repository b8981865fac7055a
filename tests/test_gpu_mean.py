"""The Ref. [8] mode on the device (kmc_mean_run, Sec. II.3) against the oracle's
mean mode, which is pinned by the two-state Boltzmann equilibrium.

Tolerance: both sides run the same FP64 recurrence; their roots, energies and
exponentials differ by rounding only (a few ulp), and the occupation update is
a contraction, so the recorded <m_z> agree to 1e-12.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs, kmc

pytestmark = pytest.mark.gpu
KB = 1.380649e-23


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()


def _batch():
    lyss = [inputs.make_lysosome(100, 12e-9, 0.05, Keff=1.3e4, T=300.0, seed=1),   # superparamagnetic
            inputs.make_lysosome(77, 20e-9, 0.05, Keff=1.3e4, T=300.0, seed=2),    # blocked
            inputs.make_lysosome(33, 16e-9, 0.05, Keff=2e4, T=0.0, seed=3),        # T = 0
            inputs.make_lysosome(40, 14e-9, 0.05, Keff=3e4, Ms=8e5, T=310.0, seed=4)]
    lyss[1].vol = lyss[1].vol * np.linspace(0.7, 1.3, lyss[1].n)  # polydisperse
    return lyss


def test_mean_mode_matches_oracle():
    lyss = _batch()
    H = [0.02, 0.04, 0.03, 0.06]
    f, S, periods, discard = 1e5, 60, 3, 1
    g = kmc.kmc_mean_run(lyss, H, f, S, periods, discard)
    assert g.shape == (len(lyss), S * (periods - discard))
    for l, ly in enumerate(lyss):
        o = oracle.mean_run(ly.axis, ly.vol, ly.Ms, ly.Keff, ly.T, ly.tau0, H[l], f, S, periods,
                            discard)
        np.testing.assert_allclose(g[l], o, rtol=0, atol=1e-12)
    # a broadcast amplitude gives the same as a repeated one
    g1 = kmc.kmc_mean_run(lyss[:2], 0.03, f, S, 2, 1)
    g2 = kmc.kmc_mean_run(lyss[:2], [0.03, 0.03], f, S, 2, 1)
    assert np.array_equal(g1, g2)


def test_mean_mode_two_state_equilibrium():
    # superparamagnetic NPs with axes along +-z relax within a step, so every
    # recorded step sits at <m_z> = tanh(M_S V B / k_B T)
    d, K, T, Ms = 8e-9, 1.3e4, 300.0, 1e6
    V = math.pi * d ** 3 / 6
    axis = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 0, 1.0]])
    lys = inputs.Lysosome(pos=np.zeros((3, 3)) + np.arange(3)[:, None] * 1e-7, axis=axis,
                          vol=np.full(3, V), Ms=Ms, Keff=K, T=T, tau0=1e-10, d=d)
    Hmax, f, S = 0.020, 1e5, 200
    g = kmc.kmc_mean_run([lys], Hmax, f, S, 2, 1)[0]
    H = Hmax * np.cos(2 * np.pi * np.arange(S) / S)
    np.testing.assert_allclose(g, np.tanh(Ms * V * H / (KB * T)), rtol=0, atol=1e-9)


def test_mean_mode_large_batch_is_deterministic():
    lys = inputs.make_lysosome(3000, 14e-9, 0.1, Keff=2e4, seed=9)
    a = kmc.kmc_mean_run([lys, lys], 0.02, 1e5, 40, 2, 1)
    b = kmc.kmc_mean_run([lys, lys], 0.02, 1e5, 40, 2, 1)
    assert np.array_equal(a, b)
    assert np.array_equal(a[0], a[1])
    o = oracle.mean_run(lys.axis, lys.vol, lys.Ms, lys.Keff, lys.T, lys.tau0, 0.02, 1e5, 40, 2, 1)
    np.testing.assert_allclose(a[0], o, rtol=0, atol=1e-12)


def test_mean_mode_errors():
    lys = inputs.make_lysosome(10, 12e-9, 0.05, seed=1)
    for args in [(0.02, 0.0, 10, 2, 1), (0.02, 1e5, 0, 2, 1), (0.02, 1e5, 10, 1, 2),
                 ([0.02, 0.03], 1e5, 10, 2, 1), (float("nan"), 1e5, 10, 2, 1)]:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_mean_run([lys], *args)
        assert e.value.status == kmc.KMC_EINVAL
    assert kmc.kmc_mean_run([lys], 0.02, 1e5, 10, 2, 2).size == 0
