"""The paper's own validation of the method, run on the GPU path (Sec. II.3):
in the non-interacting limit the kMC sample mean of the FP32-mixed step must
follow the Ref. [8] mean-magnetisation mode (the exact expectation of the same
jump process), for superparamagnetic and blocked NPs; and at zero field the
number of jumps must follow the Neel rate, P = (1 - exp(-2 nu0 e^{-KV/kT} t)) / 2
per step (the mean time between jumps is twice the Neel time, Sec. II.2).

Bounds are statistical: N independent NPs, m_z in [-1, 1], so the sample mean
at a step lies within 5 / sqrt(N) of its expectation; jump counts within 5
binomial standard deviations."""
import math

import numpy as np
import pytest

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


def _isolated(n, d, K, seed, T=300.0):
    # NPs 2 um apart: their dipolar fields are ~1e-8 T, far below the applied one
    side = int(math.ceil(n ** (1 / 3)))
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    rng = np.random.Generator(np.random.PCG64(seed))
    return inputs.Lysosome(pos=g * 2e-6, axis=inputs.random_axes(n, rng),
                           vol=np.full(n, inputs.sphere_volume(d)), Ms=1e6, Keff=K, T=T,
                           tau0=1e-10, d=d)


@pytest.mark.parametrize("d,H,is_open", [(10e-9, 0.03, False),  # KV/kT = 1.6: superparamagnetic
                                         (13e-9, 0.02, True),   # KV/kT = 7.2: lagging loop
                                         (20e-9, 0.03, True)])  # KV/kT = 13: blocked, H > H_K
def test_kmc_follows_the_mean_mode(d, H, is_open):
    n = 4096
    lys = _isolated(n, d, 1.3e4, seed=int(d * 1e9))
    f, S, periods, discard = 1e5, 100, 3, 1
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_run(ctx, H, f, S, periods, discard, 17)
    sample = kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, 0)
    area = kmc.kmc_read(ctx, kmc.KMC_READ_AREA, 0)[0]
    kmc.kmc_destroy(ctx)
    mean = kmc.kmc_mean_run([lys], H, f, S, periods, discard)[0]
    # |m_z| <= 1 per NP: the standard error of the sample mean is at most 1/sqrt(n)
    err = np.abs(sample - mean)
    assert np.max(err) < 5.0 / math.sqrt(n)
    assert np.mean(err) < 1.5 / math.sqrt(n)
    if is_open:  # superparamagnetic NPs relax within a step: no area beyond noise
        assert area > 0


def test_zero_field_jump_rate():
    n, S, d, K, T = 4096, 50, 17.5e-9, 1.3e4, 300.0  # KV/kT = 8.8, P = 0.23
    lys = _isolated(n, d, K, seed=3, T=T)
    f = 1e5
    t_step = 1.0 / (f * S)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_run(ctx, 0.0, f, S, 2, 0, 5)
    jumps = kmc.kmc_read(ctx, kmc.KMC_READ_COUNTERS, 0)[0]
    kmc.kmc_destroy(ctx)
    V = inputs.sphere_volume(d)
    P = 0.5 * (1.0 - math.exp(-2.0 * math.exp(-K * V / (KB * T)) / 1e-10 * t_step))
    trials = n * S * 2
    expect = trials * P
    assert 0.01 < P < 0.5
    assert abs(jumps - expect) < 5.0 * math.sqrt(trials * P * (1 - P))
