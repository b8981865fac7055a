"""The persistent period (kmc_persistent = 2): one cooperative launch per
field period, each block keeping its work item and a bounded grid barrier
between the steps. The step is the same code with the same cosine as the
per-step launches, so whole runs must give the same bits at the same warps,
tile and chunk. The grid barrier's failure path is tested without a fault: a
block that does not arrive makes the others give up after 1 ms, and the call
reports KMC_ETIMEOUT with the context still usable."""
import numpy as np
import pytest

from paper_1407_2737_gb300 import inputs, kmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()


OUTPUTS = (kmc.KMC_READ_LOOP_M, kmc.KMC_READ_MOMENTS, kmc.KMC_READ_NP_ENERGY,
           kmc.KMC_READ_DHDIP, kmc.KMC_READ_COUNTERS)


def _run(lyss, H, persist, shape, S=40, periods=3):
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_targets_per_lane(ctx, 1)
    kmc.kmc_cluster_split(ctx, 1)
    kmc.kmc_persistent(ctx, persist)
    kmc.kmc_tuning(ctx, *shape)
    kmc.kmc_run(ctx, H, 1e5, S, periods, 1, 12)
    kmc.kmc_sync(ctx)
    out = [kmc.kmc_read(ctx, w, l) for l in range(len(lyss)) for w in OUTPUTS]
    used = kmc.kmc_persistent(ctx)
    kmc.kmc_destroy(ctx)
    return out, used


@pytest.mark.parametrize("shape", [(4, 64, 0), (4, 128, 512), (8, 64, 0)])
def test_persistent_period_gives_the_bits_of_the_step_launches(shape):
    lyss = [inputs.make_lysosome(n, 12e-9, 0.06, seed=20 + n) for n in (700, 100, 333)]
    H = [0.015, 0.02, 0.012]
    ref, off = _run(lyss, H, 1, shape)
    got, on = _run(lyss, H, 2, shape)
    assert (off, on) == (1, 2)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    assert got[4][0] > 0  # the runs flipped NPs


def test_persistent_period_at_the_100_np_workload():
    lyss, run = inputs.config_small(seed=0)
    ref, _ = _run(lyss, [run["mu0Hmax"]], 1, (4, 64, 0), S=run["S"], periods=4)
    got, _ = _run(lyss, [run["mu0Hmax"]], 2, (4, 64, 0), S=run["S"], periods=4)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


def test_grid_barrier_timeout_is_reported_and_the_context_stays_usable():
    lyss = [inputs.make_lysosome(n, 12e-9, 0.06, seed=40 + n) for n in (300, 200)]
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_targets_per_lane(ctx, 1)
    kmc.kmc_persistent(ctx, 2)
    kmc.kmc_tuning(ctx, 4, 64, 0)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_debug_grid_stall(ctx)
    assert e.value.status == kmc.KMC_ETIMEOUT
    kmc.kmc_run(ctx, [0.02, 0.02], 1e5, 20, 2, 1, 3)  # runs on after the stall
    kmc.kmc_sync(ctx)
    m = np.concatenate([kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l) for l in range(2)])
    np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=2e-6)
    kmc.kmc_destroy(ctx)


def test_persistent_period_refusals():
    (ly,), _ = inputs.config_large50000(seed=0)
    ctx = kmc.kmc_create([ly], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_targets_per_lane(ctx, 1)
    kmc.kmc_persistent(ctx, 2)
    kmc.kmc_tuning(ctx, 4, 256, 512)  # 1563 groups x 49 parts: far more than resident
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_run(ctx, 0.04, 1e5, 10, 1, 0, 1)
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)
    small = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    c32 = kmc.kmc_create([small], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_persistent(c32, 1)
    kmc.kmc_targets_per_lane(c32, 1)
    kmc.kmc_tuning(c32, 4, 64, 0)
    with pytest.raises(kmc.KmcError) as e:  # the hook needs the persistent period
        kmc.kmc_debug_grid_stall(c32)
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(c32)
    c64 = kmc.kmc_create([small], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    with pytest.raises(kmc.KmcError):
        kmc.kmc_persistent(c64, 2)
    kmc.kmc_destroy(c64)
