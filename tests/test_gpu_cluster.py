"""The cluster split (kmc_cluster_split = 2): when every target group's sources
are split into exactly two parts, the two parts run as the two CTAs of a
thread-block cluster and exchange their sums through distributed shared
memory instead of global memory. The second part's sums reach the first as
the same floats and are added in the same order, so fields, draws and whole
runs must be the same bits as with the exchange through global memory."""
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


def _lysosomes():
    # 1000, 750, 550 and 515 source records: two parts of at most 512 each
    return [inputs.make_lysosome(n, 12e-9, 0.06, seed=70 + n) for n in (2000, 1500, 1100, 1030)]


def _run(lyss, cl, shape, H):
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_targets_per_lane(ctx, 1)
    kmc.kmc_cluster_split(ctx, cl)
    kmc.kmc_tuning(ctx, *shape)
    kmc.kmc_run(ctx, H, 1e5, 40, 3, 1, 4)
    kmc.kmc_sync(ctx)
    out = [kmc.kmc_read(ctx, w, l) for l in range(len(lyss)) for w in OUTPUTS]
    used = kmc.kmc_cluster_split(ctx)
    kmc.kmc_destroy(ctx)
    return out, used


@pytest.mark.parametrize("shape", [(4, 256, 1024), (8, 128, 1024), (4, 64, 1024)])
def test_cluster_split_gives_the_same_bits(shape):
    lyss = _lysosomes()
    H = [0.015, 0.02, 0.012, 0.018]
    ref, off = _run(lyss, 1, shape, H)
    got, on = _run(lyss, 2, shape, H)
    assert (off, on) == (1, 2)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


def test_cluster_split_debug_step_fields():
    lyss = _lysosomes()
    rng = np.random.default_rng(9)
    m = np.concatenate([l.axis + 0.3 * rng.normal(size=(l.n, 3)) for l in lyss])
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    out = []
    for cl in (1, 2):
        ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
        kmc.kmc_targets_per_lane(ctx, 1)
        kmc.kmc_cluster_split(ctx, cl)
        kmc.kmc_tuning(ctx, 4, 256, 1024)
        out.append(kmc.kmc_debug_step(ctx, [0.01, -0.02, 0.0, 0.015], 5e-8, 2, 31, m))
        kmc.kmc_destroy(ctx)
    for key in ("B_dip", "dE", "P", "u", "m_out"):
        assert np.array_equal(out[0][key], out[1][key]), key


def test_cluster_split_needs_two_parts_per_group():
    lyss = _lysosomes()
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_targets_per_lane(ctx, 1)
    kmc.kmc_cluster_split(ctx, 2)
    with pytest.raises(kmc.KmcError) as e:  # unsplit sources: refused by the shape check
        kmc.kmc_tuning(ctx, 4, 256, 0)
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_tuning(ctx, 4, 256, 512)  # up to four parts: refused when the plan is built
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_run(ctx, 0.02, 1e5, 20, 1, 0, 1)
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)
    ly = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    ctx = kmc.kmc_create([ly], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    with pytest.raises(kmc.KmcError):
        kmc.kmc_cluster_split(ctx, 2)
    kmc.kmc_destroy(ctx)
