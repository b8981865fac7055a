"""Replicas per lane: sets of identical lysosomes (the same sample run with
different random streams, as seed averages are) stepped together, each staged
source record's geometry serving every lysosome of the set.

With four replicas per lane (four warps, one per lysosome; or eight or
sixteen, two or four per lysosome), and with two replicas on four or eight
warps, every lysosome's sums are formed by the same operations in the same
order as with one target per lane and as many warps, and its update is the
same code run by one warp or a group of two or four, so whole runs must give
the same bits. With two replicas on two warps (records interleaved over two
warps) the summation order differs: the fields are checked against the oracle
within the FP32 field tolerance of the other tests (1e-5 of rms)."""
import numpy as np
import pytest

import oracle
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


def _run(lyss, rpl, shape, H, periods=3):
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_replicas_per_lane(ctx, rpl)
    kmc.kmc_tuning(ctx, *shape)
    kmc.kmc_run(ctx, H, 1e5, 40, periods, 1, 6)
    out = [kmc.kmc_read(ctx, w, l) for l in range(len(lyss)) for w in OUTPUTS]
    used = kmc.kmc_replicas_per_lane(ctx)
    kmc.kmc_destroy(ctx)
    return out, used


@pytest.mark.parametrize("tile,chunk", [(64, 0), (32, 128), (128, 256)])
def test_four_replicas_per_lane_give_the_bits_of_one_target_per_lane(tile, chunk):
    """Eight replicas of a 300-NP lysosome (a ragged last group of 12 targets),
    each at its own amplitude: two sets of four, against one target per lane
    with four warps at the same tile and source split."""
    ly = inputs.make_lysosome(300, 12e-9, 0.06, seed=81)
    lyss = inputs.replicate(ly, 8)
    H = [0.015 + 0.002 * q for q in range(8)]
    ref, used1 = _run(lyss, 1, (4, tile, chunk), H)
    got, used4 = _run(lyss, 4, (4, tile, chunk), H)
    assert (used1, used4) == (1, 4)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("wpr,rpl,tile,chunk", [(4, 4, 64, 0), (4, 4, 32, 128), (4, 2, 128, 256),
                                              (4, 2, 64, 0), (2, 2, 64, 0), (2, 2, 128, 256),
                                              (2, 4, 32, 128), (2, 4, 64, 0)])
def test_warp_groups_per_replica_give_the_bits_of_one_target_per_lane(wpr, rpl, tile, chunk):
    """Two or four warps per replica (wpr rpl warps; each replica's steps
    iii-vii run by its own group of wpr warps on named barriers) against one
    target per lane with as many warps, at the same tile and source split."""
    ly = inputs.make_lysosome(300, 12e-9, 0.06, seed=83)
    lyss = inputs.replicate(ly, 8)
    H = [0.012 + 0.003 * q for q in range(8)]
    ref, used1 = _run(lyss, 1, (wpr * rpl, tile, chunk), H)
    got, usedr = _run(lyss, rpl, (wpr * rpl, tile, chunk), H)
    assert (used1, usedr) == (1, rpl)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("rpl", [2, 4])
def test_replica_fields_match_the_oracle(rpl):
    ly = inputs.make_lysosome(700, 14e-9, 0.10, Keff=2e4, seed=82)
    lyss = inputs.replicate(ly, 4)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_replicas_per_lane(ctx, rpl)
    kmc.kmc_tuning(ctx, rpl, 64, 256)
    rng = np.random.default_rng(rpl)
    m = np.concatenate([oracle.initial_moments(ly.axis) + 0.3 * rng.normal(size=(ly.n, 3))
                        for _ in range(4)])
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    m = m.astype(np.float32).astype(np.float64)
    g = kmc.kmc_debug_step(ctx, [0.01, -0.02, 0.015, 0.0], 5e-8, 3, 44, m)
    kmc.kmc_destroy(ctx)
    for l in range(4):
        sl = slice(l * ly.n, (l + 1) * ly.n)
        B = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m[sl])
        rms = np.sqrt(np.mean(np.sum(B ** 2, axis=1)))
        assert np.max(np.linalg.norm(g["B_dip"][sl] - B, axis=1)) <= 1e-5 * rms
        assert np.array_equal(g["u"][sl], [oracle.uniform(3, 44, i, l) for i in range(ly.n)])
    np.testing.assert_allclose(np.linalg.norm(g["m_out"], axis=1), 1.0, atol=2e-6)


def test_replicas_are_refused_where_the_lysosomes_differ():
    a = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    b = inputs.make_lysosome(100, 12e-9, 0.05, seed=2)
    cases = [([a, b, a, b], kmc.KMC_FP32_MIXED, 2),       # neighbours differ
             (inputs.replicate(a, 6), kmc.KMC_FP32_MIXED, 4),  # 6 is no multiple of 4
             (inputs.replicate(a, 4), kmc.KMC_FP64_PLAIN, 4)]
    for lyss, prec, rpl in cases:
        ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_replicas_per_lane(ctx, rpl)
        assert e.value.status == kmc.KMC_EINVAL
        kmc.kmc_destroy(ctx)
    ctx = kmc.kmc_create(inputs.replicate(a, 6), kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_replicas_per_lane(ctx, 2)  # 6 = 3 sets of two
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_tuning(ctx, 16, 64, 0)  # two replicas take two, four or eight warps
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)
