"""A batch shaped like the paper's batched workload (lognormal NP counts, d, K_eff,
concentration and field amplitude drawn per lysosome) through one context, with
each lysosome at its own amplitude.

Near the switching field the FP32 scan can see de/dth change sign spuriously at
a node where it nearly vanishes; such targets are rescanned in FP64, so a long
batched run must finish without the extrema error, with unit moments and the
counters of a physical run."""
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


def test_batched_lysosomes_each_at_its_own_amplitude():
    lyss, run = inputs.config_batched(n_lys=128, seed=0)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_run(ctx, run["mu0Hmax"], run["f"], run["S"], 3, 1, run["seed"])
    kmc.kmc_sync(ctx)  # raises on a device error
    for l in (0, 17, 127):
        m = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l)
        np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=2e-6)
        assert np.all(np.isfinite(kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, l)))
    flips = sum(kmc.kmc_read(ctx, kmc.KMC_READ_COUNTERS, l)[0] for l in range(len(lyss)))
    assert flips > 0
    kmc.kmc_destroy(ctx)


def test_a_lysosome_in_a_chained_batch_matches_it_alone():
    """A batch runs its lysosomes as parallel chains of step kernels; each
    lysosome's trajectory is the one it has alone (same index 0, same shape)."""
    a = inputs.make_lysosome(100, 12e-9, 0.05, seed=21)
    others = [inputs.make_lysosome(333, 14e-9, 0.08, seed=22),
              inputs.make_lysosome(57, 10e-9, 0.05, seed=23),
              inputs.make_lysosome(250, 12e-9, 0.05, seed=24)]
    out = []
    for lyss in ([a], [a] + others):
        ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
        kmc.kmc_tuning(ctx, 4, 64, 0)
        kmc.kmc_run(ctx, 0.02, 1e5, 40, 3, 1, 9)
        out.append([kmc.kmc_read(ctx, w, 0) for w in (kmc.KMC_READ_LOOP_M, kmc.KMC_READ_MOMENTS,
                                                       kmc.KMC_READ_NP_ENERGY,
                                                       kmc.KMC_READ_COUNTERS)])
        kmc.kmc_destroy(ctx)
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_fp64_chained_batch_flip_for_flip():
    """FP64-plain batch (three chains, one amplitude per lysosome): each
    lysosome's trajectory, loop, energies and dipolar record follow the oracle
    run of that lysosome (same Philox stream index) flip for flip."""
    lyss = [inputs.make_lysosome(60, 12e-9, 0.05, seed=51),
            inputs.make_lysosome(130, 14e-9, 0.08, Keff=2e4, seed=52),
            inputs.make_lysosome(33, 10e-9, 0.05, seed=53)]
    H = [0.02, 0.03, 0.015]
    f, S, periods, discard, seed = 1e5, 50, 3, 1, 4
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    kmc.kmc_run(ctx, H, f, S, periods, discard, seed)
    compared = 0
    for l, ly in enumerate(lyss):
        o = oracle.run(ly, l, H[l], f, S, periods, discard, seed)
        if o["counters"]["near"] > 0:
            continue  # a near-threshold draw may legitimately split the trajectories
        compared += 1
        assert kmc.kmc_read(ctx, kmc.KMC_READ_COUNTERS, l)[0] == o["counters"]["flips"]
        np.testing.assert_allclose(kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, l), o["loop_M"],
                                   rtol=0, atol=1e-11)
        np.testing.assert_allclose(kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l), o["m"],
                                   rtol=0, atol=1e-11)
        E = kmc.kmc_read(ctx, kmc.KMC_READ_NP_ENERGY, l)
        np.testing.assert_allclose(E, o["E_diss"] / (periods - discard), rtol=1e-9,
                                   atol=1e-12 * np.abs(o["E_diss"]).max())
        scale = np.abs(o["dHdip"]).max()
        np.testing.assert_allclose(kmc.kmc_read(ctx, kmc.KMC_READ_DHDIP, l), o["dHdip"],
                                   rtol=0, atol=1e-11 * scale)
    kmc.kmc_destroy(ctx)
    assert compared >= 2


def _batch4():
    return [inputs.make_lysosome(n, 12e-9, 0.05, seed=60 + q) for q, n in enumerate([180, 90, 333, 45])]


def test_chained_batch_on_a_caller_stream_gives_the_same_bits():
    torch = pytest.importorskip("torch")
    out = []
    for use_stream in (False, True):
        ctx = kmc.kmc_create(_batch4(), kmc.KMC_FP32_MIXED, center=np.zeros(3))
        kmc.kmc_tuning(ctx, 4, 64, 0)
        st = torch.cuda.Stream() if use_stream else None
        if st is not None:
            kmc.kmc_set_stream(ctx, st.cuda_stream)
        kmc.kmc_run(ctx, [0.02, 0.03, 0.025, 0.015], 1e5, 40, 3, 1, 2)
        out.append([kmc.kmc_read(ctx, w, l) for l in range(4)
                    for w in (kmc.KMC_READ_LOOP_M, kmc.KMC_READ_MOMENTS, kmc.KMC_READ_COUNTERS)])
        kmc.kmc_destroy(ctx)
    for x, y in zip(*out):
        assert np.array_equal(x, y)


def test_chained_batch_checkpoint_resume_is_bit_identical(tmp_path):
    H = [0.02, 0.03, 0.025, 0.015]
    for prec in (kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED):
        a = kmc.kmc_create(_batch4(), prec, center=np.zeros(3))
        kmc.kmc_run(a, H, 1e5, 40, 3, 0, 8)
        kmc.kmc_run(a, H, 1e5, 40, 2, 0, 8)
        ref = [kmc.kmc_read(a, w, l) for l in range(4)
               for w in (kmc.KMC_READ_MOMENTS, kmc.KMC_READ_LOOP_M)]
        kmc.kmc_destroy(a)
        b = kmc.kmc_create(_batch4(), prec, center=np.zeros(3))
        kmc.kmc_run(b, H, 1e5, 40, 3, 0, 8)
        p = str(tmp_path / ("batch%d.bin" % prec))
        kmc.kmc_save(b, p)
        kmc.kmc_destroy(b)
        c = kmc.kmc_create(_batch4(), prec, center=np.zeros(3))
        kmc.kmc_load(c, p)
        kmc.kmc_run(c, H, 1e5, 40, 2, 0, 8)
        got = [kmc.kmc_read(c, w, l) for l in range(4)
               for w in (kmc.KMC_READ_MOMENTS, kmc.KMC_READ_LOOP_M)]
        kmc.kmc_destroy(c)
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)


def test_two_and_three_targets_per_lane_give_the_same_bits():
    """The multi-target kernels (64- or 96-target groups, two or three per lane)
    form every target's sums with the same operations in the same order as the
    one-target kernel and run the same update: identical outputs at the same
    shape, including ragged last groups and split source ranges. With 8 or 16
    warps and two targets per lane the two parts update side by side, each on
    half of the warps."""
    lyss = [inputs.make_lysosome(n, 12e-9, 0.05, seed=70 + q) for q, n in enumerate([700, 97, 33, 1])]
    for shape in [(4, 64, 0), (4, 128, 256), (8, 64, 128), (8, 128, 0), (16, 64, 256)]:
        out = []
        for tpl in (1, 2, 3):
            ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
            kmc.kmc_targets_per_lane(ctx, tpl)
            kmc.kmc_tuning(ctx, *shape)
            assert kmc.kmc_targets_per_lane(ctx) == tpl
            kmc.kmc_run(ctx, [0.02, 0.03, 0.025, 0.01], 1e5, 40, 3, 1, 3)
            out.append([kmc.kmc_read(ctx, w, l) for l in range(len(lyss))
                        for w in (kmc.KMC_READ_LOOP_M, kmc.KMC_READ_MOMENTS,
                                  kmc.KMC_READ_NP_ENERGY, kmc.KMC_READ_DHDIP,
                                  kmc.KMC_READ_COUNTERS)])
            kmc.kmc_destroy(ctx)
        for other in out[1:]:
            for x, y in zip(out[0], other):
                assert np.array_equal(x, y), shape
    lys64 = inputs.make_lysosome(40, 12e-9, 0.05, seed=1)
    ctx = kmc.kmc_create([lys64], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    for tpl in (2, 3):
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_targets_per_lane(ctx, tpl)
        assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)
