"""The symmetric pair form (kmc_pair_form = 2): every unordered pair of NPs is
formed once and serves both (T_ij and T_ji share d, r^2, the rsqrt and the
powers of 1/r); pairs inside a row group of cells run in the ordered form.

The summation order differs from the ordered kernels', so the fields are
checked against the oracle within the FP32 field tolerance of the other tests
(max_i |dB_i| <= 1e-5 rms_i |B_i|), steps iii-vii against the oracle's update
fed the GPU's own field (the tolerances of tests/test_gpu_workloads.py), and
draws bit for bit. Cases: ragged lysosomes (1, 2, 63, 64, 65 NPs: empty and
partial cells and row groups) at every field-kernel shape and several source
splits, the 50 000-NP lysosome, the 512-lysosome batch, and whole runs, which
must be deterministic and give each lysosome the bits it gets alone."""
import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs, kmc
from test_gpu_workloads import check_update, perturbed, rms

pytestmark = pytest.mark.gpu
SYM = kmc.FORM_SYMMETRIC


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()


def _pin(ctx, warps, cells, chunk, upd=1):
    kmc.kmc_pair_form(ctx, SYM)
    kmc.kmc_targets_per_lane(ctx, 2 * cells)
    kmc.kmc_sym_update(ctx, upd)
    kmc.kmc_tuning(ctx, warps, 32, chunk)


# (warps, cells per warp, source NPs per field item, update kernel: 1 = a warp
# per update item, 2 = a block)
SHAPES = [(4, 1, 0, 1), (4, 1, 64, 1), (4, 1, 256, 1), (4, 2, 0, 1), (4, 2, 128, 1),
          (8, 1, 0, 1), (8, 1, 192, 1), (2, 2, 0, 1), (2, 2, 320, 1),
          (4, 2, 0, 2), (4, 2, 128, 2), (8, 1, 192, 2), (2, 2, 64, 2)]


@pytest.mark.parametrize("warps,cells,chunk,upd", SHAPES)
def test_fields_of_ragged_lysosomes(warps, cells, chunk, upd):
    sizes = (1, 2, 63, 64, 65, 300, 1100)
    lyss = [inputs.make_lysosome(n, 12e-9, 0.05 if n > 2 else 0.01, seed=60 + n) for n in sizes]
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    _pin(ctx, warps, cells, chunk, upd)
    rng = np.random.default_rng(warps * 10 + cells + chunk)
    m = np.concatenate([perturbed(l.axis, rng, 0.3) for l in lyss])
    m = m.astype(np.float32).astype(np.float64)
    H = [0.01 * (q % 3) - 0.01 for q in range(len(lyss))]
    g = kmc.kmc_debug_step(ctx, H, 5e-8, 3, 71, m)
    assert kmc.kmc_pair_form(ctx) == SYM and kmc.kmc_sym_update(ctx) == upd
    assert kmc.kmc_tuning(ctx) == (warps, 32, chunk)
    kmc.kmc_destroy(ctx)
    off = 0
    for l, ly in enumerate(lyss):
        sl = slice(off, off + ly.n)
        B = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m[sl])
        err = np.max(np.linalg.norm(g["B_dip"][sl] - B, axis=1))
        assert err <= 1e-5 * max(rms(B), 1e-30) or (ly.n == 1 and err == 0.0), (ly.n, err)
        assert np.array_equal(g["u"][sl], [oracle.uniform(3, 71, i, l) for i in range(ly.n)])
        off += ly.n
    np.testing.assert_allclose(np.linalg.norm(g["m_out"], axis=1), 1.0, atol=2e-6)


def test_update_against_oracle_at_2000_nps():
    (ly,) = inputs.config_single2000(replicas=1, seed=0)[0]
    ctx = kmc.kmc_create([ly], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    _pin(ctx, 4, 2, 512)
    rng = np.random.default_rng(5)
    m32 = perturbed(ly.axis, rng, 0.3).astype(np.float32).astype(np.float64)
    t_step = 1.0 / (1e5 * 200)
    g = kmc.kmc_debug_step(ctx, -0.012, t_step, 9, 123, m32)
    axes = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0)
    kmc.kmc_destroy(ctx)
    B = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m32)
    assert np.max(np.linalg.norm(g["B_dip"] - B, axis=1)) <= 1e-5 * rms(B)
    idx = np.arange(0, ly.n, 7)
    c, a = check_update(ly, axes[idx], m32[idx], g["B_dip"][idx], -0.012, t_step, g, idx)
    assert c >= 0.95 * (c + a), (c, a)


@pytest.mark.parametrize("upd", [1, 2])
def test_large_lysosome_sampled(upd):
    """50 000 NPs, 4 warps of two cells, 2048-NP source ranges, both update
    kernels."""
    (ly,), run = inputs.config_large50000(seed=0)
    ctx = kmc.kmc_create([ly], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    _pin(ctx, 4, 2, 2048, upd)
    rng = np.random.default_rng(13)
    m32 = perturbed(ly.axis, rng, 0.3).astype(np.float32).astype(np.float64)
    t_step = 1.0 / (run["f"] * run["S"])
    g = kmc.kmc_debug_step(ctx, -0.025, t_step, 2, 778, m32)
    axes = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0)
    kmc.kmc_destroy(ctx)
    # both ends of the NP order: the first and last row groups and cells
    idx = np.unique(np.concatenate([np.arange(64), np.arange(ly.n - 64, ly.n),
                                    rng.choice(ly.n, 128, replace=False)]))
    B = oracle.dipolar_field_at(ly.pos, ly.vol, ly.Ms, m32, idx)
    err = np.max(np.linalg.norm(g["B_dip"][idx] - B, axis=1)) / rms(B)
    assert err <= 1e-5, err
    assert np.array_equal(g["u"][idx], [oracle.uniform(2, 778, int(i), 0) for i in idx])
    c, a = check_update(ly, axes[idx], m32[idx], g["B_dip"][idx], -0.025, t_step, g, idx)
    assert c >= 0.95 * (c + a), (c, a)


def test_batched_workload_sampled():
    """The 512-lysosome batch with the symmetric form pinned (its shape
    autotuned): six lysosomes, 64 sampled targets each."""
    lyss, run = inputs.config_batched(n_lys=512, seed=0)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_pair_form(ctx, SYM)
    kmc.kmc_run(ctx, run["mu0Hmax"], run["f"], run["S"], 1, 0, run["seed"])  # tunes
    assert kmc.kmc_pair_form(ctx) == SYM
    m_all = np.concatenate([kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l) for l in range(512)])
    offs = np.concatenate([[0], np.cumsum([l.n for l in lyss])])
    t_step = 1.0 / (run["f"] * run["S"])
    Hs = np.asarray(run["mu0Hmax"]) * -0.6
    g = kmc.kmc_debug_step(ctx, Hs, t_step, 17, 3002, m_all)
    kmc.kmc_destroy(ctx)
    ns = np.array([l.n for l in lyss])
    rng = np.random.default_rng(2)
    picks = [int(np.argmax(ns)), int(np.argmin(ns))] + [int(x) for x in rng.choice(512, 4, replace=False)]
    for l in picks:
        ly = lyss[l]
        idx = np.sort(rng.choice(ly.n, min(64, ly.n), replace=False))
        B = oracle.dipolar_field_at(ly.pos, ly.vol, ly.Ms, m_all[offs[l]:offs[l + 1]], idx)
        err = np.max(np.linalg.norm(g["B_dip"][offs[l] + idx] - B, axis=1)) / rms(B)
        assert err <= 1e-5, (l, ly.n, err)


OUTPUTS = (kmc.KMC_READ_LOOP_M, kmc.KMC_READ_MOMENTS, kmc.KMC_READ_NP_ENERGY,
           kmc.KMC_READ_DHDIP, kmc.KMC_READ_COUNTERS)


def _run(lyss, H, shape):
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    _pin(ctx, *shape)
    kmc.kmc_run(ctx, H, 1e5, 40, 3, 1, 8)
    kmc.kmc_sync(ctx)
    out = [[kmc.kmc_read(ctx, w, l) for w in OUTPUTS] for l in range(len(lyss))]
    kmc.kmc_destroy(ctx)
    return out


@pytest.mark.parametrize("shape", [(4, 1, 128, 1), (4, 2, 0, 1), (4, 2, 256, 2)])
def test_runs_are_deterministic_and_independent_of_the_batch(shape):
    lyss = [inputs.make_lysosome(n, 12e-9, 0.06, seed=90 + n) for n in (700, 300, 1300)]
    H = [0.015, 0.02, 0.012]
    a = _run(lyss, H, shape)
    b = _run(lyss, H, shape)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
    # the first lysosome alone (its random streams follow its index, 0 in both)
    alone = _run(lyss[:1], H[:1], shape)
    for u, v in zip(a[0], alone[0]):
        assert np.array_equal(u, v)
    assert a[0][4][0] > 0  # the run flipped NPs


def test_refusals():
    ly = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    ctx = kmc.kmc_create([ly], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    with pytest.raises(kmc.KmcError):
        kmc.kmc_pair_form(ctx, SYM)
    kmc.kmc_destroy(ctx)
    ctx = kmc.kmc_create([ly], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_pair_form(ctx, SYM)
    for bad in ((8, 32, 0, 4), (4, 32, 100, 2), (16, 32, 0, 2)):
        kmc.kmc_targets_per_lane(ctx, bad[3])
        with pytest.raises(kmc.KmcError):
            kmc.kmc_tuning(ctx, *bad[:3])
    with pytest.raises(kmc.KmcError):
        kmc.kmc_targets_per_lane(ctx, 3)
    kmc.kmc_pair_form(ctx, kmc.FORM_ORDERED)
    with pytest.raises(kmc.KmcError):
        kmc.kmc_targets_per_lane(ctx, 4)
    kmc.kmc_destroy(ctx)
