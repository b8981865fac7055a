"""kmc_regenerate (Sec. II.4: fresh axes and positions between loops) against the
oracle's regeneration draws, which are pinned by the uniform distributions they
sample. The GPU draws the same Philox numbers; sin, cos and sqrt may differ in
the last bit between the two math libraries, hence 1e-15 relative."""
import math

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


def _pair_of_lattices():
    a = inputs.lattice_nodes_lysosome(500, 14e-9, 0.1, seed=1)
    b = inputs.lattice_nodes_lysosome(333, 12e-9, 0.05, Keff=2e4, seed=2)
    return [a, b]


def _unit(v):
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("prec", [kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED])
def test_regenerate_matches_oracle(prec):
    lyss = _pair_of_lattices()
    ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
    seed, loop = 12345, 7
    dis = [inputs.max_disorder(14e-9, 0.1), inputs.max_disorder(12e-9, 0.05)]
    for l in range(2):
        kmc.kmc_regenerate(ctx, l, kmc.KMC_REGEN_AXES | kmc.KMC_REGEN_POSITIONS, dis[l], seed, loop)
    atol_axis = 1e-15 if prec == kmc.KMC_FP64_PLAIN else 6e-8
    for l, ly in enumerate(lyss):
        p = kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, l)
        po = oracle.regen_positions(ly.pos, dis[l], seed, loop, l)
        np.testing.assert_allclose(p, po, rtol=0, atol=1e-15 * np.abs(po).max())
        a = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, l)
        ao = _unit(oracle.regen_axes(ly.n, seed, loop, l))
        np.testing.assert_allclose(a, ao, rtol=0, atol=atol_axis)
        m = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l)
        np.testing.assert_array_equal(m, a * np.where(a[:, 2] >= 0, 1.0, -1.0)[:, None])
    kmc.kmc_destroy(ctx)


def test_regenerated_state_gives_the_oracle_field():
    # FP64: after regeneration the device holds the drawn geometry and the
    # restarted moments in every array the step reads
    lyss = _pair_of_lattices()
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    seed, loop = 9, 3
    dis = inputs.max_disorder(14e-9, 0.1)
    kmc.kmc_regenerate(ctx, -1, kmc.KMC_REGEN_AXES | kmc.KMC_REGEN_POSITIONS, dis, seed, loop)
    m_all = np.concatenate([kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l) for l in range(2)])
    g = kmc.kmc_debug_step(ctx, 0.01, 5e-8, 1, 0, m_all)
    o = 0
    for l, ly in enumerate(lyss):
        pos = oracle.regen_positions(ly.pos, dis, seed, loop, l)
        m = m_all[o:o + ly.n]
        B = oracle.dipolar_field(pos, ly.vol, ly.Ms, m)
        scale = np.abs(B).max()
        np.testing.assert_allclose(g["B_dip"][o:o + ly.n], B, rtol=0, atol=1e-12 * scale)
        o += ly.n
    kmc.kmc_destroy(ctx)


def test_regenerate_parts_and_determinism():
    lyss = _pair_of_lattices()
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    a0 = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0)
    kmc.kmc_regenerate(ctx, 0, kmc.KMC_REGEN_POSITIONS, 1e-9, 5, 0)
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0), a0)
    p1 = kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0)
    assert np.all(np.linalg.norm(p1 - lyss[0].pos, axis=1) <= 1e-9 * (1 + 1e-12))
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 1), lyss[1].pos)
    kmc.kmc_regenerate(ctx, 0, kmc.KMC_REGEN_AXES, 0.0, 5, 0)
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0), p1)
    a1 = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0)
    # the same (seed, loop) redraws the same sample; positions stay around the nodes
    kmc.kmc_regenerate(ctx, 0, kmc.KMC_REGEN_AXES | kmc.KMC_REGEN_POSITIONS, 1e-9, 5, 0)
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 0), a1)
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0), p1)
    # a run and the shell profile see the new geometry
    kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 1, 0)
    prof = kmc.kmc_shell_profile(ctx, 0, 0.0, 4, 0)
    count, _, R = oracle.shell_profile(p1, lyss[0].vol, np.zeros(3), 0.0, 4,
                                       np.zeros((lyss[0].n, 1)))
    np.testing.assert_array_equal(prof["count"], count)
    assert prof["radius"] == pytest.approx(R, rel=1e-15)
    kmc.kmc_destroy(ctx)


def test_regenerate_errors():
    lys = inputs.lattice_nodes_lysosome(40, 14e-9, 0.1)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    for args in [(1, 1, 0.0), (-2, 1, 0.0), (0, 0, 0.0), (0, 4, 0.0), (0, 2, -1e-9),
                 (0, 2, float("inf"))]:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_regenerate(ctx, args[0], args[1], args[2], 1, 0)
        assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)


# --- random sequential addition on the device ---------------------------------

@pytest.mark.parametrize("prec", [kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED])
def test_rsa_matches_the_oracle(prec):
    """Same candidate stream, same sequential rule: the same candidates are kept
    (candidate count exact), positions to the last bits of sin and cos."""
    lyss = [inputs.make_lysosome(150, 12e-9, 0.05, seed=5),
            inputs.make_lysosome(2000, 14e-9, 0.10, seed=6)]
    ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
    for lys, R, d, seed, loop in [(0, 60e-9, 12e-9, 9, 1), (1, inputs.lysosome_radius(2000, 14e-9, 0.1),
                                                             14e-9, 21, 3)]:
        used = kmc.kmc_regenerate_rsa(ctx, lys, R, d, seed, loop)
        o, ou = oracle.rsa(lyss[lys].n, R, d, seed, loop, lys)
        assert used == ou and used > lyss[lys].n
        np.testing.assert_allclose(kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, lys), o,
                                   rtol=0, atol=1e-15 * R)
    # the moments restart along the axes, and a run on the new positions goes through
    m = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, 1)
    ax = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, 1)
    np.testing.assert_allclose(np.abs(np.sum(m * ax, axis=1)), 1.0, atol=2e-6)
    assert np.all(m[:, 2] >= -1e-7)
    kmc.kmc_run(ctx, 0.02, 1e5, 40, 2, 1, 7)
    assert np.all(np.isfinite(kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, 1)))
    kmc.kmc_destroy(ctx)


def test_rsa_packing_at_20000():
    spatial = pytest.importorskip("scipy.spatial")
    n, d, c = 20000, 12e-9, 0.10
    R = inputs.lysosome_radius(n, d, c)
    # n NPs far apart at creation; the addition gives them their places
    lys = inputs.Lysosome(pos=np.zeros((n, 3)) + np.arange(n)[:, None] * 1e-6,
                          axis=inputs.random_axes(n, np.random.default_rng(2)),
                          vol=np.full(n, inputs.sphere_volume(d)), Ms=1e6, Keff=1.3e4, T=300.0,
                          tau0=1e-10, d=d)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    used = kmc.kmc_regenerate_rsa(ctx, 0, R, d, 4, 1)
    p = kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0)
    kmc.kmc_destroy(ctx)
    assert used >= n
    assert np.linalg.norm(p, axis=1).max() <= (R - d / 2) * (1 + 1e-12)
    dmin, _ = spatial.cKDTree(p).query(p, k=2)
    assert dmin[:, 1].min() >= d * (1 - 1e-12)


def test_rsa_rejects_bad_arguments_and_reports_a_packing_too_dense():
    lys = inputs.make_lysosome(300, 12e-9, 0.05, seed=3)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    before = kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0)
    for R, d in [(10e-9, 30e-9), (1e-7, 0.0), (float("nan"), 1e-8)]:
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_regenerate_rsa(ctx, 0, R, d, 1, 1)
        assert e.value.status == kmc.KMC_EINVAL
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_regenerate_rsa(ctx, 1, 1e-7, 1e-8, 1, 1)
    assert e.value.status == kmc.KMC_EINVAL
    # 300 spheres of 12 nm cannot fit in a 40 nm sphere
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_regenerate_rsa(ctx, 0, 40e-9, 12e-9, 1, 1, max_candidates=20000)
    assert e.value.status == kmc.KMC_ESTATE
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_POSITIONS, 0), before)
    kmc.kmc_destroy(ctx)
