"""Parity of the per-NP analysis outputs of the CUDA path (through the C ABI)
with the oracle: Delta_Hdip (Eq. 6, KMC_READ_DHDIP), the local concentration
phi_N (Eq. 8, kmc_local_concentration) and the radial shell profile of Fig. 8
(kmc_shell_profile).

Tolerances: Eq. 6 is a difference of dipolar fields, so it inherits the field
tolerances of the step (FP64: ~1e-12 of the field scale on an identical
trajectory; FP32-mixed: 1e-5 of the rms field per evaluation, two evaluations
per period). phi_N is one FP64 distance and a cube, both sides exact to a few
ulp (1e-13 relative). Shell counts are exact; shell means carry the per-NP
tolerances.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs, kmc

pytestmark = pytest.mark.gpu
MU0 = 4e-7 * math.pi


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()


def _gpu_run(lyss, prec, H, f, S, periods, discard, seed):
    ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
    kmc.kmc_run(ctx, H, f, S, periods, discard, seed)
    return ctx


@pytest.mark.parametrize("S", [200, 7])
def test_dhdip_fp64_flip_for_flip(S):
    (lys,), run = inputs.config_small(seed=0)
    periods, discard = 5, 2
    ctx = _gpu_run([lys], kmc.KMC_FP64_PLAIN, run["mu0Hmax"], run["f"], S, periods, discard, 3)
    g = kmc.kmc_read(ctx, kmc.KMC_READ_DHDIP, 0)
    flips = kmc.kmc_read(ctx, kmc.KMC_READ_COUNTERS, 0)[0]
    kmc.kmc_destroy(ctx)
    o = oracle.run(lys, 0, run["mu0Hmax"], run["f"], S, periods, discard, 3)
    if o["counters"]["near"] > 0:
        pytest.skip("a near-threshold draw occurred; trajectories may legitimately split")
    assert flips == o["counters"]["flips"]
    scale = np.abs(o["dHdip"]).max()
    assert scale > 0
    np.testing.assert_allclose(g, o["dHdip"], rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("prec,tol", [(kmc.KMC_FP64_PLAIN, 1e-12), (kmc.KMC_FP32_MIXED, 1e-5)])
@pytest.mark.parametrize("bond,sign", [((0.0, 0.0, 1.0), 4.0), ((1.0, 0.0, 0.0), -2.0)])
def test_dhdip_saturated_pair_closed_form(prec, tol, bond, sign):
    # two NPs with axes along z, T = 0, driven far past switching: the field of
    # one on the other is +2c (bond along z) or -c (bond across) times m, with
    # c = mu0 M_S V / (4 pi r^3), so Eq. 6 gives 4c or -2c
    d, sep = 20e-9, 30e-9
    lys = inputs.Lysosome(pos=np.array([[0.0, 0.0, 0.0], np.array(bond) * sep]),
                          axis=np.tile([0.0, 0.0, 1.0], (2, 1)),
                          vol=np.full(2, inputs.sphere_volume(d)), Ms=1e6, Keff=1e4, T=0.0,
                          tau0=1e-10, d=d)
    c = MU0 * lys.Ms * lys.vol[0] / (4.0 * math.pi * sep ** 3)
    ctx = _gpu_run([lys], prec, 0.1, 1e5, 40, 3, 1, 7)
    g = kmc.kmc_read(ctx, kmc.KMC_READ_DHDIP, 0)
    kmc.kmc_destroy(ctx)
    np.testing.assert_allclose(g, sign * c, rtol=tol)


def test_dhdip_fp32_on_the_gpu_trajectory():
    # FP32 moments drift from the FP64 ones, so Eq. 6 is checked on the GPU's
    # own state: S = 2 (step 0 at +Hmax, step 1 at -Hmax), one unrecorded
    # period, then one recorded period from the moments m0 read back. The GPU's
    # own fields at the two steps (debug steps from m0 and from its result m1)
    # must give the recorded value (bookkeeping), and the oracle's fields from
    # m0 and m1 must agree within the FP32 field tolerance (parity).
    lys = inputs.make_lysosome(300, 14e-9, 0.05, Keff=2e4, T=300.0, seed=4)
    H, f, S, seed = 0.02, 1e5, 2, 1
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_run(ctx, H, f, S, 1, 1, seed)
    m0 = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, 0)
    kmc.kmc_run(ctx, H, f, S, 1, 0, seed)
    g = kmc.kmc_read(ctx, kmc.KMC_READ_DHDIP, 0)
    t_step = 1.0 / (f * S)
    d0 = kmc.kmc_debug_step(ctx, H, t_step, seed, 2, m0)
    d1 = kmc.kmc_debug_step(ctx, -H, t_step, seed, 3, d0["m_out"])
    kmc.kmc_destroy(ctx)
    np.testing.assert_allclose(g, d0["B_dip"][:, 2] - d1["B_dip"][:, 2], rtol=1e-6,
                               atol=1e-9 * np.abs(g).max())
    B0 = oracle.dipolar_field(lys.pos, lys.vol, lys.Ms, m0)
    B1 = oracle.dipolar_field(lys.pos, lys.vol, lys.Ms, d0["m_out"])
    rms = np.sqrt(np.mean(np.sum(B0 ** 2, axis=1)))
    assert np.max(np.abs(g - (B0[:, 2] - B1[:, 2]))) <= 2 * 1e-5 * rms


@pytest.mark.parametrize("prec", [kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED])
def test_local_concentration_matches_oracle(prec):
    # 1501 NPs: an odd count (an FP32 padding record) and a ragged last block
    lys = inputs.make_lysosome(1501, 12e-9, 0.08, seed=21)
    small = inputs.make_lysosome(3, 12e-9, 0.01, seed=2)
    ctx = kmc.kmc_create([small, lys], prec, center=np.zeros(3))
    for N in (1, 20, kmc.KMC_PHI_MAX_N):
        g = kmc.kmc_local_concentration(ctx, 1, N)
        o = oracle.local_concentration(lys.pos, lys.vol, N)
        np.testing.assert_allclose(g, o, rtol=1e-13, atol=0)
    g = kmc.kmc_local_concentration(ctx, 0, 2)
    np.testing.assert_allclose(g, oracle.local_concentration(small.pos, small.vol, 2), rtol=1e-13)
    kmc.kmc_destroy(ctx)


def test_local_concentration_lattice_closed_form():
    # simple cubic, spacing a: the 19th-26th neighbours of an interior site are
    # at a sqrt3, so phi_20 = 3 * 20 V / (4 pi (a sqrt3)^3) there
    a, d = 25e-9, 12e-9
    lys = inputs.lattice_lysosome(9, a, d)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    g = kmc.kmc_local_concentration(ctx, 0, 20)
    kmc.kmc_destroy(ctx)
    centre = int(np.argmin(np.sum(lys.pos ** 2, axis=1)))
    V = lys.vol[centre]
    assert g[centre] == pytest.approx(3 * 20 * V / (4 * math.pi * (a * math.sqrt(3)) ** 3),
                                      rel=1e-13)


def test_local_concentration_full_size_sampled():
    (lys,), _ = inputs.config_large50000(seed=0)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    g = kmc.kmc_local_concentration(ctx, 0, 20)
    kmc.kmc_destroy(ctx)
    rng = np.random.default_rng(5)
    idx = rng.choice(lys.n, 24, replace=False)
    o = oracle.local_concentration_at(lys.pos, lys.vol, 20, idx)
    np.testing.assert_allclose(g[idx], o, rtol=1e-13)
    assert np.all(np.isfinite(g)) and np.all(g > 0)
    r = np.linalg.norm(lys.pos, axis=1)
    skin = r > lys.radius - 1.5 * lys.d  # within one diameter of the outermost centres
    assert g[r < 0.5 * lys.radius].mean() > 1.3 * g[skin].mean()


def test_shell_profile_matches_oracle():
    (lys,), run = inputs.config_small(seed=0)
    S, periods, discard, seed = 100, 4, 1, 5
    ctx = _gpu_run([lys], kmc.KMC_FP64_PLAIN, run["mu0Hmax"], run["f"], S, periods, discard, seed)
    prof = kmc.kmc_shell_profile(ctx, 0, 0.0, 5, 20)
    prof_R = kmc.kmc_shell_profile(ctx, 0, lys.radius, 10, 0)
    kmc.kmc_destroy(ctx)
    o = oracle.run(lys, 0, run["mu0Hmax"], run["f"], S, periods, discard, seed)
    if o["counters"]["near"] > 0:
        pytest.skip("a near-threshold draw occurred; trajectories may legitimately split")
    nper = periods - discard
    area = o["E_diss"] / nper / lys.vol
    phi = oracle.local_concentration(lys.pos, lys.vol, 20)
    vals = np.stack([area, o["dHdip"], phi], axis=1)
    count, mean, R = oracle.shell_profile(lys.pos, lys.vol, np.zeros(3), 0.0, 5, vals)
    assert prof["radius"] == pytest.approx(R, rel=1e-15)
    np.testing.assert_array_equal(prof["count"], count)
    a_scale = np.abs(area).max()
    np.testing.assert_allclose(prof["area"], mean[:, 0], rtol=1e-9, atol=1e-12 * a_scale)
    np.testing.assert_allclose(prof["dHdip"], mean[:, 1], rtol=0,
                               atol=1e-11 * np.abs(o["dHdip"]).max())
    np.testing.assert_allclose(prof["phi"], mean[:, 2], rtol=1e-13)
    count, mean, R = oracle.shell_profile(lys.pos, lys.vol, np.zeros(3), lys.radius, 10, vals)
    assert prof_R["radius"] == lys.radius
    np.testing.assert_array_equal(prof_R["count"], count)
    assert np.all(prof_R["phi"] == 0.0)
    assert prof_R["count"].sum() == lys.n


def test_local_errors():
    lys = inputs.make_lysosome(50, 12e-9, 0.05, seed=1)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    for N in (0, 50, kmc.KMC_PHI_MAX_N + 1):
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_local_concentration(ctx, 0, N)
        assert e.value.status == kmc.KMC_EINVAL
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_local_concentration(ctx, 1, 5)
    assert e.value.status == kmc.KMC_EINVAL
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_shell_profile(ctx, 0, 0.0, 4, 5)
    assert e.value.status == kmc.KMC_ESTATE
    kmc.kmc_run(ctx, 0.02, 1e5, 10, 1, 0, 0)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_shell_profile(ctx, 0, 0.0, 0, 5)
    assert e.value.status == kmc.KMC_EINVAL
    assert kmc.kmc_shell_profile(ctx, 0, 0.0, 3, 5)["count"].sum() == 50
    kmc.kmc_destroy(ctx)
