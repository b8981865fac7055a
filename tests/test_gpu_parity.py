"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (derived from the arithmetic, FP64 path):
* dipolar field: |dB_i| <= 1e-12 * sum_j |term_ij| (the two sides sum the same
  terms in different orders; each rounding is <= 2^-53 of a partial sum), the
  reading of a "1e-12 relative" FP64 field bound for a sum whose terms cancel;
  where they cancel by at most a factor 4, also |dB_i| <= 1e-12 |B_i|;
* barriers: |d(E3 - E_a)| <= 1e-12 |E3 - E_a| + 1e-14 E_scale, E_scale =
  K_eff V + M_S V |B| (each energy carries a few ulp of E_scale);
* jump probabilities: |dP| <= 1e-12 P + 1e-13;
* draws: bit for bit; moments: 1e-12, except NPs whose draw lies within 1e-9
  of P (counted as near-threshold, where the decision may differ).
FP32-mixed path: field error max_i |dB_i| / rms_i |B_i| <= 1e-5, SAR within
1 % of the oracle's over 32 seeds with common random numbers.
"""
import math
import os

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


def perturbed_moments(axis, rng, amp=0.3):
    m = oracle.initial_moments(axis) + amp * rng.normal(size=axis.shape)
    return m / np.linalg.norm(m, axis=1, keepdims=True)


def abs_term_sum(lys, m):
    """sum_j |term_ij| of Eq. 1 (per target), the scale of the summation error."""
    d = lys.pos[None, :, :] - lys.pos[:, None, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    w = MU0 * lys.Ms * lys.vol / (4 * math.pi)
    return (3.0 + 1.0) * (w[None, :] / r ** 3).sum(axis=1)


def oracle_steps(lyss, m_all, Hs, t_step, seed, step):
    outs, o = [], 0
    for l, ly in enumerate(lyss):
        outs.append(oracle.step(ly, l, m_all[o:o + ly.n], Hs[l], t_step, seed, step))
        o += ly.n
    cat = {k: np.concatenate([x[k] for x in outs]) for k in outs[0]}
    return cat


def ragged_batch(seed=0):
    sizes = [1, 2, 33, 100, 31, 257]
    lyss = [inputs.make_lysosome(n, 12e-9, 0.05 if n > 2 else 0.01, Ms=1e6, Keff=1.3e4,
                                 T=300.0, tau0=1e-10, seed=seed * 10 + q)
            for q, n in enumerate(sizes)]
    lyss[3].T = 0.0          # one lysosome at T = 0
    lyss[4].Keff = 2.6e4     # another material
    lyss[5].Ms = 8e5
    return lyss


@pytest.mark.parametrize("prec", [kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED])
def test_draws_are_bit_exact(prec):
    lyss = ragged_batch(1)
    ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
    m = np.concatenate([oracle.initial_moments(l.axis) for l in lyss])
    for seed, step in [(0, 0), (123456789, 5), ((1 << 40) + 3, (1 << 33) + 7)]:
        g = kmc.kmc_debug_step(ctx, np.full(len(lyss), 0.01), 5e-8, seed, step, m)
        o, expect = 0, []
        for l, ly in enumerate(lyss):
            expect += [oracle.uniform(seed, step, i, l) for i in range(ly.n)]
        assert np.array_equal(g["u"], np.array(expect))


@pytest.mark.parametrize("tile,warps,chunk", [(64, 4, 0), (128, 8, 64), (32, 16, 128),
                                              (64, 4, 192)])
def test_fp64_step_parity(tile, warps, chunk):
    lyss = ragged_batch(2)
    rng = np.random.default_rng(3)
    m = np.concatenate([perturbed_moments(l.axis, rng) for l in lyss])
    Hs = np.array([0.012, -0.02, 0.0, 0.018, -0.005, 0.03])
    t_step = 1 / (1e5 * 200)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    kmc.kmc_tuning(ctx, warps, tile, chunk)
    g = kmc.kmc_debug_step(ctx, Hs, t_step, 11, 1000, m)
    o = oracle_steps(lyss, m, Hs, t_step, 11, 1000)
    off = 0
    worst = 0.0
    for ly in lyss:
        sl = slice(off, off + ly.n)
        off += ly.n
        scale = abs_term_sum(ly, m[sl])
        tol = 1e-12 * scale
        dB = np.abs(g["B_dip"][sl] - o["B_dip"][sl])
        assert np.all(dB <= tol[:, None] + 1e-300)
        # relative to |B_i| where the terms cancel by at most a factor 4: the
        # summation error is then below n u sum_j |term_ij| <= 4 n u |B_i|, n <= 257
        Bn = np.linalg.norm(o["B_dip"][sl], axis=1)
        ok = (Bn > 0.0) & (Bn >= 0.25 * scale)  # a lone NP has no field at all
        rel = np.linalg.norm(dB, axis=1)[ok] / Bn[ok]
        if rel.size:
            worst = max(worst, float(rel.max()))
            assert rel.max() <= 1e-12
    print("FP64 field: max |dB_i| / |B_i| = %.2e (NPs without heavy cancellation)" % worst)
    assert np.array_equal(g["n_min"], o["n_min"])
    two = o["n_min"] == 2
    vols = np.concatenate([l.vol for l in lyss])
    Kv = np.concatenate([np.full(l.n, l.Keff) for l in lyss]) * vols
    Ms = np.concatenate([np.full(l.n, l.Ms) for l in lyss])
    Bt = np.linalg.norm(o["B_dip"] + np.repeat(Hs, [l.n for l in lyss])[:, None] * [0, 0, 1],
                        axis=1)
    Escale = Kv + Ms * vols * Bt
    err = np.abs(g["dE"] - o["dE"])[two]
    assert np.all(err <= 1e-12 * np.abs(o["dE"][two]) + 1e-14 * Escale[two][:, None])
    assert np.all(np.abs(g["P"] - o["P"]) <= 1e-12 * o["P"] + 1e-13)
    same = o["near"] == 0
    assert np.max(np.abs(g["m_out"][same] - o["m_out"][same])) < 1e-12
    assert np.array_equal(g["flipped"][same], o["flipped"][same])
    assert np.array_equal(g["degenerate"], o["degenerate"])


def test_fp32_shapes_agree_and_are_deterministic():
    """Every launch shape (warps, tile, source split) gives the same FP32 fields
    within FP32 rounding, and one shape run twice gives identical bits."""
    lyss = ragged_batch(4)
    rng = np.random.default_rng(8)
    m = np.concatenate([perturbed_moments(l.axis, rng) for l in lyss])
    Hs = np.full(len(lyss), 0.01)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    outs = []
    for shape in [(4, 64, 0), (8, 128, 0), (4, 32, 64), (16, 64, 128), (8, 64, 192)]:
        kmc.kmc_tuning(ctx, *shape)
        outs.append(kmc.kmc_debug_step(ctx, Hs, 5e-8, 2, 9, m))
    again = kmc.kmc_debug_step(ctx, Hs, 5e-8, 2, 9, m)
    for k in ("B_dip", "P", "m_out", "dE"):
        assert np.array_equal(again[k], outs[-1][k])
    rms = np.sqrt(np.mean(np.sum(outs[0]["B_dip"] ** 2, axis=1)))
    for o in outs[1:]:
        assert np.max(np.abs(o["B_dip"] - outs[0]["B_dip"])) < 2e-6 * rms
        assert np.array_equal(o["u"], outs[0]["u"])


def test_fp32_field_error_and_state():
    (lys,), run = inputs.config_single2000(replicas=1, seed=4)
    rng = np.random.default_rng(5)
    m = perturbed_moments(lys.axis, rng, 0.5)
    t_step = 1 / (run["f"] * run["S"])
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    g = kmc.kmc_debug_step(ctx, 0.015, t_step, 3, 42, m)
    # the GPU path computes with float32 moments: give the oracle the same state
    m32 = m.astype(np.float32).astype(np.float64)
    o = oracle.step(lys, 0, m32, 0.015, t_step, 3, 42)
    rms = np.sqrt(np.mean(np.sum(o["B_dip"] ** 2, axis=1)))
    err = np.max(np.linalg.norm(g["B_dip"] - o["B_dip"], axis=1)) / rms
    assert err <= 1e-5, err
    assert np.array_equal(g["u"], o["u"])
    # probabilities: FP32 field and extrema, FP64 exponent
    assert np.max(np.abs(g["P"] - o["P"])) < 2e-3
    agree = np.mean(np.all(np.abs(g["m_out"] - o["m_out"]) < 1e-4, axis=1))
    assert agree > 0.995
    np.testing.assert_allclose(np.linalg.norm(g["m_out"], axis=1), 1.0, atol=2e-6)


def _run_both(lyss, prec, run, periods, discard, seed):
    ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
    kmc.kmc_run(ctx, run["mu0Hmax"], run["f"], run["S"], periods, discard, seed)
    res = dict(loop=[kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, l) for l in range(len(lyss))],
               E=[kmc.kmc_read(ctx, kmc.KMC_READ_NP_ENERGY, l) for l in range(len(lyss))],
               m=[kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l) for l in range(len(lyss))],
               sar=[kmc.kmc_read(ctx, kmc.KMC_READ_SAR, l)[0] for l in range(len(lyss))],
               cnt=[kmc.kmc_read(ctx, kmc.KMC_READ_COUNTERS, l) for l in range(len(lyss))],
               H=kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_H, 0))
    kmc.kmc_destroy(ctx)
    return res


def test_fp64_trajectory_flip_for_flip():
    (lys,), run = inputs.config_small(seed=0)
    periods, discard = 6, 2
    g = _run_both([lys], kmc.KMC_FP64_PLAIN, run, periods, discard, 0)
    o = oracle.run(lys, 0, run["mu0Hmax"], run["f"], run["S"], periods, discard, 0)
    if o["counters"]["near"] > 0:
        pytest.skip("a near-threshold draw occurred; trajectories may legitimately split")
    assert g["cnt"][0][0] == o["counters"]["flips"]
    np.testing.assert_allclose(g["loop"][0], o["loop_M"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(g["H"], o["loop_H"], rtol=1e-15, atol=0)
    np.testing.assert_allclose(g["m"][0], o["m"], rtol=0, atol=1e-11)
    nper = periods - discard
    np.testing.assert_allclose(g["E"][0], o["E_diss"] / nper, rtol=1e-9,
                               atol=1e-12 * np.abs(o["E_diss"]).max())
    assert abs(g["sar"][0] - o["sar"]) <= 1e-9 * abs(o["sar"]) + 1e-9


def test_fp32_sar_within_one_percent_over_32_seeds():
    """32 replicas of one lysosome (each its own random stream); oracle in FP64,
    GPU in FP32-mixed; the mean SAR agrees within 1 %."""
    lys = inputs.make_lysosome(100, 20e-9, 0.02, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10,
                               seed=7)
    reps = 32
    S, periods, discard, H, f = 100, 4, 1, 0.04, 1e5
    run = dict(mu0Hmax=H, f=f, S=S)
    g = _run_both(inputs.replicate(lys, reps), kmc.KMC_FP32_MIXED, run, periods, discard, 9)
    sar_o = [oracle.run(lys, r, H, f, S, periods, discard, 9, nthreads=8)["sar"]
             for r in range(reps)]
    mg, mo = float(np.mean(g["sar"])), float(np.mean(sar_o))
    assert mo > 0
    assert abs(mg - mo) / mo < 0.01, (mg, mo)


def test_checkpoint_resume_is_bit_identical(tmp_path):
    (lys,), run = inputs.config_small(seed=1)
    for prec in (kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED):
        a = kmc.kmc_create([lys], prec, center=np.zeros(3))
        kmc.kmc_run(a, 0.02, 1e5, 50, 3, 0, 5)
        kmc.kmc_run(a, 0.02, 1e5, 50, 2, 0, 5)
        ref_m = kmc.kmc_read(a, kmc.KMC_READ_MOMENTS)
        ref_loop = kmc.kmc_read(a, kmc.KMC_READ_LOOP_M)
        b = kmc.kmc_create([lys], prec, center=np.zeros(3))
        kmc.kmc_run(b, 0.02, 1e5, 50, 3, 0, 5)
        p = str(tmp_path / ("ck%d.bin" % prec))
        kmc.kmc_save(b, p)
        c = kmc.kmc_create([lys], prec, center=np.zeros(3))
        kmc.kmc_load(c, p)
        assert kmc.kmc_info(c)["global_step"] == 150
        kmc.kmc_run(c, 0.02, 1e5, 50, 2, 0, 5)
        assert np.array_equal(kmc.kmc_read(c, kmc.KMC_READ_MOMENTS), ref_m)
        assert np.array_equal(kmc.kmc_read(c, kmc.KMC_READ_LOOP_M), ref_loop)


def test_errors_and_capacity(tmp_path):
    (lys,), run = inputs.config_small(seed=2)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_read(ctx, kmc.KMC_READ_SAR)
    assert e.value.status == kmc.KMC_ESTATE
    kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 1, 0)
    L = kmc.lib()
    import ctypes as C
    n = C.c_int64()
    buf = np.zeros(3)
    st = L.kmc_read(ctx.handle, kmc.KMC_READ_LOOP_M, 0, buf.ctypes.data_as(C.POINTER(C.c_double)),
                    3, C.byref(n))
    assert st == kmc.KMC_ECAPACITY and n.value == 20
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 3, 0)
    assert e.value.status == kmc.KMC_EINVAL
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a checkpoint")
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_load(ctx, str(bad))
    assert e.value.status == kmc.KMC_EIO
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_read(ctx, kmc.KMC_READ_SAR, 5)
    assert e.value.status == kmc.KMC_EINVAL
    # a checkpoint whose moment is damaged (NaN, or no longer of unit length)
    # is refused and leaves the context's moments as they were
    good = tmp_path / "good.bin"
    kmc.kmc_save(ctx, str(good))
    m_before = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS)
    raw = bytearray(good.read_bytes())
    first = 8 + 3 * 4 + 2 * 8 + 4 * 1  # magic, int32 header, int64 header, the NP counts
    for bad_x in (float("nan"), 2.0):
        dmg = bytearray(raw)
        dmg[first:first + 4] = np.float32(bad_x).tobytes()  # x of NP 0 (float4 records)
        bad.write_bytes(bytes(dmg))
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_load(ctx, str(bad))
        assert e.value.status == kmc.KMC_EINVAL and "unit vector" in str(e.value)
        assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS), m_before)
    kmc.kmc_load(ctx, str(good))
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS), m_before)


def test_full_size_sampled():
    """The 8 x 2000-NP workload in the launch shape the benchmark uses: sampled
    fields against the oracle one target at a time, draws bit-exact, steps
    iii-vii of the sampled targets against the oracle's update fed the GPU's
    field (the tolerances of tests/test_gpu_workloads.py), invariants
    everywhere: after one recorded period every lysosome's per-NP energies add
    up to the area of its recorded M(H) loop."""
    from test_gpu_workloads import check_update
    lyss, run = inputs.config_single2000(replicas=8, seed=0)
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_run(ctx, run["mu0Hmax"], run["f"], run["S"], 1, 0, run["seed"])  # tunes, warms
    # that recorded period, every lysosome: the per-NP energies add up to the
    # area of the recorded M(H) loop (Sec. III.2.a), M_(-1) being the initial
    # state (moments along the float32 axes, m_z >= 0)
    H = kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_H, 0)
    for l in range(8):
        ly = lyss[l]
        M = kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, l)
        E = kmc.kmc_read(ctx, kmc.KMC_READ_NP_ENERGY, l)
        vtot = float(ly.vol.sum())
        mz0 = np.abs(kmc.kmc_read(ctx, kmc.KMC_READ_AXES, l).reshape(-1, 3)[:, 2])
        dM = M - np.concatenate([[float(np.dot(ly.vol, mz0)) / vtot], M[:-1]])
        scale = ly.Ms * vtot * np.sum(np.abs(H) * np.abs(dM))
        assert abs(E.sum() - ly.Ms * vtot * np.sum(H * dM)) <= 1e-9 * scale, l
    m_all = np.concatenate([kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, l) for l in range(8)])
    t_step = 1 / (run["f"] * run["S"])
    g = kmc.kmc_debug_step(ctx, 0.02, t_step, 1, 200, m_all)
    rng = np.random.default_rng(0)
    compared = ambiguous = 0
    for l in (0, 7):
        idx = rng.choice(2000, 64, replace=False)
        m = m_all[2000 * l:2000 * (l + 1)]
        B = oracle.dipolar_field_at(lyss[l].pos, lyss[l].vol, lyss[l].Ms, m, idx)
        Bg = g["B_dip"][2000 * l + idx]
        rms = np.sqrt(np.mean(np.sum(B ** 2, axis=1)))
        assert np.max(np.linalg.norm(Bg - B, axis=1)) / rms <= 1e-5
        assert np.array_equal(g["u"][2000 * l + idx],
                              [oracle.uniform(1, 200, int(i), l) for i in idx])
        axes = kmc.kmc_read(ctx, kmc.KMC_READ_AXES, l)
        m32 = m.astype(np.float32).astype(np.float64)
        c, a = check_update(lyss[l], axes[idx], m32[idx], Bg, 0.02, t_step, g, 2000 * l + idx)
        compared += c
        ambiguous += a
    kmc.kmc_destroy(ctx)
    assert compared >= 0.95 * (compared + ambiguous), (compared, ambiguous)
    np.testing.assert_allclose(np.linalg.norm(g["m_out"], axis=1), 1.0, atol=2e-6)
    assert np.all((g["P"] >= 0) & (g["P"] <= 1))
