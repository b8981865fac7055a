"""T = 0 Stoner-Wohlfarth limits of the oracle (Sec. II.1 step vii "T = 0";
Sec. III.2.c) and the SAR conversion of Sec. III.2.a.

* Axes along the field: the moment reverses at the anisotropy field
  mu0 H_K = 2 K_eff / M_S (within one field step).
* Axes uniform on the sphere: coercive field 0.479 H_K and remanence M_S / 2
  (textbook Stoner-Wohlfarth), and dimensionless area A / K_eff = 2, the value
  the paper gives for randomly oriented NPs at low concentration.
* 10^4 J/m^3 at 100 kHz and rho = 5200 kg/m^3 is 192 W/g.
* The per-NP energies: exact in the isolated square-loop limit, and with
  dipolar coupling their sum is the area of the recorded M(H) loop.
"""
import math

import numpy as np

import oracle
from paper_1407_2737_gb300 import inputs
from test_oracle_dynamics import read_paper_values

MS = 1e6


def _far_apart(axis, d, **kw):
    n = len(axis)
    pos = np.zeros((n, 3))
    pos[:, 0] = np.arange(n) * 1e-3
    vol = np.full(n, math.pi * d ** 3 / 6)
    return inputs.Lysosome(pos=pos, axis=np.asarray(axis, float), vol=vol, Ms=MS, d=d,
                           **kw)


def fibonacci_sphere(n):
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    r = np.sqrt(1 - z * z)
    ph = math.pi * (1 + math.sqrt(5)) * k
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


def test_aligned_axes_switch_at_HK():
    K = 1.3e4
    BK = 2 * K / MS
    lys = _far_apart([[0, 0, 1.0], [0, 0, -1.0]], 20e-9, Keff=K, T=0.0, tau0=1e-10)
    S = 2000
    Hmax = 1.5 * BK
    out = oracle.run(lys, 0, Hmax, 1e5, S, 2, 1, seed=0)
    H, M = out["loop_H"], out["loop_M"]
    k = np.arange(S)
    desc = (k > 0) & (k < S // 2)
    first_neg = np.where(desc & (M < 0))[0][0]
    dH = Hmax * 2 * math.pi / S
    assert abs(-H[first_neg] - BK) <= dH
    asc = k >= S // 2
    first_pos = np.where(asc & (M > 0))[0][0]
    assert abs(H[first_pos] - BK) <= dH
    # square loop of height 2 M_S and width 2 H_K: A = 4 M_S mu0 H_K = 8 K_eff
    assert abs(out["area"] / (4 * MS * BK) - 1) < 0.01


def test_random_axes_loop(golden_dir):
    vals = read_paper_values(golden_dir)
    K = 1.3e4
    BK = 2 * K / MS
    axis = fibonacci_sphere(600)
    lys = _far_apart(axis, 20e-9, Keff=K, T=0.0, tau0=1e-10)
    S = 1600
    out = oracle.run(lys, 0, 2.0 * BK, 1e5, S, 2, 1, seed=0, nthreads=8)
    H, M = out["loop_H"], out["loop_M"]
    half = S // 2
    # descending branch: +Hmax -> -Hmax
    Hd, Md = H[:half + 1], M[:half + 1]
    i = np.where(Md < 0)[0][0]
    Hc = Hd[i - 1] + (Hd[i] - Hd[i - 1]) * (0 - Md[i - 1]) / (Md[i] - Md[i - 1])
    assert abs(-Hc / BK - 0.479) < 0.01
    j = np.where(Hd < 0)[0][0]
    Mr = Md[j - 1] + (Md[j] - Md[j - 1]) * (0 - Hd[j - 1]) / (Hd[j] - Hd[j - 1])
    assert abs(Mr - 0.5) < 0.01
    # A / K_eff = 2 (Sec. III.2.c)
    assert abs(out["area"] / K - vals["area_over_K_low_conc"]) < 0.03
    # the area is the enclosed area of the recorded M(H) loop
    loop_area = MS * np.sum(H * (M - np.roll(M, 1)))
    assert abs(loop_area / out["area"] - 1) < 0.02


def test_sar_conversion(golden_dir):
    v = read_paper_values(golden_dir)
    s = oracle.sar(v["sar_area_J_m3"], v["sar_f_Hz"], v["sar_rho_kg_m3"])  # W/kg
    assert abs(s / 1000.0 - v["sar_W_per_g"]) < 0.5


def test_per_np_energy_of_isolated_square_loops():
    # The per-NP split of the loop area (reading 12) in the limit where every
    # reading agrees: isolated NPs, axes along +-z, T = 0. Each moment starts at
    # m_z = +1, drops to -1 at the first step of the descending half whose field
    # lies beyond -H_K and returns at the first ascending step beyond +H_K, so
    # per period E_i = mu0 M_S V (H_up * 2 + H_down * (-2)) with those two field
    # samples.
    K = 1.3e4
    BK = 2 * K / MS
    lys = _far_apart([[0, 0, 1.0], [0, 0, -1.0], [0, 0, 1.0]], 16e-9, Keff=K, T=0.0,
                     tau0=1e-10)
    S, periods, discard = 400, 3, 1
    Hmax = 1.72 * BK  # every sample at least 1 % away from +-H_K
    out = oracle.run(lys, 0, Hmax, 1e5, S, periods, discard, seed=0)
    H, M = out["loop_H"][:S], out["loop_M"][:S]
    # no field sample sits where the grid could miss the vanishing well
    assert np.all(np.abs(np.abs(H) / BK - 1) > 1e-3)
    k_down = np.where(M < 0)[0][0]
    k_up = k_down + np.where(M[k_down:] > 0)[0][0]
    assert H[k_down] < -BK and H[k_down - 1] >= -BK
    assert H[k_up] > BK and H[k_up - 1] <= BK
    E = MS * lys.vol * 2.0 * (H[k_up] - H[k_down])
    nper = periods - discard
    np.testing.assert_allclose(out["E_diss"] / nper, E, rtol=1e-12)


def test_per_np_energies_sum_to_the_loop_area_with_interactions():
    # Sec. III.2.a defines the heating through the area of the M(H) loop. With
    # strong dipolar coupling the split between NPs is a reading (reading 12),
    # but the total is not: sum_i V_i dm_z,i over a step is V_tot dM over that
    # step, so the per-NP energies must add up to M_S V_tot sum_k mu0H_k
    # (M_k - M_(k-1)) of the recorded loop, M_(-1) being the volume-weighted
    # m_z before the first recorded step. A dropped volume weight, a shifted
    # field index or a wrong sign in the per-NP accumulation breaks it.
    lys = inputs.make_lysosome(60, 14e-9, 0.2, Ms=MS, Keff=2e4, T=300.0, tau0=1e-10,
                               seed=7)
    lys.vol = lys.vol * np.random.default_rng(1).uniform(0.6, 1.0, lys.n)  # polydisperse
    mz0 = oracle.initial_moments(lys.axis)[:, 2]
    vtot = float(lys.vol.sum())
    S, periods = 120, 2
    out = oracle.run(lys, 0, 0.03, 1e5, S, periods, 0, seed=3)
    H, M = out["loop_H"], out["loop_M"]
    assert out["counters"]["flips"] > 0  # thermal jumps happened on the way
    M_prev = np.concatenate([[float(np.dot(lys.vol, mz0)) / vtot], M[:-1]])
    loop = MS * vtot * np.sum(H * (M - M_prev))
    scale = MS * vtot * np.sum(np.abs(H) * np.abs(M - M_prev))
    total = float(out["E_diss"].sum())
    assert abs(total - loop) <= 1e-12 * scale, (total, loop, scale)
    # the same total as the area per unit volume and cycle
    assert abs(out["area"] * vtot * periods - total) <= 1e-12 * scale
    # dipolar coupling moves the individual NPs' shares: they are not all alike
    assert np.std(out["E_diss"] / lys.vol) > 0
