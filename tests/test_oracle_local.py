"""Pins of the oracle's per-NP analysis outputs:

* Eq. 6 (Sec. III.2.b): Delta_Hdip = mu0 H_dip,z(+mu0Hmax) - mu0 H_dip,z(-mu0Hmax),
  recorded by the oracle's run. Pinned by closed forms of the field of a
  saturated pair (parallel bond: +, perpendicular bond: -) and by re-deriving it
  in numpy from a trajectory taken one oracle step at a time.
* Eq. 8 (Sec. III.5): phi_N = 3 N V / (4 pi r_N^3), pinned by the neighbour
  shells of simple-cubic and body-centred-cubic lattices.
* The radial shell profile of Fig. 8, pinned by hand-placed NPs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs

MU0 = 4e-7 * math.pi


def _pair(bond, sep, d=20e-9, Keff=1e4, Ms=1e6):
    pos = np.array([[0.0, 0.0, 0.0], bond * sep])
    return inputs.Lysosome(pos=pos, axis=np.tile([0.0, 0.0, 1.0], (2, 1)),
                           vol=np.full(2, inputs.sphere_volume(d)), Ms=Ms, Keff=Keff, T=0.0,
                           tau0=1e-10, d=d)


@pytest.mark.parametrize("bond,sign", [(np.array([0.0, 0.0, 1.0]), 4.0),
                                       (np.array([1.0, 0.0, 0.0]), -2.0)])
def test_dhdip_saturated_pair_closed_form(bond, sign):
    # Two NPs with easy axes along z, T = 0, driven well past the switching
    # field mu0 H_K = 2 K / M_S (20 mT here) by 100 mT: both sit at +z at +Hmax
    # and at -z at -Hmax. The field of one on the other is
    # mu0 M_S V / (4 pi r^3) (3 (m.e) e - m): +2 c m along the bond, -c m
    # across it, so Delta = 2 * (2 c) or 2 * (-c).
    sep = 30e-9
    lys = _pair(bond, sep)
    c = MU0 * lys.Ms * lys.vol[0] / (4.0 * math.pi * sep ** 3)
    out = oracle.run(lys, 0, 0.1, 1e5, 40, 3, 1, 7)
    np.testing.assert_allclose(out["dHdip"], sign * c, rtol=1e-12)
    assert out["counters"]["flips"] == 0  # T = 0: the wells move, no jumps


def test_dhdip_zero_for_one_step_period():
    # S = 1: the +Hmax and -Hmax steps coincide (k = S/2 = 0), so Eq. 6 is 0
    lys = _pair(np.array([0.0, 0.0, 1.0]), 30e-9)
    out = oracle.run(lys, 0, 0.1, 1e5, 1, 4, 1, 7)
    assert np.all(out["dHdip"] == 0.0)


@pytest.mark.parametrize("S", [6, 7])
def test_dhdip_rederived_from_stepped_trajectory(S):
    # The run's bookkeeping (which steps, which sign, discard, average) against
    # a numpy restatement over single oracle steps at T = 300 K (same draws).
    lys = inputs.make_lysosome(24, 14e-9, 0.1, Keff=1.5e4, seed=5)
    f, periods, discard, seed, Hmax = 1e5, 3, 1, 11, 0.03
    out = oracle.run(lys, 0, Hmax, f, S, periods, discard, seed)
    m = oracle.initial_moments(lys.axis)
    t_step = 1.0 / (f * S)
    acc = np.zeros(lys.n)
    for p in range(periods):
        for k in range(S):
            H = Hmax * math.cos(2.0 * math.pi * k / S)
            st = oracle.step(lys, 0, m, H, t_step, seed, p * S + k)
            if p >= discard:
                if k == 0:
                    acc += st["B_dip"][:, 2]
                if k == S // 2:
                    acc -= st["B_dip"][:, 2]
            m = st["m_out"]
    acc /= periods - discard
    np.testing.assert_allclose(out["dHdip"], acc, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(out["m"], m)
    assert np.any(acc != 0.0)


def _cubic(n_side, a, basis):
    g = np.arange(n_side)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    pts = np.concatenate([cells + np.asarray(b, dtype=np.float64) for b in basis])
    return pts * a


def _phi(N, V, r):
    return 3.0 * N * V / (4.0 * math.pi * r ** 3)


def test_phi_simple_cubic_neighbour_shells():
    # simple cubic, spacing a: 6 neighbours at a, 12 at a sqrt2, 8 at a sqrt3,
    # 6 at 2a around an interior site
    a, V = 25e-9, 1.1e-24
    pos = _cubic(7, a, [(0, 0, 0)])
    vol = np.full(len(pos), V)
    centre = int(np.argmin(np.sum((pos - 3 * a) ** 2, axis=1)))
    for N, r in [(1, a), (6, a), (7, a * math.sqrt(2)), (18, a * math.sqrt(2)),
                 (19, a * math.sqrt(3)), (20, a * math.sqrt(3)), (26, a * math.sqrt(3)),
                 (27, 2 * a), (32, 2 * a)]:
        phi = oracle.local_concentration(pos, vol, N)
        assert phi[centre] == pytest.approx(_phi(N, V, r), rel=1e-14), N
    # a corner site has 3 neighbours at a, 3 at a sqrt2, 1 at a sqrt3, 3 at 2a
    corner = int(np.argmin(np.sum(pos ** 2, axis=1)))
    for N, r in [(3, a), (4, a * math.sqrt(2)), (6, a * math.sqrt(2)), (7, a * math.sqrt(3)),
                 (8, 2 * a), (10, 2 * a)]:
        phi = oracle.local_concentration(pos, vol, N)
        assert phi[corner] == pytest.approx(_phi(N, V, r), rel=1e-14), N


def test_phi_bcc_and_volume_of_the_site():
    # body-centred cubic, cube edge a: 8 neighbours at a sqrt3 / 2, 6 at a
    a = 30e-9
    pos = _cubic(6, a, [(0, 0, 0), (0.5, 0.5, 0.5)])
    rng = np.random.default_rng(3)
    vol = rng.uniform(0.5e-24, 2e-24, len(pos))  # phi uses the site's own V
    centre = int(np.argmin(np.sum((pos - 2.5 * a) ** 2, axis=1)))
    phi8 = oracle.local_concentration(pos, vol, 8)
    phi14 = oracle.local_concentration(pos, vol, 14)
    assert phi8[centre] == pytest.approx(_phi(8, vol[centre], a * math.sqrt(3) / 2), rel=1e-14)
    assert phi14[centre] == pytest.approx(_phi(14, vol[centre], a), rel=1e-14)


def test_phi_near_surface_lower_than_core():
    # Sec. III.4-5: NPs near the membrane have fewer neighbours
    lys = inputs.make_lysosome(1500, 12e-9, 0.1, seed=2)
    phi = oracle.local_concentration(lys.pos, lys.vol, 20)
    r = np.linalg.norm(lys.pos, axis=1) / lys.radius
    core, skin = phi[r < 0.5], phi[r > 0.9]
    assert core.mean() > 1.4 * skin.mean()
    # the core's local concentration is near the lysosome's c
    assert 0.7 * lys.c < np.median(core) < 1.5 * lys.c


def test_phi_rejects_bad_N():
    pos = np.eye(3)
    with pytest.raises(ValueError):
        oracle.local_concentration(pos, np.ones(3), 0)
    with pytest.raises(ValueError):
        oracle.local_concentration(pos, np.ones(3), 3)


def test_shell_profile_hand_placed():
    R, ns = 100e-9, 10
    radii = (np.arange(ns) + 0.5) * R / ns
    dirs = np.array([[1, 0, 0], [0, -1, 0], [0, 0, 1], [-1, 0, 0], [0, 1, 0]] * 2, float)
    c = np.array([1e-9, -2e-9, 3e-9])
    pos = c + radii[:, None] * dirs
    vol = np.full(ns, 1e-25)
    vals = np.stack([np.arange(ns, dtype=float), -np.arange(ns, dtype=float)], axis=1)
    count, mean, Rused = oracle.shell_profile(pos, vol, c, R, ns, vals)
    assert Rused == R
    np.testing.assert_array_equal(count, np.ones(ns))
    np.testing.assert_allclose(mean, vals, rtol=0, atol=0)
    # 5 shells over the same NPs: pairs of them, volume-weighted means
    vol2 = np.tile([1.0, 3.0], ns // 2) * 1e-25
    count, mean, _ = oracle.shell_profile(pos, vol2, c, R, 5, vals)
    np.testing.assert_array_equal(count, np.full(5, 2.0))
    expect = (vals[0::2] * 1.0 + vals[1::2] * 3.0) / 4.0
    np.testing.assert_allclose(mean, expect, rtol=1e-15)


def test_shell_profile_enclosing_radius_and_outside():
    d = 10e-9
    V = inputs.sphere_volume(d)
    pos = np.array([[0.0, 0.0, 0.0], [40e-9, 0.0, 0.0], [0.0, 0.0, -70e-9]])
    vol = np.full(3, V)
    vals = np.array([[1.0], [2.0], [3.0]])
    count, mean, Rused = oracle.shell_profile(pos, vol, np.zeros(3), 0.0, 4, vals)
    assert Rused == pytest.approx(70e-9 + d / 2, rel=1e-15)
    np.testing.assert_array_equal(count, [1, 0, 1, 1])
    np.testing.assert_array_equal(mean[:, 0], [1.0, 0.0, 2.0, 3.0])
    # an NP outside the given radius goes to the last shell
    count, mean, _ = oracle.shell_profile(pos, vol, np.zeros(3), 60e-9, 5, vals)
    np.testing.assert_array_equal(count, [1, 0, 0, 1, 1])
    np.testing.assert_array_equal(mean[:, 0], [1.0, 0.0, 0.0, 2.0, 3.0])
