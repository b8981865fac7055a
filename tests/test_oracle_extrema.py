"""Pins of the oracle's extremum search on Eq. 2 (Sec. II.1, step iv).

Checks: the zero-field profile (minima along the easy axis, maxima across it,
barrier K_eff V); the Stoner-Wohlfarth astroid, which says when two minima
exist; a brute-force fine scan of Eq. 2 on many random (field, angle) pairs;
the switching field H_K = 2 K_eff / (mu0 M_S) for a field along the axis."""
import math

import numpy as np
import pytest

import oracle

MS = 1e6
K = 1.3e4
V = math.pi * (12e-9) ** 3 / 6
BK = 2 * K / MS  # mu0 H_K, T


def E_eq2(th, B, phi):
    return K * V * np.sin(th) ** 2 - MS * V * B * np.cos(th - phi)


def test_zero_field():
    ex = oracle.extrema(K, MS, V, 0.0, 0.7)
    mins = sorted(t for t, e, m in ex if m)
    maxs = sorted(t for t, e, m in ex if not m)
    assert len(mins) == 2 and len(maxs) == 2
    assert min(abs(mins[0]), abs(mins[0] - 2 * math.pi)) < 1e-12
    assert abs(mins[1] - math.pi) < 1e-12
    np.testing.assert_allclose(maxs, [math.pi / 2, 3 * math.pi / 2], atol=1e-12)
    Emax = [e for t, e, m in ex if not m]
    Emin = [e for t, e, m in ex if m]
    np.testing.assert_allclose(min(Emax) - np.array(Emin), K * V, rtol=1e-12)


def astroid(h, phi):
    return h ** (2 / 3) * (abs(math.sin(phi)) ** (2 / 3) + abs(math.cos(phi)) ** (2 / 3))


def test_astroid_counts():
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(3000):
        h = rng.uniform(0, 1.6)
        phi = rng.uniform(0, 2 * math.pi)
        a = astroid(h, phi)
        if abs(a - 1) < 0.02:
            continue  # two extrema may share one grid cell near the astroid
        ex = oracle.extrema(K, MS, V, h * BK, phi)
        nmin = sum(m for _, _, m in ex)
        assert nmin == (2 if a < 1 else 1), (h, phi)
        assert len(ex) == 2 * nmin
        checked += 1
    assert checked > 2500


def test_against_brute_force_scan():
    rng = np.random.default_rng(1)
    th = np.linspace(0, 2 * math.pi, 2_000_001)[:-1]
    step = th[1] - th[0]
    for _ in range(40):
        h = rng.uniform(0, 1.4)
        phi = rng.uniform(0, math.pi)
        if abs(astroid(h, phi) - 1) < 0.02:
            continue
        E = E_eq2(th, h * BK, phi)
        Em, Ep = np.roll(E, 1), np.roll(E, -1)
        bmin = np.where((E < Em) & (E <= Ep))[0]
        bmax = np.where((E > Em) & (E >= Ep))[0]
        ex = oracle.extrema(K, MS, V, h * BK, phi)
        omin = sorted(t for t, e, m in ex if m)
        omax = sorted(t for t, e, m in ex if not m)
        assert len(omin) == len(bmin) and len(omax) == len(bmax)

        def circ(a, b):
            d = abs(a - b) % (2 * math.pi)
            return min(d, 2 * math.pi - d)

        for tb in th[bmin]:
            assert min(circ(tb, t) for t in omin) <= 1.5 * step
        for tb in th[bmax]:
            assert min(circ(tb, t) for t in omax) <= 1.5 * step
        for t, e, m in ex:
            # the energy is Eq. 2 at the root and the root is stationary
            assert abs(e - E_eq2(t, h * BK, phi)) <= 1e-12 * K * V
            dE = K * V * math.sin(2 * t) + MS * V * h * BK * math.sin(t - phi)
            assert abs(dE) < 1e-12 * K * V


@pytest.mark.parametrize("phi", [0.0, math.pi])
def test_switching_field_along_axis(phi):
    """For a field along the easy axis the far minimum disappears at H_K."""
    below = oracle.extrema(K, MS, V, 0.995 * BK, phi)
    above = oracle.extrema(K, MS, V, 1.005 * BK, phi)
    assert sum(m for _, _, m in below) == 2
    assert sum(m for _, _, m in above) == 1
    t_min = [t for t, e, m in above if m][0]
    # the surviving minimum lies along the field
    assert min(abs(t_min - phi), abs(t_min - phi - 2 * math.pi)) < 1e-10


def _plane(axis, B):
    bh = B / np.linalg.norm(B)
    ep = bh - (bh @ axis) * axis
    ep /= np.linalg.norm(ep)
    return ep, math.acos(np.clip(bh @ axis, -1, 1))


def test_barriers_use_the_lower_maximum():
    """dE of steps iv/vi against a brute-force scan: barrier top = the lower of
    the two maxima, for both wells."""
    rng = np.random.default_rng(4)
    th = np.linspace(0, 2 * math.pi, 400_001)[:-1]
    done = 0
    while done < 25:
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        B = rng.normal(size=3) * 0.4 * BK
        ep, phi = _plane(axis, B)
        h = np.linalg.norm(B) / BK
        if abs(astroid(h, phi) - 1) < 0.05 or astroid(h, phi) > 1:
            continue
        E = E_eq2(th, np.linalg.norm(B), phi)
        Em, Ep = np.roll(E, 1), np.roll(E, -1)
        emin = E[(E < Em) & (E <= Ep)]
        emax = E[(E > Em) & (E >= Ep)]
        assert len(emin) == 2 and len(emax) == 2
        r = oracle.np_update(axis, axis, B, K, MS, V, 300.0, 1e-10, 1e-9, 0.999)
        expect = sorted(emax.min() - emin)
        np.testing.assert_allclose(sorted(r["dE"]), expect, rtol=1e-6)
        assert abs(emax.max() - emax.min()) > 1e-3 * K * V  # the choice matters
        done += 1


def test_fall_follows_the_energy_profile():
    """Steps iii and v against brute-force steepest descent from the projected
    moment on a fine grid (T = 0, so no jump)."""
    rng = np.random.default_rng(6)
    for _ in range(60):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        B = rng.normal(size=3) * 0.5 * BK
        m_old = rng.normal(size=3)
        m_old /= np.linalg.norm(m_old)
        ep, phi = _plane(axis, B)
        Bm = np.linalg.norm(B)
        t = math.atan2(m_old @ ep, m_old @ axis)
        dt = 1e-5

        def dEdt(x):
            return K * V * math.sin(2 * x) + MS * V * Bm * math.sin(x - phi)

        g0 = dEdt(t)
        if abs(g0) < 1e-4 * K * V:
            continue  # too close to a maximum to call
        direction = -1.0 if g0 > 0 else 1.0
        for _ in range(700_000):
            if dEdt(t + direction * dt) * direction > 0:
                break
            t += direction * dt
        expect = math.cos(t) * axis + math.sin(t) * ep
        r = oracle.np_update(axis, m_old, B, K, MS, V, 0.0, 1e-10, 1e-9, 0.5)
        np.testing.assert_allclose(r["m_new"], expect, atol=3e-5)
