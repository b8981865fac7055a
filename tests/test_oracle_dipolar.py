"""Pins of the oracle's dipolar field, Eq. 1 (Sec. II.1).

Closed forms of the point-dipole field (on the axis of a dipole 2 w / r^3, on
its equator -w / r^3, with w = mu0 M_S V / 4 pi), their superposition for
three NPs, the cubic symmetry of a lattice sphere, reciprocity, and the field
as the numerical gradient of the magnetic scalar potential."""
import math

import numpy as np

import oracle
from paper_1407_2737_gb300 import inputs

MU0 = 4e-7 * math.pi
MS = 1e6
D = 12e-9
V = math.pi * D ** 3 / 6


def w(vol=V):
    return MU0 * MS * vol / (4 * math.pi)


def test_two_coaxial_and_broadside():
    r = 1.7 * D
    pos = np.array([[0, 0, 0], [0, 0, r]], float)
    vol = np.array([V, V])
    # moments along the bond: the field on each is 2 w / r^3 along the moment
    B = oracle.dipolar_field(pos, vol, MS, np.array([[0, 0, 1], [0, 0, 1]], float))
    np.testing.assert_allclose(B[0], [0, 0, 2 * w() / r ** 3], rtol=1e-14, atol=0)
    np.testing.assert_allclose(B[1], [0, 0, 2 * w() / r ** 3], rtol=1e-14, atol=0)
    # moments across the bond: -w / r^3 along the moment
    B = oracle.dipolar_field(pos, vol, MS, np.array([[1, 0, 0], [0, 1, 0]], float))
    np.testing.assert_allclose(B[0], [0, -w() / r ** 3, 0], rtol=1e-14, atol=1e-30)
    np.testing.assert_allclose(B[1], [-w() / r ** 3, 0, 0], rtol=1e-14, atol=1e-30)


def test_source_volume_is_the_sources():
    r = 2.0 * D
    pos = np.array([[0, 0, 0], [0, 0, r]], float)
    vol = np.array([V, 3 * V])
    B = oracle.dipolar_field(pos, vol, MS, np.array([[0, 0, 1], [0, 0, 1]], float))
    np.testing.assert_allclose(B[0, 2], 2 * w(3 * V) / r ** 3, rtol=1e-14)
    np.testing.assert_allclose(B[1, 2], 2 * w(V) / r ** 3, rtol=1e-14)


def test_three_nps_right_triangle():
    r = 1.3 * D
    pos = np.array([[0, 0, 0], [r, 0, 0], [0, r, 0]], float)
    vol = np.full(3, V)
    # all moments along z: every pair is broadside
    B = oracle.dipolar_field(pos, vol, MS, np.tile([0.0, 0, 1], (3, 1)))
    s2 = 2 * math.sqrt(2)
    np.testing.assert_allclose(B[0], [0, 0, -2 * w() / r ** 3], rtol=1e-13, atol=1e-30)
    np.testing.assert_allclose(B[1], [0, 0, -w() / r ** 3 - w() / (s2 * r ** 3)],
                               rtol=1e-13, atol=1e-30)
    # all moments along x: at NP 0, NP 1 is coaxial and NP 2 broadside
    B = oracle.dipolar_field(pos, vol, MS, np.tile([1.0, 0, 0], (3, 1)))
    np.testing.assert_allclose(B[0], [w() / r ** 3, 0, 0], rtol=1e-13, atol=1e-25)
    # at NP 2: NP 0 broadside (-w/r^3 x), NP 1 at 45 degrees: w (1/2, -3/2, 0)/(2 sqrt2 r^3)
    expect = np.array([-w() / r ** 3 + 0.5 * w() / (s2 * r ** 3),
                       -1.5 * w() / (s2 * r ** 3), 0.0])
    np.testing.assert_allclose(B[2], expect, rtol=1e-13, atol=1e-25)


def test_cubic_lattice_sphere_centre_is_field_free():
    lys = inputs.lattice_lysosome(n_side=12, spacing=1.5 * D, d=D)
    m = np.tile([0.0, 0, 1], (lys.n, 1))
    B = oracle.dipolar_field(lys.pos, lys.vol, MS, m)
    centre = int(np.argmin(np.linalg.norm(lys.pos, axis=1)))
    assert np.linalg.norm(lys.pos[centre]) == 0.0
    nearest = w() / (1.5 * D) ** 3
    assert np.linalg.norm(B[centre]) < 1e-12 * nearest
    # off-centre sites do feel a field (the check is not vacuous)
    assert np.max(np.linalg.norm(B, axis=1)) > 0.1 * nearest


def test_reciprocity():
    """m_i . B_i(from j) = m_j . B_j(from i): the pair tensor is symmetric."""
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(2, 3)) * 2 * D
    m = inputs.random_axes(2, rng)
    vol = np.array([V, V])
    B = oracle.dipolar_field(pos, vol, MS, m)
    assert abs(m[0] @ B[0] - m[1] @ B[1]) < 1e-13 * abs(m[0] @ B[0]) + 1e-30


def test_field_is_minus_gradient_of_scalar_potential():
    """mu0 H = -mu0 grad psi, psi(r) = sum_j M_S V_j m_j . (r - r_j) / (4 pi |r - r_j|^3),
    differentiated numerically (4th-order central differences)."""
    lys = inputs.make_lysosome(30, D, 0.1, seed=11)
    rng = np.random.default_rng(5)
    m = inputs.random_axes(lys.n, rng)
    B = oracle.dipolar_field(lys.pos, lys.vol, MS, m)

    def psi(i, r):
        s = 0.0
        for j in range(lys.n):
            if j == i:
                continue
            dvec = r - lys.pos[j]
            s += MS * lys.vol[j] * (m[j] @ dvec) / (4 * math.pi * np.linalg.norm(dvec) ** 3)
        return s

    h = 1e-3 * D
    for i in range(0, lys.n, 3):
        g = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            r = lys.pos[i]
            g[a] = (-psi(i, r + 2 * e) + 8 * psi(i, r + e) - 8 * psi(i, r - e)
                    + psi(i, r - 2 * e)) / (12 * h)
        np.testing.assert_allclose(B[i], -MU0 * g, rtol=0, atol=1e-7 * np.linalg.norm(B[i]) + 1e-12 * w() / D ** 3)


def test_field_at_subset_matches_full():
    lys = inputs.make_lysosome(60, D, 0.1, seed=12)
    m = inputs.random_axes(lys.n, np.random.default_rng(1))
    B = oracle.dipolar_field(lys.pos, lys.vol, MS, m)
    idx = np.array([0, 7, 59, 7])
    np.testing.assert_array_equal(oracle.dipolar_field_at(lys.pos, lys.vol, MS, m, idx), B[idx])
