"""Pins of the oracle's sample regeneration between loops (Sec. II.4): fresh easy
axes uniform on the sphere, and fresh positions drawn around the nodes of a
simple-cubic lattice with a displacement of uniform direction and a length
uniform on [0, disorder], the disorder being as large as it can be without two
neighbours overlapping.

Pinned by the moments of the uniform distribution on the sphere, Kolmogorov-
Smirnov tests of z, azimuth and displacement length against their exact
distributions, and a brute-force overlap check at maximal disorder."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs

scipy_stats = pytest.importorskip("scipy.stats")


def test_axes_uniform_on_sphere():
    n = 20000
    a = oracle.regen_axes(n, seed=3, loop=7, lys=2)
    np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-15)
    # E[a] = 0 (sd sqrt(1/3n)); E[a_i^2] = 1/3 (sd of z^2 for z ~ U(-1,1) is sqrt(4/45))
    assert np.all(np.abs(a.mean(axis=0)) < 4.0 * math.sqrt(1.0 / (3 * n)))
    assert np.all(np.abs((a ** 2).mean(axis=0) - 1.0 / 3.0) < 4.0 * math.sqrt(4.0 / 45.0 / n))
    assert abs(np.mean(a[:, 0] * a[:, 1])) < 4.0 * math.sqrt(1.0 / 15.0 / n)
    # z ~ U(-1, 1) (Archimedes) and azimuth ~ U(0, 2 pi)
    assert scipy_stats.kstest(a[:, 2], "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    az = np.mod(np.arctan2(a[:, 1], a[:, 0]), 2 * math.pi)
    assert scipy_stats.kstest(az, "uniform", args=(0.0, 2 * math.pi)).pvalue > 1e-3


def test_draws_are_keyed():
    a = oracle.regen_axes(50, seed=1, loop=0)
    assert np.array_equal(a, oracle.regen_axes(50, seed=1, loop=0))
    for other in [oracle.regen_axes(50, seed=2, loop=0), oracle.regen_axes(50, seed=1, loop=1),
                  oracle.regen_axes(50, seed=1, loop=0, lys=1)]:
        assert not np.any(np.all(a == other, axis=1))
    # positions and axes come from different counters
    p = oracle.regen_positions(np.zeros((50, 3)), 1.0, seed=1, loop=0)
    d = p / np.linalg.norm(p, axis=1, keepdims=True)
    assert not np.any(np.all(np.abs(d - a) < 1e-12, axis=1))


def test_displacement_length_and_direction():
    n, dis = 20000, 3e-9
    nodes = np.random.default_rng(0).normal(size=(n, 3)) * 1e-7
    p = oracle.regen_positions(nodes, dis, seed=5, loop=2)
    dv = p - nodes
    r = np.linalg.norm(dv, axis=1)
    assert np.all(r <= dis * (1 + 1e-12))
    assert scipy_stats.kstest(r / dis, "uniform").pvalue > 1e-3
    assert scipy_stats.kstest(dv[:, 2] / r, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    assert np.array_equal(oracle.regen_positions(nodes, 0.0, seed=5, loop=2), nodes)


def test_maximal_disorder_never_overlaps():
    d, c = 14e-9, 0.1
    lys = inputs.lattice_nodes_lysosome(2000, d, c, seed=1)
    dis = inputs.max_disorder(d, c)
    from scipy.spatial import cKDTree
    for loop in range(3):
        p = oracle.regen_positions(lys.pos, dis, seed=11, loop=loop)
        dist, _ = cKDTree(p).query(p, k=2)
        assert dist[:, 1].min() >= d * (1 - 1e-12)
    # a larger disorder does overlap somewhere: the bound is the right one
    p = oracle.regen_positions(lys.pos, 1.5 * dis, seed=11, loop=0)
    dist, _ = cKDTree(p).query(p, k=2)
    assert dist[:, 1].min() < d
