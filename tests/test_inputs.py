"""Invariants of the seeded synthetic lysosomes (random sequential addition
inside a sphere, Sec. II.1 / III.1)."""
import math

import numpy as np
import pytest
from scipy.spatial.distance import pdist

from paper_1407_2737_gb300 import inputs


def test_rsa_invariants():
    for n, d, c in [(300, 12e-9, 0.05), (2000, 14e-9, 0.10), (1500, 8e-9, 0.20)]:
        L = inputs.make_lysosome(n, d, c, seed=n)
        assert L.n == n
        assert pdist(L.pos).min() >= d * (1 - 1e-7)
        assert np.linalg.norm(L.pos, axis=1).max() <= L.radius - d / 2 + 1e-6 * d
        assert abs(n * math.pi * d ** 3 / 6 / (4 / 3 * math.pi * L.radius ** 3) - c) < 1e-12
        np.testing.assert_allclose(np.linalg.norm(L.axis, axis=1), 1.0, atol=1e-14)
        v = L.pos / d
        assert np.all(v.astype(np.float32).astype(np.float64) * d == L.pos)


def test_seeded_and_distinct():
    a = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    b = inputs.make_lysosome(100, 12e-9, 0.05, seed=1)
    c = inputs.make_lysosome(100, 12e-9, 0.05, seed=2)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.axis, b.axis)
    assert not np.array_equal(a.pos, c.pos)


def test_batched_workload_shape():
    lys, run = inputs.config_batched(n_lys=16, seed=3)
    ns = np.array([L.n for L in lys])
    assert np.all((ns >= 200) & (ns <= 10000))
    assert len(run["mu0Hmax"]) == 16
    assert np.all((run["mu0Hmax"] >= 0.010) & (run["mu0Hmax"] <= 0.080))


def test_lattice_nodes_lysosome():
    # the n simple-cubic nodes of cell a = d (pi / 6c)^(1/3) nearest the centre
    d, c, n = 14e-9, 0.1, 2000
    lys = inputs.lattice_nodes_lysosome(n, d, c, seed=3)
    a = inputs.lattice_spacing(d, c)
    assert lys.n == n
    assert a ** 3 * c == pytest.approx(math.pi * d ** 3 / 6, rel=1e-12)
    g = lys.pos / a
    np.testing.assert_allclose(g, np.round(g), atol=1e-9)
    assert len({tuple(x) for x in np.round(g).astype(int)}) == n
    r = np.linalg.norm(lys.pos, axis=1)
    # every node left out lies no nearer than the farthest one kept
    assert r.max() == pytest.approx(lys.radius, rel=0.05)
    assert inputs.max_disorder(d, c) == pytest.approx(0.5 * (a - d), rel=1e-12)
    np.testing.assert_allclose(np.linalg.norm(lys.axis, axis=1), 1.0, atol=1e-12)
