"""Pins of the oracle's random sequential addition (Sec. II.4; the configs place
lysosomes by it): the candidate stream is uniform in the ball, every keep and
every rejection follows from the candidates by brute force, and a dilute packing
keeps the first n candidates."""
import math

import numpy as np
import pytest

import oracle


def _candidates(k, R, d, seed, loop, lys=0):
    return np.array([oracle.rsa_candidate(R, d, seed, loop, c, lys) for c in range(k)])


def test_candidates_are_uniform_in_the_ball():
    scipy_stats = pytest.importorskip("scipy.stats")
    R, d = 1e-6, 2e-8
    p = _candidates(6000, R, d, seed=5, loop=2)
    Rb = R - d / 2
    r = np.linalg.norm(p, axis=1)
    assert r.max() <= Rb * (1 + 1e-15)
    # uniform in the ball: (r / Rb)^3 uniform on [0, 1]; directions uniform on the sphere
    assert scipy_stats.kstest((r / Rb) ** 3, "uniform").pvalue > 1e-3
    e = p / r[:, None]
    assert scipy_stats.kstest((e[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    az = (np.arctan2(e[:, 1], e[:, 0]) + math.pi) / (2 * math.pi)
    assert scipy_stats.kstest(az, "uniform").pvalue > 1e-3
    np.testing.assert_allclose(p.mean(axis=0), 0.0, atol=4 * Rb / math.sqrt(len(p)))


def test_every_keep_and_rejection_by_brute_force():
    n, R, d = 150, 60e-9, 12e-9  # 15 % volume fraction: some candidates are rejected
    pos, used = oracle.rsa(n, R, d, seed=9, loop=1, lys=3)
    cand = _candidates(used, R, d, seed=9, loop=1, lys=3)
    kept = []
    for c in range(used):
        p = cand[c]
        ok = all(np.sum((p - q) ** 2) >= d * d for q in kept)
        if ok:
            kept.append(p)
    assert len(kept) == n and used > n
    np.testing.assert_array_equal(np.array(kept), pos)
    # the packing: no two closer than d, all inside R - d/2
    diff = pos[:, None, :] - pos[None, :, :]
    dist = np.sqrt(np.sum(diff ** 2, axis=2)) + np.eye(n) * 1e9
    assert dist.min() >= d * (1 - 1e-12)
    assert np.linalg.norm(pos, axis=1).max() <= (R - d / 2) * (1 + 1e-15)


def test_dilute_limit_keeps_the_first_candidates():
    R, d = 1e-6, 1e-12
    pos, used = oracle.rsa(40, R, d, seed=3, loop=7)
    assert used == 40
    np.testing.assert_array_equal(pos, _candidates(40, R, d, seed=3, loop=7))


def test_streams_differ_by_loop_and_lysosome_and_run_out():
    R, d = 80e-9, 10e-9
    a, _ = oracle.rsa(20, R, d, seed=1, loop=1)
    b, _ = oracle.rsa(20, R, d, seed=1, loop=2)
    c, _ = oracle.rsa(20, R, d, seed=1, loop=1, lys=1)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    with pytest.raises(RuntimeError):
        oracle.rsa(2000, R, d, seed=1, loop=1, max_candidates=5000)  # cannot fit 2000
