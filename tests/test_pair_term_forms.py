"""The algebra behind the FP32 pair loop, checked on the CPU against the
oracle's Eq. 1.

Each FP32 source record holds t_j = 3 w_j m_j and n_j = -w_j m_j beside the
position, and a pair adds q^3 (u d + n_j) with d = r_j - r_i, q = 1/|d| and
u = (t_j . d) q^2. That is Eq. 1's term w_j (3 (m_j . d) d / |d|^5 - m_j / |d|^3)
rearranged. Here the rearranged sum is formed in FP64 with numpy and must
agree with the oracle's field to rounding; the same sum with the factor 3 or
the sign of n dropped must not."""
import math

import numpy as np

import oracle

MU0 = 4e-7 * math.pi


def _sample(n, seed):
    rng = np.random.default_rng(seed)
    pos = []
    while len(pos) < n:  # NPs of 10-20 nm, never overlapping, in a 0.3 um ball
        p = rng.uniform(-1.5e-7, 1.5e-7, 3)
        if np.linalg.norm(p) < 1.5e-7 and all(np.linalg.norm(p - q) > 2.2e-8 for q in pos):
            pos.append(p)
    pos = np.array(pos)
    d = rng.uniform(10e-9, 20e-9, n)
    vol = math.pi / 6.0 * d ** 3
    m = rng.normal(size=(n, 3))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    return pos, vol, m


def _fused_field(pos, vol, Ms, m, three=3.0, n_sign=-1.0):
    """mu0 H_dip in T from the record form: sum_j q^3 (u d + n_j)."""
    w = MU0 * Ms * vol / (4.0 * math.pi)  # T m^3 per unit moment
    t = three * w[:, None] * m
    nn = n_sign * w[:, None] * m
    B = np.zeros_like(pos)
    for i in range(len(pos)):
        d = pos - pos[i]
        r2 = np.einsum("ij,ij->i", d, d)
        r2[i] = 1.0  # the self term is dropped below
        q = 1.0 / np.sqrt(r2)
        u = np.einsum("ij,ij->i", t, d) * q * q
        term = (q ** 3)[:, None] * (u[:, None] * d + nn)
        term[i] = 0.0
        B[i] = term.sum(axis=0)
    return B


def test_record_form_equals_eq1():
    pos, vol, m = _sample(300, 7)
    Ms = 4.8e5
    ref = oracle.dipolar_field(pos, vol, Ms, m)
    B = _fused_field(pos, vol, Ms, m)
    scale = np.max(np.linalg.norm(ref, axis=1))
    assert scale > 0
    assert np.max(np.abs(B - ref)) <= 1e-12 * scale


def test_record_form_detects_a_wrong_factor_or_sign():
    pos, vol, m = _sample(120, 8)
    Ms = 4.8e5
    ref = oracle.dipolar_field(pos, vol, Ms, m)
    scale = np.max(np.linalg.norm(ref, axis=1))
    for three, n_sign in ((1.0, -1.0), (3.0, 1.0), (-3.0, 1.0)):
        B = _fused_field(pos, vol, Ms, m, three=three, n_sign=n_sign)
        assert np.max(np.abs(B - ref)) > 1e-2 * scale, (three, n_sign)
