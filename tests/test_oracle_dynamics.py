"""Pins of the oracle's steps iii-vii and of whole runs (Sec. II.1-II.3).

* Eq. 5 against the worked example of Fig. 1(b): nu1 = 1 Hz, nu2 = 0.2 Hz give
  the long-time probability 0.166 and initial slopes equal to the rates.
* Zero field: the jump probability per step is (1 - exp(-2 nu t)) / 2 and the
  mean time between jumps is twice the Neel relaxation time 1 / (2 nu).
* Two-state (Neel) equilibrium of superparamagnetic NPs with axes along the
  field: <m_z> = tanh(M_S V mu0 H / k T), for the Ref. [8] mode exactly and
  for the kMC sample mean within its statistical error.
* The kMC sample mean follows the Ref. [8] mode out of equilibrium.
* Invariants of one step on a real lysosome.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs

KB = 1.380649e-23
MS = 1e6


def read_paper_values(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "paper_values.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def _fig1b_np(golden_dir):
    """An NP with its axis along a field chosen so that the deep well (theta = 0)
    has escape rate nu2 and the shallow well (theta = pi) escape rate nu1.
    With h = M_S B / (2 K): barriers K V (1 + h)^2 and K V (1 - h)^2."""
    vals = read_paper_values(golden_dir)
    nu1, nu2 = vals["fig1b_nu1_Hz"], vals["fig1b_nu2_Hz"]
    h = 0.1
    a = math.log(nu1 / nu2) / (4 * h)        # K V / k T
    nu0 = nu1 * math.exp(a * (1 - h) ** 2)
    T, K, V = 300.0, 1e4, None
    V = a * KB * T / K
    B = 2 * K * h / MS
    return vals, dict(K=K, V=V, T=T, tau0=1 / nu0, B=B, nu1=nu1, nu2=nu2)


def test_fig1b_worked_example(golden_dir):
    vals, p = _fig1b_np(golden_dir)
    axis = np.array([0.3, -0.2, 0.9])
    axis /= np.linalg.norm(axis)
    B = p["B"] * axis
    # start in the deep well theta = 0 (escape rate nu2): P(t -> inf) = nu2/(nu1+nu2)
    r = oracle.np_update(axis, axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], 1e4, 0.99)
    assert r["n_min"] == 2
    assert abs(r["P"] - vals["fig1b_P_inf"]) < 1e-3        # the printed 0.166
    # initial slopes are the rates (tangents at the origin of Fig. 1(b))
    t = 1e-7
    r2 = oracle.np_update(axis, axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], t, 0.99)
    assert abs(r2["P"] / t - p["nu2"]) < 1e-6
    r1 = oracle.np_update(axis, -axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], t, 0.99)
    assert abs(r1["P"] / t - p["nu1"]) < 1e-6
    # from the shallow well the long-time probability to leave is nu1/(nu1+nu2)
    r3 = oracle.np_update(axis, -axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], 1e4, 0.99)
    assert abs(r3["P"] - (1 - vals["fig1b_P_inf"])) < 1e-3
    # u < P jumps, u >= P stays (step vii)
    assert oracle.np_update(axis, axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], 1e4,
                            0.10)["flipped"]
    assert not oracle.np_update(axis, axis, B, p["K"], MS, p["V"], p["T"], p["tau0"], 1e4,
                                0.20)["flipped"]


def test_zero_field_jump_probability():
    d, K, T = 10e-9, 1.3e4, 300.0
    V = math.pi * d ** 3 / 6
    nu = 1e10 * math.exp(-K * V / (KB * T))
    axis = np.array([0.0, 0.6, 0.8])
    for t in [1e-12, 1e-9, 1e-7, 1e-5]:
        r = oracle.np_update(axis, axis, np.zeros(3), K, MS, V, T, 1e-10, t, 0.5)
        exact = 0.5 * -math.expm1(-2 * nu * t)
        assert abs(r["P"] - exact) <= 1e-13 * exact
        np.testing.assert_allclose(r["dE"], [K * V, K * V], rtol=1e-12)


def _far_apart(n, axis, d, **kw):
    """n NPs on a line 1 mm apart: dipolar fields below 1e-18 T."""
    pos = np.zeros((n, 3))
    pos[:, 0] = np.arange(n) * 1e-3
    vol = np.full(n, math.pi * d ** 3 / 6)
    return inputs.Lysosome(pos=pos, axis=np.asarray(axis, float), vol=vol, Ms=MS,
                           d=d, **kw)


def test_neel_mean_time_between_jumps():
    """Zero field, many steps: the jump count matches rate nu, i.e. the mean
    time between jumps is 1/nu = twice the Neel time 1/(2 nu)."""
    d, K, T, tau0 = 11e-9, 1.3e4, 300.0, 1e-10
    V = math.pi * d ** 3 / 6
    nu = math.exp(-K * V / (KB * T)) / tau0
    n, S, periods = 50, 400, 4
    f = 1.0 / (S * 0.02 / nu)       # P per step ~ 0.02
    lys = _far_apart(n, np.tile([0.0, 0, 1], (n, 1)), d, Keff=K, T=T, tau0=tau0)
    out = oracle.run(lys, 0, 0.0, f, S, periods, 0, seed=5, nthreads=4)
    t_step = 1 / (f * S)
    p = 0.5 * -math.expm1(-2 * nu * t_step)
    steps = n * S * periods
    flips = out["counters"]["flips"]
    assert abs(flips - steps * p) < 4.5 * math.sqrt(steps * p * (1 - p))
    mean_time_between = steps * t_step / flips
    tau_neel = 1 / (2 * nu)
    assert abs(mean_time_between / (2 * tau_neel) - 1) < 0.05


def test_two_state_equilibrium_mean_mode():
    """Superparamagnetic NPs (relaxation much faster than a step) with axes along
    z: the Ref. [8] mode gives the Boltzmann two-state value at every step
    where both wells exist."""
    d, K, T = 8e-9, 1.3e4, 300.0
    V = math.pi * d ** 3 / 6
    n = 3
    axis = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 0, 1.0]])
    vol = np.full(n, V)
    Hmax, f, S = 0.020, 1e5, 200
    M = oracle.mean_run(axis, vol, MS, K, T, 1e-10, Hmax, f, S, 2, 1)
    H = Hmax * np.cos(2 * np.pi * np.arange(S) / S)
    assert np.all(MS * np.abs(H) / (2 * K) < 1)
    expect = np.tanh(MS * V * H / (KB * T))
    np.testing.assert_allclose(M, expect, rtol=0, atol=1e-9)


def test_two_state_equilibrium_kmc_sample_mean():
    d, K, T = 8e-9, 1.3e4, 300.0
    V = math.pi * d ** 3 / 6
    n, S = 400, 40
    axis = np.tile([0.0, 0, 1], (n, 1))
    axis[::2] *= -1
    lys = _far_apart(n, axis, d, Keff=K, T=T, tau0=1e-10)
    Hmax, f = 0.020, 1e5
    out = oracle.run(lys, 0, Hmax, f, S, 3, 1, seed=17, nthreads=4)
    H = out["loop_H"]
    expect = np.tanh(MS * V * H / (KB * T))
    sigma = np.sqrt((1 - expect ** 2) / n)
    z = (out["loop_M"] - expect) / sigma
    assert np.max(np.abs(z)) < 4.5
    assert abs(np.mean(z)) < 4.5 / math.sqrt(len(z)) * 1.5


def test_kmc_follows_mean_mode_out_of_equilibrium():
    """Random axes, K V / k T ~ 8: a lagging loop. The kMC mean over NPs stays
    within its statistical band around the Ref. [8] mode."""
    d, K, T = 13e-9, 1.3e4, 300.0
    n, S = 600, 100
    rng = np.random.default_rng(2)
    lys = _far_apart(n, inputs.random_axes(n, rng), d, Keff=K, T=T, tau0=1e-10)
    Hmax, f = 0.020, 1e5
    out = oracle.run(lys, 0, Hmax, f, S, 3, 1, seed=23, nthreads=4)
    M = oracle.mean_run(lys.axis, lys.vol, MS, K, T, 1e-10, Hmax, f, S, 3, 1)
    # |m_z| <= 1 per NP, so the standard error of the mean is at most 1/sqrt(n)
    err = np.abs(out["loop_M"] - M)
    assert np.max(err) < 5.0 / math.sqrt(n)
    assert np.mean(err) < 1.5 / math.sqrt(n)
    # the loop is open: the area is well above its noise
    assert out["area"] > 0


def test_step_invariants():
    (lys,), run = inputs.config_small(seed=3)
    m0 = oracle.initial_moments(lys.axis)
    # move the moments off the axes so the projection step matters
    rng = np.random.default_rng(9)
    m = m0 + 0.3 * rng.normal(size=m0.shape)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    out = oracle.step(lys, 0, m, 0.012, 1 / (run["f"] * run["S"]), 0, 1234)
    mn = out["m_out"]
    np.testing.assert_allclose(np.linalg.norm(mn, axis=1), 1.0, rtol=0, atol=1e-14)
    Bt = out["B_dip"] + np.array([0, 0, 0.012])
    # m_new lies in the plane of the axis and the total field
    normal = np.cross(lys.axis, Bt)
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    assert np.max(np.abs(np.einsum("ij,ij->i", normal, mn))) < 1e-12
    # without a jump the moment only goes downhill from its projection
    E = lambda mm: (lys.Keff * lys.vol * (1 - np.einsum("ij,ij->i", mm, lys.axis) ** 2)
                    - MS * lys.vol * np.einsum("ij,ij->i", Bt, mm))
    proj = m - np.einsum("ij,ij->i", m, normal)[:, None] * normal
    proj /= np.linalg.norm(proj, axis=1, keepdims=True)
    stay = out["flipped"] == 0
    assert np.all(E(mn)[stay] <= E(proj)[stay] + 1e-12 * lys.Keff * lys.vol[stay])
    assert np.all((out["P"] >= 0) & (out["P"] <= 1))
    assert np.all(out["P"][out["n_min"] == 1] == 0)
    assert np.all(out["flipped"][out["n_min"] == 1] == 0)


def test_T0_skips_jumps():
    (lys,), run = inputs.config_small(seed=4)
    lys.T = 0.0
    out = oracle.run(lys, 0, 0.02, run["f"], run["S"], 2, 1, seed=1)
    assert out["counters"]["flips"] == 0
