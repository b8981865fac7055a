"""Plain FP64 CPU oracle of the kinetic Monte-Carlo hysteresis method of
Tan, Carrey & Respaud (arXiv:1407.2737, Sec. II, Eqs. 1-5).

TEST INFRASTRUCTURE. This package checks the CUDA library; it is not part of
it. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it. It shares no code with the CUDA
path and never imports it. The arithmetic lives in ``kmc_oracle.c`` (plain C,
FP64, compiled with ``-ffp-contract=off`` so that every product and sum is
rounded as written); this module only builds that file and marshals arrays.

Parity status (see ``kmc_oracle.h``): every entry point is pinned by the tests
under ``tests/test_oracle_*.py`` except the split of the loop area between the
NPs of one lysosome, which is "parity unpinned": the paper fixes only the
lysosome total.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkmc_oracle.so")
_lock = threading.Lock()
_lib = None

GRID = 200


def build(force: bool = False) -> str:
    """Compile ``kmc_oracle.c`` into ``_build/libkmc_oracle.so`` (gcc, FP64,
    OpenMP when the compiler has it). Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(_SRC[:-1] + "h"))):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class _Lys(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", C.POINTER(C.c_double)),
                ("axis", C.POINTER(C.c_double)), ("vol", C.POINTER(C.c_double)),
                ("Ms", C.c_double), ("Keff", C.c_double), ("T", C.c_double),
                ("tau0", C.c_double)]


class _NpRes(C.Structure):
    _fields_ = [("m_new", C.c_double * 3), ("dE", C.c_double * 2),
                ("P", C.c_double), ("u", C.c_double), ("n_min", C.c_int32),
                ("flipped", C.c_int32), ("near", C.c_int32),
                ("degenerate", C.c_int32)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.kmc_oracle_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.kmc_oracle_uniform.argtypes = [C.c_uint64, C.c_int64, C.c_int32, C.c_int32]
            L.kmc_oracle_uniform.restype = C.c_double
            L.kmc_oracle_dipolar_field.argtypes = [C.c_int32, _D, _D, C.c_double, _D, _D]
            L.kmc_oracle_dipolar_field_at.argtypes = [C.c_int32, _D, _D, C.c_double, _D,
                                                      C.c_int32, _I32, _D]
            L.kmc_oracle_extrema.argtypes = [C.c_double] * 5 + [_D, _D, _I32]
            L.kmc_oracle_extrema.restype = C.c_int32
            L.kmc_oracle_np_update.argtypes = [_D, _D, _D] + [C.c_double] * 7 + [
                C.POINTER(_NpRes)]
            L.kmc_oracle_np_update.restype = C.c_int32
            L.kmc_oracle_step.argtypes = [C.POINTER(_Lys), C.c_int32, _D, C.c_double,
                                          C.c_double, C.c_uint64, C.c_int64, _D, _D,
                                          _D, _D, _D, _I32]
            L.kmc_oracle_step.restype = C.c_int32
            L.kmc_oracle_run.argtypes = [C.POINTER(_Lys), C.c_int32, _D, C.c_double,
                                         C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_uint64, C.c_int64, C.c_int32, _D, _D, _D,
                                         _D, _I64]
            L.kmc_oracle_run.restype = C.c_int32
            L.kmc_oracle_area.argtypes = [C.c_int32, _D, _D, C.c_int32]
            L.kmc_oracle_area.restype = C.c_double
            L.kmc_oracle_sar.argtypes = [C.c_double] * 3
            L.kmc_oracle_sar.restype = C.c_double
            L.kmc_oracle_mean_run.argtypes = [C.c_int32, _D, _D] + [C.c_double] * 6 + [
                C.c_int32] * 3 + [_D]
            L.kmc_oracle_mean_run.restype = C.c_int32
            L.kmc_oracle_local_concentration.argtypes = [C.c_int32, _D, _D, C.c_int32, _D]
            L.kmc_oracle_local_concentration.restype = C.c_int32
            L.kmc_oracle_local_concentration_at.argtypes = [C.c_int32, _D, _D, C.c_int32,
                                                            C.c_int32, _I32, _D]
            L.kmc_oracle_local_concentration_at.restype = C.c_int32
            L.kmc_oracle_shell_profile.argtypes = [C.c_int32, _D, _D, _D, C.c_double,
                                                   C.c_int32, C.c_int32, _D, _D, _D]
            L.kmc_oracle_shell_profile.restype = C.c_double
            L.kmc_oracle_regen_axes.argtypes = [C.c_int32, C.c_uint64, C.c_uint32, C.c_int32, _D]
            L.kmc_oracle_regen_axes.restype = None
            L.kmc_oracle_regen_positions.argtypes = [C.c_int32, _D, C.c_double, C.c_uint64,
                                                     C.c_uint32, C.c_int32, _D]
            L.kmc_oracle_regen_positions.restype = None
            L.kmc_oracle_rsa_candidate.argtypes = [C.c_double, C.c_double, C.c_uint64,
                                                   C.c_uint32, C.c_int64, C.c_int32, _D]
            L.kmc_oracle_rsa_candidate.restype = None
            L.kmc_oracle_rsa.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                         C.c_uint32, C.c_int32, C.c_int64, _D]
            L.kmc_oracle_rsa.restype = C.c_int64
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _lys_struct(lys):
    pos = _f64(lys.pos, (-1, 3))
    axis = _f64(lys.axis, (-1, 3))
    vol = _f64(lys.vol, (-1,))
    s = _Lys(len(vol), _dp(pos), _dp(axis), _dp(vol), float(lys.Ms), float(lys.Keff),
             float(lys.T), float(lys.tau0))
    return s, (pos, axis, vol)


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().kmc_oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform(seed, step, np_index, lys_index):
    """53-bit uniform draw in [0, 1) for (seed, step, NP, lysosome)."""
    return float(lib().kmc_oracle_uniform(C.c_uint64(seed), C.c_int64(step),
                                          C.c_int32(np_index), C.c_int32(lys_index)))


def dipolar_field(pos, vol, Ms, m):
    """Eq. 1: mu0*H_dip (T) on every NP; pos (n,3) m, vol (n,) m^3, m (n,3)."""
    pos = _f64(pos, (-1, 3))
    vol = _f64(vol, (-1,))
    m = _f64(m, (-1, 3))
    B = np.zeros_like(pos)
    lib().kmc_oracle_dipolar_field(len(vol), _dp(pos), _dp(vol), float(Ms), _dp(m), _dp(B))
    return B


def dipolar_field_at(pos, vol, Ms, m, idx):
    """Eq. 1 at the listed target NPs only; returns (len(idx), 3) in T."""
    pos = _f64(pos, (-1, 3))
    vol = _f64(vol, (-1,))
    m = _f64(m, (-1, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    B = np.zeros((len(idx), 3))
    lib().kmc_oracle_dipolar_field_at(len(vol), _dp(pos), _dp(vol), float(Ms), _dp(m),
                                      len(idx), idx.ctypes.data_as(_I32), _dp(B))
    return B


def extrema(Keff, Ms, V, B, phi):
    """Step iv: list of (theta, E, is_min) found by the 200-point scan + Newton."""
    th = np.zeros(4)
    E = np.zeros(4)
    im = np.zeros(4, dtype=np.int32)
    n = lib().kmc_oracle_extrema(float(Keff), float(Ms), float(V), float(B), float(phi),
                                 _dp(th), _dp(E), im.ctypes.data_as(_I32))
    if n < 0:
        raise RuntimeError("more than four extrema")
    return [(float(th[q]), float(E[q]), bool(im[q])) for q in range(n)]


def np_update(axis, m_old, Btot, Keff, Ms, V, T, tau0, t_step, u):
    """Steps iii-vii for one NP; returns a dict."""
    a = _f64(axis, (3,))
    m = _f64(m_old, (3,))
    b = _f64(Btot, (3,))
    r = _NpRes()
    rc = lib().kmc_oracle_np_update(_dp(a), _dp(m), _dp(b), float(Keff), float(Ms),
                                    float(V), float(T), float(tau0), float(t_step),
                                    float(u), C.byref(r))
    if rc != 0:
        raise RuntimeError("np_update failed")
    return dict(m_new=np.array(r.m_new[:]), dE=np.array(r.dE[:]), P=r.P, u=r.u,
                n_min=r.n_min, flipped=bool(r.flipped), near=bool(r.near),
                degenerate=bool(r.degenerate))


def step(lys, lys_index, m_in, mu0Hext, t_step, seed, step_index):
    """One synchronous kMC step of one lysosome (steps i-vii for every NP)."""
    s, keep = _lys_struct(lys)
    n = s.n
    m_in = _f64(m_in, (n, 3))
    out = dict(m_out=np.zeros((n, 3)), B_dip=np.zeros((n, 3)), dE=np.zeros((n, 2)),
               P=np.zeros(n), u=np.zeros(n), flags=np.zeros(n, dtype=np.int32))
    rc = lib().kmc_oracle_step(C.byref(s), int(lys_index), _dp(m_in), float(mu0Hext),
                               float(t_step), C.c_uint64(seed), C.c_int64(step_index),
                               _dp(out["m_out"]), _dp(out["B_dip"]), _dp(out["dE"]),
                               _dp(out["P"]), _dp(out["u"]),
                               out["flags"].ctypes.data_as(_I32))
    if rc != 0:
        raise RuntimeError("oracle step failed (%d)" % rc)
    del keep
    out["n_min"] = out["flags"] & 3
    out["flipped"] = (out["flags"] >> 2) & 1
    out["near"] = (out["flags"] >> 3) & 1
    out["degenerate"] = (out["flags"] >> 4) & 1
    return out


def initial_moments(axis):
    """Initial state: m = +/- easy axis with m_z >= 0 (saturated by +H_max)."""
    a = _f64(axis, (-1, 3))
    sign = np.where(a[:, 2] >= 0.0, 1.0, -1.0)
    return a * sign[:, None]


def run(lys, lys_index, mu0Hmax, f, S, periods, discard, seed, m=None, step0=0,
        nthreads=1):
    """A whole kMC run of one lysosome; returns m, E_diss, dHdip (Eq. 6, T),
    loop_H, loop_M, counters, area (J/m^3 per cycle) and sar (W/kg)."""
    s, keep = _lys_struct(lys)
    n = s.n
    m = initial_moments(lys.axis) if m is None else _f64(m, (n, 3)).copy()
    nrec = max(0, S * (periods - discard))
    E = np.zeros(n)
    dH = np.zeros(n)
    lH = np.zeros(max(nrec, 1))
    lM = np.zeros(max(nrec, 1))
    cnt = np.zeros(4, dtype=np.int64)
    rc = lib().kmc_oracle_run(C.byref(s), int(lys_index), _dp(m), float(mu0Hmax), float(f),
                              int(S), int(periods), int(discard), C.c_uint64(seed),
                              C.c_int64(step0), int(nthreads), _dp(E), _dp(dH), _dp(lH), _dp(lM),
                              cnt.ctypes.data_as(_I64))
    if rc != 0:
        raise RuntimeError("oracle run failed (%d)" % rc)
    nper = max(0, periods - discard)
    area = lib().kmc_oracle_area(n, _dp(keep[2]), _dp(E), nper)
    rho = float(getattr(lys, "rho", 5200.0))
    del keep
    return dict(m=m, E_diss=E, dHdip=dH, loop_H=lH[:nrec], loop_M=lM[:nrec],
                counters=dict(flips=int(cnt[0]), near=int(cnt[1]), monostable=int(cnt[2]),
                              degenerate=int(cnt[3])),
                area=float(area), sar=float(lib().kmc_oracle_sar(area, float(f), rho)))


def area(vol, E_diss, n_periods):
    vol = _f64(vol, (-1,))
    E = _f64(E_diss, (-1,))
    return float(lib().kmc_oracle_area(len(vol), _dp(vol), _dp(E), int(n_periods)))


def sar(area_J_m3, f, rho):
    """SAR = A f / rho in W/kg (Sec. III.2.a)."""
    return float(lib().kmc_oracle_sar(float(area_J_m3), float(f), float(rho)))


def mean_run(axis, vol, Ms, Keff, T, tau0, mu0Hmax, f, S, periods, discard):
    """Ref. [8] mode: the mean moment from well probabilities (no sampling,
    no interactions); returns the volume-weighted mean m_z per recorded step."""
    axis = _f64(axis, (-1, 3))
    vol = _f64(vol, (-1,))
    nrec = max(0, S * (periods - discard))
    lM = np.zeros(max(nrec, 1))
    rc = lib().kmc_oracle_mean_run(len(vol), _dp(axis), _dp(vol), float(Ms), float(Keff),
                                   float(T), float(tau0), float(mu0Hmax), float(f), int(S),
                                   int(periods), int(discard), _dp(lM))
    if rc != 0:
        raise RuntimeError("oracle mean_run failed (%d)" % rc)
    return lM[:nrec]


def local_concentration(pos, vol, N):
    """Eq. 8: phi_N per NP from the distance to its N-th nearest neighbour."""
    pos = _f64(pos, (-1, 3))
    vol = _f64(vol, (-1,))
    phi = np.zeros(len(vol))
    rc = lib().kmc_oracle_local_concentration(len(vol), _dp(pos), _dp(vol), int(N), _dp(phi))
    if rc != 0:
        raise ValueError("oracle local_concentration failed (%d)" % rc)
    return phi


def local_concentration_at(pos, vol, N, idx):
    """Eq. 8 at the listed NPs only."""
    pos = _f64(pos, (-1, 3))
    vol = _f64(vol, (-1,))
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    phi = np.zeros(len(idx))
    rc = lib().kmc_oracle_local_concentration_at(len(vol), _dp(pos), _dp(vol), int(N), len(idx),
                                                 idx.ctypes.data_as(_I32), _dp(phi))
    if rc != 0:
        raise ValueError("oracle local_concentration_at failed (%d)" % rc)
    return phi


def shell_profile(pos, vol, center, R, n_shells, values):
    """Radial profile (Fig. 8): per shell the NP count and the volume-weighted
    mean of each column of values ([n][n_val]); returns (count, mean, R used)."""
    pos = _f64(pos, (-1, 3))
    vol = _f64(vol, (-1,))
    val = _f64(values, (len(vol), -1))
    c = _f64(center, (3,))
    count = np.zeros(int(n_shells))
    mean = np.zeros((int(n_shells), val.shape[1]))
    r = lib().kmc_oracle_shell_profile(len(vol), _dp(pos), _dp(vol), _dp(c), float(R),
                                       int(n_shells), val.shape[1], _dp(val), _dp(count),
                                       _dp(mean))
    if r < 0:
        raise ValueError("oracle shell_profile failed (%g)" % r)
    return count, mean, float(r)


def rsa_candidate(radius, d, seed, loop, c, lys=0):
    """Candidate c of the RSA stream: a point uniform in the ball of radius
    radius - d/2 (m)."""
    out = np.zeros(3)
    lib().kmc_oracle_rsa_candidate(float(radius), float(d), C.c_uint64(seed), C.c_uint32(loop),
                                   C.c_int64(c), int(lys), _dp(out))
    return out


def rsa(n, radius, d, seed, loop, lys=0, max_candidates=None):
    """Random sequential addition of n spheres of diameter d in the sphere of
    the given radius, from the candidate stream; returns (positions [n][3],
    candidates used). Raises if max_candidates (default 1000 n) run out."""
    pos = np.zeros((int(n), 3))
    cap = int(max_candidates if max_candidates is not None else 1000 * max(int(n), 1))
    used = lib().kmc_oracle_rsa(int(n), float(radius), float(d), C.c_uint64(seed), C.c_uint32(loop),
                                int(lys), C.c_int64(cap), _dp(pos))
    if used < 0:
        raise RuntimeError("RSA ran out of candidates")
    return pos, int(used)


def regen_axes(n, seed, loop, lys=0):
    """Fresh easy axes for loop `loop` (Sec. II.4), uniform on the sphere."""
    axis = np.zeros((int(n), 3))
    lib().kmc_oracle_regen_axes(int(n), C.c_uint64(seed), C.c_uint32(loop), int(lys), _dp(axis))
    return axis


def regen_positions(nodes, disorder, seed, loop, lys=0):
    """Fresh positions around the nodes (Sec. II.4): a uniform direction and a
    distance uniform on [0, disorder]."""
    nodes = _f64(nodes, (-1, 3))
    pos = np.zeros_like(nodes)
    lib().kmc_oracle_regen_positions(len(nodes), _dp(nodes), float(disorder), C.c_uint64(seed),
                                     C.c_uint32(loop), int(lys), _dp(pos))
    return pos
