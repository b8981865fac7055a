"""Thin Python binding of libkmc (include/kmc.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: each step of the kMC path runs in the CUDA kernels
of ``csrc/``. Loading fails loudly if ``_build/libkmc.so`` is missing
(build it with ``python -m paper_1407_2737_gb300.build``); there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KMC_LIB_PATH selects another build of the same library (the KMC_DEBUG one)
LIB_PATH = os.environ.get("KMC_LIB_PATH") or os.path.join(_HERE, "_build", "libkmc.so")

KMC_OK, KMC_EINVAL, KMC_ENOMEM, KMC_ECUDA, KMC_ETIMEOUT, KMC_ESTATE, KMC_ECAPACITY, \
    KMC_EIO = range(8)
KMC_FP64_PLAIN, KMC_FP32_MIXED = 0, 1
(KMC_READ_LOOP_H, KMC_READ_LOOP_M, KMC_READ_NP_ENERGY, KMC_READ_AREA, KMC_READ_SAR,
 KMC_READ_MOMENTS, KMC_READ_COUNTERS, KMC_READ_DHDIP, KMC_READ_POSITIONS,
 KMC_READ_AXES) = range(10)
KMC_REGEN_AXES, KMC_REGEN_POSITIONS = 1, 2

STATUS_NAMES = {0: "KMC_OK", 1: "KMC_EINVAL", 2: "KMC_ENOMEM", 3: "KMC_ECUDA",
                4: "KMC_ETIMEOUT", 5: "KMC_ESTATE", 6: "KMC_ECAPACITY", 7: "KMC_EIO"}

# the entry points declared in include/kmc.h
EXPORTS = ("kmc_create", "kmc_set_stream", "kmc_run", "kmc_read", "kmc_sync",
           "kmc_debug_step", "kmc_save", "kmc_load", "kmc_info", "kmc_tuning", "kmc_destroy",
           "kmc_last_error", "kmc_dipolar_field_noalloc", "kmc_local_concentration",
           "kmc_shell_profile", "kmc_mean_run", "kmc_regenerate", "kmc_debug_stall",
           "kmc_regenerate_rsa", "kmc_targets_per_lane", "kmc_plan_items",
           "kmc_replicas_per_lane", "kmc_pair_form", "kmc_plan_sym", "kmc_cluster_split",
           "kmc_sym_update", "kmc_persistent", "kmc_debug_grid_stall")
KMC_NOALLOC_MAX_N = 8192
KMC_MAX_CHAINS = 8  # parallel step-kernel chains of a batch (kmc_run)
KMC_ITEM_FIELDS = 8  # per work item in kmc_plan_items
KMC_SYM_FIELDS = 8  # per field and update item in kmc_plan_sym
KMC_CELL = 64  # NPs per cell of the symmetric pair form
FORM_ORDERED, FORM_SYMMETRIC = 1, 2  # kmc_pair_form
KMC_PHI_MAX_N = 64
# KMC_READ_COUNTERS slots
(CNT_JUMPS, CNT_NEAR, CNT_ONE_MIN, CNT_FALLBACK, CNT_RESCAN, CNT_POLISH,
 CNT_NONFINITE) = range(7)


class KmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class kmc_lysosome(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", C.POINTER(C.c_double)),
                ("axis", C.POINTER(C.c_double)), ("vol", C.POINTER(C.c_double)),
                ("center", C.POINTER(C.c_double)), ("Ms", C.c_double), ("Keff", C.c_double),
                ("T", C.c_double), ("tau0", C.c_double), ("rho", C.c_double)]


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libkmc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libkmc is not built (%s missing); run "
                                   "`python -m paper_1407_2737_gb300.build`" % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp = C.c_void_p
            L.kmc_create.argtypes = [C.POINTER(kmc_lysosome), C.c_int32, C.c_int, C.POINTER(vp)]
            L.kmc_set_stream.argtypes = [vp, vp]
            L.kmc_run.argtypes = [vp, _D, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                                  C.c_int32, C.c_uint64]
            L.kmc_read.argtypes = [vp, C.c_int32, C.c_int32, _D, C.c_int64, _I64]
            L.kmc_sync.argtypes = [vp]
            L.kmc_debug_step.argtypes = [vp, _D, C.c_double, C.c_uint64, C.c_int64, _D, _D, _D,
                                         _D, _D, _D, _I32]
            L.kmc_save.argtypes = [vp, C.c_char_p]
            L.kmc_load.argtypes = [vp, C.c_char_p]
            L.kmc_info.argtypes = [vp, _I64, _I32, _I64]
            L.kmc_tuning.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, _I32, _I32, _I32]
            L.kmc_dipolar_field_noalloc.argtypes = [C.c_int32, vp, vp, vp, C.c_double, _D,
                                                    C.c_double, vp, vp, vp]
            L.kmc_local_concentration.argtypes = [vp, C.c_int32, C.c_int32, _D, C.c_int64,
                                                  _I64]
            L.kmc_shell_profile.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, C.c_int32, _D,
                                            C.c_int64, _I64, _D]
            L.kmc_mean_run.argtypes = [C.POINTER(kmc_lysosome), C.c_int32, _D, C.c_int32,
                                       C.c_double, C.c_int32, C.c_int32, C.c_int32, _D,
                                       C.c_int64, _I64]
            L.kmc_regenerate.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, C.c_uint64,
                                         C.c_uint32]
            L.kmc_debug_stall.argtypes = [vp]
            L.kmc_targets_per_lane.argtypes = [vp, C.c_int32, _I32]
            L.kmc_replicas_per_lane.argtypes = [vp, C.c_int32, _I32]
            L.kmc_pair_form.argtypes = [vp, C.c_int32, _I32]
            L.kmc_cluster_split.argtypes = [vp, C.c_int32, _I32]
            L.kmc_sym_update.argtypes = [vp, C.c_int32, _I32]
            L.kmc_persistent.argtypes = [vp, C.c_int32, _I32]
            L.kmc_debug_grid_stall.argtypes = [vp]
            L.kmc_plan_sym.argtypes = [_I32, C.c_int32, C.c_int32, C.c_int32, _I32, C.c_int64,
                                       _I64, _I32, C.c_int64, _I64, _I64, _I32, _I32, _I32]
            L.kmc_plan_items.argtypes = [_I32, C.c_int32, C.c_int, C.c_int32, C.c_int32,
                                         C.c_int32, C.c_int32, _I32, C.c_int64, _I64, _I32,
                                         _I32]
            L.kmc_regenerate_rsa.argtypes = [vp, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                             C.c_uint32, C.c_int64, _I64]
            L.kmc_destroy.argtypes = [vp]
            L.kmc_destroy.restype = None
            L.kmc_last_error.argtypes = []
            L.kmc_last_error.restype = C.c_char_p
            for name in EXPORTS:
                if name not in ("kmc_destroy", "kmc_last_error"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def kmc_last_error():
    return lib().kmc_last_error().decode()


def _check(status):
    if status != KMC_OK:
        raise KmcError(status, kmc_last_error())


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _lysosome_arrays(ly, q):
    """pos [n][3], axis [n][3] and vol [n] of lysosome q as contiguous float64,
    refused (KMC_EINVAL) unless all three describe the same n NPs: the C side
    takes n from vol and reads n rows of the others."""
    pos = _f64(ly.pos)
    axis = _f64(ly.axis)
    vol = _f64(ly.vol).reshape(-1)
    n = vol.shape[0]
    if pos.size != 3 * n or axis.size != 3 * n:
        raise KmcError(KMC_EINVAL, "lysosome %d: pos (%d values) and axis (%d) must hold 3 per "
                       "NP for %d volumes" % (q, pos.size, axis.size, n))
    return pos.reshape(n, 3), axis.reshape(n, 3), vol


class Context:
    """An opened kmc_ctx; keeps the host arrays it was built from alive."""

    def __init__(self, handle, sizes):
        self.handle = C.c_void_p(handle)
        self.sizes = list(sizes)
        self.n_total = int(sum(sizes))

    def __del__(self):
        try:
            kmc_destroy(self)
        except Exception:
            pass


def kmc_create(lysosomes, precision=KMC_FP32_MIXED, center=None):
    """kmc_create over a list of objects with pos, axis, vol, Ms, Keff, T, tau0
    (and optional rho) attributes. center: None (centroid) or a (3,) origin used
    for every lysosome."""
    L = lib()
    keep = []
    arr = (kmc_lysosome * len(lysosomes))()
    cen = None if center is None else _f64(center, (3,))
    for q, ly in enumerate(lysosomes):
        pos, axis, vol = _lysosome_arrays(ly, q)
        keep += [pos, axis, vol]
        arr[q] = kmc_lysosome(len(vol), _dp(pos), _dp(axis), _dp(vol), _dp(cen), float(ly.Ms),
                              float(ly.Keff), float(ly.T), float(ly.tau0),
                              float(getattr(ly, "rho", 5200.0)))
    h = C.c_void_p()
    _check(L.kmc_create(arr, len(lysosomes), int(precision), C.byref(h)))
    return Context(h.value, [int(np.asarray(ly.vol).shape[0]) for ly in lysosomes])


def kmc_mean_run(lysosomes, mu0Hmax, f, steps_per_period, periods, discard_periods):
    """Ref. [8] mode on the device: returns [n_lys][S * (periods - discard)]
    volume-weighted mean m_z after each recorded step."""
    keep = []
    arr = (kmc_lysosome * len(lysosomes))()
    for q, ly in enumerate(lysosomes):
        pos, axis, vol = _lysosome_arrays(ly, q)
        keep += [pos, axis, vol]
        arr[q] = kmc_lysosome(len(vol), _dp(pos), _dp(axis), _dp(vol), None, float(ly.Ms),
                              float(ly.Keff), float(ly.T), float(ly.tau0),
                              float(getattr(ly, "rho", 5200.0)))
    H = _f64(np.atleast_1d(mu0Hmax), (-1,))
    n_rec = int(steps_per_period) * (int(periods) - int(discard_periods))
    out = np.zeros(max(n_rec * len(lysosomes), 1))
    n = C.c_int64(0)
    _check(lib().kmc_mean_run(arr, len(lysosomes), _dp(H), len(H), float(f),
                              int(steps_per_period), int(periods), int(discard_periods),
                              _dp(out), len(out), C.byref(n)))
    del keep
    return out[:int(n.value)].reshape(len(lysosomes), -1)


def kmc_regenerate(ctx, lys, what, disorder, seed, loop):
    """Redraw axes and/or positions of lysosome `lys` (-1: all) on the device."""
    _check(lib().kmc_regenerate(ctx.handle, int(lys), int(what), float(disorder),
                                C.c_uint64(int(seed)), C.c_uint32(int(loop))))


def kmc_regenerate_rsa(ctx, lys, radius, diameter, seed, loop, max_candidates=0):
    """Random sequential addition of lysosome `lys` on the device; returns the
    number of candidates used."""
    used = C.c_int64(0)
    _check(lib().kmc_regenerate_rsa(ctx.handle, int(lys), float(radius), float(diameter),
                                    C.c_uint64(int(seed)), C.c_uint32(int(loop)),
                                    int(max_candidates), C.byref(used)))
    return int(used.value)


def kmc_plan_items(n, precision, tpl=1, chunk=0, blocks_per_sm=5, n_sms=0):
    """The work items kmc_run launches for lysosomes of n[l] NPs (host only, no
    GPU): returns (items, chain_cut), items an int32 array [n_items, 8] of
    (lysosome, first target, targets, group, first record, end record, part,
    parts) and chain_cut the list of chain boundaries into items."""
    nn = np.ascontiguousarray(n, dtype=np.int32)
    cnt = C.c_int64()
    nch = C.c_int32()
    cut = np.zeros(KMC_MAX_CHAINS + 1, dtype=np.int32)
    args = (nn.ctypes.data_as(_I32), len(nn), int(precision), int(tpl), int(chunk),
            int(blocks_per_sm), int(n_sms))
    status = lib().kmc_plan_items(*args, None, 0, C.byref(cnt), cut.ctypes.data_as(_I32),
                                  C.byref(nch))
    if status != KMC_ECAPACITY:
        _check(status)
    items = np.zeros((max(cnt.value, 1), KMC_ITEM_FIELDS), dtype=np.int32)
    _check(lib().kmc_plan_items(*args, items.ctypes.data_as(_I32), cnt.value, C.byref(cnt),
                                cut.ctypes.data_as(_I32), C.byref(nch)))
    return items[:cnt.value], [int(x) for x in cut[:nch.value + 1]]


def kmc_plan_sym(n, gc, src_cells=0):
    """The symmetric pair form's plan for lysosomes of n[l] NPs (host only, no
    GPU): returns (items, upd, n_rev, cut_items, cut_upd). items: int32
    [n_items, 8] of (lysosome, row group, first source cell, end source cell
    (-1, -1: diagonal item), forward slot, first reverse slot of the
    lysosome, 0, 0); upd: int32 [n_upd, 8] of (lysosome, first target,
    targets, first forward slot, forward slots, first reverse slot, reverse
    slots, first target minus the row group's first NP)."""
    nn = np.ascontiguousarray(n, dtype=np.int32)
    ni, nu, nr = C.c_int64(), C.c_int64(), C.c_int64()
    nch = C.c_int32()
    ci = np.zeros(KMC_MAX_CHAINS + 1, dtype=np.int32)
    cu = np.zeros(KMC_MAX_CHAINS + 1, dtype=np.int32)
    head = (nn.ctypes.data_as(_I32), len(nn), int(gc), int(src_cells))
    tail = (C.byref(nr), ci.ctypes.data_as(_I32), cu.ctypes.data_as(_I32), C.byref(nch))
    status = lib().kmc_plan_sym(*head, None, 0, C.byref(ni), None, 0, C.byref(nu), *tail)
    if status != KMC_ECAPACITY:
        _check(status)
    items = np.zeros((max(ni.value, 1), KMC_SYM_FIELDS), dtype=np.int32)
    upd = np.zeros((max(nu.value, 1), KMC_SYM_FIELDS), dtype=np.int32)
    _check(lib().kmc_plan_sym(*head, items.ctypes.data_as(_I32), ni.value, C.byref(ni),
                              upd.ctypes.data_as(_I32), nu.value, C.byref(nu), *tail))
    return (items[:ni.value], upd[:nu.value], int(nr.value),
            [int(x) for x in ci[:nch.value + 1]], [int(x) for x in cu[:nch.value + 1]])


def kmc_pair_form(ctx, form=None):
    """Pins the FP32 pair form (FORM_ORDERED or FORM_SYMMETRIC; 0 = autotuned)
    or, with no argument, returns the form in use."""
    r = C.c_int32()
    _check(lib().kmc_pair_form(ctx.handle, -1 if form is None else int(form), C.byref(r)))
    return int(r.value)


def kmc_persistent(ctx, mode=None):
    """Pins the persistent period (1 = off, 2 = on: one cooperative launch per
    field period with a grid barrier between steps; 0 = autotuned) or, with no
    argument, returns the value in use."""
    r = C.c_int32()
    _check(lib().kmc_persistent(ctx.handle, -1 if mode is None else int(mode), C.byref(r)))
    return int(r.value)


def kmc_debug_grid_stall(ctx):
    """Failure-detection hook of the persistent period: raises
    KmcError(KMC_ETIMEOUT) when the stalled grid barrier runs out as designed."""
    _check(lib().kmc_debug_grid_stall(ctx.handle))


def kmc_sym_update(ctx, mode=None):
    """Pins the symmetric form's update kernel (1 = one warp per update item,
    2 = one block; 0 = autotuned) or, with no argument, returns the one in
    use."""
    r = C.c_int32()
    _check(lib().kmc_sym_update(ctx.handle, -1 if mode is None else int(mode), C.byref(r)))
    return int(r.value)


def kmc_cluster_split(ctx, mode=None):
    """Pins the FP32 one-target kernel's cluster split (1 = off, 2 = on: each
    group's two source parts as a two-CTA cluster; 0 = autotuned) or, with no
    argument, returns the value in use."""
    r = C.c_int32()
    _check(lib().kmc_cluster_split(ctx.handle, -1 if mode is None else int(mode), C.byref(r)))
    return int(r.value)


def kmc_targets_per_lane(ctx, tpl=None):
    """Pins the FP32 kernel's targets per lane (1, 2 or 3 ordered; 2 or 4 in
    the symmetric form; 0 = autotuned) or, with no argument, returns the value
    in use."""
    t = C.c_int32()
    _check(lib().kmc_targets_per_lane(ctx.handle, -1 if tpl is None else int(tpl), C.byref(t)))
    return int(t.value)


def kmc_replicas_per_lane(ctx, rpl=None):
    """Pins the FP32 kernel's replicas per lane (1 = off, 2 or 4 for sets of
    identical consecutive lysosomes; 0 = autotuned) or, with no argument,
    returns the value in use."""
    r = C.c_int32()
    _check(lib().kmc_replicas_per_lane(ctx.handle, -1 if rpl is None else int(rpl), C.byref(r)))
    return int(r.value)


def kmc_debug_stall(ctx):
    """Failure-detection hook: raises KmcError(KMC_ETIMEOUT) when the stalled
    waits run out as designed."""
    _check(lib().kmc_debug_stall(ctx.handle))


def kmc_set_stream(ctx, stream_handle):
    _check(lib().kmc_set_stream(ctx.handle, C.c_void_p(stream_handle or 0)))


def kmc_run(ctx, mu0Hmax, f, steps_per_period, periods, discard_periods, seed):
    amps = _f64(np.atleast_1d(mu0Hmax), (-1,))
    _check(lib().kmc_run(ctx.handle, _dp(amps), len(amps), float(f), int(steps_per_period),
                         int(periods), int(discard_periods), C.c_uint64(int(seed))))


def kmc_sync(ctx):
    _check(lib().kmc_sync(ctx.handle))


def kmc_read(ctx, what, lys=0):
    L = lib()
    n = C.c_int64(0)
    st = L.kmc_read(ctx.handle, int(what), int(lys), None, 0, C.byref(n))
    if st not in (KMC_OK, KMC_ECAPACITY):
        _check(st)
    buf = np.zeros(max(int(n.value), 1))
    _check(L.kmc_read(ctx.handle, int(what), int(lys), _dp(buf), len(buf), C.byref(n)))
    out = buf[:int(n.value)]
    if what in (KMC_READ_MOMENTS, KMC_READ_POSITIONS, KMC_READ_AXES):
        return out.reshape(-1, 3)
    return out


def kmc_debug_step(ctx, mu0Hext, t_step, seed, step, m_in):
    N = ctx.n_total
    H = _f64(np.broadcast_to(np.atleast_1d(mu0Hext), (len(ctx.sizes),)), (-1,))
    m_in = _f64(m_in, (N, 3))
    out = dict(m_out=np.zeros((N, 3)), B_dip=np.zeros((N, 3)), dE=np.zeros((N, 2)),
               P=np.zeros(N), u=np.zeros(N), flags=np.zeros(N, dtype=np.int32))
    _check(lib().kmc_debug_step(ctx.handle, _dp(H), float(t_step), C.c_uint64(int(seed)),
                                int(step), _dp(m_in), _dp(out["m_out"]), _dp(out["B_dip"]),
                                _dp(out["dE"]), _dp(out["P"]), _dp(out["u"]),
                                out["flags"].ctypes.data_as(_I32)))
    f = out["flags"]
    out.update(n_min=f & 3, flipped=(f >> 2) & 1, near=(f >> 3) & 1, degenerate=(f >> 4) & 1,
               rescan=(f >> 5) & 1, polish=(f >> 6) & 1, nonfinite=(f >> 7) & 1)
    return out


def kmc_save(ctx, path):
    _check(lib().kmc_save(ctx.handle, os.fsencode(path)))


def kmc_load(ctx, path):
    _check(lib().kmc_load(ctx.handle, os.fsencode(path)))


def kmc_info(ctx):
    n = C.c_int64()
    nl = C.c_int32()
    s = C.c_int64()
    _check(lib().kmc_info(ctx.handle, C.byref(n), C.byref(nl), C.byref(s)))
    return dict(n_total=n.value, n_lys=nl.value, global_step=s.value)


def kmc_tuning(ctx, warps=None, tile=None, chunk=0):
    """Sets the launch shape (warps and tile given; 0 = autotune) or, with no
    arguments, returns the shape in use as (warps, tile, chunk)."""
    w, t, c = C.c_int32(), C.c_int32(), C.c_int32()
    if warps is None and tile is None:
        _check(lib().kmc_tuning(ctx.handle, -1, -1, -1, C.byref(w), C.byref(t), C.byref(c)))
    else:
        _check(lib().kmc_tuning(ctx.handle, int(warps), int(tile), int(chunk), C.byref(w),
                                C.byref(t), C.byref(c)))
    return int(w.value), int(t.value), int(c.value)


def kmc_dipolar_field_noalloc(n, pos_dev, m_dev, vol_dev, Ms, center, length, B_dev,
                              stream_handle=0, status_dev=0):
    """Calls the no-allocation field entry point. pos_dev, m_dev, vol_dev and
    B_dev are device addresses (integers, e.g. a tensor's data_ptr()) of
    caller-owned float64 buffers; status_dev the address of a caller-owned
    int32 that receives the call's device-side status (0: none); center is a
    host (3,) origin in m."""
    cen = _f64(center, (3,))
    _check(lib().kmc_dipolar_field_noalloc(int(n), C.c_void_p(pos_dev), C.c_void_p(m_dev),
                                           C.c_void_p(vol_dev), float(Ms), _dp(cen),
                                           float(length), C.c_void_p(B_dev),
                                           C.c_void_p(status_dev or 0),
                                           C.c_void_p(stream_handle or 0)))


def kmc_local_concentration(ctx, lys, N):
    """Eq. 8: phi_N of every NP of lysosome `lys` (computed on the device)."""
    n = C.c_int64(0)
    L = lib()
    st = L.kmc_local_concentration(ctx.handle, int(lys), int(N), None, 0, C.byref(n))
    if st not in (KMC_OK, KMC_ECAPACITY):
        _check(st)
    buf = np.zeros(max(int(n.value), 1))
    _check(L.kmc_local_concentration(ctx.handle, int(lys), int(N), _dp(buf), len(buf),
                                     C.byref(n)))
    return buf[:int(n.value)]


def kmc_shell_profile(ctx, lys, radius, n_shells, N):
    """Radial profile of the last run: dict of per-shell count, area (J/m^3 per
    cycle), dHdip (T) and phi_N, and the radius R used (m)."""
    out = np.zeros(4 * int(n_shells))
    n = C.c_int64(0)
    R = C.c_double(0.0)
    _check(lib().kmc_shell_profile(ctx.handle, int(lys), float(radius), int(n_shells), int(N),
                                   _dp(out), len(out), C.byref(n), C.byref(R)))
    t = out.reshape(-1, 4)
    return dict(count=t[:, 0].copy(), area=t[:, 1].copy(), dHdip=t[:, 2].copy(),
                phi=t[:, 3].copy(), radius=float(R.value))


def kmc_destroy(ctx):
    if ctx is not None and ctx.handle is not None and ctx.handle.value:
        lib().kmc_destroy(ctx.handle)
        ctx.handle = C.c_void_p(0)
