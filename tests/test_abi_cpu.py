"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/kmc.h declares, and rejects bad arguments
before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1407_2737_gb300 import build as kbuild
from paper_1407_2737_gb300 import inputs, kmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    kbuild.build()
    return kmc.lib()


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(kmc_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    names = declared_entry_points()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(kmc.EXPORTS)


def test_bad_arguments_are_rejected_on_the_host(L):
    h = C.c_void_p()
    assert L.kmc_create(None, 1, 0, C.byref(h)) == kmc.KMC_EINVAL
    assert "lysosome" in kmc.kmc_last_error()
    lys = inputs.make_lysosome(10, 12e-9, 0.05, seed=0)
    lys.Ms = -1.0
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_create([lys])
    assert e.value.status == kmc.KMC_EINVAL
    lys = inputs.make_lysosome(10, 12e-9, 0.05, seed=0)
    lys.vol = np.zeros(10)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_create([lys])
    assert e.value.status == kmc.KMC_EINVAL
    assert L.kmc_run(None, None, 0, 0.0, 0, 0, 0, 0) == kmc.KMC_EINVAL
    assert L.kmc_read(None, 0, 0, None, 0, None) == kmc.KMC_EINVAL
    assert L.kmc_sync(None) == kmc.KMC_EINVAL
    L.kmc_destroy(None)  # NULL-safe


def _bad(field):
    lys = inputs.make_lysosome(10, 12e-9, 0.05, seed=0)
    if field == "empty":
        lys.pos, lys.axis, lys.vol = np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0)
    elif field == "nan_pos":
        lys.pos = lys.pos.copy()
        lys.pos[3, 1] = np.nan
    elif field == "zero_axis":
        lys.axis = lys.axis.copy()
        lys.axis[7] = 0.0
    elif field == "inf_axis":
        lys.axis = lys.axis.copy()
        lys.axis[0, 2] = np.inf
    elif field == "neg_vol":
        lys.vol = lys.vol.copy()
        lys.vol[2] = -lys.vol[2]
    elif field == "short_pos":
        lys.pos = lys.pos[:9]
    elif field == "long_axis":
        lys.axis = np.concatenate([lys.axis, lys.axis[:1]])
    else:
        setattr(lys, field[0], field[1])
    return lys


@pytest.mark.parametrize("field", ["empty", "nan_pos", "zero_axis", "inf_axis", "neg_vol",
                                   "short_pos", "long_axis", ("Ms", 0.0), ("Ms", np.inf),
                                   ("Keff", -1.0), ("Keff", np.nan), ("T", -1.0),
                                   ("tau0", 0.0), ("tau0", np.nan)],
                         ids=str)
def test_bad_lysosomes_are_rejected_before_any_device_call(L, field):
    """Each bad lysosome is refused with KMC_EINVAL, on the host, in both
    precisions and in the mean mode: validation comes before the device is
    looked for, so a machine without a GPU gives the same answer."""
    lys = _bad(field)
    for prec in (kmc.KMC_FP64_PLAIN, kmc.KMC_FP32_MIXED):
        with pytest.raises(kmc.KmcError) as e:
            kmc.kmc_create([inputs.make_lysosome(5, 12e-9, 0.05, seed=1), lys], prec)
        assert e.value.status == kmc.KMC_EINVAL, (field, str(e.value))
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_mean_run([lys], 0.02, 1e5, 20, 2, 1)
    assert e.value.status == kmc.KMC_EINVAL, (field, str(e.value))


def test_no_device_is_an_error_not_a_fallback(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lys = inputs.make_lysosome(10, 12e-9, 0.05, seed=0)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_create([lys])
    assert e.value.status == kmc.KMC_ECUDA


def test_header_constants_match_the_binding():
    text = "".join(open(os.path.join(ROOT, "include", fn)).read()
                   for fn in sorted(os.listdir(os.path.join(ROOT, "include"))) if fn.endswith(".h"))
    defs = re.findall(r"#define\s+(KMC_\w+)\s+(\d+)", text)
    assert len(defs) >= 2
    for name, value in defs:
        assert getattr(kmc, name) == int(value), name


def test_every_context_entry_point_rejects_a_null_context(L):
    """Each entry point that takes a context answers a NULL one with
    KMC_EINVAL before any device call; the context-free ones check their
    sizes and pointers on the host too."""
    def neutral(t):
        if t in (C.c_int32, C.c_int, C.c_int64, C.c_uint64, C.c_uint32):
            return 0
        if t is C.c_double:
            return 0.0
        return None
    checked = 0
    for name in kmc.EXPORTS:
        f = getattr(L, name)
        at = getattr(f, "argtypes", None)
        if name == "kmc_destroy" or not at or at[0] is not C.c_void_p:
            continue
        assert f(None, *[neutral(t) for t in at[1:]]) == kmc.KMC_EINVAL, name
        checked += 1
    assert checked >= 14
    big = kmc.KMC_NOALLOC_MAX_N + 1
    cen = np.zeros(3)
    cp = cen.ctypes.data_as(C.POINTER(C.c_double))
    assert L.kmc_dipolar_field_noalloc(0, 1, 1, 1, 1e6, cp, 1e-8, 1, None, None) == kmc.KMC_ECAPACITY
    assert L.kmc_dipolar_field_noalloc(big, 1, 1, 1, 1e6, cp, 1e-8, 1, None, None) == kmc.KMC_ECAPACITY
    assert L.kmc_dipolar_field_noalloc(4, None, 1, 1, 1e6, cp, 1e-8, 1, None, None) == kmc.KMC_EINVAL
    assert L.kmc_dipolar_field_noalloc(4, 1, 1, 1, -1.0, cp, 1e-8, 1, None, None) == kmc.KMC_EINVAL
    assert L.kmc_mean_run(None, 0, None, 0, 0.0, 0, 0, 0, None, 0, None) == kmc.KMC_EINVAL


def test_debug_build_compiles_and_exports_the_same_entry_points():
    """The KMC_DEBUG build (bounds checks on the device) is a separate library
    with the same ABI; here it is only built and inspected (no GPU)."""
    lib = kbuild.build(debug=True)
    assert lib != kbuild.LIB and os.path.exists(lib)
    D = C.CDLL(lib)
    for n in declared_entry_points():
        assert hasattr(D, n), n
