"""The KMC_DEBUG build of the library (every work item, staged tile and Newton
bracket checked against its bounds on the device; a failed check skips the
access and kmc_sync reports KMC_ESTATE with the check's site) on the small and
ragged cases where index arithmetic goes wrong first: lysosomes of 1, 2, 3 and
33 NPs and one tile of sources minus one, exactly and plus one, in both
precisions, one and two targets per lane, whole and split source ranges, and
the symmetric pair form's field and update items over empty, partial and whole
cells and row groups, and the cluster split. Every launch must pass its checks, and the results must
still match the oracle.

The debug library is loaded in a child process (KMC_LIB_PATH), so that it does
not replace the release build in this one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1407_2737_gb300 import inputs, kmc

def rms(B):
    return float(np.sqrt(np.mean(np.sum(B ** 2, axis=1)))) or 1.0

checked = 0
for prec, tile, sizes in ((kmc.KMC_FP32_MIXED, 64, (1, 2, 3, 33, 127, 128, 129)),
                          (kmc.KMC_FP64_PLAIN, 64, (1, 2, 3, 33, 63, 64, 65))):
    lyss = [inputs.make_lysosome(n, 12e-9, 0.05 if n > 3 else 0.01, seed=40 + n) for n in sizes]
    # (targets per lane, warps): with 8 warps the two parts update side by side
    tpls = ((1, 4), (2, 4), (2, 8)) if prec == kmc.KMC_FP32_MIXED else ((1, 4),)
    for tpl, warps in tpls:
        for chunk in (0, 128):
            ctx = kmc.kmc_create(lyss, prec, center=np.zeros(3))
            if prec == kmc.KMC_FP32_MIXED:
                kmc.kmc_targets_per_lane(ctx, tpl)
            kmc.kmc_tuning(ctx, warps, tile, chunk)
            rng = np.random.default_rng(tpl * 10 + chunk)
            m = np.concatenate([oracle.initial_moments(l.axis) + 0.3 * rng.normal(size=(l.n, 3))
                                for l in lyss])
            m /= np.linalg.norm(m, axis=1, keepdims=True)
            m = m.astype(np.float32).astype(np.float64)
            g = kmc.kmc_debug_step(ctx, np.full(len(lyss), 0.015), 5e-8, 3, 21, m)
            off = 0
            for l, ly in enumerate(lyss):
                B = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m[off:off + ly.n])
                err = np.max(np.linalg.norm(g["B_dip"][off:off + ly.n] - B, axis=1))
                tol = (1e-5 if prec == kmc.KMC_FP32_MIXED else 1e-11) * rms(B)
                assert err <= tol, (prec, tpl, chunk, ly.n, err)
                off += ly.n
            kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 1, 5)
            kmc.kmc_sync(ctx)  # raises KMC_ESTATE if a bounds check failed
            kmc.kmc_destroy(ctx)
            checked += 1
# the symmetric pair form: field and update items, cells and row groups
lyss = [inputs.make_lysosome(n, 12e-9, 0.05 if n > 3 else 0.01, seed=50 + n)
        for n in (1, 2, 63, 64, 65, 129, 600)]
for warps, cells, chunk, upd in ((4, 1, 0, 1), (4, 1, 64, 1), (4, 2, 128, 1), (8, 1, 0, 1),
                                 (2, 2, 64, 1), (4, 2, 128, 2), (8, 1, 64, 2)):
    ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
    kmc.kmc_pair_form(ctx, kmc.FORM_SYMMETRIC)
    kmc.kmc_targets_per_lane(ctx, 2 * cells)
    kmc.kmc_sym_update(ctx, upd)
    kmc.kmc_tuning(ctx, warps, 32, chunk)
    rng = np.random.default_rng(warps + cells + chunk)
    m = np.concatenate([oracle.initial_moments(l.axis) + 0.3 * rng.normal(size=(l.n, 3))
                        for l in lyss])
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    m = m.astype(np.float32).astype(np.float64)
    g = kmc.kmc_debug_step(ctx, np.full(len(lyss), 0.015), 5e-8, 3, 21, m)
    off = 0
    for l, ly in enumerate(lyss):
        B = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m[off:off + ly.n])
        err = np.max(np.linalg.norm(g["B_dip"][off:off + ly.n] - B, axis=1))
        assert err <= 1e-5 * rms(B) or ly.n == 1, ("sym", warps, cells, chunk, ly.n, err)
        off += ly.n
    kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 1, 5)
    kmc.kmc_sync(ctx)
    kmc.kmc_destroy(ctx)
    checked += 1
# the cluster split: two-CTA clusters over groups of exactly two source parts
lyss = [inputs.make_lysosome(n, 12e-9, 0.05, seed=30 + n) for n in (2000, 1030)]
ctx = kmc.kmc_create(lyss, kmc.KMC_FP32_MIXED, center=np.zeros(3))
kmc.kmc_targets_per_lane(ctx, 1)
kmc.kmc_cluster_split(ctx, 2)
kmc.kmc_tuning(ctx, 4, 128, 1024)
kmc.kmc_run(ctx, 0.02, 1e5, 20, 2, 1, 5)
kmc.kmc_sync(ctx)
kmc.kmc_destroy(ctx)
checked += 1
print("debug build: %d contexts passed their bounds checks" % checked)
'''


def test_small_and_ragged_cases_pass_the_debug_bounds_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    lib = kbuild.build(debug=True)
    env = dict(os.environ, KMC_LIB_PATH=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "passed their bounds checks" in r.stdout
