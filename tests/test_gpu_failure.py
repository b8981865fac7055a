"""Failure detection without a GPU fault: a step whose staged copies can never
complete (each tile waits for 16 bytes more than it receives) must end its
bounded waits, report KMC_ETIMEOUT through the device error word, write no
state, and leave the context usable."""
import time

import numpy as np
import pytest

from paper_1407_2737_gb300 import inputs, kmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()


def _run(ctx):
    kmc.kmc_run(ctx, 0.02, 1e5, 50, 2, 1, 3)
    return (kmc.kmc_read(ctx, kmc.KMC_READ_LOOP_M, 0), kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, 0))


def test_stalled_waits_report_timeout_and_leave_the_context_usable():
    lys = inputs.make_lysosome(150, 12e-9, 0.05, seed=3)
    ref = kmc.kmc_create([lys], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    loop_ref, m_ref = _run(ref)
    kmc.kmc_destroy(ref)

    ctx = kmc.kmc_create([lys], kmc.KMC_FP64_PLAIN, center=np.zeros(3))
    m0 = kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, 0)
    t = time.perf_counter()
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_debug_stall(ctx)
    assert e.value.status == kmc.KMC_ETIMEOUT
    assert time.perf_counter() - t < 5.0  # 1 ms waits, not the 2 s production limit
    assert np.array_equal(kmc.kmc_read(ctx, kmc.KMC_READ_MOMENTS, 0), m0)  # nothing written
    loop, m = _run(ctx)  # the context carries on as if nothing had happened
    assert np.array_equal(loop, loop_ref)
    assert np.array_equal(m, m_ref)
    kmc.kmc_destroy(ctx)


def test_stall_hook_is_fp64_only():
    lys = inputs.make_lysosome(40, 12e-9, 0.05, seed=1)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_debug_stall(ctx)
    assert e.value.status == kmc.KMC_EINVAL
    kmc.kmc_destroy(ctx)
