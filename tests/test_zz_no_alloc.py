"""kmc_dipolar_field_noalloc: the dipolar field for callers that cannot
allocate device memory (a framework's memory pool, memory reserved up front,
device pointers handed in by a caller). The buffers here are allocated by the
test, playing that caller; the entry point itself allocates nothing and works
in its static scratch array. Its fields must match those of the library's
regular path (kmc_debug_step on a context) within the FP32 field tolerance of
the other tests, on two calls in a row (the second reuses the scratch the first
left behind).

The file name makes pytest collect it last."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2737_gb300 import inputs, kmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1407_2737_gb300 import build as kbuild
    kbuild.build()
    return torch


def test_noalloc_field_matches_regular_path(torch_cuda):
    torch = torch_cuda
    # 1501 NPs: odd count (padding record), a ragged last group of 29 targets,
    # and source ranges split over two items per group
    lys = inputs.make_lysosome(1501, 12e-9, 0.08, seed=21)
    n = lys.n
    length = (6.0 * float(np.mean(lys.vol)) / math.pi) ** (1.0 / 3.0)
    ctx = kmc.kmc_create([lys], kmc.KMC_FP32_MIXED, center=np.zeros(3))
    dev = torch.device("cuda")
    pos_d = torch.tensor(lys.pos, dtype=torch.float64, device=dev).contiguous()
    vol_d = torch.tensor(lys.vol, dtype=torch.float64, device=dev).contiguous()
    rng = np.random.default_rng(4)
    for call in range(2):
        m = oracle.initial_moments(lys.axis) + 0.4 * rng.normal(size=(n, 3))
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        m = m.astype(np.float32).astype(np.float64)  # the state both paths hold
        ref = kmc.kmc_debug_step(ctx, 0.0, 5e-8, 1, call, m)["B_dip"]
        m_d = torch.tensor(m, dtype=torch.float64, device=dev).contiguous()
        B_d = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        kmc.kmc_dipolar_field_noalloc(n, pos_d.data_ptr(), m_d.data_ptr(), vol_d.data_ptr(),
                                      lys.Ms, np.zeros(3), length, B_d.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        B = B_d.cpu().numpy()
        assert np.all(np.isfinite(B))
        rms = np.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
        err = np.max(np.linalg.norm(B - ref, axis=1)) / rms
        assert err <= 1e-5, (call, err)
    kmc.kmc_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_dipolar_field_noalloc(kmc.KMC_NOALLOC_MAX_N + 1, 1, 1, 1, 1e6, np.zeros(3),
                                      1e-8, 1, 0)
    assert e.value.status == kmc.KMC_ECAPACITY
    assert "8192" in str(e.value)
