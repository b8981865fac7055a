"""kmc_dipolar_field_noalloc: the dipolar field for callers that cannot
allocate device memory -- code running inside another framework's memory pool,
processes that reserve all device memory up front, or libraries that are only
handed device pointers by their caller. Such a caller owns every buffer; the
entry point itself allocates nothing and works in one static scratch array that
all calls share.

Checked here through the C ABI: the field against the FP64 oracle (Eq. 1 on the
float32 frame's geometry) within the FP32 field tolerance of the other tests,
1e-5 of rms, on two calls in a row for every size (the second call reuses the
scratch the first left behind); that a call changes neither torch's allocation
count nor the device's free memory; that host memory is refused before any
launch; and that a staging wait that runs out is reported through the
caller's status word with NaN in the field, after which the next call is
correct again.

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


def _call(torch, n, pos_d, m_d, vol_d, Ms, length, B_d, status_d=None):
    kmc.kmc_dipolar_field_noalloc(n, pos_d.data_ptr(), m_d.data_ptr(), vol_d.data_ptr(), Ms,
                                  np.zeros(3), length, B_d.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream,
                                  status_d.data_ptr() if status_d is not None else 0)


def _moments(axis, rng):
    m = oracle.initial_moments(axis) + 0.4 * rng.normal(size=axis.shape)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    return m.astype(np.float32).astype(np.float64)  # what the float32 records hold


@pytest.mark.parametrize("n", [1, 7, 1024, 1501, kmc.KMC_NOALLOC_MAX_N])
def test_noalloc_field_matches_the_oracle(torch_cuda, n):
    """n = 1 (no other NP: zero field), 7 (one ragged group), 1024 (one source
    part), 1501 (odd count, ragged last group, two parts) and the maximum 8192
    (eight parts, every scratch region full)."""
    torch = torch_cuda
    ly = inputs.make_lysosome(n, 12e-9, 0.08 if n > 7 else 0.02, seed=21 + n)
    dev = torch.device("cuda")
    pos_d = torch.tensor(ly.pos, dtype=torch.float64, device=dev).contiguous()
    vol_d = torch.tensor(ly.vol, dtype=torch.float64, device=dev).contiguous()
    status_d = torch.full((1,), -1, dtype=torch.int32, device=dev)
    rng = np.random.default_rng(4)
    for call in range(2):
        m = _moments(ly.axis, rng)
        ref = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m)
        m_d = torch.tensor(m, dtype=torch.float64, device=dev).contiguous()
        B_d = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        _call(torch, n, pos_d, m_d, vol_d, ly.Ms, ly.d, B_d, status_d)
        torch.cuda.synchronize()
        B = B_d.cpu().numpy()
        assert int(status_d.item()) == kmc.KMC_OK
        assert np.all(np.isfinite(B))
        if n == 1:
            assert np.all(B == 0.0)
            continue
        rms = np.sqrt(np.mean(np.sum(ref ** 2, axis=1)))
        err = np.max(np.linalg.norm(B - ref, axis=1)) / rms
        assert err <= 1e-5, (n, call, err)


def test_noalloc_call_allocates_nothing(torch_cuda):
    torch = torch_cuda
    n = 4000
    ly = inputs.make_lysosome(n, 12e-9, 0.08, seed=5)
    dev = torch.device("cuda")
    pos_d = torch.tensor(ly.pos, dtype=torch.float64, device=dev).contiguous()
    vol_d = torch.tensor(ly.vol, dtype=torch.float64, device=dev).contiguous()
    m_d = torch.tensor(oracle.initial_moments(ly.axis), dtype=torch.float64, device=dev)
    B_d = torch.empty((n, 3), dtype=torch.float64, device=dev)
    _call(torch, n, pos_d, m_d, vol_d, ly.Ms, ly.d, B_d)  # first call on this device
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    _call(torch, n, pos_d, m_d, vol_d, ly.Ms, ly.d, B_d)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_host_memory_and_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    n = 64
    ly = inputs.make_lysosome(n, 12e-9, 0.05, seed=6)
    dev = torch.device("cuda")
    pos_h = np.ascontiguousarray(ly.pos)
    vol_d = torch.tensor(ly.vol, dtype=torch.float64, device=dev)
    m_d = torch.tensor(oracle.initial_moments(ly.axis), dtype=torch.float64, device=dev)
    B_d = torch.full((n, 3), 7.0, dtype=torch.float64, device=dev)
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_dipolar_field_noalloc(n, pos_h.ctypes.data, m_d.data_ptr(), vol_d.data_ptr(),
                                      ly.Ms, np.zeros(3), ly.d, B_d.data_ptr(), 0)
    assert e.value.status == kmc.KMC_EINVAL and "pos" in str(e.value)
    torch.cuda.synchronize()
    assert torch.all(B_d == 7.0)  # nothing ran
    with pytest.raises(kmc.KmcError) as e:
        kmc.kmc_dipolar_field_noalloc(kmc.KMC_NOALLOC_MAX_N + 1, 1, 1, 1, 1e6, np.zeros(3),
                                      1e-8, 1, 0)
    assert e.value.status == kmc.KMC_ECAPACITY
    assert "8192" in str(e.value)


def test_noalloc_timeout_is_reported_and_the_next_call_is_correct(torch_cuda, monkeypatch):
    """With KMC_FAULT=noalloc_stall every staging wait expects 16 bytes more
    than its copy delivers and gives up after 1 ms (every copy has landed, no
    kernel faults or hangs): the status word reads KMC_ETIMEOUT and the field
    is NaN. The next call, without the fault, gives the oracle's field."""
    torch = torch_cuda
    n = 1501
    ly = inputs.make_lysosome(n, 12e-9, 0.08, seed=9)
    dev = torch.device("cuda")
    pos_d = torch.tensor(ly.pos, dtype=torch.float64, device=dev).contiguous()
    vol_d = torch.tensor(ly.vol, dtype=torch.float64, device=dev).contiguous()
    m = _moments(ly.axis, np.random.default_rng(2))
    m_d = torch.tensor(m, dtype=torch.float64, device=dev).contiguous()
    status_d = torch.full((1,), -1, dtype=torch.int32, device=dev)
    B_d = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    monkeypatch.setenv("KMC_FAULT", "noalloc_stall")
    _call(torch, n, pos_d, m_d, vol_d, ly.Ms, ly.d, B_d, status_d)
    torch.cuda.synchronize()
    assert int(status_d.item()) == kmc.KMC_ETIMEOUT
    assert torch.all(torch.isnan(B_d))
    monkeypatch.delenv("KMC_FAULT")
    _call(torch, n, pos_d, m_d, vol_d, ly.Ms, ly.d, B_d, status_d)
    torch.cuda.synchronize()
    assert int(status_d.item()) == kmc.KMC_OK
    ref = oracle.dipolar_field(ly.pos, ly.vol, ly.Ms, m)
    rms = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    assert np.max(np.linalg.norm(B_d.cpu().numpy() - ref, axis=1)) <= 1e-5 * rms
