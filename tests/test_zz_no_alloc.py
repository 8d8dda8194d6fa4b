"""cascade_forward_fixed_scratch: the forward for callers that cannot call
cudaMalloc (a plugin inside a host framework whose memory pool owns all device
memory, or a latency-bound path where an allocation could synchronise the
GPU).  Its workspace is a fixed 32 MiB device array inside the library.

Checked through the C ABI against cascade_forward with a caller workspace
filled with NaN, so that a read of any workspace byte the call did not write
first shows up in y.  Both paths run the same deterministic kernels, so y
must be equal bit for bit, on two calls in a row with different inputs,
after the shared array was left holding another plan's data (another m,
batch and input scale).  The §3 schedule, the work-efficient schedule and a
plan that keeps its stage outputs are covered; for the last, a backward
after a fixed-scratch forward still uses the caller-workspace forward's
states.  A batch whose workspace exceeds the array is refused.  This file is
collected last and builds what it needs, so it passes both alone in a fresh
process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import _abi, cascade
    return torch, _abi, cascade


def fixed_forward(torch, _abi, c, u, y):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = c.lib.cascade_forward_fixed_scratch(c.plan, C.c_void_p(u.data_ptr()),
                                             C.c_void_p(y.data_ptr()), stream)
    assert st == _abi.CASCADE_OK, c.lib.cascade_last_error(c.plan)


def dirty_the_array(torch, _abi, cascade):
    """Leave another plan's states (m = 256, large inputs) in the shared array."""
    w = wl.precision_form(m=256, L=2500, batch=2, N=11)
    c = cascade.from_workload(w, precision="bf16_split")
    assert c.workspace_size() <= (32 << 20)
    u = torch.full((w.rows, 1), 1e3, dtype=torch.float32, device="cuda")
    y = torch.empty((w.rows, 1), dtype=torch.float32, device="cuda")
    fixed_forward(torch, _abi, c, u, y)
    torch.cuda.synchronize()
    assert c.device_error() == 0
    c.close()


@pytest.mark.parametrize("flag", ["default", "scan", "save_states"])
def test_fixed_scratch_forward_matches_workspace_forward(mods, flag):
    torch, _abi, cascade = mods
    flags = {"default": 0, "scan": _abi.CASCADE_FLAG_SCAN,
             "save_states": _abi.CASCADE_FLAG_SAVE_STATES}[flag]
    dirty_the_array(torch, _abi, cascade)
    w = wl.precision_form(m=128, L=1000, batch=3, N=9)
    c = cascade.from_workload(w, precision="bf16_split", flags=flags)
    assert c.workspace_size() <= (32 << 20)
    rng = np.random.default_rng(11)
    for call in range(2):
        u = torch.as_tensor(rng.standard_normal((w.rows, 1)).astype(np.float32), device="cuda")
        c.workspace().fill_(0xFF)                  # NaN in every BF16 / FP32 plane
        y_ref = c.forward(u)                       # existing entry point, caller workspace
        y_fix = torch.full_like(y_ref, float("nan"))
        fixed_forward(torch, _abi, c, u, y_fix)
        torch.cuda.synchronize()
        assert c.device_error() == 0
        a = y_fix.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.all(np.isfinite(b)), f"call {call}: the forward read unwritten workspace"
        assert np.array_equal(a, b), (call, float(np.max(np.abs(a - b))))
        if flag == "save_states":
            # the backward refers to the caller-workspace forward, not to the
            # states the fixed-scratch call left in the shared array
            dy = torch.as_tensor(rng.standard_normal((w.rows, 1)).astype(np.float32),
                                 device="cuda")
            g1 = c.backward(u, dy)
            c.forward(u)
            g2 = c.backward(u, dy)
            torch.cuda.synchronize()
            for k in g1:
                assert torch.equal(g1[k], g2[k]), k


def test_fixed_scratch_rejects_oversized_batch(mods):
    torch, _abi, cascade = mods
    w = wl.precision_form(m=256, L=16384, batch=2, N=13)     # 2^15 rows x 256 x 8 B > 32 MiB
    c = cascade.from_workload(w, precision="bf16_split")
    assert c.workspace_size() > (32 << 20)
    u = torch.zeros((w.rows, 1), dtype=torch.float32, device="cuda")
    y = torch.zeros((w.rows, 1), dtype=torch.float32, device="cuda")
    st = c.lib.cascade_forward_fixed_scratch(c.plan, C.c_void_p(u.data_ptr()),
                                             C.c_void_p(y.data_ptr()), None)
    assert st == _abi.CASCADE_ERR_UNSUPPORTED
    assert b"fixed scratch" in c.lib.cascade_last_error(c.plan)
