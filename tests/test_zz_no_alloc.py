"""cascade_forward_fixed_scratch: the forward for callers that cannot call
cudaMalloc (a plugin inside a host framework whose memory pool owns all device
memory, or a latency-bound path where an allocation could synchronise the
GPU).  Its workspace is a fixed 32 MiB device array inside the library.

Checked through the C ABI against cascade_forward (caller-provided workspace)
on two calls in a row with different inputs, within the BF16-split tolerance
of the parity tests; a batch whose workspace exceeds the array is refused.
This file is collected last, and it builds what it needs, so it passes both
alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from _parity import OUT_EPS, TOL, rel_errors

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


def test_fixed_scratch_forward_matches_workspace_forward(mods):
    torch, _abi, cascade = mods
    w = wl.precision_form(m=128, L=1500, batch=3, N=10)
    c = cascade.from_workload(w, precision="bf16_split")
    assert c.workspace_size() <= (32 << 20)
    lib = c.lib
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(11)
    for call in range(2):
        u_np = rng.standard_normal((w.rows, 1)).astype(np.float32)
        u = torch.as_tensor(u_np, device="cuda")
        y_ref = c.forward(u)                       # existing entry point, torch workspace
        y_fix = torch.full_like(y_ref, float("nan"))
        st = lib.cascade_forward_fixed_scratch(c.plan, C.c_void_p(u.data_ptr()),
                                               C.c_void_p(y_fix.data_ptr()), stream)
        assert st == _abi.CASCADE_OK, lib.cascade_last_error(c.plan)
        torch.cuda.synchronize()
        assert c.device_error() == 0
        a = y_fix.double().cpu().numpy()
        b = y_ref.double().cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: unwritten outputs"
        w.u = u_np.astype(np.float64)
        ey, ecx = rel_errors(w, a, b, OUT_EPS["bf16_split"])
        assert ey <= TOL["bf16_split"] and ecx <= TOL["bf16_split"], (call, ey, ecx)


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
