"""Error paths of the C ABI on a GPU: status codes for bad arguments and call
order, and the bounded-wait self-test (a wait that nothing completes gives up
with CASCADE_ERR_TIMEOUT and the context stays usable)."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import _abi
    return _abi


def test_bounded_wait_times_out(abi):
    import torch
    lib = abi.lib()
    assert lib.cascade_selftest_timeout(2000) == abi.CASCADE_ERR_TIMEOUT
    x = torch.ones(10, device="cuda")
    assert float((x * 2).sum()) == 20.0          # context still usable


def test_bad_descriptors(abi):
    lib = abi.lib()
    plan = abi.cascade_plan_t()
    for kw, code in [(dict(m=0), abi.CASCADE_ERR_INVALID_ARG),
                     (dict(precision=7), abi.CASCADE_ERR_INVALID_ARG),
                     (dict(m=100, precision=abi.CASCADE_BF16_SPLIT), abi.CASCADE_ERR_UNSUPPORTED),
                     (dict(m=48, precision=abi.CASCADE_FP32), abi.CASCADE_ERR_UNSUPPORTED)]:
        base = dict(m=64, p=1, q=1, nsys=1, N=3, precision=abi.CASCADE_FP64, max_len=100,
                    flags=0, max_rows=100, eps=0.0)
        base.update(kw)
        d = abi.cascade_desc_t(**base)
        assert lib.cascade_plan_create(C.byref(plan), C.byref(d)) == code
        assert not plan.value


def test_call_order_and_batch_validation(abi):
    from paper_2411_17729_gb300 import cascade
    c = cascade.Cascade(8, 1, 1, N=3, precision="fp64", max_len=50, max_rows=100)
    offs = np.array([0, 10], np.int64)
    st = c.lib.cascade_set_batch(c.plan, offs.ctypes.data_as(C.POINTER(C.c_int64)), 1, None)
    assert st == abi.CASCADE_ERR_STATE
    w = wl.small_system(m=8, p=1, q=1, lengths=(10,), N=3)
    c.set_system_discrete(w.Abar, w.B, w.C, w.D)
    for bad in ([0, 60], [1, 5], [0, 5, 3], [0, 40, 120]):
        o = np.array(bad, np.int64)
        st = c.lib.cascade_set_batch(c.plan, o.ctypes.data_as(C.POINTER(C.c_int64)), len(o) - 1, None)
        assert st == abi.CASCADE_ERR_INVALID_ARG, bad
    c.set_batch([0, 10])
    ws = c.workspace()
    st = c.lib.cascade_forward(c.plan, None, None, C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert st == abi.CASCADE_ERR_INVALID_ARG


def test_misaligned_rows_rejected(abi):
    """u, y, dy and du move through some paths in 16-byte words: a pointer off
    that alignment is refused with CASCADE_ERR_INVALID_ARG before anything is
    launched, and the plan stays usable (an aligned forward then matches)."""
    import torch
    from paper_2411_17729_gb300 import cascade
    from paper_2411_17729_gb300.cascade import _stream
    w = wl.small_system(m=128, p=16, q=16, lengths=(300, 77), N=8, seed=2, radius=0.97,
                        precision="bf16_split")
    c = cascade.from_workload(w, precision="bf16_split", flags=abi.CASCADE_FLAG_SAVE_STATES)
    rows, p, q = w.rows, w.p, w.q
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    y_ref = c.forward(u).clone()
    ub = torch.zeros(rows * p + 4, dtype=torch.float32, device="cuda")
    yb = torch.zeros(rows * q + 4, dtype=torch.float32, device="cuda")
    ub[1:1 + rows * p].copy_(u.reshape(-1))
    odd_u, odd_y = C.c_void_p(ub.data_ptr() + 4), C.c_void_p(yb.data_ptr() + 4)
    ok_u, ok_y = C.c_void_p(u.data_ptr()), C.c_void_p(yb.data_ptr())
    ws = c.workspace()
    wsp, n = C.c_void_p(ws.data_ptr()), ws.numel()
    lib = c.lib
    E = abi.CASCADE_ERR_INVALID_ARG
    assert lib.cascade_forward(c.plan, odd_u, ok_y, wsp, n, _stream()) == E
    assert lib.cascade_forward(c.plan, ok_u, odd_y, wsp, n, _stream()) == E
    assert lib.cascade_forward_fixed_scratch(c.plan, odd_u, ok_y, _stream()) == E
    h_u, h_y = u.cpu(), torch.empty((rows, q))
    assert lib.cascade_forward_host(c.plan, C.c_void_p(h_u.data_ptr()), C.c_void_p(h_y.data_ptr()),
                                    odd_u, ok_y, wsp, n, _stream()) == E
    dy = torch.ones((rows, q), device="cuda")
    du = torch.empty(rows * p + 4, device="cuda")
    assert lib.cascade_backward(c.plan, ok_u, C.c_void_p(dy.data_ptr()), C.c_void_p(du.data_ptr() + 4),
                                None, None, None, None, None, None, wsp, n, _stream()) == E
    torch.cuda.synchronize()
    assert c.device_error() == 0
    y = c.forward(u)
    torch.cuda.synchronize()
    assert torch.equal(y, y_ref)
