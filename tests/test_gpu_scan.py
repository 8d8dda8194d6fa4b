"""GPU parity of the work-efficient schedule (CASCADE_FLAG_SCAN: up-sweep and
down-sweep over the powers Abar^(2^k), about 2L products per sequence, as the
abstract and §6 count them) against the CPU FP64 oracle's cascade, which it
equals up to rounding when 2^(N+1) >= L.  Same bars as the stage schedule:
2e-3 (BF16 split) and 1e-5 (FP32) on y and on Cx = y - Du."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import TOL, SeqGate, cast_inputs, gate, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import cascade
    return cascade


def scan_products(L):
    """Products by powers the schedule makes for one sequence of length L:
    odd rows of the first level, then up-sweep levels 1..K-1 and down-sweep
    levels K-2..0 (K = ceil(log2 L))."""
    K = int(np.ceil(np.log2(L))) if L > 1 else 0
    n = L // 2
    n += sum(L // 2 ** (k + 1) for k in range(1, K))
    n += sum((L - 2 ** k) // 2 ** (k + 1) for k in range(K - 1) if L > 2 ** k)
    return n


def run(lib, w, precision, flags):
    import torch
    c = lib.from_workload(w, precision=precision, flags=flags)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    y = c.forward(u)
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    return c, y.double().cpu().numpy()


def matvecs(c):
    import ctypes
    n = ctypes.c_int64()
    c._check(c.lib.cascade_get_matvec_count(c.plan, ctypes.byref(n)))
    return n.value


LENGTHS = (1, 2, 3, 4, 5, 64, 127, 128, 129, 255, 256, 257, 1000, 2048, 3001)


@pytest.mark.parametrize("precision,m,q", [("bf16_split", 128, 2), ("bf16_split", 256, 2),
                                           ("fp32", 128, 2), ("fp32", 64, 2),
                                           ("bf16_split", 128, 6), ("bf16_split", 64, 1),
                                           ("bf16_split", 192, 4)])
def test_scan_matches_oracle(lib, precision, m, q):
    """Ragged lengths around every power of two the tiles and levels meet
    (1 .. 3001), two systems, MIMO.  With q <= 4 the down-sweep levels form y
    in their epilogue (rows 2^t - 1 separately); q = 6 takes the separate
    output pass."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SCAN
    w = wl.differentiation_form(m=m, p=3, q=q, L=8, batch=len(LENGTHS), N=11, delta=1e-2)
    w.offsets = np.concatenate([[0], np.cumsum(LENGTHS)]).astype(np.int64)
    w.u = np.random.default_rng(21).standard_normal((int(w.offsets[-1]), 3))
    w.sys_of_seq = (np.arange(len(LENGTHS)) % 2).astype(np.int32)
    w.A = np.concatenate([w.A, w.A])
    w.delta = np.array([1e-2, 3e-2])
    for k in ("B", "C", "D"):
        setattr(w, k, np.concatenate([getattr(w, k), 0.7 * getattr(w, k)]))
    w = cast_inputs(w, precision)
    c, y = run(lib, w, precision, CASCADE_FLAG_SCAN)
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y, yo, precision)
    # operation count: about 2L, never above it (abstract, §6)
    want = sum(scan_products(L) for L in LENGTHS)
    assert matvecs(c) == want
    assert want <= sum(oracle.matvec_counts(11, L)["paper_bound"] for L in LENGTHS)


@pytest.mark.parametrize("precision,m,q", [("bf16_split", 256, 1), ("bf16_split", 128, 3),
                                           ("fp32", 128, 1), ("fp32", 64, 4)])
def test_scan_even_rows_on_chip(lib, precision, m, q):
    """p = 1 with the output fused: the first level stores only the odd rows
    and row 0, and the last down-sweep level forms the even rows' v^(1) =
    Bbar u from u.  Same results, bit for bit, as the path that stores every
    row (CASCADE_FLAG_NO_FUSED_FIRST), and oracle parity."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_FIRST, CASCADE_FLAG_SCAN
    if q == 1:
        w = wl.precision_form(m=m, L=8, batch=len(LENGTHS), N=11)
    else:
        w = wl.differentiation_form(m=m, p=1, q=q, L=8, batch=len(LENGTHS), N=11, delta=1e-2)
    w.offsets = np.concatenate([[0], np.cumsum(LENGTHS)]).astype(np.int64)
    w.u = np.random.default_rng(23).standard_normal((int(w.offsets[-1]), 1))
    w = cast_inputs(w, precision)
    c1, y1 = run(lib, w, precision, CASCADE_FLAG_SCAN)
    c2, y2 = run(lib, w, precision, CASCADE_FLAG_SCAN | CASCADE_FLAG_NO_FUSED_FIRST)
    assert c1.first_fused() and not c2.first_fused()
    assert np.array_equal(y1, y2)
    yo = oracle.cascade_forward(w, N_per_seq=c1.seq_N())
    gate(w, y1, yo, precision)


def test_scan_autotuned_levels(lib):
    """The autotuner's per-level shapes on the work-efficient schedule (keys k
    for up-sweep levels, 100 + k for down-sweep levels) keep oracle parity,
    and setting the saved shapes again gives the same output bit for bit."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SCAN
    w = cast_inputs(wl.precision_form(m=128, L=8, batch=len(LENGTHS), N=11), "bf16_split")
    w.offsets = np.concatenate([[0], np.cumsum(LENGTHS)]).astype(np.int64)
    w.u = np.random.default_rng(24).standard_normal((int(w.offsets[-1]), 1))
    c = lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_SCAN)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    shape = c.autotune(u, reps=1)
    per = c.stage_shapes()
    K = int(np.ceil(np.log2(max(LENGTHS))))
    assert per and set(per) <= set(range(1, K)) | set(range(100, 100 + K))
    y1 = c.forward(u).double().cpu().numpy()
    assert c.device_error() == 0
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y1, yo, "bf16_split")
    c.set_kernel_shape(*shape)
    c.set_stage_shapes(per)
    assert c.stage_shapes() == per
    assert np.array_equal(y1, c.forward(u).double().cpu().numpy())


def test_stage_schedule_count(lib):
    """The stage schedule's count is the oracle's sum_k (L - 2^k)^+ per sequence."""
    w = wl.precision_form(m=64, L=8, batch=len(LENGTHS), N=12)
    w.offsets = np.concatenate([[0], np.cumsum(LENGTHS)]).astype(np.int64)
    w.u = np.random.default_rng(22).standard_normal((int(w.offsets[-1]), 1))
    w = cast_inputs(w, "bf16_split")
    c, _ = run(lib, w, "bf16_split", 0)
    Ns = c.seq_N()
    assert matvecs(c) == sum(oracle.matvec_counts(int(N), L)["executed"]
                             for N, L in zip(Ns, LENGTHS))


def test_scan_equals_stage_schedule(lib):
    """Both schedules on the same batch agree to the rounding of the format."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SCAN
    w = cast_inputs(wl.precision_form(m=256, L=4096, batch=6, N=11), "bf16_split")
    _, y1 = run(lib, w, "bf16_split", 0)
    _, y2 = run(lib, w, "bf16_split", CASCADE_FLAG_SCAN)
    yo = oracle.cascade_forward(w)
    gate(w, y1, yo, "bf16_split", what="stages")
    gate(w, y2, yo, "bf16_split", what="scan")
    e12 = rel_errors(w, y2, y1)
    assert max(e12[0], e12[2]) <= TOL["bf16_split"], e12


def test_scan_precision_form_full_size(lib):
    """64 sequences x 16384 steps, m = 256, N = 13 (the benchmark's
    configuration) on the work-efficient schedule: every sequence in full
    against the oracle, element-wise and in norm."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SCAN
    w = cast_inputs(wl.precision_form(), "bf16_split")
    c, y = run(lib, w, "bf16_split", CASCADE_FLAG_SCAN)
    assert matvecs(c) == 64 * scan_products(16384)
    g = SeqGate("bf16_split")
    for i in range(w.nseq):
        sl = w.seq(i)
        Abar, Bbar, C, D = oracle.system_matrices(w, int(w.sys_of_seq[i]))
        uu = w.u[sl]
        yo = oracle.cascade_forward_seq(Abar, Bbar, C, D, uu, 13)
        g.add(y[sl], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
    g.check()


def test_scan_refuses_truncation_and_backward(lib):
    """2^(N+1) < L has no work-efficient form here (UNSUPPORTED), and the
    schedule keeps no stage outputs for a backward (INVALID_ARG)."""
    from paper_2411_17729_gb300._abi import (CASCADE_FLAG_SAVE_STATES, CASCADE_FLAG_SCAN,
                                             CascadeError)
    w = cast_inputs(wl.precision_form(m=64, L=1000, batch=2, N=4), "bf16_split")
    with pytest.raises(CascadeError):
        lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_SCAN)
    w2 = cast_inputs(wl.precision_form(m=64, L=100, batch=2, N=9), "bf16_split")
    with pytest.raises(CascadeError):
        lib.from_workload(w2, precision="bf16_split",
                          flags=CASCADE_FLAG_SCAN | CASCADE_FLAG_SAVE_STATES)


def test_scan_graph_replay_bitwise(lib):
    """The work-efficient schedule replayed as a CUDA graph (the timed path of the
    benchmark) gives the direct launches' output bit for bit, over three replays."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_GRAPH, CASCADE_FLAG_SCAN
    w = cast_inputs(wl.precision_form(m=256, L=4096, batch=5, N=11), "bf16_split")
    _, y1 = run(lib, w, "bf16_split", CASCADE_FLAG_SCAN)
    c = lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_SCAN | CASCADE_FLAG_GRAPH)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda()
    y = torch.empty((w.rows, w.q), dtype=torch.float32, device="cuda")
    for _ in range(3):
        y.zero_()
        c.forward(u, y)
        torch.cuda.synchronize()
        assert c.device_error() == 0
        assert np.array_equal(y.double().cpu().numpy(), y1)
