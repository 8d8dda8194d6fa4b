"""Seeded random sweep of small configurations through the C ABI against the
CPU FP64 oracle: precision, m, p, q, the number of systems and which
sequence uses which, sequence lengths (empty, one step, ragged, across tile
boundaries), N (truncated or complete), discrete or continuous systems, the
§3 or the work-efficient schedule, and, for plans that keep their stage
outputs, the backward.  Each configuration is gated element-wise and in norm
at its path's bar; a failure names the configuration's seed."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate, gate_grads

pytestmark = pytest.mark.gpu

LENGTH_POOL = (0, 1, 2, 3, 17, 127, 128, 129, 255, 300, 1000, 1537, 2500)


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import cascade
    return cascade


def draw(seed):
    """One configuration: (workload, precision, schedule, keep states)."""
    rng = np.random.default_rng(1000 + seed)
    precision = ("bf16_split", "fp32", "fp64")[seed % 3]
    if precision == "bf16_split":
        m = int(rng.choice([64, 128, 192, 256, 320]))
    elif precision == "fp32":
        m = int(rng.choice([32, 64, 96, 128, 160]))
    else:
        m = int(rng.choice([3, 8, 24, 40]))
    p = int(rng.choice([1, 2, 3, 4, 16]))
    q = int(rng.choice([1, 2, 4, 5, 16]))
    nsys = int(rng.integers(1, 4))
    nseq = int(rng.integers(1, 6))
    lengths = [int(x) for x in rng.choice(LENGTH_POOL, size=nseq)]
    if sum(lengths) == 0:
        lengths[0] = 129
    scan = precision != "fp64" and seed % 4 == 1
    keep = not scan and seed % 4 == 2
    # the work-efficient schedule needs a complete cascade (2^(N+1) >= L)
    N = 12 if scan else int(rng.integers(0, 13))
    w = wl.small_system(m=m, p=p, q=q, lengths=lengths, N=N, seed=seed, nsys=nsys,
                        radius=float(rng.choice([0.9, 0.99, 1.0005])),
                        discrete=bool(seed % 2), delta=0.05, precision=precision)
    w.sys_of_seq = rng.integers(0, nsys, size=nseq).astype(np.int32)
    return cast_inputs(w, precision), precision, scan, keep


@pytest.mark.parametrize("seed", range(64))
def test_random_configuration(lib, seed):
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SAVE_STATES, CASCADE_FLAG_SCAN
    w, precision, scan, keep = draw(seed)
    flags = (CASCADE_FLAG_SCAN if scan else 0) | (CASCADE_FLAG_SAVE_STATES if keep else 0)
    c = lib.from_workload(w, precision=precision, flags=flags)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    y = c.forward(u)
    dy = np.random.default_rng(seed).standard_normal((w.rows, w.q))
    g = c.backward(u, torch.as_tensor(dy, dtype=dt).cuda().contiguous()) if keep else None
    torch.cuda.synchronize()
    assert c.device_error() == 0, (seed, c.lib.cascade_last_error(c.plan))
    Ns = c.seq_N()
    cfg = f"{precision} m={w.m} p={w.p} q={w.q} L={[int(x) for x in w.lengths]} N={Ns}"
    try:
        gate(w, y.double().cpu().numpy(), oracle.cascade_forward(w, N_per_seq=Ns), precision,
             what=f"y m{w.m}")
    except AssertionError as e:
        raise AssertionError(f"seed {seed}: {cfg}: {e}") from None
    if keep:
        ref = oracle.cascade_backward(w, dy, N_per_seq=Ns)
        gate_grads(w, {k: v.double().cpu().numpy() for k, v in g.items()}, ref, precision)
    c.close()


FLAG_POOL = (0, 1, 9, 17, 100, 129, 255, 777, 1500, 2600)


def draw_flags(seed):
    """One configuration over the plan flags: the schedule and what the
    backward keeps, graph replay, the diagnostic switches that route around a
    fused kernel, the wide fused output, the zero-order hold, the dense
    set-up of a lower-triangular A; and the entry point (device forward, the
    host-buffer forward, or two forwards on the same buffers)."""
    from paper_2411_17729_gb300 import _abi as A
    rng = np.random.default_rng(5000 + seed)
    precision = ("bf16_split", "bf16_split", "fp32", "fp64")[seed % 4]
    m = int(rng.choice({"bf16_split": [64, 128, 256, 320, 512], "fp32": [32, 64, 128],
                        "fp64": [5, 16, 33]}[precision]))
    p = int(rng.choice([1, 1, 3, 16]))
    q = int(rng.choice([1, 4, 16, 32]))
    mode = str(rng.choice(["none", "save", "recompute", "scan"]))
    if precision == "fp64" and mode == "scan":
        mode = "none"
    flags = {"none": 0, "save": A.CASCADE_FLAG_SAVE_STATES, "recompute": A.CASCADE_FLAG_RECOMPUTE,
             "scan": A.CASCADE_FLAG_SCAN}[mode]
    for f in (A.CASCADE_FLAG_GRAPH, A.CASCADE_FLAG_NO_FUSED_OUTPUT, A.CASCADE_FLAG_NO_FUSED_FIRST,
              A.CASCADE_FLAG_NO_FUSED_STAGES, A.CASCADE_FLAG_FUSE_WIDE_OUTPUT):
        if rng.random() < 0.3:
            flags |= f
    discrete = bool(rng.integers(2))
    lengths = [int(x) for x in rng.choice(FLAG_POOL, size=int(rng.integers(1, 5)))]
    if sum(lengths) == 0:
        lengths[0] = 255
    N = 12 if mode == "scan" else int(rng.integers(3, 13))
    w = wl.small_system(m=m, p=p, q=q, lengths=lengths, N=N, seed=seed, nsys=int(rng.integers(1, 3)),
                        radius=float(rng.choice([0.95, 0.999])), discrete=discrete, delta=0.05,
                        precision=precision)
    if not discrete:
        if rng.random() < 0.5:
            w.A = np.tril(w.A)
            if rng.random() < 0.5:
                flags |= A.CASCADE_FLAG_DENSE_SETUP
        if rng.random() < 0.3:
            w.discretisation = "zoh"
    entry = str(rng.choice(["forward", "host", "twice"]))
    return cast_inputs(w, precision), precision, mode, flags, entry


@pytest.mark.parametrize("seed", range(48))
def test_random_flags(lib, seed):
    import torch
    w, precision, mode, flags, entry = draw_flags(seed)
    c = lib.from_workload(w, precision=precision, flags=flags)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    y = c.forward(u)
    if entry == "twice":                       # a graph plan replays its recorded launches
        y1 = y.clone()
        c.forward(u, y)
        torch.cuda.synchronize()
        assert torch.equal(y, y1), seed
    elif entry == "host":
        h_u = u.cpu().pin_memory()
        h_y = torch.full((w.rows, w.q), float("nan"), dtype=dt).pin_memory()
        c.forward_host(h_u, h_y)
        torch.cuda.synchronize()
        assert torch.equal(h_y, y.cpu()), seed
    dy = np.random.default_rng(seed).standard_normal((w.rows, w.q))
    keep = mode in ("save", "recompute")
    if keep:
        if entry == "host":                   # the backward refers to the last forward
            c.forward(u, y)
        g = c.backward(u, torch.as_tensor(dy, dtype=dt).cuda().contiguous())
    torch.cuda.synchronize()
    assert c.device_error() == 0, (seed, c.lib.cascade_last_error(c.plan))
    Ns = c.seq_N()
    cfg = (f"{precision} m={w.m} p={w.p} q={w.q} L={[int(x) for x in w.lengths]} N={Ns} "
           f"mode={mode} flags={flags} entry={entry} "
           f"{getattr(w, 'discretisation', 'trapezoid') if w.Abar is None else 'discrete'}")
    try:
        gate(w, y.double().cpu().numpy(), oracle.cascade_forward(w, N_per_seq=Ns), precision,
             what=f"y m{w.m}")
        if keep:
            ref = oracle.cascade_backward(w, dy, N_per_seq=Ns)
            gate_grads(w, {k: v.double().cpu().numpy() for k, v in g.items()}, ref, precision)
    except AssertionError as e:
        raise AssertionError(f"seed {seed}: {cfg}: {e}") from None
    c.close()
