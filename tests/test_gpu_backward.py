"""GPU parity of the reverse-mode derivative (through the C ABI) against the
CPU FP64 oracle's adjoint, plus central finite differences through the GPU's
own FP64 forward.  Bars, per sequence for du and per system for the
system-matrix gradients, as the relative Frobenius error and element-wise
(max |g - g_o| / max |g_o|): 1e-10 for the FP64 path, 1e-5 for FP32, 2e-3
for the BF16 split."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate_grads

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


def gpu_grads(lib, w, precision, dy, flags=None):
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SAVE_STATES
    c = lib.from_workload(w, precision=precision,
                          flags=CASCADE_FLAG_SAVE_STATES if flags is None else flags)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    y = c.forward(u)
    g = c.backward(u, torch.as_tensor(dy, dtype=dt).cuda().contiguous())
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    return c, y.double().cpu().numpy(), {k: v.double().cpu().numpy() for k, v in g.items()}


def compare(w, c, g, dy, precision):
    ref = oracle.cascade_backward(w, dy, N_per_seq=c.seq_N())
    return gate_grads(w, g, ref, precision)


@pytest.mark.parametrize("discrete", [True, False])
def test_fp64_backward_matches_oracle(lib, discrete):
    w = wl.small_system(m=9, p=2, q=3, lengths=(20, 0, 37, 1, 70), N=6, nsys=2, seed=3,
                        radius=0.97, discrete=discrete, delta=0.2, precision="fp64")
    dy = np.random.default_rng(1).standard_normal((w.rows, w.q))
    c, _, g = gpu_grads(lib, w, "fp64", dy)
    compare(w, c, g, dy, "fp64")


def test_fp64_backward_truncated_and_growing(lib):
    """N below log2 L and spectral radius above one."""
    w = wl.small_system(m=7, p=3, q=2, lengths=(100, 41), N=3, seed=5, radius=1.03)
    dy = np.random.default_rng(2).standard_normal((w.rows, w.q))
    c, _, g = gpu_grads(lib, w, "fp64", dy)
    compare(w, c, g, dy, "fp64")


def test_fp64_backward_finite_differences_on_gpu(lib):
    """Directional derivatives of sum(dy * y) by central differences (h = 1e-6)
    through the GPU's FP64 forward agree with the GPU backward."""
    import torch
    w = wl.small_system(m=6, p=2, q=2, lengths=(30, 17), N=4, seed=7, radius=0.95,
                        discrete=False, delta=0.1, precision="fp64")
    rng = np.random.default_rng(4)
    dy = rng.standard_normal((w.rows, w.q))
    c, _, g = gpu_grads(lib, w, "fp64", dy)
    u = torch.as_tensor(w.u).cuda()

    def loss(**over):
        kw = dict(A=w.A, B=w.B, C=w.C, D=w.D)
        kw.update(over)
        c2 = lib.from_workload(w, precision="fp64")
        c2.set_system_continuous(kw["A"], kw["B"], w.delta, kw["C"], kw["D"])
        uu = torch.as_tensor(over.get("u", w.u)).cuda()
        return float(np.sum(dy * c2.forward(uu).cpu().numpy()))

    h = 1e-6
    for name, X, grad in (("A", w.A, g["dA"]), ("B", w.B, g["dB"]), ("C", w.C, g["dC"]),
                          ("D", w.D, g["dD"]), ("u", w.u, g["du"])):
        E = rng.standard_normal(X.shape)
        fd = (loss(**{name: X + h * E}) - loss(**{name: X - h * E})) / (2 * h)
        an = float(np.sum(grad * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)


@pytest.mark.parametrize("precision,m", [("bf16_split", 128), ("fp32", 128), ("bf16_split", 256),
                                         ("fp32", 64)])
def test_tc_backward_matches_oracle(lib, precision, m):
    """MIMO HiPPO system, ragged lengths, continuous (gradients to A and B)."""
    w = wl.differentiation_form(m=m, p=4, q=4, L=8, batch=4, N=10, delta=1e-2)
    lengths = (700, 129, 1, 300)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(5).standard_normal((int(w.offsets[-1]), 4))
    w = cast_inputs(w, precision)
    dy = np.random.default_rng(6).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, precision, dy)
    compare(w, c, g, dy, precision)


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_tc_backward_discrete_multisystem(lib, precision):
    """Discrete systems (orthogonal plus low rank), two systems, truncated N."""
    w = wl.large_form(m=128, p=3, q=2, L=600, batch=3, N=6)
    w.sys_of_seq = np.array([0, 1, 0], np.int32)
    w.Abar = np.concatenate([w.Abar, 0.98 * w.Abar[:, ::-1, :]])
    for k in ("B", "C", "D"):
        setattr(w, k, np.concatenate([getattr(w, k), 0.5 * getattr(w, k)]))
    w = cast_inputs(w, precision)
    dy = np.random.default_rng(8).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, precision, dy)
    compare(w, c, g, dy, precision)


def test_autograd_function(lib):
    """torch.autograd through CascadeFunction gives the plan's gradients."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SAVE_STATES
    w = wl.small_system(m=64, p=2, q=2, lengths=(300, 77), N=8, seed=9, radius=0.99,
                        discrete=False, delta=0.05, precision="bf16_split")
    w = cast_inputs(w, "bf16_split")
    c = lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_SAVE_STATES)
    dev = torch.device("cuda")
    A = torch.tensor(w.A, device=dev, requires_grad=True)
    B = torch.tensor(w.B, device=dev, requires_grad=True)
    C = torch.tensor(w.C, device=dev, requires_grad=True)
    D = torch.tensor(w.D, device=dev, requires_grad=True)
    u = torch.tensor(w.u, dtype=torch.float32, device=dev, requires_grad=True)
    delta = torch.tensor(w.delta, device=dev)
    y = lib.CascadeFunction.apply(c, u, A, B, C, D, delta)
    dy = torch.randn_like(y)
    (y * dy).sum().backward()
    dy_np = dy.double().cpu().numpy()
    ref = oracle.cascade_backward(w, dy_np, N_per_seq=c.seq_N())
    g = {k: t.grad.double().cpu().numpy()
         for t, k in ((A, "dA"), (B, "dB"), (C, "dC"), (D, "dD"), (u, "du"))}
    gate_grads(w, g, ref, "bf16_split")


def test_backward_requires_saved_states(lib):
    import torch
    from paper_2411_17729_gb300._abi import CascadeError
    w = wl.small_system(m=64, lengths=(100,), N=5, precision="bf16_split")
    c = lib.from_workload(w, precision="bf16_split")
    u = torch.zeros((w.rows, w.p), dtype=torch.float32, device="cuda")
    c.forward(u)
    with pytest.raises(CascadeError):
        c.backward(u, torch.zeros((w.rows, w.q), dtype=torch.float32, device="cuda"))


def test_differentiation_form_full_size(lib):
    """m = 256, p = q = 16, 32 sequences x 8192 steps, N = 12, BF16 split,
    stage outputs recomputed from checkpoints, gradients to u, A (through the
    squaring chain and Eq. 4.2), B, C, D against the oracle's FP64 adjoint over
    the whole batch."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_RECOMPUTE
    w = cast_inputs(wl.differentiation_form(), "bf16_split")
    dy = np.random.default_rng(10).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, "bf16_split", dy, flags=CASCADE_FLAG_RECOMPUTE)
    compare(w, c, g, dy, "bf16_split")


def test_large_form_backward_full_length(lib):
    """The large form at full length: one sequence of 65536 steps, m = 1024,
    p = q = 64, Abar = 0.9999 Q + rank-4 E, N = 15 (every stage, shifts up to
    2^15, dAbar through 15 levels of the squaring chain), BF16 split with
    stage outputs recomputed from checkpoints, as the benchmark's
    forward + backward runs them.  Every gradient against the oracle's FP64
    adjoint, element-wise and in norm."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_RECOMPUTE
    w = wl.large_form(batch=1)
    w = cast_inputs(w, "bf16_split")
    dy = np.random.default_rng(26).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, "bf16_split", dy, flags=CASCADE_FLAG_RECOMPUTE)
    assert np.all(c.seq_N() == 15)
    compare(w, c, g, dy, "bf16_split")


def test_large_form_backward_reduced_length(lib):
    """The large form's shapes (m = 1024, p = q = 64, Abar = 0.9999 Q + rank-4 E,
    N = 15 clipped to the length) on one 3000-step sequence: every gradient
    (u, Abar through the squaring chain, Bbar, C, D) against the oracle's
    FP64 adjoint."""
    w = wl.large_form(L=3000, batch=1)
    w = cast_inputs(w, "bf16_split")
    dy = np.random.default_rng(16).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, "bf16_split", dy)
    compare(w, c, g, dy, "bf16_split")


@pytest.mark.parametrize("p,q", [(1, 1), (8, 2), (16, 16), (3, 20), (64, 64)])
def test_tc_backward_mimo_shapes(lib, p, q):
    """Input and output widths across the projection and reduction kernels:
    one narrow side (register-tiled reductions, one or two shifts per pass)
    and wide ones (tiled reductions), ragged lengths."""
    w = wl.differentiation_form(m=128, p=p, q=q, L=8, batch=3, N=9, delta=1e-2)
    lengths = (300, 129, 1)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(11).standard_normal((int(w.offsets[-1]), p))
    w = cast_inputs(w, "bf16_split")
    dy = np.random.default_rng(12).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, "bf16_split", dy)
    compare(w, c, g, dy, "bf16_split")


@pytest.mark.parametrize("precision,m", [("bf16_split", 128), ("fp32", 64), ("fp64", 24)])
def test_recompute_matches_saved_states(lib, precision, m):
    """Checkpointed stage outputs (CASCADE_FLAG_RECOMPUTE) give the same
    forward output and gradients, bit for bit, as keeping every stage output,
    and both match the oracle.  Lengths give per-sequence N from 0 to 10, so
    segments of several stages, of one stage, and sequences that stop inside a
    segment all occur."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_RECOMPUTE, CASCADE_FLAG_SAVE_STATES
    if precision == "fp64":
        w = wl.small_system(m=m, p=2, q=3, lengths=(700, 129, 1, 300, 2000), N=10, nsys=2,
                            seed=13, radius=0.97, discrete=False, delta=0.05)
    else:
        w = wl.differentiation_form(m=m, p=2, q=3, L=8, batch=5, N=10, delta=1e-2)
        lengths = (700, 129, 1, 300, 2000)
        w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        w.u = np.random.default_rng(14).standard_normal((int(w.offsets[-1]), 2))
        w = cast_inputs(w, precision)
    dy = np.random.default_rng(15).standard_normal((w.rows, w.q))
    if precision != "fp64":
        dy = dy.astype(np.float32).astype(np.float64)
    c1, y1, g1 = gpu_grads(lib, w, precision, dy, flags=CASCADE_FLAG_SAVE_STATES)
    c2, y2, g2 = gpu_grads(lib, w, precision, dy, flags=CASCADE_FLAG_RECOMPUTE)
    c0 = lib.from_workload(w, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    y0 = c0.forward(torch.as_tensor(w.u, dtype=dt).cuda().contiguous()).double().cpu().numpy()
    assert np.array_equal(y0, y1) and np.array_equal(y1, y2)
    assert c2.workspace_size() < c1.workspace_size()
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k
    compare(w, c2, g2, dy, precision)


@pytest.mark.parametrize("m,p,q", [(512, 1, 1), (256, 2, 4), (128, 4, 1)])
def test_first_stage_adjoint_one_pass(lib, m, p, q):
    """du, R1 and R2 from one pass over W^(1) (p, q <= 4): one or two 8-column groups
    per lane, ragged lengths (rows past a sequence end inside a tile, a one-row
    sequence), two systems."""
    w = wl.differentiation_form(m=m, p=p, q=q, L=8, batch=4, N=10, delta=1e-2, seed=17)
    lengths = (1, 129, 700, 300)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(18).standard_normal((int(w.offsets[-1]), p))
    w.sys_of_seq = np.array([0, 1, 0, 1], np.int32)
    w.A = np.concatenate([w.A, w.A])
    w.delta = np.array([1e-2, 2e-2])
    for k in ("B", "C", "D"):
        setattr(w, k, np.concatenate([getattr(w, k), 0.8 * getattr(w, k)]))
    w = cast_inputs(w, "bf16_split")
    dy = np.random.default_rng(19).standard_normal((w.rows, q)).astype(np.float32).astype(np.float64)
    c, _, g = gpu_grads(lib, w, "bf16_split", dy)
    compare(w, c, g, dy, "bf16_split")


@pytest.mark.parametrize("lengths", [(0, 0), (130, 0, 7)])
def test_backward_overwrites_every_output(lib, lengths):
    """The backward writes each requested gradient in full: outputs filled with
    NaN before the call come back as the oracle's gradients (all zero for a
    batch of no rows, which needs no u, dy or workspace)."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SAVE_STATES
    from paper_2411_17729_gb300.cascade import _ptr, _stream
    w = wl.small_system(m=64, p=2, q=3, lengths=lengths, N=8, nsys=2, seed=11, radius=0.98,
                        discrete=False, delta=0.1, precision="bf16_split")
    w = cast_inputs(w, "bf16_split")
    c = lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_SAVE_STATES)
    m, p, q, ns = w.m, w.p, w.q, c.nsys
    shapes = {"dAbar": (ns, m, m), "dBbar": (ns, m, p), "dC": (ns, q, m), "dD": (ns, q, p),
              "dA": (ns, m, m), "dB": (ns, m, p)}
    out = {k: torch.full(s, float("nan"), dtype=torch.float64, device="cuda")
           for k, s in shapes.items()}
    dy = np.random.default_rng(4).standard_normal((w.rows, q))
    if w.rows:
        u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
        c.forward(u)
        dyt = torch.as_tensor(dy, dtype=torch.float32).cuda().contiguous()
        du = torch.full((w.rows, p), float("nan"), dtype=torch.float32, device="cuda")
        ws = c.workspace()
        args = (_ptr(u), _ptr(dyt), _ptr(du), _ptr(ws), ws.numel())
    else:
        du = None
        args = (None, None, None, None, 0)
    c._check(c.lib.cascade_backward(c.plan, args[0], args[1], args[2], _ptr(out["dAbar"]),
                                    _ptr(out["dBbar"]), _ptr(out["dC"]), _ptr(out["dD"]),
                                    _ptr(out["dA"]), _ptr(out["dB"]), args[3], args[4],
                                    _stream()))
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    for k, v in g.items():
        assert np.isfinite(v).all(), k
    if not w.rows:
        for k, v in g.items():
            assert not v.any(), k
        return
    g["du"] = du.double().cpu().numpy()
    compare(w, c, g, dy, "bf16_split")
