"""GPU parity of the forward cascade (through the C ABI) against the CPU FP64
oracle, on the same seeded inputs.

Bars, per sequence and maxed over sequences, on y and on Cx = y - Du, both as
the relative Frobenius error and element-wise (max |y - y_o| / max |y_o|):
1e-12 for the FP64 path, 1e-5 for FP32 (three TF32 products), 2e-3 for the
BF16 split.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import TOL, SeqGate, cast_inputs, gate, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import cascade
    return cascade


def run_gpu(cascade, w, precision, flags=0, N=None):
    import torch
    c = cascade.from_workload(w, precision=precision, flags=flags, N=N)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    y = c.forward(u)
    torch.cuda.synchronize()
    err = c.device_error()
    assert err == 0, f"device error word {err}: {c.lib.cascade_last_error(c.plan)}"
    return c, y.double().cpu().numpy()


def check(cascade, w, precision, flags=0):
    w = cast_inputs(w, precision)
    c, y = run_gpu(cascade, w, precision, flags)
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y, yo, precision)
    return c, y, yo


# ------------------------------------------------------------ FP64 path
@pytest.mark.parametrize("m,p,q", [(1, 1, 1), (5, 2, 3), (64, 1, 1), (70, 3, 2)])
def test_fp64_small_ragged(lib, m, p, q):
    w = wl.small_system(m=m, p=p, q=q, lengths=(1, 2, 3, 0, 64, 65, 200, 1000), N=12, nsys=2,
                        seed=m, radius=0.98, precision="fp64")
    check(lib, w, "fp64")


def test_fp64_plain_hippo_workload(lib):
    """HiPPO-LegS m = 64, L = 4096, N = 11: equals the recursion (1.2)."""
    w = wl.plain_fp64()
    c, y, yo = check(lib, w, "fp64")
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    yr, _ = oracle.recursion_forward_seq(Abar, Bbar, C, D, w.u)
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-12


@pytest.mark.parametrize("N", [0, 1, 3])
def test_fp64_truncated(lib, N):
    """N + 1 < log2 L: the truncated polynomial, not the recursion."""
    w = wl.small_system(m=9, p=2, q=2, lengths=(100, 37), N=N, seed=4, radius=1.03)
    check(lib, w, "fp64")


def test_fp64_recursion_kernel(lib):
    import torch
    w = wl.small_system(m=33, p=2, q=3, lengths=(50, 0, 7), N=10, seed=5, radius=0.9)
    c = lib.from_workload(w, precision="fp64")
    y = c.recursion(torch.as_tensor(w.u).cuda()).cpu().numpy()
    for i in range(w.nseq):
        sl = w.seq(i)
        if sl.stop == sl.start:
            continue
        Abar, Bbar, C, D = oracle.system_matrices(w, int(w.sys_of_seq[i]))
        yr, _ = oracle.recursion_forward_seq(Abar, Bbar, C, D, w.u[sl])
        assert np.max(np.abs(y[sl] - yr)) <= 1e-12 * max(1, np.max(np.abs(yr)))


# ------------------------------------------------------------ system prep
def test_discretisation_and_powers(lib):
    """Eq. (4.2) and the squaring chain on the device vs the oracle (dense
    continuous A, pivoting exercised)."""
    w = wl.small_system(m=48, p=3, q=2, lengths=(10,), N=6, seed=2, discrete=False, delta=0.3,
                        nsys=3)
    c = lib.from_workload(w, precision="fp64", N=6, max_len=200)
    for s in range(3):
        Abar, Bbar, C, D = oracle.system_matrices(w, s)
        P = oracle.squaring_chain(Abar, 6)
        G = c.powers(s, 6).cpu().numpy()
        for k in range(7):
            assert np.max(np.abs(G[k] - P[k])) <= 1e-12 * max(1.0, np.max(np.abs(P[k])))


def test_hippo_paper_example_powers(lib):
    """§4 example (1-based HiPPO, m = 100, delta = 5e-4): device powers match
    the oracle's to 1e-12 and the (0,0) entry of Abar^(2^15) is d_1^(2^15)."""
    import math
    m = 100
    A = wl.hippo_legs(m, base=1)[None]
    B = wl.hippo_legs_B(m, base=1)[None]
    w = wl.Workload(name="paper", m=m, p=1, q=1, N=15, precision="fp64",
                    offsets=np.array([0, 4], np.int64), u=np.ones((4, 1)), B=B,
                    C=np.ones((1, 1, m)), D=np.zeros((1, 1, 1)), sys_of_seq=np.zeros(1, np.int32),
                    A=A, delta=np.array([5e-4]))
    c = lib.from_workload(w, precision="fp64", N=15, max_len=1 << 16)
    G = c.powers(0, 15).cpu().numpy()
    Abar, _, _, _ = oracle.system_matrices(w, 0)
    P = oracle.squaring_chain(Abar, 15)
    for k in range(16):
        assert np.max(np.abs(G[k] - P[k])) <= 1e-12 * np.max(np.abs(P[k]))
    assert abs(G[15][0, 0] - math.exp(-(2 ** 16) * math.atanh(5e-4))) < 1e-11 * G[15][0, 0]


def test_accuracy_rule_matches_oracle(lib):
    w = wl.batching_form(nseq=6, Lmin=100, Lmax=3000, m=64)
    c = lib.from_workload(w, precision="fp32")
    Abar, _, _, _ = oracle.system_matrices(w, 0)
    assert int(c.N()[0]) == oracle.choose_N(Abar, int(w.lengths.max()), w.eps)
    for i, L in enumerate(w.lengths):
        assert c.seq_N()[i] == oracle.effective_N(int(c.N()[0]), int(L))
    # a contracting system reaches eps before covering the length
    w2 = wl.small_system(m=32, lengths=(5000,), seed=1, radius=0.5, precision="fp32")
    w2.N, w2.eps = -1, 1e-6
    c2 = lib.from_workload(w2, precision="fp32")
    Abar2, _, _, _ = oracle.system_matrices(w2, 0)
    assert int(c2.N()[0]) == oracle.choose_N(Abar2, 5000, 1e-6) < 11


# ------------------------------------------------------------ tensor-core paths
@pytest.mark.parametrize("precision,m", [("bf16_split", 64), ("bf16_split", 128),
                                         ("bf16_split", 256), ("fp32", 32), ("fp32", 128),
                                         ("fp32", 256)])
def test_tc_hippo_ragged(lib, precision, m):
    """HiPPO-LegS with per-sequence step sizes, ragged lengths spanning
    several 128-row tiles, empty and one-step sequences."""
    lengths = (1, 2, 127, 128, 129, 0, 1000, 3000)
    w = wl.precision_form(m=m, L=8, batch=len(lengths), N=12)
    rng = np.random.default_rng(7)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = rng.standard_normal((int(w.offsets[-1]), 1))
    w.precision = precision
    check(lib, w, precision)


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
@pytest.mark.parametrize("p,q", [(1, 1), (4, 4), (3, 16), (2, 20)])
def test_tc_mimo(lib, precision, p, q):
    """MIMO systems: fused output for q <= 16, separate output kernel above."""
    w = wl.differentiation_form(m=128, p=p, q=q, L=700, batch=3, N=9, delta=1e-2)
    check(lib, w, precision)


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_tc_large_m_multiblock(lib, precision):
    """m = 512: two N-blocks per tile, output kernel path."""
    w = wl.large_form(m=512, p=2, q=3, L=600, batch=2, N=9)
    check(lib, w, precision)


@pytest.mark.parametrize("precision,m", [("bf16_split", 2048), ("fp32", 1024)])
def test_tc_wide_state(lib, precision, m):
    """Wide states: m = 2048 with BF16 pairs (eight N-blocks of 256 per tile),
    m = 1024 with TF32 pairs (eight of 128), ragged sequences, p = 16, q = 20.
    (The TF32 pair's tensor-core sums truncate once per 8-term K step, so its
    error grows with m: at m = 2048 it measured 1.5e-5, above the 1e-5 bar.)"""
    w = wl.large_form(m=m, p=16, q=20, L=8, batch=2, N=8)
    w.offsets = np.array([0, 300, 300 + 173], dtype=np.int64)
    w.u = np.random.default_rng(31).standard_normal((473, 16))
    check(lib, w, precision)


@pytest.mark.parametrize("precision,wide", [("bf16_split", False), ("fp64", False),
                                            ("bf16_split", True)])
def test_forward_host_matches_device_forward(lib, precision, wide):
    """cascade_forward_host (host u in, host y out, synchronous) gives the
    device forward's y bit for bit, repeatedly, from page-locked and ordinary
    host memory.  wide: p = q = 16 at m = 512, where u's copies overlap the
    first-stage projection and y's the output projection, chunk by chunk."""
    import torch
    if wide:
        w = wl.large_form(m=512, p=16, q=16, L=8, batch=3, N=9)
        w.offsets = np.array([0, 700, 700 + 1, 700 + 1 + 1300], dtype=np.int64)
        w.u = np.random.default_rng(41).standard_normal((2001, 16))
        w = cast_inputs(w, precision)
    else:
        w = cast_inputs(wl.precision_form(m=128 if precision != "fp64" else 24, L=700, batch=3,
                                          N=9), precision)
    c = lib.from_workload(w, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    y_dev = c.forward(u).cpu()
    for pin in (True, False):
        h_u = torch.as_tensor(w.u, dtype=dt).contiguous()
        h_y = torch.full((w.rows, w.q), float("nan"), dtype=dt)
        if pin:
            h_u, h_y = h_u.pin_memory(), h_y.pin_memory()
        for _ in range(2):
            c.forward_host(h_u, h_y)
            assert torch.equal(h_y, y_dev)
    assert c.device_error() == 0


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_tc_unfused_matches_fused(lib, precision):
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_OUTPUT
    w = wl.precision_form(m=128, L=900, batch=3, N=9)
    w = cast_inputs(w, precision)
    _, y1 = run_gpu(lib, w, precision)
    _, y2 = run_gpu(lib, w, precision, flags=CASCADE_FLAG_NO_FUSED_OUTPUT)
    fy, _, ey, _ = rel_errors(w, y1, y2)
    assert fy < 1e-5 and ey < 1e-5, (fy, ey)


@pytest.mark.parametrize("precision,m,p,q", [("bf16_split", 256, 1, 1), ("bf16_split", 128, 1, 4),
                                             ("fp32", 128, 1, 4), ("bf16_split", 512, 1, 3),
                                             ("fp32", 64, 1, 1), ("bf16_split", 192, 1, 2)])
def test_first_stage_on_chip(lib, precision, m, p, q):
    """Stage 1 forming v^(1) = Bbar u_l + Abar Bbar u_(l-1) on chip gives the
    results of the path that writes v^(1) to memory bit for bit, and matches
    the oracle.  Ragged lengths with sequences too short for a stage 1 (their
    v^(1) is still written), one system per sequence."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_FIRST
    lengths = (3, 1, 127, 128, 129, 2, 700, 1000)
    if q == 1:
        w = wl.precision_form(m=m, L=8, batch=len(lengths), N=10)
    else:
        w = wl.differentiation_form(m=m, p=p, q=q, L=8, batch=len(lengths), N=10, delta=1e-2)
    rng = np.random.default_rng(11)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = rng.standard_normal((int(w.offsets[-1]), p))
    w.precision = precision
    c, y1, yo = check(lib, w, precision)
    assert c.first_fused()
    w2 = cast_inputs(w, precision)
    c2, y2 = run_gpu(lib, w2, precision, flags=CASCADE_FLAG_NO_FUSED_FIRST)
    assert not c2.first_fused()
    assert np.array_equal(y1, y2)
    # without sequences shorter than 3 steps no first-stage launch remains
    w3 = cast_inputs(w, precision)
    keep = [i for i, L in enumerate(lengths) if L >= 3]
    w3 = w3.subset(keep)
    launches = []
    for flags in (0, CASCADE_FLAG_NO_FUSED_FIRST):
        c3 = lib.from_workload(w3, precision=precision, flags=flags)
        u3 = torch.as_tensor(w3.u, dtype=torch.float32).cuda().contiguous()
        c3.forward(u3)
        torch.cuda.synchronize()
        n0 = c3.lib.cascade_launch_count()
        c3.forward(u3)
        torch.cuda.synchronize()
        launches.append(c3.lib.cascade_launch_count() - n0)
        assert c3.device_error() == 0
    assert launches[0] == launches[1] - 1, launches


def test_output_fused_query(lib):
    """cascade_get_output_fused: y formed in the last stage's epilogue for
    q <= 4 when a stage tile spans all columns (not FP64, not opted out)."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_OUTPUT
    cases = [(128, 1, 1, "bf16_split", 0, True), (128, 4, 4, "fp32", 0, True),
             (128, 3, 16, "bf16_split", 0, False), (512, 2, 3, "bf16_split", 0, False),
             (64, 1, 1, "fp64", 0, False),
             (128, 1, 1, "bf16_split", CASCADE_FLAG_NO_FUSED_OUTPUT, False)]
    for m, p, q, precision, flags, want in cases:
        c = lib.Cascade(m, p, q, N=8, precision=precision, flags=flags, max_len=1024)
        assert c.output_fused() == want, (m, p, q, precision, flags)
        c.close()


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_tc_truncation_and_growth(lib, precision):
    """Spectral radius above one with N below log2 L (truncated polynomial)."""
    w = wl.small_system(m=64, p=2, q=2, lengths=(1000, 513), N=4, seed=3, radius=1.002,
                        precision=precision)
    check(lib, w, precision)


def test_graph_replay_matches(lib):
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_GRAPH
    w = cast_inputs(wl.precision_form(m=128, L=1000, batch=3, N=9), "bf16_split")
    _, y1 = run_gpu(lib, w, "bf16_split")
    c = lib.from_workload(w, precision="bf16_split", flags=CASCADE_FLAG_GRAPH)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda()
    y = torch.empty((w.rows, 1), dtype=torch.float32, device="cuda")
    for _ in range(3):
        y.zero_()
        c.forward(u, y)
        torch.cuda.synchronize()
        assert np.array_equal(y.double().cpu().numpy(), y1)


# ------------------------------------------------------------ full-size
def test_precision_form_full_size(lib):
    """64 sequences x 16384 steps, m = 256, N = 13, BF16 split (the launch
    configuration the benchmark times): every sequence in full against the
    oracle, element-wise and in norm."""
    w = cast_inputs(wl.precision_form(), "bf16_split")
    c, y = run_gpu(lib, w, "bf16_split")
    Ns = c.seq_N()
    assert np.all(Ns == 13)
    g = SeqGate("bf16_split")
    for i in range(w.nseq):
        sl = w.seq(i)
        Abar, Bbar, C, D = oracle.system_matrices(w, int(w.sys_of_seq[i]))
        uu = w.u[sl]
        yo = oracle.cascade_forward_seq(Abar, Bbar, C, D, uu, 13)
        g.add(y[sl], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
    g.check()


def test_large_form_full_size(lib):
    """m = 1024, p = q = 64, 8 sequences x 65536 steps, N = 15, Abar = 0.9999 Q
    + rank-4 E, BF16 split (four N-blocks per tile), in the launch
    configuration the benchmark times.  The last sequence, whose rows sit at
    the highest offsets of the 2 GiB state planes, is checked in full
    (every stage, shifts up to 2^15); 192-step prefixes of the other seven
    (the cascade is causal, so a prefix run with the same N gives the same
    rows)."""
    w = cast_inputs(wl.large_form(), "bf16_split")
    c, y = run_gpu(lib, w, "bf16_split")
    assert np.all(c.seq_N() == 15)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    powers = oracle.squaring_chain(Abar, 15)
    g = SeqGate("bf16_split")
    for i in range(w.nseq):
        sl = w.seq(i)
        n = sl.stop - sl.start if i == w.nseq - 1 else 192
        uu = w.u[sl][:n]
        yo = oracle.cascade_forward_seq(Abar, Bbar, C, D, uu, 15, powers=powers)
        g.add(y[sl][:n], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
    g.check()


def test_batching_form_full_size(lib):
    """512 sequences of uneven length (log-uniform in [1024, 65536], 8.85e6
    rows), m = 128, p = q = 4, Abar = 1.000001 x trapezoid(HiPPO-LegS, 5e-7)
    (spectral radius above one), N per sequence from eps = 1e-6, FP32 path.
    The oracle recomputes the four shortest and the two longest sequences in
    full, and 512-step prefixes of 16 others, with the N the library chose
    for each."""
    w = cast_inputs(wl.batching_form(), "fp32")
    c, y = run_gpu(lib, w, "fp32")
    Ns = c.seq_N()
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    assert int(c.N()[0]) == oracle.choose_N(Abar, int(w.lengths.max()), w.eps)
    for i, L in enumerate(w.lengths):
        assert Ns[i] == oracle.effective_N(int(c.N()[0]), int(L))
    order = np.argsort(w.lengths)
    picks = ([(int(i), None) for i in order[:4]] + [(int(i), None) for i in order[-2:]]
             + [(int(i), 512) for i in order[4::31][:16]])
    g = SeqGate("fp32")
    for i, n in picks:
        sl = w.seq(i)
        uu = w.u[sl] if n is None else w.u[sl][:n]
        yo = oracle.cascade_forward_seq(Abar, Bbar, C, D, uu, int(Ns[i]))
        g.add(y[sl][: len(uu)], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
    g.check()


@pytest.mark.parametrize("precision", ["fp32", "bf16_split"])
def test_batching_form_cx_only(lib, precision):
    """The batching-form system with D = 0, so y = Cx exactly and the gate
    measures the cascade itself (with D != 0, Du dominates y at delta = 5e-7):
    24 uneven sequences up to 8192 steps, spectral radius above one."""
    w = wl.batching_form(nseq=24, Lmax=8192)
    w.D = np.zeros_like(w.D)
    check(lib, w, precision)


@pytest.mark.parametrize("precision,m", [("bf16_split", 256), ("fp32", 128), ("bf16_split", 512)])
def test_autotuned_shape_keeps_parity(lib, precision, m):
    """Every kernel shape the autotuner may pick gives the same results; the
    chosen one is valid and keeps oracle parity."""
    import torch
    w = cast_inputs(wl.precision_form(m=m, L=1200, batch=4, N=10), precision)
    c = lib.from_workload(w, precision=precision)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda()
    stages, ring, group = c.autotune(u)
    assert 2 <= stages <= 8 and ring in (2, 4, 6, 8) and group in (1, 2) and ring % group == 0
    # the per-stage choices: one for each stage 1..N with tiles, all valid shapes
    per = c.stage_shapes()
    assert set(per) <= set(range(1, 11)) and len(per) >= 1
    for s_, r_, g_ in per.values():
        assert 2 <= s_ <= 8 and r_ in (2, 4, 6, 8) and g_ in (1, 2) and r_ % (2 * g_) == 0
    y = c.forward(u).double().cpu().numpy()
    assert c.device_error() == 0
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y, yo, precision)
    # an explicit shape applies to every stage; saved per-stage shapes come back
    c.set_kernel_shape(stages, ring, group)
    assert c.stage_shapes() == {}
    c.set_stage_shapes(per)
    assert c.stage_shapes() == per
    y2 = c.forward(u).double().cpu().numpy()
    assert np.array_equal(y, y2)


@pytest.mark.parametrize("precision,m", [("bf16_split", 256), ("bf16_split", 128), ("fp32", 128),
                                         ("fp32", 64), ("bf16_split", 512)])
def test_every_kernel_shape(lib, precision, m):
    """Each kernel shape that fits (operand stages x ring slots x chunks per
    step) matches the oracle on ragged sequences; shapes that do not fit, or
    whose ring slots cannot be split evenly between the two epilogue groups,
    are refused."""
    import torch
    from paper_2411_17729_gb300._abi import CascadeError
    lengths = (1, 130, 700, 257)
    w = wl.precision_form(m=m, L=8, batch=len(lengths), N=10)
    rng = np.random.default_rng(3)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = rng.standard_normal((int(w.offsets[-1]), 1))
    w = cast_inputs(w, precision)
    c = lib.from_workload(w, precision=precision)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda()
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    tried = 0
    for group in (1, 2):
        for ring in (2, 4, 6, 8):
            for stages in (2, 3, 4, 5, 6):
                try:
                    c.set_kernel_shape(stages, ring, group)
                except CascadeError:
                    continue
                tried += 1
                y = c.forward(u).double().cpu().numpy()
                assert c.device_error() == 0
                gate(w, y, yo, precision, what=f"{stages}/{ring}/{group}")
    assert tried >= 5
    with pytest.raises(CascadeError):
        c.set_kernel_shape(2, 5, 2)          # ring not a multiple of the step
    with pytest.raises(CascadeError):
        c.set_kernel_shape(2, 6, 2)          # ring slots not split evenly over the two groups


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_many_items_per_block(lib, precision):
    """40 sequences x 2048 steps: every block of the persistent stage kernel
    walks several tiles per stage, pass-through tiles (all sources before the
    sequence start) interleaved with computed ones."""
    w = wl.precision_form(m=128, L=2048, batch=40, N=10)
    c, y, yo = check(lib, w, precision)


@pytest.mark.parametrize("deltas", ["small", "large"])
@pytest.mark.parametrize("discrete", [False, True])
def test_lower_triangular_setup(lib, discrete, deltas):
    """HiPPO-LegS is lower-triangular: the set-up then solves Eq. (4.2) by forward
    elimination without row exchanges over the non-zero triangle, and squares
    with a triangular product.  Abar and every power come out exactly
    lower-triangular and match the oracle.  With small steps, where the dense
    set-up (CASCADE_FLAG_DENSE_SETUP) exchanges no rows either, powers and
    outputs are the dense set-up's bit for bit; with steps up to 0.3 (row
    exchanges in the dense elimination) the outputs pass the parity gate."""
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_DENSE_SETUP
    w = wl.precision_form(m=256, L=1500, batch=4, N=10)
    w.delta = np.array([1e-4, 3e-4, 1e-3, 2e-3]) if deltas == "small" else \
        np.array([1e-4, 1e-2, 0.1, 0.3])
    if discrete:
        mats = [oracle.system_matrices(w, s) for s in range(4)]
        w.Abar = np.stack([np.tril(mt[0]) for mt in mats])   # drop LAPACK's round-off fill-in
        w.B = np.stack([mt[1] for mt in mats])
        w.A, w.delta = None, None
    w = cast_inputs(w, "bf16_split")
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda()
    out = []
    for flags in (0, CASCADE_FLAG_DENSE_SETUP):
        c = lib.from_workload(w, precision="bf16_split", flags=flags)
        P = [c.powers(s, 10).cpu().numpy() for s in range(4)]
        y = c.forward(u).double().cpu().numpy()
        torch.cuda.synchronize()
        assert c.device_error() == 0
        out.append((P, y, c))
    for s in range(4):
        for k in range(11):
            assert np.all(np.triu(out[0][0][s][k], 1) == 0.0), (s, k)
        Abar, _, _, _ = oracle.system_matrices(w, s)
        P = oracle.squaring_chain(Abar, 10)
        for k in range(11):
            err = np.max(np.abs(out[0][0][s][k] - P[k])) / np.max(np.abs(P[k]))
            assert err <= 1e-12 * 2 ** k, (s, k, err)
        if deltas == "small" or discrete:
            assert np.array_equal(out[0][0][s], out[1][0][s]), s
    if deltas == "small" or discrete:
        assert np.array_equal(out[0][1], out[1][1])
    yo = oracle.cascade_forward(w, N_per_seq=out[0][2].seq_N())
    gate(w, out[0][1], yo, "bf16_split")
