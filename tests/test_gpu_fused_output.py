"""GPU parity of the output y = C v + D u (end of §3) formed on the tensor cores
inside the last stage (BF16 split, p and q multiples of 16, q <= 64; m <= 256
by default, wider m with CASCADE_FLAG_FUSE_WIDE_OUTPUT): the
finished state chunks the stage kernel stages for its store are the A operand
of a second tcgen05 product with C, the first column block adds D u, and with
m above one column block the partial sums over the blocks are added in order.

Checked against the oracle (element-wise and in norm, the usual bars), against
the separate projection pass (CASCADE_FLAG_NO_FUSED_OUTPUT) to FP32 rounding,
and, for plans that keep their stage outputs, the backward's gradients equal
those after the separate pass bit for bit (the stored final states are the same).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate, gate_grads, rel_errors

pytestmark = pytest.mark.gpu

LENGTHS = (1, 127, 128, 129, 0, 300, 1000, 2049)


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17729_gb300 import build
    build()
    from paper_2411_17729_gb300 import cascade
    return cascade


def two_systems(m, p, q, N=11, lengths=LENGTHS, seed=41):
    """Discrete systems (orthogonal plus low rank, and its reversal scaled by
    0.98), ragged lengths with empty, one-step and tile-edge sequences."""
    w = wl.large_form(m=m, p=p, q=q, L=8, batch=len(lengths), N=N, seed=seed)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(seed).standard_normal((int(w.offsets[-1]), p))
    w.sys_of_seq = (np.arange(len(lengths)) % 2).astype(np.int32)
    w.Abar = np.concatenate([w.Abar, 0.98 * w.Abar[:, ::-1, :]])
    for k in ("B", "C", "D"):
        setattr(w, k, np.concatenate([getattr(w, k), 0.5 * getattr(w, k)]))
    return cast_inputs(w, "bf16_split")


def wide(m):
    """The flag that fuses the output when m spans several column blocks."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_FUSE_WIDE_OUTPUT
    return CASCADE_FLAG_FUSE_WIDE_OUTPUT if m > 256 else 0


def forward(lib, w, flags=0):
    import torch
    c = lib.from_workload(w, precision="bf16_split", flags=flags)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    y = c.forward(u)
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    return c, y.double().cpu().numpy()


def test_output_fused_query(lib):
    """cascade_get_output_fused for the tensor-core form of the fused output."""
    from paper_2411_17729_gb300._abi import (CASCADE_FLAG_FUSE_WIDE_OUTPUT,
                                             CASCADE_FLAG_NO_FUSED_OUTPUT, CASCADE_FLAG_SCAN)
    cases = [(256, 16, 16, "bf16_split", 0, True), (128, 16, 64, "bf16_split", 0, True),
             (1024, 64, 64, "bf16_split", 0, False), (512, 32, 48, "bf16_split", 0, False),
             (1024, 64, 64, "bf16_split", CASCADE_FLAG_FUSE_WIDE_OUTPUT, True),
             (512, 32, 48, "bf16_split", CASCADE_FLAG_FUSE_WIDE_OUTPUT, True),
             (256, 16, 80, "bf16_split", 0, False), (128, 16, 16, "fp32", 0, False),
             (256, 3, 16, "bf16_split", 0, False),
             (256, 16, 16, "bf16_split", CASCADE_FLAG_NO_FUSED_OUTPUT, False),
             (256, 16, 16, "bf16_split", CASCADE_FLAG_SCAN, False)]
    for m, p, q, precision, flags, want in cases:
        c = lib.Cascade(m, p, q, N=8, precision=precision, flags=flags, max_len=1024)
        assert c.output_fused() == want, (m, p, q, precision, flags)
        c.close()


@pytest.mark.parametrize("m,p,q", [(128, 16, 16), (256, 16, 16), (256, 32, 48), (192, 16, 32),
                                   (512, 16, 64), (256, 64, 64), (1024, 64, 64)])
def test_fused_output_matches_oracle_and_separate_pass(lib, m, p, q):
    """One to four column blocks, q from 16 to 64, p up to 64 (two (u, D)
    chunks), ragged lengths, two systems."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_OUTPUT
    w = two_systems(m, p, q)
    c1, y1 = forward(lib, w, wide(m))
    assert c1.output_fused()
    c2, y2 = forward(lib, w, CASCADE_FLAG_NO_FUSED_OUTPUT)
    assert not c2.output_fused()
    yo = oracle.cascade_forward(w, N_per_seq=c1.seq_N())
    gate(w, y1, yo, "bf16_split", what="fused")
    gate(w, y2, yo, "bf16_split", what="pass")
    fy, _, ey, _ = rel_errors(w, y1, y2)
    assert fy < 1e-5 and ey < 1e-5, (fy, ey)


@pytest.mark.parametrize("m,N", [(512, 4), (256, 3)])
def test_fused_output_truncated(lib, m, N):
    """A truncated cascade (2^(N+1) < L): every sequence's last stage is N."""
    w = two_systems(m, 16, 32, N=N)
    c, y = forward(lib, w, wide(m))
    assert c.output_fused()
    gate(w, y, oracle.cascade_forward(w, N_per_seq=c.seq_N()), "bf16_split")


def test_fused_output_many_tiles_per_block(lib):
    """40 sequences x 2048 steps at m = 512: every block of the persistent last
    stage walks many tiles, both column blocks of each, fused copies (all
    sources before the sequence start) interleaved with computed tiles."""
    w = two_systems(512, 16, 64, lengths=(2048,) * 40)
    c, y = forward(lib, w, wide(512))
    assert c.output_fused()
    gate(w, y, oracle.cascade_forward(w, N_per_seq=c.seq_N()), "bf16_split")


@pytest.mark.parametrize("m,p,q", [(256, 16, 16), (512, 32, 64)])
def test_fused_output_backward_bitwise(lib, m, p, q):
    """Plans that keep their stage outputs: the fused last stage still stores
    v^(N+1), so the backward after it gives the gradients of the backward after
    the separate pass bit for bit, and they match the oracle's adjoint."""
    import torch
    from paper_2411_17729_gb300._abi import (CASCADE_FLAG_NO_FUSED_OUTPUT,
                                             CASCADE_FLAG_RECOMPUTE, CASCADE_FLAG_SAVE_STATES)
    w = two_systems(m, p, q, N=10)
    dy = np.random.default_rng(43).standard_normal((w.rows, q)).astype(np.float32)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    grads = []
    for flags in (CASCADE_FLAG_SAVE_STATES, CASCADE_FLAG_SAVE_STATES | CASCADE_FLAG_NO_FUSED_OUTPUT,
                  CASCADE_FLAG_RECOMPUTE):
        c = lib.from_workload(w, precision="bf16_split", flags=flags | wide(m))
        c.forward(u)
        g = c.backward(u, torch.as_tensor(dy).cuda())
        torch.cuda.synchronize()
        assert c.device_error() == 0
        grads.append({k: v.double().cpu().numpy() for k, v in g.items()})
    for k in grads[0]:
        assert np.array_equal(grads[0][k], grads[1][k]), k
        assert np.array_equal(grads[0][k], grads[2][k]), k
    ref = oracle.cascade_backward(w, dy.astype(np.float64), N_per_seq=c.seq_N())
    gate_grads(w, grads[0], ref, "bf16_split")


def test_differentiation_form_forward_full_size(lib):
    """The differentiation workload's forward at full size (m = 256, p = q = 16,
    32 x 8192, N = 12), output formed on the tensor cores in the last stage:
    every sequence against the oracle, and the separate projection pass on the
    same inputs agrees with it to rounding."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_OUTPUT
    from _parity import SeqGate
    w = cast_inputs(wl.differentiation_form(), "bf16_split")
    c1, y1 = forward(lib, w)
    assert c1.output_fused()
    c2, y2 = forward(lib, w, CASCADE_FLAG_NO_FUSED_OUTPUT)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    powers = oracle.squaring_chain(Abar, 12)
    g1, g2 = SeqGate("bf16_split", "fused"), SeqGate("bf16_split", "pass")
    for i in range(w.nseq):
        sl = w.seq(i)
        uu = w.u[sl]
        yo = oracle.cascade_forward_seq(Abar, Bbar, C, D, uu, 12, powers=powers)
        g1.add(y1[sl], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
        g2.add(y2[sl], yo, uu @ D.T, np.abs(uu) @ np.abs(D).T)
    e1, e2 = g1.check(), g2.check()
    fy, _, ey, _ = rel_errors(w, y1, y2)
    assert fy < 1e-5 and ey < 1e-5, (fy, ey, e1, e2)
