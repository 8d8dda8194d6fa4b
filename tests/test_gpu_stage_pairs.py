"""GPU parity of stage pairs: stages k and k + 1 of the §3 schedule run as one
launch over an interleaved tile list, the second stage's tiles waiting for the
blocks that store the first stage's rows they read (the middle states go
through memory as with separate launches).  Checked bit for bit against the
same plan with one launch per stage (CASCADE_FLAG_NO_STAGE_PAIRS) and against
the oracle (element-wise and in norm)."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate

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


def hippo(m, lengths, q=1, N=13, seed=61):
    """HiPPO-LegS with one trapezoidal step per sequence (log-uniform in
    [1e-4, 1e-1]); lengths multiples of 128."""
    if q == 1:
        w = wl.precision_form(m=m, L=8, batch=len(lengths), N=N, seed=seed)
    else:
        w = wl.differentiation_form(m=m, p=1, q=q, L=8, batch=len(lengths), N=N, delta=1e-2,
                                    seed=seed)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(seed).standard_normal((int(w.offsets[-1]), 1))
    return cast_inputs(w, "bf16_split")


def forward(lib, w, flags=0, reps=1):
    import torch
    c = lib.from_workload(w, precision="bf16_split", flags=flags)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    ys = []
    for _ in range(reps):
        ys.append(c.forward(u).double().cpu().numpy())
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    return c, ys[-1] if reps == 1 else ys


def flag(name):
    from paper_2411_17729_gb300 import _abi
    return getattr(_abi, name)


@pytest.mark.parametrize("m,extra", [(256, 0), (128, 0), (256, "CASCADE_FLAG_NO_FUSED_STAGES"),
                                     (256, "CASCADE_FLAG_NO_FUSED_STAGES|"
                                           "CASCADE_FLAG_NO_FUSED_FIRST")])
def test_pairs_bitwise_and_oracle(lib, m, extra):
    """Lengths 128 .. 2048 (per-sequence N from 6 to 10, so some sequences end
    on the first stage of a pair and form y there); pairs from stage 4 (after
    the fused first stages), 2 (stage 1 forms v^(1) on chip) or 1."""
    fl = 0
    for n in (extra.split("|") if extra else []):
        fl |= flag(n)
    w = hippo(m, (128, 256, 384, 512, 1024, 1152, 2048, 1920))
    c1, y1 = forward(lib, w, fl)
    pairs = c1.stage_pairs()
    assert pairs, "no stage pairs for an eligible batch"
    first = 4 if not fl else (2 if fl == flag("CASCADE_FLAG_NO_FUSED_STAGES") else 1)
    assert pairs[0] == first, pairs
    c2, y2 = forward(lib, w, fl | flag("CASCADE_FLAG_NO_STAGE_PAIRS"))
    assert c2.stage_pairs() == []
    assert np.array_equal(y1, y2), np.max(np.abs(y1 - y2))
    gate(w, y1, oracle.cascade_forward(w, N_per_seq=c1.seq_N()), "bf16_split", what="pairs")


def test_pairs_long_list_repeated_and_graph(lib):
    """64 sequences x 2048 steps: lists longer than the grid (the lag and the
    place holders), several forwards in a row (the launch count advances) and
    graph replays, all bit for bit those of separate launches."""
    w = hippo(256, (2048,) * 64, N=10)
    c0, y0 = forward(lib, w, flag("CASCADE_FLAG_NO_STAGE_PAIRS"))
    c1, ys = forward(lib, w, 0, reps=3)
    assert c1.stage_pairs()
    for y in ys:
        assert np.array_equal(y, y0)
    c2, ys = forward(lib, w, flag("CASCADE_FLAG_GRAPH"), reps=3)
    for y in ys:
        assert np.array_equal(y, y0)
    yo = oracle.cascade_forward(w, N_per_seq=c1.seq_N())
    gate(w, y0, yo, "bf16_split", what="pairs")


def test_pairs_output_fused_q3(lib):
    """q = 3 (the output formed in the epilogue of the last stage, which may be
    the second stage of a pair or the first)."""
    w = hippo(256, (1024, 2048, 1536), q=3)
    c1, y1 = forward(lib, w)
    assert c1.stage_pairs()
    c2, y2 = forward(lib, w, flag("CASCADE_FLAG_NO_STAGE_PAIRS"))
    assert np.array_equal(y1, y2)
    gate(w, y1, oracle.cascade_forward(w, N_per_seq=c1.seq_N()), "bf16_split", what="pairs")


def test_pairs_when(lib):
    """Pairs apply to forward-only BF16-pair plans on the §3 schedule with
    m <= 256 whose sequences are multiples of 128 steps long."""
    w = hippo(256, (1024, 2048))
    for fl in ("CASCADE_FLAG_NO_STAGE_PAIRS", "CASCADE_FLAG_SAVE_STATES", "CASCADE_FLAG_SCAN",
               "CASCADE_FLAG_RECOMPUTE"):
        c = lib.from_workload(w, precision="bf16_split", flags=flag(fl))
        assert c.stage_pairs() == [], fl
        c.close()
    c = lib.from_workload(w, precision="bf16_split")
    assert c.stage_pairs() == [4, 6, 8]        # N_i = 9, 10: stages 4..10
    c.close()
    c = lib.from_workload(hippo(256, (1024, 2000)), precision="bf16_split")
    assert c.stage_pairs() == []               # 2000 is not a multiple of 128
    c.close()
    c = lib.from_workload(w, precision="fp32")
    assert c.stage_pairs() == []
    c.close()
    c = lib.from_workload(hippo(512, (1024, 2048)), precision="bf16_split")
    assert c.stage_pairs() == []               # two column blocks per tile
    c.close()
