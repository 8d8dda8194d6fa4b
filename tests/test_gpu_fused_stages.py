"""GPU parity of stages 1, 2, 3 of the §3 schedule run as one pass over
overlapping windows of 128 time steps with the states on chip (v^(1) formed
from u, each stage one tcgen05 contraction, FP32 states between the stages,
v^(4) the only state written).  Checked against the oracle (element-wise and
in norm) and against the same plan with the stages as separate launches
(CASCADE_FLAG_NO_FUSED_STAGES) to rounding: the fused pass keeps FP32 states
between the stages where the separate launches store BF16 pairs."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate, rel_errors

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


def hippo(m, lengths, q=1, N=12, seed=51):
    """HiPPO-LegS, one trapezoidal step per sequence (log-uniform in [1e-4,
    1e-1]), ragged lengths."""
    if q == 1:
        w = wl.precision_form(m=m, L=8, batch=len(lengths), N=N, seed=seed)
    else:
        w = wl.differentiation_form(m=m, p=1, q=q, L=8, batch=len(lengths), N=N, delta=1e-2,
                                    seed=seed)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(seed).standard_normal((int(w.offsets[-1]), 1))
    return cast_inputs(w, "bf16_split")


def forward(lib, w, flags=0):
    import torch
    c = lib.from_workload(w, precision="bf16_split", flags=flags)
    u = torch.as_tensor(w.u, dtype=torch.float32).cuda().contiguous()
    y = c.forward(u)
    torch.cuda.synchronize()
    assert c.device_error() == 0, c.lib.cascade_last_error(c.plan)
    return c, y.double().cpu().numpy()


LENGTHS = (17, 100, 113, 114, 115, 127, 128, 129, 228, 229, 1000, 3001)


@pytest.mark.parametrize("m,q", [(256, 1), (128, 1), (256, 3), (128, 4)])
def test_fused_stages_match_oracle_and_separate_launches(lib, m, q):
    """Lengths around the window step (114 rows) and the tile size, the
    shortest that still runs four stages (17), two step sizes per system."""
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_NO_FUSED_STAGES
    w = hippo(m, LENGTHS, q=q)
    c1, y1 = forward(lib, w)
    assert c1.fused_stages() == 3
    c2, y2 = forward(lib, w, CASCADE_FLAG_NO_FUSED_STAGES)
    assert c2.fused_stages() == 0
    yo = oracle.cascade_forward(w, N_per_seq=c1.seq_N())
    gate(w, y1, yo, "bf16_split", what="fused")
    gate(w, y2, yo, "bf16_split", what="launch")
    fy, fcx, ey, ecx = rel_errors(w, y1, y2)
    assert max(fy, ey) < 1e-5, (fy, ey)


def test_fused_stages_many_windows_per_block(lib):
    """40 sequences x 4096 steps: every block walks many windows."""
    w = hippo(256, (4096,) * 40)
    c, y = forward(lib, w)
    assert c.fused_stages() == 3
    gate(w, y, oracle.cascade_forward(w, N_per_seq=c.seq_N()), "bf16_split")


def test_fused_stages_when(lib):
    """The pass applies to forward-only plans with p = 1, m = 128 or 256, BF16
    pairs, on the §3 schedule, when every sequence runs more than 3 stages."""
    from paper_2411_17729_gb300._abi import (CASCADE_FLAG_NO_FUSED_STAGES, CASCADE_FLAG_SAVE_STATES,
                                             CASCADE_FLAG_SCAN)
    w = hippo(256, (300, 500))
    for flags, want in ((0, 3), (CASCADE_FLAG_NO_FUSED_STAGES, 0), (CASCADE_FLAG_SAVE_STATES, 0),
                        (CASCADE_FLAG_SCAN, 0)):
        c = lib.from_workload(w, precision="bf16_split", flags=flags)
        assert c.fused_stages() == want, flags
        c.close()
    c = lib.from_workload(hippo(256, (300, 16)), precision="bf16_split")    # N = 3 for 16 steps
    assert c.fused_stages() == 0
    c.close()
    c = lib.from_workload(hippo(256, (300, 500)), precision="fp32")
    assert c.fused_stages() == 0
    c.close()
    c = lib.from_workload(hippo(512, (300, 500)), precision="bf16_split")
    assert c.fused_stages() == 0
    c.close()
