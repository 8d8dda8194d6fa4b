"""CPU checks of the bench's roofline arithmetic: the stage-GEMM flop count it
reports for a whole forward equals the §3 schedule's matrix-vector products
as the oracle counts them (times 6 m^2 for the three split products, stage 0
excluded: it runs inside the first projection), and the bound it names
follows the kernel's arithmetic intensity (HBM at m = 256, tensor at m = 1024)."""
import types

import numpy as np
import pytest

import oracle
import workloads as wl


class FakePlan:
    """The plan queries stage_roofline makes, answered from the workload."""

    def __init__(self, w, fused_stages=0, first_fused=False, output_fused=True):
        self._N = np.array([oracle.effective_N(w.N, int(L)) for L in w.lengths])
        self._J, self._first, self._out = fused_stages, first_fused, output_fused

    def seq_N(self):
        return self._N

    def fused_stages(self):
        return self._J

    def first_fused(self):
        return self._first

    def output_fused(self):
        return self._out


def roofline(w, plan, ms_per_launch=1.0):
    import bench
    Ns = plan.seq_N()
    first = 1 if plan.fused_stages() == 0 else plan.fused_stages() + 1
    stage_ms = {k: [ms_per_launch] for k in range(first, int(Ns.max()) + 1)}
    if plan.fused_stages() or plan.first_fused():
        stage_ms[1] = [ms_per_launch]
    args = types.SimpleNamespace(steps=1, cur_workload="test", seqs=0)
    return bench.stage_roofline(w, plan, stage_ms, "bf16_split", args)


@pytest.mark.parametrize("fused", [0, 3])
def test_all_stage_flops_match_the_oracle_count(fused):
    w = wl.precision_form(m=64, L=8, batch=4, N=11)
    w.offsets = np.array([0, 1, 700, 700 + 4096, 700 + 4096 + 2000], dtype=np.int64)
    w.u = np.zeros((int(w.offsets[-1]), 1))
    plan = FakePlan(w, fused_stages=fused)
    roof = roofline(w, plan)
    products = 0
    for L, N in zip(w.lengths, plan.seq_N()):
        products += oracle.matvec_counts(int(N), int(L))["executed"] - max(int(L) - 1, 0)
    assert roof["all_stages"]["flops_per_step"] == 6 * w.m * w.m * products


def test_bound_follows_intensity():
    for m, want in ((256, "hbm"), (1024, "tensor")):
        w = wl.precision_form(m=m, L=4096, batch=2, N=11)
        w.u = np.zeros((w.rows, 1))
        roof = roofline(w, FakePlan(w))
        assert roof["bound"] == want, (m, roof["intensity_flop_per_byte"])
        assert (roof["intensity_flop_per_byte"] > roof["ridge_flop_per_byte"]) == (want == "tensor")
