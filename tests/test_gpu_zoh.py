"""GPU parity of the zero-order-hold discretisation (§5, CASCADE_FLAG_ZOH):
the device's FP64 exponential against the oracle's (scipy) one, the cascade
on the resulting systems, and gradients to A and B through the Frechet
derivative of the exponential."""
import numpy as np
import pytest

import oracle
import workloads as wl
from _parity import cast_inputs, gate, gate_grads

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


def zoh_small(m=24, p=3, q=2, lengths=(70, 1, 33), delta=0.3, nsys=2, seed=31):
    w = wl.small_system(m=m, p=p, q=q, lengths=lengths, N=8, nsys=nsys, seed=seed,
                        discrete=False, delta=delta)
    w.delta = np.array([delta, 2.5 * delta][:nsys])
    w.discretisation = "zoh"
    return w


def test_zoh_powers_and_forward_fp64(lib):
    """Abar = exp(delta A) to 1e-12 against scipy, for two step sizes (one
    needing several squarings), and the FP64 cascade on the ZOH systems."""
    import torch
    w = zoh_small()
    c = lib.from_workload(w, precision="fp64")
    for s in range(w.nsys):
        Ab, Bb = oracle.discretise_zoh(w.A[s], w.B[s], float(w.delta[s]))
        P0 = c.powers(s, 0)[0].cpu().numpy()
        assert np.linalg.norm(P0 - Ab) <= 1e-12 * np.linalg.norm(Ab)
    y = c.forward(torch.as_tensor(w.u).cuda()).cpu().numpy()
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y, yo, "fp64")


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_zoh_hippo_tensor_cores(lib, precision):
    """HiPPO-LegS m = 128 with per-sequence steps in [1e-4, 1e-1] discretised
    by the zero-order hold, tensor-core forward."""
    import torch
    w = wl.precision_form(m=128, L=1500, batch=4, N=10)
    w.discretisation = "zoh"
    w = cast_inputs(w, precision)
    c = lib.from_workload(w, precision=precision)
    y = c.forward(torch.as_tensor(w.u, dtype=torch.float32).cuda()).double().cpu().numpy()
    yo = oracle.cascade_forward(w, N_per_seq=c.seq_N())
    gate(w, y, yo, precision)


def grads(lib, w, precision, dy):
    import torch
    from paper_2411_17729_gb300._abi import CASCADE_FLAG_SAVE_STATES
    c = lib.from_workload(w, precision=precision, flags=CASCADE_FLAG_SAVE_STATES)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = torch.as_tensor(w.u, dtype=dt).cuda().contiguous()
    c.forward(u)
    g = c.backward(u, torch.as_tensor(dy, dtype=dt).cuda().contiguous())
    torch.cuda.synchronize()
    assert c.device_error() == 0
    ref = oracle.cascade_backward(w, dy, N_per_seq=c.seq_N())
    return {k: v.double().cpu().numpy() for k, v in g.items()}, ref


def test_zoh_backward_fp64(lib):
    """dA, dB through the exponential's Frechet derivative (and every other
    gradient) against the oracle's FP64 adjoint."""
    w = zoh_small(m=12, p=2, q=3, lengths=(40, 17), delta=0.4)
    dy = np.random.default_rng(32).standard_normal((w.rows, w.q))
    g, ref = grads(lib, w, "fp64", dy)
    gate_grads(w, g, ref, "fp64")


def test_zoh_backward_bf16(lib):
    w = wl.differentiation_form(m=128, p=4, q=4, L=8, batch=3, N=9, delta=2e-2)
    lengths = (300, 129, 1)
    w.offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    w.u = np.random.default_rng(33).standard_normal((int(w.offsets[-1]), 4))
    w.discretisation = "zoh"
    w = cast_inputs(w, "bf16_split")
    dy = np.random.default_rng(34).standard_normal((w.rows, w.q)).astype(np.float32).astype(np.float64)
    g, ref = grads(lib, w, "bf16_split", dy)
    gate_grads(w, g, ref, "bf16_split")
