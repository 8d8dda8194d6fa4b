"""CPU checks of the parity gates themselves (tests/_parity.py): the
allowance for the delivered y's rounding admits an output evaluated exactly
as the kernels evaluate it (FP32), and a fault planted in one element of one
128-row tile is caught element-wise where the norm alone would pass it."""
import numpy as np

from _parity import OUT_EPS, TOL, seq_errors


def _fp32_output(Cx, D, u):
    """y = Cx + D u with the D u products added one by one in FP32."""
    y = Cx.astype(np.float32)
    for j in range(u.shape[1]):
        y = (y + (D[:, j].astype(np.float32)[None, :] * u[:, j:j + 1].astype(np.float32))).astype(np.float32)
    return y.astype(np.float64)


def test_fp32_evaluation_of_du_is_within_the_allowance():
    rng = np.random.default_rng(5)
    L, p, q = 20000, 4, 4
    u = rng.standard_normal((L, p)).astype(np.float32).astype(np.float64)
    D = rng.standard_normal((q, p)) / np.sqrt(128)
    Cx = 1e-4 * rng.standard_normal((L, q))          # Cx small beside Du, as at delta = 5e-7
    yo = Cx + u @ D.T
    yg = _fp32_output(Cx, D, u)
    fy, fcx, ey, ecx = seq_errors(yg, yo, u @ D.T, OUT_EPS["fp32"], np.abs(u) @ np.abs(D).T)
    assert ecx == 0.0 and fcx == 0.0, (fcx, ecx)
    # an error of 1e-4 max |Cx| at one element is still seen on Cx
    yg[777, 2] += 1e-4 * np.max(np.abs(Cx)) + 8 * 2.0 ** -24 * (abs(yo[777, 2]) + np.abs(u[777]) @ np.abs(D[2]))
    _, _, _, ecx = seq_errors(yg, yo, u @ D.T, OUT_EPS["fp32"], np.abs(u) @ np.abs(D).T)
    assert ecx >= 0.99e-4, ecx


def test_a_fault_in_one_tile_is_caught_element_wise():
    rng = np.random.default_rng(6)
    L, q = 16384, 1
    yo = rng.standard_normal((L, q))
    yg = yo * (1 + 1e-6 * rng.standard_normal((L, q)))
    yg[4096:4224] *= 1.02                              # one 128-row tile 2 % off
    fy, _, ey, _ = seq_errors(yg, yo)
    assert fy <= TOL["bf16_split"] < ey, (fy, ey)
