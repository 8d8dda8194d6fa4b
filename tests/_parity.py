"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def cast_inputs(w, precision):
    """Inputs as the CUDA path sees them: float32 u for the tensor-core
    precisions (the oracle then runs on the same float32 values)."""
    if precision == "fp64":
        return w
    w.u = w.u.astype(np.float32).astype(np.float64)
    return w


# Unit roundoff of the output element type: Cx = y - Du is recovered from the
# delivered y, so its error cannot fall below the rounding of y itself.
OUT_EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "bf16_split": 2.0 ** -24}


def rel_errors(w, y, yo, out_eps=0.0):
    """Per-sequence relative Frobenius errors of y and of Cx = y - Du, maxed
    over sequences (empty sequences skipped).  The Cx error is taken beyond
    an allowance of 2 * out_eps * ||y|| for the rounding of y to its output
    format (zero by default)."""
    ey, ecx = 0.0, 0.0
    for i in range(w.nseq):
        sl = w.seq(i)
        if sl.stop == sl.start:
            continue
        s = int(w.sys_of_seq[i])
        D = w.D[min(s, w.D.shape[0] - 1)]
        Du = w.u[sl] @ D.T
        ny = np.linalg.norm(yo[sl])
        ncx = np.linalg.norm(yo[sl] - Du)
        if ny > 0:
            ey = max(ey, np.linalg.norm(y[sl] - yo[sl]) / ny)
        if ncx > 0:
            d = np.linalg.norm((y[sl] - Du) - (yo[sl] - Du)) - 2.0 * out_eps * ny
            ecx = max(ecx, max(d, 0.0) / ncx)
    return ey, ecx


TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16_split": 2e-3}
