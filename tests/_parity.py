"""Helpers shared by the GPU parity tests (no method arithmetic here).

Every comparison of a GPU result with the oracle goes through ``gate`` (or
``gate_arrays``), which checks two things per sequence (per system for the
system-matrix gradients) and records the worst values for the run's summary:

  * the relative Frobenius error ||x - x_o|| / ||x_o||, and for outputs also
    on Cx = y - Du (so that Du cannot hide a broken cascade);
  * the element-wise error max |x - x_o| / max |x_o| (for outputs also on
    Cx), so that a fault confined to one 128-row tile (a wrong shift, mask or
    ring slot) cannot hide in the norm of a long sequence.

Both must stay within the path's bar: 1e-12 (FP64), 1e-5 (FP32), 2e-3
(BF16 split) for outputs; 1e-10, 1e-5, 2e-3 for gradients.
"""
import os

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

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16_split": 2e-3}
GTOL = {"fp64": 1e-10, "fp32": 1e-5, "bf16_split": 2e-3}

# (test id, what, frob y, frob Cx, elem y, elem Cx, bar) of every gate, for the
# summary the conftest prints at the end of the run
RESULTS = []


def _test_id():
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def seq_errors(yg, yo, Du=None, out_eps=0.0, absDu=None):
    """Errors of one sequence (rows = time): (frob y, frob Cx, elem y, elem Cx).
    The Cx errors are taken beyond an allowance for the rounding of the
    delivered y: 2 out_eps ||y|| in norm; element-wise, per element,
    (p + 2) out_eps (|y| + |D| |u|) when absDu = |u| |D|^T is given (y's last
    rounding and the p products of D u evaluated in the output type; p = the
    width of u), else 2 out_eps max |y|.  Without Du the Cx errors are those
    of y."""
    d = yg - yo
    ny, my = np.linalg.norm(yo), np.max(np.abs(yo)) if yo.size else 0.0
    nd, md = np.linalg.norm(d), np.max(np.abs(d)) if d.size else 0.0
    fy = nd / ny if ny > 0 else nd
    ey = md / my if my > 0 else md
    if Du is None:
        return fy, fy, ey, ey
    cx = yo - Du
    ncx, mcx = np.linalg.norm(cx), np.max(np.abs(cx)) if cx.size else 0.0
    fcx = max(nd - 2.0 * out_eps * ny, 0.0) / ncx if ncx > 0 else 0.0
    if absDu is not None and d.size:
        pw = absDu.shape[1] if absDu.ndim > 1 else 1
        excess = np.max(np.maximum(np.abs(d) - (pw + 2) * out_eps * (np.abs(yo) + absDu), 0.0))
    else:
        excess = max(md - 2.0 * out_eps * my, 0.0)
    ecx = excess / mcx if mcx > 0 else 0.0
    return fy, fcx, ey, ecx


def record(what, errs, bar):
    RESULTS.append((_test_id(), what) + tuple(float(e) for e in errs) + (float(bar),))


def rel_errors(w, y, yo, out_eps=0.0):
    """(frob y, frob Cx, elem y, elem Cx), each maxed over the sequences of a
    packed workload (empty sequences skipped)."""
    worst = np.zeros(4)
    for i in range(w.nseq):
        sl = w.seq(i)
        if sl.stop == sl.start:
            continue
        s = int(w.sys_of_seq[i])
        D = w.D[min(s, w.D.shape[0] - 1)]
        Du = w.u[sl] @ D.T
        absDu = np.abs(w.u[sl]) @ np.abs(D).T
        worst = np.maximum(worst, seq_errors(y[sl], yo[sl], Du, out_eps, absDu))
    return tuple(worst)


def gate(w, y, yo, precision, what="y", tol=None):
    """Assert the four errors of a packed output against the path's bar and
    record them.  Returns them."""
    errs = rel_errors(w, y, yo, OUT_EPS[precision])
    bar = TOL[precision] if tol is None else tol
    record(what, errs, bar)
    assert all(e <= bar for e in errs), (what, errs, bar)
    return errs


class SeqGate:
    """Accumulates per-sequence errors of sampled full-size checks, then
    asserts and records the worst."""

    def __init__(self, precision, what="y"):
        self.precision, self.what = precision, what
        self.worst = np.zeros(4)

    def add(self, yg, yo, Du, absDu=None):
        self.worst = np.maximum(self.worst, seq_errors(yg, yo, Du, OUT_EPS[self.precision], absDu))

    def check(self):
        bar = TOL[self.precision]
        record(self.what, self.worst, bar)
        assert all(e <= bar for e in self.worst), (self.what, tuple(self.worst), bar)
        return tuple(self.worst)


def grad_errors(w, g, ref):
    """Per gradient: (frob, elem), maxed over sequences for du (rows = time)
    and over systems for the system-matrix gradients."""
    out = {}
    for k, v in g.items():
        r = ref[k]
        worst = np.zeros(2)
        if k == "du":
            for i in range(w.nseq):
                sl = w.seq(i)
                if sl.stop == sl.start:
                    continue
                fy, _, ey, _ = seq_errors(v[sl], r[sl])
                worst = np.maximum(worst, (fy, ey))
        else:
            for s in range(r.shape[0]):
                fy, _, ey, _ = seq_errors(v[s], r[s])
                worst = np.maximum(worst, (fy, ey))
        out[k] = tuple(worst)
    return out


def gate_grads(w, g, ref, precision, tol=None):
    bar = GTOL[precision] if tol is None else tol
    errs = grad_errors(w, g, ref)
    for k, (f, e) in errs.items():
        record(k, (f, f, e, e), bar)
    bad = {k: e for k, e in errs.items() if not (e[0] <= bar and e[1] <= bar)}
    assert not bad, (bad, errs, bar)
    return errs
