"""Tensor-level wrapper over the C ABI: device memory and streams come from
PyTorch, every computation from libcascade.so.  Argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Cascade:
    """One plan of the C ABI: systems (Abar or (A, delta)), a packed batch, and
    forward / backward over it.  Tensors passed in must live on the current
    CUDA device; system matrices are float64 with a leading system axis."""

    def __init__(self, m, p, q, nsys=1, N=-1, eps=0.0, precision="bf16_split", max_len=1 << 16,
                 max_rows=1 << 20, flags=0, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the cascade library needs a CUDA device")
        self.lib = _abi.lib()
        self.m, self.p, self.q, self.nsys = m, p, q, nsys
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        d = _abi.cascade_desc_t(m=m, p=p, q=q, nsys=nsys, N=N, precision=_abi.PRECISIONS[precision],
                                max_len=max_len, flags=flags, max_rows=max_rows, eps=eps)
        self.plan = _abi.cascade_plan_t()
        with torch.cuda.device(self.device):
            _abi.check(self.lib.cascade_plan_create(C.byref(self.plan), C.byref(d)))
        self._ws = None
        self.continuous = False

    def close(self):
        if self.plan:
            self.lib.cascade_plan_destroy(self.plan)
            self.plan = _abi.cascade_plan_t()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        _abi.check(st, self.plan)

    @staticmethod
    def _dev64(x, device):
        x = np.array(x, dtype=np.float64, copy=True) if isinstance(x, np.ndarray) else x
        return torch.as_tensor(x, dtype=torch.float64).to(device).contiguous()

    def set_system_continuous(self, A, B, delta, C_, D, abar_scale=None, stream=None):
        t = [self._dev64(x, self.device) for x in (A, B, delta, C_, D)]
        sc = None if abar_scale is None else self._dev64(abar_scale, self.device)
        self._check(self.lib.cascade_set_system_continuous(self.plan, _ptr(t[0]), _ptr(t[1]),
                                                           _ptr(t[2]), _ptr(sc), _ptr(t[3]),
                                                           _ptr(t[4]), _stream(stream)))
        self.continuous = True

    def set_system_discrete(self, Abar, Bbar, C_, D, stream=None):
        t = [self._dev64(x, self.device) for x in (Abar, Bbar, C_, D)]
        self._check(self.lib.cascade_set_system_discrete(self.plan, *[_ptr(x) for x in t],
                                                         _stream(stream)))
        self.continuous = False

    def set_batch(self, offsets, sys_of_seq=None):
        offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        nseq = len(offs) - 1
        sys_arr = None
        if sys_of_seq is not None:
            sys_arr = np.ascontiguousarray(np.asarray(sys_of_seq, dtype=np.int32))
        self._check(self.lib.cascade_set_batch(
            self.plan, offs.ctypes.data_as(C.POINTER(C.c_int64)), nseq,
            None if sys_arr is None else sys_arr.ctypes.data_as(C.POINTER(C.c_int32))))
        self.rows = int(offs[-1]) if nseq > 0 else 0
        self.nseq = nseq

    def N(self):
        out = (C.c_int32 * self.nsys)()
        self._check(self.lib.cascade_get_N(self.plan, out))
        return np.array(out[:], dtype=np.int32)

    def seq_N(self):
        out = (C.c_int32 * max(self.nseq, 1))()
        self._check(self.lib.cascade_get_seq_N(self.plan, out))
        return np.array(out[: self.nseq], dtype=np.int32)

    def powers(self, sys, kmax, stream=None):
        out = torch.empty((kmax + 1, self.m, self.m), dtype=torch.float64, device=self.device)
        self._check(self.lib.cascade_get_powers(self.plan, sys, kmax, _ptr(out), _stream(stream)))
        return out

    def output_fused(self):
        """True when y = C v + D u is formed in the last stage's epilogue."""
        f = C.c_int32()
        self._check(self.lib.cascade_get_output_fused(self.plan, C.byref(f)))
        return bool(f.value)

    def workspace_size(self):
        n = C.c_size_t()
        self._check(self.lib.cascade_workspace_size(self.plan, C.byref(n)))
        return n.value

    def workspace(self):
        need = self.workspace_size()
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def forward(self, u, y=None, stream=None):
        assert u.dtype == self.dtype and u.is_contiguous() and u.shape == (self.rows, self.p)
        if y is None:
            y = torch.empty((self.rows, self.q), dtype=self.dtype, device=self.device)
        ws = self.workspace()
        self._check(self.lib.cascade_forward(self.plan, _ptr(u), _ptr(y), _ptr(ws), ws.numel(),
                                             _stream(stream)))
        return y

    def forward_host(self, h_u, h_y, d_u=None, d_y=None, stream=None):
        """The forward from host memory to host memory (cascade_forward_host):
        h_u [rows, p] and h_y [rows, q] CPU tensors (page-locked for full-speed
        copies), d_u, d_y device staging tensors (allocated when omitted).
        Returns h_y once y is there."""
        for t, n in ((h_u, self.p), (h_y, self.q)):
            assert t.device.type == "cpu" and t.dtype == self.dtype and t.is_contiguous()
            assert t.shape == (self.rows, n)
        if d_u is None:
            d_u = torch.empty((self.rows, self.p), dtype=self.dtype, device=self.device)
        if d_y is None:
            d_y = torch.empty((self.rows, self.q), dtype=self.dtype, device=self.device)
        ws = self.workspace()
        self._check(self.lib.cascade_forward_host(self.plan, _ptr(h_u), _ptr(h_y), _ptr(d_u),
                                                  _ptr(d_y), _ptr(ws), ws.numel(),
                                                  _stream(stream)))
        return h_y

    def backward(self, u, dy, stream=None, want=("du", "dAbar", "dBbar", "dC", "dD", "dA", "dB")):
        """Gradients of sum(dy * y) for the last forward (plan created with
        CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE).  Returns a dict of
        tensors; dA, dB only for continuous systems."""
        assert dy.dtype == self.dtype and dy.is_contiguous() and dy.shape == (self.rows, self.q)
        f64 = dict(dtype=torch.float64, device=self.device)
        m, p, q, ns = self.m, self.p, self.q, self.nsys
        out = {}
        if "du" in want:
            out["du"] = torch.empty((self.rows, p), dtype=self.dtype, device=self.device)
        shapes = {"dAbar": (ns, m, m), "dBbar": (ns, m, p), "dC": (ns, q, m), "dD": (ns, q, p)}
        if self.continuous:
            shapes.update({"dA": (ns, m, m), "dB": (ns, m, p)})
        for k, shp in shapes.items():
            if k in want:
                out[k] = torch.empty(shp, **f64)   # the library writes every entry
        ws = self.workspace()
        g = lambda k: _ptr(out.get(k))
        self._check(self.lib.cascade_backward(self.plan, _ptr(u), _ptr(dy), g("du"), g("dAbar"),
                                              g("dBbar"), g("dC"), g("dD"), g("dA"), g("dB"),
                                              _ptr(ws), ws.numel(), _stream(stream)))
        return out

    def recursion(self, u, y=None, stream=None):
        assert u.dtype == torch.float64 and u.is_contiguous()
        if y is None:
            y = torch.empty((self.rows, self.q), dtype=torch.float64, device=self.device)
        self._check(self.lib.cascade_recursion_forward(self.plan, _ptr(u), _ptr(y), _stream(stream)))
        return y

    def autotune(self, u, y=None, reps=2, stream=None):
        """Pick the fastest tensor-core kernel shape for the current batch
        (returns (stages, ring slots, chunks per step))."""
        if y is None:
            y = torch.empty((self.rows, self.q), dtype=self.dtype, device=self.device)
        ws = self.workspace()
        choice = (C.c_int32 * 3)()
        self._check(self.lib.cascade_autotune(self.plan, _ptr(u), _ptr(y), _ptr(ws), ws.numel(),
                                              _stream(stream), reps, choice))
        return tuple(choice[:])

    def set_kernel_shape(self, stages, ring, group):
        shape = (C.c_int32 * 3)(stages, ring, group)
        self._check(self.lib.cascade_set_kernel_shape(self.plan, shape))

    def first_fused(self):
        """True when the current batch forms first-stage values v^(1) on chip."""
        f = C.c_int32()
        self._check(self.lib.cascade_get_first_fused(self.plan, C.byref(f)))
        return bool(f.value)

    def fused_stages(self):
        """Leading stages 1 .. J that the forward runs as one pass with the states
        on chip (0: none)."""
        j = C.c_int32()
        self._check(self.lib.cascade_get_fused_stages(self.plan, C.byref(j)))
        return j.value

    def stage_shapes(self):
        """{entry: (stages, ring slots, chunks per step)} chosen per stage by autotune
        (entry k: stage k; work-efficient schedule: up-sweep level k, 100 + k: down-sweep
        level k)."""
        n = C.c_int32()
        self._check(self.lib.cascade_get_stage_shapes(self.plan, 0, None, C.byref(n)))
        cap = n.value
        buf = (C.c_int32 * max(3 * cap, 1))()
        self._check(self.lib.cascade_get_stage_shapes(self.plan, cap, buf, C.byref(n)))
        return {k: tuple(buf[3 * k:3 * k + 3]) for k in range(min(cap, n.value))
                if buf[3 * k] > 0}

    def set_stage_shapes(self, shapes):
        """Per-stage shapes {entry: (stages, ring slots, chunks per step)}, as
        stage_shapes() returns them; {} clears them."""
        n = (max(shapes) + 1) if shapes else 0
        buf = (C.c_int32 * max(3 * n, 1))()
        for k, v in shapes.items():
            buf[3 * k:3 * k + 3] = list(v)
        self._check(self.lib.cascade_set_stage_shapes(self.plan, n, buf))

    def enable_stage_timing(self, on=True):
        self._check(self.lib.cascade_enable_stage_timing(self.plan, 1 if on else 0))

    def stage_times(self, cap=64):
        ks = (C.c_int32 * cap)()
        ms = (C.c_float * cap)()
        n = C.c_int32()
        self._check(self.lib.cascade_get_stage_times(self.plan, cap, ks, ms, C.byref(n)))
        k = min(cap, n.value)
        return list(zip(ks[:k], ms[:k]))

    def device_error(self):
        code = C.c_int32()
        self._check(self.lib.cascade_get_device_error(self.plan, C.byref(code)))
        return code.value


def from_workload(w, precision=None, flags=0, N=None, max_len=None, device=None):
    """Plan for a ``workloads.Workload`` with its systems and batch set."""
    prec = precision or w.precision
    if getattr(w, "discretisation", "trapezoid") == "zoh" and w.Abar is None:
        flags |= _abi.CASCADE_FLAG_ZOH
    casc = Cascade(w.m, w.p, w.q, nsys=w.nsys, N=w.N if N is None else N, eps=w.eps,
                   precision=prec, max_len=int(max_len or max(1, int(w.lengths.max(initial=1)))),
                   max_rows=max(w.rows, 1), flags=flags, device=device)
    nsys = w.nsys
    rep = lambda x: np.broadcast_to(x, (nsys,) + x.shape[1:]) if x.shape[0] == 1 else x
    if w.Abar is not None:
        casc.set_system_discrete(rep(w.Abar), rep(w.B), rep(w.C), rep(w.D))
    else:
        delta = np.broadcast_to(w.delta, (nsys,)) if len(w.delta) == 1 else w.delta
        sc = None if w.abar_scale is None else (np.broadcast_to(w.abar_scale, (nsys,))
                                                if len(w.abar_scale) == 1 else w.abar_scale)
        casc.set_system_continuous(rep(w.A), rep(w.B), delta, rep(w.C), rep(w.D), abar_scale=sc)
    casc.set_batch(w.offsets, w.sys_of_seq)
    return casc


class CascadeFunction(torch.autograd.Function):
    """y = cascade(u; A or Abar, B or Bbar, C, D) as a differentiable op.

    apply(casc, u, A, B, C, D, delta=None): with ``delta`` the system is
    continuous (A, B discretised by Eq. 4.2 on the device), otherwise A, B are
    Abar, Bbar.  ``casc`` is a Cascade plan created with
    CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE whose batch is already
    set; system tensors are
    float64 [nsys, ...] on the plan's device.  Gradients flow to u, A (through
    the squaring chain, and the discretisation when continuous), B, C and D.
    """

    @staticmethod
    def forward(ctx, casc, u, A, B, C_, D, delta=None):
        if delta is None:
            casc.set_system_discrete(A.detach(), B.detach(), C_.detach(), D.detach())
        else:
            casc.set_system_continuous(A.detach(), B.detach(), delta.detach(), C_.detach(),
                                       D.detach())
        u = u.contiguous()
        y = casc.forward(u)
        ctx.casc = casc
        ctx.continuous = delta is not None
        ctx.save_for_backward(u)
        return y

    @staticmethod
    def backward(ctx, dy):
        (u,) = ctx.saved_tensors
        g = ctx.casc.backward(u, dy.contiguous().to(u.dtype))
        gA = g["dA"] if ctx.continuous else g["dAbar"]
        gB = g["dB"] if ctx.continuous else g["dBbar"]
        return None, g["du"], gA, gB, g["dC"], g["dD"], None
