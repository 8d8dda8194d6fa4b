"""Seeded input generators (HiPPO-shaped linear time-invariant systems).

Every generator takes an explicit ``seed`` and draws from
``numpy.random.default_rng(seed)`` in a fixed order, so the oracle and the
CUDA path see bit-identical inputs.  Floating-point inputs are produced in
float64; a caller that feeds a float32 kernel casts them and hands the *same*
cast values (promoted back to float64) to the oracle.

Shapes follow the problem statement of §1 (Eq. 1.1): A is m x m, B is m x p,
C is q x m, D is q x p.  Sequences are stored time-major and packed: u has
shape [sum_i L_i, p], with int64 ``offsets`` (length nseq+1) marking where
each sequence starts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "hippo_legs", "hippo_legs_B", "haar_orthogonal", "Workload",
    "plain_fp64", "precision_form", "batching_form", "differentiation_form",
    "large_form", "small_system", "WORKLOADS",
]


def hippo_legs(m: int, base: int = 0) -> np.ndarray:
    """Continuous HiPPO-LegS state matrix of §4, Eq. (4.1).

    A[n, k] = -sqrt(2n+1) sqrt(2k+1) for n > k, -(n+1) for n == k, 0 above,
    with the row/column labels n, k running over base .. base+m-1.  The
    worked example of §4 uses labels 1..m (its printed eigenvalues need
    that); the usual HiPPO-LegS form labels 0..m-1.
    """
    idx = np.arange(base, base + m, dtype=np.float64)
    r = np.sqrt(2.0 * idx + 1.0)
    A = -np.outer(r, r)
    A = np.tril(A, -1)
    A[np.diag_indices(m)] = -(idx + 1.0)
    return A


def hippo_legs_B(m: int, base: int = 0) -> np.ndarray:
    """HiPPO-LegS input vector B_n = sqrt(2n+1), as an m x 1 matrix."""
    idx = np.arange(base, base + m, dtype=np.float64)
    return np.sqrt(2.0 * idx + 1.0).reshape(m, 1)


def haar_orthogonal(rng: np.random.Generator, m: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian, signs fixed by diag(R)."""
    G = rng.standard_normal((m, m))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


@dataclass
class Workload:
    """One batch of sequences together with the systems that filter them.

    Either ``A`` (continuous, with per-system ``delta`` and optional
    ``abar_scale``) or ``Abar`` (already discrete, Eq. 1.2) is given.
    System matrices carry a leading system axis of length ``nsys``;
    ``sys_of_seq`` maps each sequence to its system.
    """
    name: str
    m: int
    p: int
    q: int
    N: int                      # stages run are k = 0..N (-1: choose from eps)
    precision: str              # "fp64", "fp32", "bf16_split"
    offsets: np.ndarray         # int64 [nseq+1]
    u: np.ndarray               # float64 [rows, p]
    B: np.ndarray               # float64 [nsys, m, p] (continuous B, or Bbar if discrete)
    C: np.ndarray               # float64 [nsys, q, m]
    D: np.ndarray               # float64 [nsys, q, p]
    sys_of_seq: np.ndarray      # int32 [nseq]
    A: np.ndarray | None = None         # float64 [nsys, m, m] continuous
    delta: np.ndarray | None = None     # float64 [nsys]
    abar_scale: np.ndarray | None = None  # float64 [nsys] multiplies Abar after discretisation
    discretisation: str = "trapezoid"   # rule for continuous systems: "trapezoid" or "zoh"
    Abar: np.ndarray | None = None      # float64 [nsys, m, m] discrete
    eps: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def nseq(self) -> int:
        return len(self.offsets) - 1

    @property
    def nsys(self) -> int:
        return self.C.shape[0]

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def rows(self) -> int:
        return int(self.offsets[-1])

    @property
    def discrete(self) -> bool:
        return self.Abar is not None

    def seq(self, i: int) -> slice:
        return slice(int(self.offsets[i]), int(self.offsets[i + 1]))

    def subset(self, seqs) -> "Workload":
        """The same workload restricted to the listed sequences (systems kept)."""
        seqs = list(seqs)
        lens = self.lengths[seqs]
        offs = np.zeros(len(seqs) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        u = np.concatenate([self.u[self.seq(i)] for i in seqs], axis=0) if seqs else self.u[:0]
        w = Workload(**{**self.__dict__})
        w.offsets, w.u = offs, u
        w.sys_of_seq = self.sys_of_seq[seqs].copy()
        w.name = self.name + f"[{len(seqs)} seqs]"
        return w


def _offsets(lengths) -> np.ndarray:
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(np.asarray(lengths, dtype=np.int64))
    return offs


def plain_fp64(m=64, L=4096, N=11, seed=0, batch=1, delta=1.0 / 4096) -> Workload:
    """Plain FP64 cascade: HiPPO-LegS (labels 0..m-1), trapezoidal step delta,
    B_n = sqrt(2n+1), p = q = 1, C ~ N(0, 1/m), D ~ N(0, 1), u ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    A = hippo_legs(m)[None]
    B = hippo_legs_B(m)[None]
    C = rng.standard_normal((1, 1, m)) / math.sqrt(m)
    D = rng.standard_normal((1, 1, 1))
    u = rng.standard_normal((batch * L, 1))
    return Workload(name=f"plain_fp64 m={m} L={L} b={batch}", m=m, p=1, q=1, N=N,
                    precision="fp64", offsets=_offsets([L] * batch), u=u, B=B, C=C, D=D,
                    sys_of_seq=np.zeros(batch, np.int32), A=A, delta=np.array([delta]))


def precision_form(m=256, L=16384, batch=64, N=13, seed=0,
                   delta_range=(1e-4, 1e-1)) -> Workload:
    """BF16-split form: HiPPO-LegS, p = q = 1, one step size per sequence drawn
    log-uniform in ``delta_range`` (so one system per sequence), u ~ N(0, 1),
    B_n = sqrt(2n+1), C ~ N(0, 1/m), D ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(delta_range[0]), np.log(delta_range[1])
    delta = np.exp(rng.uniform(lo, hi, size=batch))
    A = np.broadcast_to(hippo_legs(m), (batch, m, m)).copy()
    B = np.broadcast_to(hippo_legs_B(m), (batch, m, 1)).copy()
    C = np.broadcast_to(rng.standard_normal((1, m)) / math.sqrt(m), (batch, 1, m)).copy()
    D = np.broadcast_to(rng.standard_normal((1, 1)), (batch, 1, 1)).copy()
    u = rng.standard_normal((batch * L, 1))
    return Workload(name=f"precision_form m={m} L={L} b={batch}", m=m, p=1, q=1, N=N,
                    precision="bf16_split", offsets=_offsets([L] * batch), u=u, B=B, C=C, D=D,
                    sys_of_seq=np.arange(batch, dtype=np.int32), A=A, delta=delta)


def batching_form(m=128, p=4, q=4, nseq=512, Lmin=1024, Lmax=65536, seed=0,
                  delta=5e-7, growth=1e-6, eps=1e-6) -> Workload:
    """Batching form: uneven sequence lengths log-uniform in [Lmin, Lmax],
    Abar = (1 + growth) * trapezoid(HiPPO-LegS, delta) so that its spectral
    radius slightly exceeds 1, B, C, D ~ N(0, 1/m), u ~ N(0, 1); N is chosen
    per sequence from the accuracy target ``eps`` (N = -1)."""
    rng = np.random.default_rng(seed)
    lens = np.floor(np.exp(rng.uniform(np.log(Lmin), np.log(Lmax), size=nseq))).astype(np.int64)
    lens = np.clip(lens, Lmin, Lmax)
    A = hippo_legs(m)[None]
    B = rng.standard_normal((1, m, p)) / math.sqrt(m)
    C = rng.standard_normal((1, q, m)) / math.sqrt(m)
    D = rng.standard_normal((1, q, p)) / math.sqrt(m)
    offs = _offsets(lens)
    u = rng.standard_normal((int(offs[-1]), p))
    return Workload(name=f"batching_form m={m} p={p} q={q} nseq={nseq}", m=m, p=p, q=q, N=-1,
                    precision="fp32", offsets=offs, u=u, B=B, C=C, D=D,
                    sys_of_seq=np.zeros(nseq, np.int32), A=A, delta=np.array([delta]),
                    abar_scale=np.array([1.0 + growth]), eps=eps)


def differentiation_form(m=256, p=16, q=16, L=8192, batch=32, N=12, seed=0,
                         delta=1e-3) -> Workload:
    """Differentiation form: HiPPO-LegS with step delta, B, C, D ~ N(0, 1/m),
    u ~ N(0, 1), MIMO p = q = 16."""
    rng = np.random.default_rng(seed)
    A = hippo_legs(m)[None]
    B = rng.standard_normal((1, m, p)) / math.sqrt(m)
    C = rng.standard_normal((1, q, m)) / math.sqrt(m)
    D = rng.standard_normal((1, q, p)) / math.sqrt(m)
    u = rng.standard_normal((batch * L, p))
    return Workload(name=f"differentiation_form m={m} p={p} q={q} L={L} b={batch}", m=m, p=p,
                    q=q, N=N, precision="bf16_split", offsets=_offsets([L] * batch), u=u,
                    B=B, C=C, D=D, sys_of_seq=np.zeros(batch, np.int32), A=A,
                    delta=np.array([delta]))


def large_form(m=1024, p=64, q=64, L=65536, batch=8, N=15, seed=0, radius=0.9999,
               rank=4, pert_var=1e-4) -> Workload:
    """Large form: Abar = radius * Q + E with Q Haar-orthogonal and E = s X Y^T
    of the given rank, X, Y ~ N(0, 1), s chosen so that every entry of E has
    variance pert_var / m.  Bbar, C, D ~ N(0, 1/m), u ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(rng, m)
    X = rng.standard_normal((m, rank))
    Y = rng.standard_normal((m, rank))
    s = math.sqrt(pert_var / (rank * m))
    Abar = (radius * Q + s * (X @ Y.T))[None]
    Bbar = rng.standard_normal((1, m, p)) / math.sqrt(m)
    C = rng.standard_normal((1, q, m)) / math.sqrt(m)
    D = rng.standard_normal((1, q, p)) / math.sqrt(m)
    u = rng.standard_normal((batch * L, p))
    return Workload(name=f"large_form m={m} p={p} q={q} L={L} b={batch}", m=m, p=p, q=q,
                    N=N, precision="bf16_split", offsets=_offsets([L] * batch), u=u,
                    B=Bbar, C=C, D=D, sys_of_seq=np.zeros(batch, np.int32), Abar=Abar)


def small_system(m=8, p=2, q=3, lengths=(37,), N=3, seed=0, nsys=1, radius=0.95,
                 discrete=True, delta=0.05, precision="fp64") -> Workload:
    """Small dense random systems for brute-force checks.

    discrete=True: Abar = radius * (random matrix normalised to spectral
    radius 1), with nonsymmetric entries; Bbar, C, D ~ N(0, 1).
    discrete=False: A is a random stable-ish continuous matrix (-I + G/sqrt(m))
    with per-system step ``delta``."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(nsys):
        G = rng.standard_normal((m, m))
        if discrete:
            rho = max(abs(np.linalg.eigvals(G)))
            mats.append(radius * G / rho)
        else:
            mats.append(-np.eye(m) + G / math.sqrt(m))
    M = np.stack(mats)
    B = rng.standard_normal((nsys, m, p))
    C = rng.standard_normal((nsys, q, m))
    D = rng.standard_normal((nsys, q, p))
    offs = _offsets(lengths)
    u = rng.standard_normal((int(offs[-1]), p))
    sys_of_seq = (np.arange(len(lengths)) % nsys).astype(np.int32)
    kw = dict(Abar=M) if discrete else dict(A=M, delta=np.full(nsys, delta))
    return Workload(name=f"small m={m} p={p} q={q}", m=m, p=p, q=q, N=N, precision=precision,
                    offsets=offs, u=u, B=B, C=C, D=D, sys_of_seq=sys_of_seq, **kw)


WORKLOADS = {
    "plain_fp64": plain_fp64,
    "precision_form": precision_form,
    "batching_form": batching_form,
    "differentiation_form": differentiation_form,
    "large_form": large_form,
}
