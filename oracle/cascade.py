"""Plain, slow, float64 restatement of the cascade (arXiv 2411.17729).

Test infrastructure only (see the package docstring).  Each function cites
the passage of the paper it restates.  Library primitives used as single
steps: ``numpy.linalg.solve`` (a linear solve), ``@`` (a matrix product).
No blocking, fusion or reordering beyond what the paper's equations state.

Notation (paper's): state dimension m, input p, output q, sequence length L,
stages n = 1 .. N+1 applying Abar^(2^(n-1)) with a time shift of 2^(n-1)
(we index them k = n-1 = 0 .. N, shift s_k = 2^k).  Vectors are stored as
rows: V[l] is the column v_l of the paper's m x L matrix V.

Readings of the paper taken here (each is listed with its reason in the
design notes):
  * the truncated product has N+1 factors, so the cascade has N+1 stages
    k = 0..N and the output is v after the last one (Eq. 2.2, §3 example
    N = 14 -> 15 matvecs; the "n = 0..N-1" of §3 is read as a slip);
  * Eq. (3.1) adds D u_l once, outside the sum;
  * v_{-1} = 0 (x_{-1} = 0 in §2 and §3): a shifted source before the start
    of a sequence is zero;
  * the accuracy rule picks the smallest N with 2^(N+1) >= L or
    ||Abar^(2^(N+1))||_F <= eps (the Frobenius norm bounds the spectral norm
    from above; the remainder identity makes this the state truncation error).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "discretise_trapezoid", "discretise_zoh", "discretise_zoh_vjp", "squaring_chain", "stage",
    "cascade_states",
    "cascade_forward_seq", "cascade_forward", "recursion_forward_seq",
    "brute_force_seq", "choose_N", "effective_N", "cascade_vjp_seq",
    "squaring_chain_vjp", "discretise_trapezoid_vjp", "cascade_backward",
    "system_matrices", "stage_count", "matvec_counts",
]


# --------------------------------------------------------------------------- §5
def _zoh_block(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Z = [[A, B], [0, 0]], (m + p) x (m + p)."""
    m, p = B.shape
    Z = np.zeros((m + p, m + p))
    Z[:m, :m] = A
    Z[:m, m:] = B
    return Z


def discretise_zoh(A: np.ndarray, B: np.ndarray, delta: float):
    """Zero-order-hold discretisation named in §5:

        Abar = exp(delta A),   Bbar = (delta A)^{-1} (exp(delta A) - I) (delta B),

    reading the printed last factor "delta A" as "delta B" (with delta A the
    units do not match and B would not enter).  Both blocks are read off one
    exponential of the block matrix delta [[A, B], [0, 0]], whose upper right
    block is int_0^delta exp(sA) ds B: that equals the formula above when A is
    invertible and needs no inverse otherwise.  scipy.linalg.expm is the step.
    """
    import scipy.linalg
    m = A.shape[0]
    E = scipy.linalg.expm(delta * _zoh_block(A, B))
    return E[:m, :m].copy(), E[:m, m:].copy()


def discretise_zoh_vjp(A, B, delta, dAbar, dBbar):
    """Adjoint of ``discretise_zoh``.  With F(Z) = exp(Z), Z = delta [[A, B],
    [0, 0]], the directional derivative is the Frechet derivative L(Z, E) and
    its adjoint is L(Z^T, G); G carries (dAbar, dBbar) in the blocks that
    Abar, Bbar occupy.  Then dA = delta dZ[:m, :m], dB = delta dZ[:m, m:].
    scipy.linalg.expm_frechet is the step."""
    import scipy.linalg
    m, p = B.shape
    Z = delta * _zoh_block(A, B)
    G = np.zeros((m + p, m + p))
    G[:m, :m] = dAbar
    G[:m, m:] = dBbar
    dZ = scipy.linalg.expm_frechet(Z.T, G, compute_expm=False)
    return delta * dZ[:m, :m], delta * dZ[:m, m:]


# --------------------------------------------------------------------------- §1
def discretise_trapezoid(A: np.ndarray, B: np.ndarray, delta: float):
    """Trapezoidal discretisation, §1 (after Eq. 1.2) and Eq. (4.2):

        Abar = (I - delta/2 A)^{-1} (I + delta/2 A),
        Bbar = delta (I - delta/2 A)^{-1} B.
    """
    m = A.shape[0]
    I = np.eye(m)
    M = I - 0.5 * delta * A
    Abar = np.linalg.solve(M, I + 0.5 * delta * A)
    Bbar = delta * np.linalg.solve(M, B)
    return Abar, Bbar


def system_matrices(w, s: int):
    """(Abar, Bbar, C, D) of system ``s`` of a workload, in float64.

    Continuous systems are discretised with Eq. (4.2) (or the zero-order hold
    of §5 when ``w.discretisation == "zoh"``); an ``abar_scale``
    multiplies Abar after discretisation (used to push the spectral radius
    above 1 for the stability experiments of §6).
    """
    if w.Abar is not None:
        Abar = np.asarray(w.Abar[min(s, w.Abar.shape[0] - 1)], dtype=np.float64)
        Bbar = np.asarray(w.B[min(s, w.B.shape[0] - 1)], dtype=np.float64)
    else:
        A = w.A[min(s, w.A.shape[0] - 1)]
        B = w.B[min(s, w.B.shape[0] - 1)]
        rule = discretise_zoh if w.discretisation == "zoh" else discretise_trapezoid
        Abar, Bbar = rule(A, B, float(w.delta[min(s, len(w.delta) - 1)]))
        if w.abar_scale is not None:
            Abar = Abar * float(w.abar_scale[min(s, len(w.abar_scale) - 1)])
    C = np.asarray(w.C[min(s, w.C.shape[0] - 1)], dtype=np.float64)
    D = np.asarray(w.D[min(s, w.D.shape[0] - 1)], dtype=np.float64)
    return Abar, Bbar, C, D


# --------------------------------------------------------------------------- §2
def squaring_chain(Abar: np.ndarray, N: int):
    """Powers Abar^(2^k), k = 0..N, by repeated squaring (end of §2, §4).

    Returns the list [P_0, ..., P_N] with P_0 = Abar and P_{k+1} = P_k P_k.
    """
    P = [np.array(Abar, dtype=np.float64)]
    for _ in range(N):
        P.append(P[-1] @ P[-1])
    return P


def choose_N(Abar: np.ndarray, L: int, eps: float, N_max: int = 62) -> int:
    """Number of stages minus one for accuracy eps (Lemma 1; remainder reading).

    Smallest N >= 0 with 2^(N+1) >= L (the truncated product then reproduces
    the full convolution over L steps, Eq. 3.1) or ||Abar^(2^(N+1))||_F <= eps.
    """
    if L <= 2:
        return 0
    P = np.array(Abar, dtype=np.float64)
    for N in range(0, N_max):
        P = P @ P                      # P = Abar^(2^(N+1))
        if 2 ** (N + 1) >= L:
            return N
        if eps > 0 and np.sqrt(np.sum(P * P)) <= eps:
            return N
    return N_max


def effective_N(N: int, L: int) -> int:
    """Stages with shift 2^k >= L do nothing (§3: the update range 2^k <= l <= L-1
    is empty), so a sequence of length L runs stages k = 0..min(N, ceil(log2 L)-1)."""
    if L <= 1:
        return 0
    return min(N, int(np.ceil(np.log2(L))) - 1)


# --------------------------------------------------------------------------- §3
def stage(V: np.ndarray, P: np.ndarray, s: int) -> np.ndarray:
    """One cascade stage, §3 Eqs. (3.2)-(3.4) and the general step:

        v^(n)_l = Abar^(2^(n-1)) v^(n-1)_{l - 2^(n-1)} + v^(n-1)_l   for 2^(n-1) <= l <= L-1,
        v^(n)_l = v^(n-1)_l                                          for 0 <= l < 2^(n-1),

    with P = Abar^(2^(n-1)) and s = 2^(n-1).
    """
    L = V.shape[0]
    out = V.copy()
    if s < L:
        out[s:] = V[s:] + V[: L - s] @ P.T
    return out


def cascade_states(powers, Bbar: np.ndarray, u: np.ndarray, keep_all: bool = False):
    """§3: v^(0)_l = Bbar u_l, then the stages with P_k = Abar^(2^k), k = 0..N.

    Returns V^(N+1) (rows = time), or the list [V^(0), ..., V^(N+1)] if keep_all.
    """
    V = np.asarray(u, dtype=np.float64) @ Bbar.T
    Vs = [V]
    for k, P in enumerate(powers):
        V = stage(V, P, 2 ** k)
        Vs.append(V)
    return Vs if keep_all else V


def cascade_forward_seq(Abar, Bbar, C, D, u, N: int, powers=None):
    """y_l = C v^(N+1)_l + D u_l (end of §3) for one sequence u of shape [L, p]."""
    if powers is None:
        powers = squaring_chain(Abar, N)
    V = cascade_states(powers[: N + 1], Bbar, u)
    return V @ C.T + np.asarray(u, dtype=np.float64) @ D.T


def cascade_forward(w, N_per_seq=None, return_states=False):
    """Oracle output y for every sequence of a workload (packed, [rows, q]).

    N_per_seq: stages per sequence (default: the workload's N, or the accuracy
    rule when N < 0, clipped by ``effective_N``).
    """
    y = np.zeros((w.rows, w.q))
    Vfin = np.zeros((w.rows, w.m)) if return_states else None
    cache = {}
    Ns = []
    for i in range(w.nseq):
        sl = w.seq(i)
        L = sl.stop - sl.start
        s = int(w.sys_of_seq[i])
        if s not in cache:
            cache[s] = system_matrices(w, s)
        Abar, Bbar, C, D = cache[s]
        if N_per_seq is not None:
            N = int(N_per_seq[i])
        else:
            N = w.N if w.N >= 0 else choose_N(Abar, int(max(w.lengths)), w.eps)
            N = effective_N(N, L)
        Ns.append(N)
        if L == 0:
            continue
        key = (s, N)
        if key not in cache:
            cache[key] = squaring_chain(Abar, N)
        V = cascade_states(cache[key], Bbar, w.u[sl])
        y[sl] = V @ C.T + w.u[sl] @ D.T
        if return_states:
            Vfin[sl] = V
    if return_states:
        return y, Vfin, np.array(Ns)
    return y


# ------------------------------------------------------------- comparison forms
def recursion_forward_seq(Abar, Bbar, C, D, u):
    """The discrete recursion of Eq. (1.2), x_{-1} = 0, one step at a time:
    x_n = Abar x_{n-1} + Bbar u_n, y_n = C x_n + D u_n.  Returns (y, x)."""
    L = u.shape[0]
    x = np.zeros(Abar.shape[0])
    X = np.zeros((L, Abar.shape[0]))
    for n in range(L):
        x = Abar @ x + Bbar @ u[n]
        X[n] = x
    return X @ C.T + u @ D.T, X


def brute_force_seq(Abar, Bbar, C, D, u, M: int):
    """Eq. (3.1) truncated to the polynomial degree M-1 of Eq. (2.2):

        y_l = sum_{j=0}^{min(l, M-1)} C Abar^j Bbar u_{l-j} + D u_l

    with every power Abar^j formed by numpy.linalg.matrix_power (independent
    of the squaring chain).  For tiny inputs only.
    """
    L = u.shape[0]
    y = u @ D.T
    for j in range(min(L, M)):
        K = C @ np.linalg.matrix_power(Abar, j) @ Bbar          # q x p
        y[j:] = y[j:] + u[: L - j] @ K.T
    return y


def stage_count(N: int, L: int) -> int:
    """Number of stages that do work for length L: k = 0..N with 2^k < L."""
    return sum(1 for k in range(N + 1) if 2 ** k < L)


def matvec_counts(N: int, L: int):
    """Matrix-vector products by Abar-powers for one sequence.

    executed: the §3 schedule, sum_k (L - 2^k)^+ (every l >= 2^k is updated);
    paper_bound: the 2L of the abstract and §6 (Abar on every entry, Abar^2 on
    every second, ...); recursion: L (Eq. 1.2).
    """
    executed = sum(max(L - 2 ** k, 0) for k in range(N + 1))
    return {"executed": executed, "paper_bound": 2 * L, "recursion": L}


# ------------------------------------------------------------------ adjoints
def cascade_vjp_seq(powers, Bbar, C, D, u, G):
    """Reverse-mode derivative of one sequence's cascade (derived from §3).

    Forward: V0 = u Bbar^T;  V_{k+1}[l] = V_k[l] + P_k V_k[l - s_k]  (l >= s_k);
             y = V_{N+1} C^T + u D^T.
    Given G = d loss / d y (shape [L, q]), returns
    (du, dP list, dBbar, dC, dD) with
        dC = sum_l G_l V_{N+1,l}^T,   dD = sum_l G_l u_l^T,   W_{N+1} = G C,
        for k = N..0:  dP_k = sum_{l >= s_k} W_{k+1}[l] V_k[l - s_k]^T,
                       W_k[l] = W_{k+1}[l] + P_k^T W_{k+1}[l + s_k]  (l + s_k < L),
        dBbar = sum_l W_0[l] u_l^T,   du = W_0 Bbar + G D.
    """
    u = np.asarray(u, dtype=np.float64)
    Vs = cascade_states(powers, Bbar, u, keep_all=True)
    L = u.shape[0]
    dC = G.T @ Vs[-1]
    dD = G.T @ u
    W = G @ C
    dP = [None] * len(powers)
    for k in range(len(powers) - 1, -1, -1):
        s = 2 ** k
        P = powers[k]
        if s < L:
            dP[k] = W[s:].T @ Vs[k][: L - s]
            Wn = W.copy()
            Wn[: L - s] = W[: L - s] + W[s:] @ P
            W = Wn
        else:
            dP[k] = np.zeros_like(P)
    dBbar = W.T @ u
    du = W @ Bbar + G @ D
    return du, dP, dBbar, dC, dD


def squaring_chain_vjp(powers, dP):
    """Adjoint of P_{k+1} = P_k P_k: dP_k += dP_{k+1} P_k^T + P_k^T dP_{k+1},
    for k = N-1 .. 0.  Returns dAbar = the total derivative w.r.t. P_0."""
    g = [x.copy() for x in dP]
    for k in range(len(powers) - 2, -1, -1):
        g[k] = g[k] + g[k + 1] @ powers[k].T + powers[k].T @ g[k + 1]
    return g[0]


def discretise_trapezoid_vjp(A, B, delta, dAbar, dBbar):
    """Adjoint of Eq. (4.2).  With M = I - delta/2 A, Nm = I + delta/2 A,
    Abar = M^{-1} Nm, Bbar = delta M^{-1} B:
        dNm = M^{-T} dAbar,  dM = -M^{-T} (dAbar Abar^T + dBbar Bbar^T),
        dA = delta/2 (dNm - dM),  dB = delta M^{-T} dBbar."""
    Abar, Bbar = discretise_trapezoid(A, B, delta)
    m = A.shape[0]
    M = np.eye(m) - 0.5 * delta * A
    MinvT = np.linalg.inv(M).T
    dNm = MinvT @ dAbar
    dM = -MinvT @ (dAbar @ Abar.T + dBbar @ Bbar.T)
    dA = 0.5 * delta * (dNm - dM)
    dB = delta * MinvT @ dBbar
    return dA, dB


def cascade_backward(w, G, N_per_seq=None):
    """Gradients of sum(G * y) for a whole workload.

    Returns a dict with du [rows, p] and, per system s, dAbar, dBbar, dC, dD
    (and dA, dB for continuous systems, through Eq. 4.2 or the zero-order
    hold; abar_scale, if any, is applied to dAbar first)."""
    out = {"du": np.zeros((w.rows, w.p))}
    nsys = w.nsys
    acc = {s: None for s in range(nsys)}
    cache = {}
    for i in range(w.nseq):
        sl = w.seq(i)
        L = sl.stop - sl.start
        if L == 0:
            continue
        s = int(w.sys_of_seq[i])
        if s not in cache:
            cache[s] = system_matrices(w, s)
        Abar, Bbar, C, D = cache[s]
        if N_per_seq is not None:
            N = int(N_per_seq[i])
        else:
            N = w.N if w.N >= 0 else choose_N(Abar, int(max(w.lengths)), w.eps)
            N = effective_N(N, L)
        powers = squaring_chain(Abar, N)
        du, dP, dBbar, dC, dD = cascade_vjp_seq(powers, Bbar, C, D, w.u[sl], G[sl])
        out["du"][sl] = du
        dAbar = squaring_chain_vjp(powers, dP)
        part = dict(dAbar=dAbar, dBbar=dBbar, dC=dC, dD=dD)
        if acc[s] is None:
            acc[s] = part
        else:
            for kk in part:
                acc[s][kk] = acc[s][kk] + part[kk]
    m, p, q = w.m, w.p, w.q
    for name, shape in (("dAbar", (m, m)), ("dBbar", (m, p)), ("dC", (q, m)), ("dD", (q, p))):
        out[name] = np.stack([acc[s][name] if acc[s] is not None else np.zeros(shape)
                              for s in range(nsys)])
    if w.Abar is None:
        dA, dB = [], []
        for s in range(nsys):
            scale = 1.0 if w.abar_scale is None else float(w.abar_scale[min(s, len(w.abar_scale) - 1)])
            vjp = discretise_zoh_vjp if w.discretisation == "zoh" else discretise_trapezoid_vjp
            dA_s, dB_s = vjp(
                w.A[min(s, w.A.shape[0] - 1)], w.B[min(s, w.B.shape[0] - 1)],
                float(w.delta[min(s, len(w.delta) - 1)]), out["dAbar"][s] * scale,
                out["dBbar"][s])
            dA.append(dA_s)
            dB.append(dB_s)
        out["dA"] = np.stack(dA)
        out["dB"] = np.stack(dB)
    return out
