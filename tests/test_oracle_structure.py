"""Whether the powers Abar^(2^k) keep the structure that §5 points to for
O(m log m) matrix-vector products: for trapezoidal HiPPO-LegS, Abar itself
has off-diagonal blocks of numerical rank one, but repeated squaring raises
that rank roughly like 2^k, so structured powers pay only for the first few
stages.  Recorded here as a check of the mathematics (CPU)."""
import numpy as np

import oracle
import workloads as wl


def offdiag_rank(P, tol):
    """Largest numerical rank (singular values above tol * ||P||_2) of the two
    off-diagonal blocks of the top-level 2 x 2 split."""
    n = P.shape[0] // 2
    nrm = np.linalg.norm(P, 2)
    r = 0
    for blk in (P[:n, n:], P[n:, :n]):
        sv = np.linalg.svd(blk, compute_uv=False)
        r = max(r, int(np.sum(sv > tol * nrm)))
    return r


def test_hippo_powers_lose_low_offdiagonal_rank():
    m = 128
    A = wl.hippo_legs(m)
    B = wl.hippo_legs_B(m).reshape(m, 1)
    Abar, _ = oracle.discretise_trapezoid(A, B, 1e-2)
    powers = oracle.squaring_chain(Abar, 6)
    ranks = [offdiag_rank(powers[k], 1e-3) for k in (0, 3, 6)]
    assert ranks[0] == 1                        # rank-one off-diagonal part of Abar
    assert ranks[1] >= 6 and ranks[2] >= 16     # grows with the power
    assert ranks[2] > ranks[1] > ranks[0], ranks
