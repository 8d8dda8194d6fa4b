"""Pins of the CPU FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against something fixed independently of it: a
value printed in the paper (tests/golden/paper_section4.json), a closed form,
a brute-force sum built from numpy.linalg.matrix_power, the recursion of
Eq. (1.2), an algebraic identity of §2, or finite differences.  The inputs
are chosen nonsymmetric, with p != q, so that a transposed operand, a
dropped term, a wrong sign or an off-by-one shift fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_section4.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ----------------------------------------------------------------- §4 example
def test_paper_hippo_eigenvalues():
    """§4: the diagonal of the discretised (1-based) HiPPO matrix runs from
    d_1 = 0.999000499750125 to d_100 = 0.9507437210436478."""
    g = golden()["hippo_example"]
    A = wl.hippo_legs(g["m"], base=g["base"])
    Abar, _ = oracle.discretise_trapezoid(A, wl.hippo_legs_B(g["m"], g["base"]), g["delta"])
    assert np.allclose(np.triu(Abar, 1), 0.0)          # stays lower-triangular
    assert abs(Abar[0, 0] - g["d_1"]) <= 2e-16
    assert abs(Abar[-1, -1] - g["d_100"]) <= 2e-16
    # closed form of a triangular trapezoid step: d_n = (1 - delta a_n/2)/(1 + delta a_n/2)
    a = np.arange(1, g["m"] + 1) + 1.0
    d = (1 - g["delta"] * a / 2) / (1 + g["delta"] * a / 2)
    assert np.max(np.abs(np.diag(Abar) - d)) <= 4e-16


def test_paper_tail_and_triangular_powers():
    """§4: d_1^(2^15) ~ 5.87548e-15; the diagonal of a power of a triangular
    matrix is the power of its diagonal.  The printed value agrees with
    exp(-2^16 atanh(delta)) = 5.875397e-15 to five significant digits, so the
    pin holds it to 2e-5 relative."""
    g = golden()["hippo_example"]
    A = wl.hippo_legs(g["m"], base=g["base"])
    Abar, _ = oracle.discretise_trapezoid(A, wl.hippo_legs_B(g["m"], g["base"]), g["delta"])
    P = oracle.squaring_chain(Abar, 15)
    assert len(P) == 16
    rel = abs(P[15][0, 0] - g["d_1_pow_2_15"]) / g["d_1_pow_2_15"]
    assert rel < 2e-5
    exact = math.exp(-(2 ** 16) * math.atanh(g["delta"]))   # d_1 = (1-delta)/(1+delta)
    assert abs(P[15][0, 0] - exact) <= 1e-12 * exact
    d = np.diag(Abar)
    for k in range(16):
        # k squarings of a rounded number amplify its relative error 2^k times
        assert np.allclose(np.diag(P[k]), d ** (2 ** k), rtol=(2 ** k + 1) * 2.3e-16,
                           atol=1e-290)
        assert np.allclose(np.triu(P[k], 1), 0.0)


def test_paper_powers_accuracy_vs_extended_precision():
    """§4: the powers Abar^(2^k) formed in double precision are accurate to
    about 1e-14.  Recompute them in extended precision (long double forward
    substitution for the triangular solve, long double products) and bound the
    float64 chain's max-norm relative error by 1e-12 (observed ~2e-13)."""
    g = golden()["hippo_example"]
    m, delta = g["m"], g["delta"]
    A = wl.hippo_legs(m, base=g["base"])
    Abar, _ = oracle.discretise_trapezoid(A, wl.hippo_legs_B(m, g["base"]), delta)
    P = oracle.squaring_chain(Abar, 15)
    ld = np.longdouble
    Al = A.astype(ld)
    M = np.eye(m, dtype=ld) - ld(delta) / 2 * Al
    Nm = np.eye(m, dtype=ld) + ld(delta) / 2 * Al
    X = np.zeros((m, m), dtype=ld)
    for i in range(m):                       # M is lower-triangular
        X[i] = (Nm[i] - M[i, :i] @ X[:i]) / M[i, i]
    Pl = X
    for k in range(16):
        err = float(np.max(np.abs(P[k] - Pl)) / np.max(np.abs(Pl)))
        assert err < 1e-12, (k, err)
        Pl = Pl @ Pl


def test_paper_stage_count_example():
    """§3: N = 14 gives degree 2^(N+1)-1 = 32767 with 15 matrix-vector products;
    the truncated cascade has N+1 stages."""
    g = golden()["stage_count_example"]
    N = g["N"]
    assert 2 ** (N + 1) - 1 == g["degree"]
    L = 10 ** 6
    assert oracle.stage_count(N, L) == g["matvecs"]
    # the impulse response of the cascade with N stages has exactly degree 2^(N+1)-1
    a, N2 = 0.5, 3
    h = oracle.cascade_forward_seq(np.array([[a]]), np.array([[1.0]]), np.array([[1.0]]),
                                   np.array([[0.0]]), np.eye(40, 1), N2)[:, 0]
    M = 2 ** (N2 + 1)
    assert np.allclose(h[:M], a ** np.arange(M), rtol=1e-15, atol=0)
    assert np.all(h[M:] == 0.0)


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a0,b,c,d,delta", [(-3.0, 1.5, -0.7, 0.3, 0.01),
                                            (-0.2, 2.0, 1.1, -1.0, 0.5),
                                            (0.4, 0.9, 1.3, 0.25, 0.02)])   # last: |abar| > 1
@pytest.mark.parametrize("N,L", [(0, 9), (2, 9), (3, 9), (5, 40), (6, 40)])
def test_scalar_closed_form(a0, b, c, d, delta, N, L):
    """m = p = q = 1, u = 1: y_l = c bbar (1 - abar^min(l+1, M)) / (1 - abar) + d
    with M = 2^(N+1), abar = (1 + delta a0/2)/(1 - delta a0/2),
    bbar = delta b / (1 - delta a0/2)."""
    abar = (1 + delta * a0 / 2) / (1 - delta * a0 / 2)
    bbar = delta * b / (1 - delta * a0 / 2)
    Abar, Bbar = oracle.discretise_trapezoid(np.array([[a0]]), np.array([[b]]), delta)
    assert abs(Abar[0, 0] - abar) <= 1e-15 * abs(abar)
    assert abs(Bbar[0, 0] - bbar) <= 1e-15 * abs(bbar)
    u = np.ones((L, 1))
    y = oracle.cascade_forward_seq(Abar, Bbar, np.array([[c]]), np.array([[d]]), u, N)[:, 0]
    M = 2 ** (N + 1)
    l = np.arange(L)
    expect = c * bbar * (1 - abar ** np.minimum(l + 1, M)) / (1 - abar) + d
    assert np.allclose(y, expect, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------- brute force
@pytest.mark.parametrize("m,p,q", [(1, 1, 1), (3, 2, 1), (5, 1, 4), (8, 3, 2)])
@pytest.mark.parametrize("L", [1, 2, 3, 17, 64])
@pytest.mark.parametrize("N", [0, 1, 2, 4, 6])
def test_brute_force_truncated_sum(m, p, q, L, N):
    """Eq. (3.1) truncated at degree 2^(N+1)-1 with every power from
    matrix_power, on tiny nonsymmetric systems (including |lambda| > 1)."""
    w = wl.small_system(m=m, p=p, q=q, lengths=(L,), N=N, seed=m * 100 + L + N, radius=1.05)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    y = oracle.cascade_forward_seq(Abar, Bbar, C, D, w.u, N)
    yb = oracle.brute_force_seq(Abar, Bbar, C, D, w.u, 2 ** (N + 1))
    scale = max(1.0, np.max(np.abs(yb)))
    assert np.max(np.abs(y - yb)) <= 1e-12 * scale


def test_dropped_stage_is_caught():
    """A cascade with one stage fewer differs from the brute-force sum: the
    brute-force pin does see the stage count."""
    w = wl.small_system(m=4, p=1, q=1, lengths=(40,), seed=3)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    y_short = oracle.cascade_forward_seq(Abar, Bbar, C, D, w.u, 3)
    yb = oracle.brute_force_seq(Abar, Bbar, C, D, w.u, 2 ** 5)
    assert np.max(np.abs(y_short - yb)) > 1e-3


# ------------------------------------------------------------- recursion
@pytest.mark.parametrize("radius", [0.5, 0.999, 1.05])
def test_recursion_equivalence(radius):
    """When 2^(N+1) >= L the cascade equals the recursion (1.2), for any
    spectral radius (the two are the same finite sum)."""
    L = 100
    w = wl.small_system(m=7, p=2, q=3, lengths=(L,), seed=11, radius=radius)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    N = int(math.ceil(math.log2(L))) - 1
    y = oracle.cascade_forward_seq(Abar, Bbar, C, D, w.u, N)
    yr, _ = oracle.recursion_forward_seq(Abar, Bbar, C, D, w.u)
    assert np.max(np.abs(y - yr)) <= 1e-11 * max(1.0, np.max(np.abs(yr)))


def test_hippo_recursion_equivalence_fp64_workload():
    """The plain FP64 workload (m = 64, L = 4096, N = 11) reduces to the
    recursion because 2^12 = 4096 >= L."""
    w = wl.plain_fp64(m=64, L=4096, N=11)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    y = oracle.cascade_forward(w)
    yr, X = oracle.recursion_forward_seq(Abar, Bbar, C, D, w.u)
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-13
    Cx, Cxr = y - w.u @ D.T, X @ C.T
    assert np.linalg.norm(Cx - Cxr) / np.linalg.norm(Cxr) < 1e-13


def test_remainder_identity():
    """For M = 2^(N+1) < L: v^(N+1)_l = x_l - Abar^M x_{l-M}, where x is the
    recursion state (x_{l-M} = 0 for l < M).  Pins the truncation itself."""
    L, N = 90, 3
    w = wl.small_system(m=6, p=2, q=2, lengths=(L,), seed=5, radius=1.02)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    V = oracle.cascade_states(oracle.squaring_chain(Abar, N), Bbar, w.u)
    _, X = oracle.recursion_forward_seq(Abar, Bbar, C, D, w.u)
    M = 2 ** (N + 1)
    AM = np.linalg.matrix_power(Abar, M)
    expect = X.copy()
    expect[M:] -= X[: L - M] @ AM.T
    assert np.max(np.abs(V - expect)) <= 1e-11 * np.max(np.abs(X))


# ------------------------------------------------------- §2 identities
@pytest.mark.parametrize("N", [0, 2, 4])
def test_product_identity_random_z(N):
    """Eq. (2.2) against its expansion: at random complex z,
    sum_{j<M} z^-j Abar^j = prod_{k<=N} (I + z^(-2^k) Abar^(2^k)).  The left
    side comes from the cascade's impulse response (Bbar = C = I, D = 0), the
    right side from matrix_power."""
    m = 5
    rng = np.random.default_rng(N)
    Abar = rng.standard_normal((m, m)) / math.sqrt(m)
    M = 2 ** (N + 1)
    L = M + 3
    I = np.eye(m)
    H = np.zeros((L, m, m))
    for j in range(m):           # impulse e_j at l = 0
        u = np.zeros((L, m))
        u[0, j] = 1.0
        H[:, :, j] = oracle.cascade_forward_seq(Abar, I, I, np.zeros((m, m)), u, N)
    assert np.all(H[M:] == 0.0)
    for z in (0.7 + 0.9j, -1.3 + 0.2j, np.exp(2.1j)):
        lhs = sum(z ** (-j) * H[j] for j in range(L))
        rhs = I.astype(complex)
        for k in range(N + 1):
            rhs = rhs @ (I + z ** (-(2 ** k)) * np.linalg.matrix_power(Abar, 2 ** k))
        assert np.max(np.abs(lhs - rhs)) <= 1e-12 * max(1.0, np.max(np.abs(rhs)))


def test_lemma1_bound_on_unit_circle():
    """Lemma 1: for gamma = ||Abar||_2 < 1 and |z| = 1,
    ||(I - z^-1 Abar)^-1 - prod_{n<=N}(I + (z^-1 Abar)^(2^n))|| <= gamma^(2^(N+1))/(1-gamma)."""
    m = 6
    rng = np.random.default_rng(7)
    G = rng.standard_normal((m, m))
    Abar = 0.9 * G / np.linalg.norm(G, 2)
    gamma = np.linalg.norm(Abar, 2)
    P = oracle.squaring_chain(Abar, 4)
    I = np.eye(m)
    for N in range(4):
        bound = gamma ** (2 ** (N + 1)) / (1 - gamma)
        for t in np.linspace(0, 2 * np.pi, 13):
            z = np.exp(1j * t)
            exact = np.linalg.inv(I - Abar / z)
            prod = I.astype(complex)
            for n in range(N + 1):
                prod = prod @ (I + z ** (-(2 ** n)) * P[n])
            assert np.linalg.norm(exact - prod, 2) <= bound * (1 + 1e-10)


# ------------------------------------------------------- accuracy rule
def test_choose_N_diagonal_closed_form():
    """For a diagonal Abar the rule's norm is sqrt(sum d_i^(2M)); the smallest
    N with that <= eps (or 2^(N+1) >= L) has a closed form."""
    d = np.array([0.99, 0.9, -0.5, 0.3])
    Abar = np.diag(d)
    for eps in (1e-2, 1e-6, 1e-12):
        N = 0
        while math.sqrt(np.sum(d ** (2 * 2 ** (N + 1)))) > eps:
            N += 1
        assert oracle.choose_N(Abar, 10 ** 9, eps) == N
        assert oracle.choose_N(Abar, 64, eps) == min(N, 5)      # 2^6 >= 64
    # spectral radius above one: no eps is reached, only the length cap
    assert oracle.choose_N(np.diag([1.0 + 1e-6, 0.5]), 5000, 1e-6) == 12   # 2^13 >= 5000


def test_choose_N_paper_example():
    """§4 example: eigenvalues alone suggest N = 14 (d_1^(2^15) ~ 6e-15), but
    ||Abar^(2^15)|| ~ 1e-9 because Abar is far from normal; the norm rule picks
    N = 14 for eps = 2e-9 and N = 15 for eps <= 1e-9."""
    g = golden()["hippo_example"]
    A = wl.hippo_legs(g["m"], base=g["base"])
    Abar, _ = oracle.discretise_trapezoid(A, wl.hippo_legs_B(g["m"], g["base"]), g["delta"])
    assert oracle.choose_N(Abar, 10 ** 9, 2e-9) == g["N_stated"]
    assert oracle.choose_N(Abar, 10 ** 9, 1e-14) == g["N_stated"] + 1


# ------------------------------------------------------------- gradients
def _loss(w, G, **over):
    """sum(G * y) for one sequence with overridden system matrices."""
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    Abar = over.get("Abar", Abar)
    Bbar = over.get("Bbar", Bbar)
    C = over.get("C", C)
    D = over.get("D", D)
    u = over.get("u", w.u)
    y = oracle.cascade_forward_seq(Abar, Bbar, C, D, u, w.N)
    return float(np.sum(G * y))


@pytest.mark.parametrize("L,N", [(23, 2), (23, 5), (8, 1)])
def test_vjp_finite_differences(L, N):
    """Central finite differences (h = 1e-6, float64) on random directions for
    every input of the cascade: u, Abar (through the squaring chain), Bbar, C, D."""
    w = wl.small_system(m=5, p=2, q=3, lengths=(L,), N=N, seed=L * 10 + N, radius=0.97)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((L, w.q))
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    powers = oracle.squaring_chain(Abar, N)
    du, dP, dBbar, dC, dD = oracle.cascade_vjp_seq(powers, Bbar, C, D, w.u, G)
    dAbar = oracle.squaring_chain_vjp(powers, dP)
    base = dict(Abar=Abar, Bbar=Bbar, C=C, D=D, u=w.u)
    grads = dict(Abar=dAbar, Bbar=dBbar, C=dC, D=dD, u=du)
    h = 1e-6
    for name, X in base.items():
        for _ in range(3):
            E = rng.standard_normal(X.shape)
            fp = _loss(w, G, **{name: X + h * E})
            fm = _loss(w, G, **{name: X - h * E})
            fd = (fp - fm) / (2 * h)
            an = float(np.sum(grads[name] * E))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)


def test_vjp_dot_product_adjoint():
    """<G, J du> = <J^T G, du> for the linear map u -> y, exact to rounding."""
    w = wl.small_system(m=6, p=3, q=2, lengths=(50,), N=4, seed=9)
    Abar, Bbar, C, D = oracle.system_matrices(w, 0)
    powers = oracle.squaring_chain(Abar, 4)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((50, 2))
    du_dir = rng.standard_normal((50, 3))
    Jd = oracle.cascade_forward_seq(Abar, Bbar, C, D, du_dir, 4, powers=powers)
    du = oracle.cascade_vjp_seq(powers, Bbar, C, D, w.u, G)[0]
    lhs, rhs = float(np.sum(G * Jd)), float(np.sum(du * du_dir))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_scalar_gradient_closed_form():
    """m = 1: d/d abar of sum_l G_l y_l = c bbar sum_l G_l sum_{1<=j<M, j<=l} j abar^(j-1) u_{l-j}."""
    L, N = 30, 3
    M = 2 ** (N + 1)
    a, b, c, d = 0.93, 0.7, -1.2, 0.4
    rng = np.random.default_rng(4)
    u = rng.standard_normal((L, 1))
    G = rng.standard_normal((L, 1))
    powers = oracle.squaring_chain(np.array([[a]]), N)
    du, dP, dBbar, dC, dD = oracle.cascade_vjp_seq(powers, np.array([[b]]), np.array([[c]]),
                                                  np.array([[d]]), u, G)
    dA = oracle.squaring_chain_vjp(powers, dP)[0, 0]
    expect = 0.0
    for l in range(L):
        for j in range(1, min(l, M - 1) + 1):
            expect += G[l, 0] * c * b * j * a ** (j - 1) * u[l - j, 0]
    assert abs(dA - expect) <= 1e-12 * abs(expect)
    # dD = sum G u, dBbar = c sum_l G_l sum_j a^j u_{l-j}
    assert abs(dD[0, 0] - float(np.sum(G * u))) <= 1e-12
    eb = sum(G[l, 0] * c * a ** j * u[l - j, 0] for l in range(L) for j in range(min(l, M - 1) + 1))
    assert abs(dBbar[0, 0] - eb) <= 1e-12 * abs(eb)


def test_discretisation_vjp_finite_differences():
    """Gradient through Eq. (4.2) to the continuous A and B (central FD)."""
    w = wl.small_system(m=4, p=2, q=2, lengths=(21,), N=3, seed=21, discrete=False, delta=0.1)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((21, 2))
    A, B, delta = w.A[0], w.B[0], float(w.delta[0])
    C, D = w.C[0], w.D[0]

    def loss(A_, B_):
        Abar, Bbar = oracle.discretise_trapezoid(A_, B_, delta)
        return float(np.sum(G * oracle.cascade_forward_seq(Abar, Bbar, C, D, w.u, 3)))

    out = oracle.cascade_backward(w, G)
    h = 1e-6
    for name, X, grad in (("A", A, out["dA"][0]), ("B", B, out["dB"][0])):
        for _ in range(3):
            E = rng.standard_normal(X.shape)
            if name == "A":
                fd = (loss(A + h * E, B) - loss(A - h * E, B)) / (2 * h)
            else:
                fd = (loss(A, B + h * E) - loss(A, B - h * E)) / (2 * h)
            an = float(np.sum(grad * E))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)


def test_packed_batch_matches_per_sequence():
    """The packed driver equals per-sequence calls, and sequences never mix."""
    w = wl.small_system(m=4, p=2, q=3, lengths=(5, 0, 17, 1, 33), N=3, nsys=2, seed=8)
    y = oracle.cascade_forward(w)
    for i in range(w.nseq):
        sl = w.seq(i)
        if sl.stop == sl.start:
            continue
        Abar, Bbar, C, D = oracle.system_matrices(w, int(w.sys_of_seq[i]))
        N = oracle.effective_N(w.N, sl.stop - sl.start)
        yi = oracle.brute_force_seq(Abar, Bbar, C, D, w.u[sl], 2 ** (N + 1))
        assert np.max(np.abs(y[sl] - yi)) <= 1e-12 * max(1.0, np.max(np.abs(yi)))


# --------------------------------------------------------------- counts by running the stages
def _rows_updated_by_stages(N, L, m=3, seed=0):
    """Rows each §3 stage k = 0..N changes, counted by running oracle.stage on
    random states with a power that has no zero row (every updated row then
    differs from its input), independently of the counting formulas."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((L, m)) + 2.0
    P = np.eye(m) + 0.25                           # positive entries, no zero row
    counts = []
    for k in range(N + 1):
        Vn = oracle.stage(V, P, 2 ** k)
        counts.append(int(np.sum(np.any(Vn != V, axis=1))))
        V = Vn
    return counts


@pytest.mark.parametrize("L", [0, 1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 64, 100])
@pytest.mark.parametrize("N", [0, 1, 2, 3, 4, 6, 8])
def test_matvec_count_and_effective_N_by_running_stages(N, L):
    """oracle.matvec_counts (executed) equals the rows the stages update, and
    oracle.effective_N is the last stage that updates a row (0 when none):
    lengths on both sides of every power of two catch a < / <= slip at
    2^k = L."""
    counts = _rows_updated_by_stages(N, L)
    assert oracle.matvec_counts(N, L)["executed"] == sum(counts)
    working = [k for k, c in enumerate(counts) if c > 0]
    assert oracle.effective_N(N, L) == (max(working) if working else 0)
    assert oracle.stage_count(N, L) == len(working)
    # every stage up to the last working one updates rows: no gaps
    assert working == list(range(len(working)))
