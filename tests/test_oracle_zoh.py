"""Pins of the oracle's zero-order-hold discretisation (§5) against what the
mathematics fixes: closed forms, the invertible-A formula of §5 computed by a
different route, exact finite sums for nilpotent A, the semigroup law, the
third-order agreement with the trapezoidal rule (its [1/1] Pade form), and
finite differences for the adjoint."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl

scipy_linalg = pytest.importorskip("scipy.linalg")


def rand_stable(rng, m):
    G = rng.standard_normal((m, m)) / math.sqrt(m)
    return G - 1.5 * np.eye(m)


@pytest.mark.parametrize("a,b,delta", [(-0.7, 1.3, 0.25), (2.0, -0.5, 0.1), (-30.0, 2.0, 1e-3)])
def test_scalar_closed_form(a, b, delta):
    Ab, Bb = oracle.discretise_zoh(np.array([[a]]), np.array([[b]]), delta)
    assert Ab[0, 0] == pytest.approx(math.exp(delta * a), rel=1e-14)
    assert Bb[0, 0] == pytest.approx(math.expm1(delta * a) / a * b, rel=1e-13)


def test_diagonal_closed_form():
    d = np.array([-3.0, -0.5, 0.2, 1.5])
    B = np.arange(8.0).reshape(4, 2) - 3.0
    delta = 0.4
    Ab, Bb = oracle.discretise_zoh(np.diag(d), B, delta)
    np.testing.assert_allclose(Ab, np.diag(np.exp(delta * d)), rtol=1e-14, atol=1e-15)
    want = (np.expm1(delta * d) / d)[:, None] * B
    np.testing.assert_allclose(Bb, want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_invertible_formula_of_section5(seed):
    """(delta A)^{-1} (exp(delta A) - I) (delta B), with exp(delta A) alone and a
    linear solve, against the block-exponential route."""
    rng = np.random.default_rng(seed)
    m, p = 7, 3
    A = rand_stable(rng, m)
    B = rng.standard_normal((m, p))
    delta = 0.3
    Ab, Bb = oracle.discretise_zoh(A, B, delta)
    E = scipy_linalg.expm(delta * A)
    np.testing.assert_allclose(Ab, E, rtol=1e-13, atol=1e-14)
    want = np.linalg.solve(delta * A, (E - np.eye(m)) @ (delta * B))
    np.testing.assert_allclose(Bb, want, rtol=1e-11, atol=1e-13)


def test_nilpotent_exact_sum():
    """A strictly upper triangular: exp(dA) and int exp(sA) ds B are finite sums."""
    rng = np.random.default_rng(3)
    m, p = 6, 2
    A = np.triu(rng.standard_normal((m, m)), 1)
    B = rng.standard_normal((m, p))
    delta = 0.7
    E = np.zeros((m, m))
    F = np.zeros((m, p))
    Ak = np.eye(m)
    for k in range(m):
        E += delta ** k * Ak / math.factorial(k)
        F += delta ** (k + 1) * Ak @ B / math.factorial(k + 1)
        Ak = Ak @ A
    Ab, Bb = oracle.discretise_zoh(A, B, delta)
    np.testing.assert_allclose(Ab, E, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(Bb, F, rtol=1e-13, atol=1e-14)


def test_semigroup_law():
    """Holding for 2 delta is holding twice: Abar(2d) = Abar(d)^2 and
    Bbar(2d) = Abar(d) Bbar(d) + Bbar(d)."""
    rng = np.random.default_rng(4)
    A = rand_stable(rng, 9)
    B = rng.standard_normal((9, 2))
    A1, B1 = oracle.discretise_zoh(A, B, 0.2)
    A2, B2 = oracle.discretise_zoh(A, B, 0.4)
    np.testing.assert_allclose(A2, A1 @ A1, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(B2, A1 @ B1 + B1, rtol=1e-12, atol=1e-14)


def test_third_order_agreement_with_trapezoid():
    """The trapezoidal Abar is the [1/1] Pade approximant of exp(delta A): the
    difference falls like delta^3 (HiPPO-LegS, m = 8)."""
    A = wl.hippo_legs(8)
    B = wl.hippo_legs_B(8).reshape(8, 1)
    errs = []
    for delta in (1e-2, 5e-3):
        Az, _ = oracle.discretise_zoh(A, B, delta)
        At, _ = oracle.discretise_trapezoid(A, B, delta)
        errs.append(np.linalg.norm(Az - At))
    assert 7.0 < errs[0] / errs[1] < 9.0, errs


def test_printed_factor_read_as_delta_B():
    """The printed last factor (delta A) would make Bbar independent of B."""
    rng = np.random.default_rng(5)
    A = rand_stable(rng, 4)
    B1 = rng.standard_normal((4, 1))
    _, Bb1 = oracle.discretise_zoh(A, B1, 0.3)
    _, Bb2 = oracle.discretise_zoh(A, 2.0 * B1, 0.3)
    np.testing.assert_allclose(Bb2, 2.0 * Bb1, rtol=1e-14)


def test_zoh_vjp_finite_differences():
    rng = np.random.default_rng(6)
    m, p, delta = 5, 2, 0.35
    A = rand_stable(rng, m)
    B = rng.standard_normal((m, p))
    GA = rng.standard_normal((m, m))
    GB = rng.standard_normal((m, p))
    dA, dB = oracle.discretise_zoh_vjp(A, B, delta, GA, GB)

    def f(A_, B_):
        Ab, Bb = oracle.discretise_zoh(A_, B_, delta)
        return float(np.sum(GA * Ab) + np.sum(GB * Bb))

    h = 1e-6
    for X, grad, name in ((A, dA, "A"), (B, dB, "B")):
        E = rng.standard_normal(X.shape)
        if name == "A":
            fd = (f(A + h * E, B) - f(A - h * E, B)) / (2 * h)
        else:
            fd = (f(A, B + h * E) - f(A, B - h * E)) / (2 * h)
        assert abs(fd - np.sum(grad * E)) <= 1e-7 * max(1.0, abs(fd)), (name, fd)


def test_zoh_workload_gradients_finite_differences():
    """cascade_backward through the zero-order hold: directional derivatives
    of sum(G * y) w.r.t. A and B by central differences."""
    w = wl.small_system(m=5, p=2, q=2, lengths=(23, 9), N=4, seed=8, discrete=False, delta=0.2)
    w.discretisation = "zoh"
    rng = np.random.default_rng(9)
    G = rng.standard_normal((w.rows, w.q))
    g = oracle.cascade_backward(w, G)

    def loss(A, B):
        w2 = w.subset(range(w.nseq))
        w2.A, w2.B = A, B
        return float(np.sum(G * oracle.cascade_forward(w2)))

    h = 1e-6
    for name in ("A", "B"):
        X = getattr(w, name)
        E = rng.standard_normal(X.shape)
        args_p = {"A": w.A, "B": w.B}
        args_m = {"A": w.A, "B": w.B}
        args_p[name] = X + h * E
        args_m[name] = X - h * E
        fd = (loss(**args_p) - loss(**args_m)) / (2 * h)
        an = float(np.sum(g["d" + name] * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)
