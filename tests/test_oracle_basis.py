"""Pins of the oracle's basis (LGL nodes/weights, differentiation matrix) and
of its Runge-Kutta coefficients against closed forms, quadrature exactness,
the SBP property and exact rational order conditions (CPU only)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lgl():
    rows = []
    with open(os.path.join(GOLDEN, "lgl_closed_forms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            N, nodes, weights = (s.strip() for s in line.split(";"))
            env = {"sqrt": math.sqrt}
            rows.append((int(N), [eval(x, env) for x in nodes.split(",")],
                         [eval(x, env) for x in weights.split(",")]))
    return rows


@pytest.mark.parametrize("N,nodes,weights", _golden_lgl())
def test_lgl_closed_forms(orc, N, nodes, weights):
    xi, w = orc.lgl(N)
    np.testing.assert_allclose(xi, nodes, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, weights, rtol=3e-16, atol=0)


@pytest.mark.parametrize("N", range(1, 9))
def test_lgl_quadrature_exact(orc, N):
    # LGL quadrature with N+1 points integrates polynomials of degree 2N-1 exactly
    xi, w = orc.lgl(N)
    for k in range(2 * N):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, xi ** k) - exact) < 4e-15
    # ...and not degree 2N (the Lobatto rule's defect), which fixes the node set
    k = 2 * N
    exact = 2.0 / (k + 1)
    assert abs(np.dot(w, xi ** k) - exact) > 1e-6


@pytest.mark.parametrize("N", range(1, 9))
def test_diff_matrix_exact_on_polynomials(orc, N):
    xi, _ = orc.lgl(N)
    D = orc.diff_matrix(N)
    for p in range(N + 1):
        lhs = D @ xi ** p
        rhs = p * xi ** (p - 1) if p > 0 else np.zeros_like(xi)
        assert np.max(np.abs(lhs - rhs)) < 2e-13 * max(1, N * N)


@pytest.mark.parametrize("N", range(1, 9))
def test_diff_matrix_matches_numpy_lagrange(orc, N):
    # independent construction: derivative of the interpolating polynomial of
    # each unit vector via numpy's polynomial fitting
    xi, _ = orc.lgl(N)
    D = orc.diff_matrix(N)
    V = np.polynomial.legendre.legvander(xi, N)
    Vd = np.stack([np.polynomial.legendre.legval(xi, np.polynomial.legendre.legder(np.eye(N + 1)[k]))
                   for k in range(N + 1)], axis=1)
    D_ref = Vd @ np.linalg.inv(V)
    assert np.max(np.abs(D - D_ref)) < 1e-12 * max(1, N * N)


@pytest.mark.parametrize("N", range(1, 9))
def test_sbp_property(orc, N):
    # summation by parts: W D + (W D)^T = B = diag(-1, 0, ..., 0, 1)
    xi, w = orc.lgl(N)
    D = orc.diff_matrix(N)
    Q = np.diag(w) @ D
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    assert np.max(np.abs(Q + Q.T - B)) < 1e-14 * max(1, N)
    # D~ = 2 D - W^-1 B has zero diagonal and W D~ is skew-symmetric
    Dt = 2 * D - np.diag(1.0 / w) @ B
    assert np.max(np.abs(np.diag(Dt))) < 1e-13 * max(1, N * N)
    S = np.diag(w) @ Dt
    assert np.max(np.abs(S + S.T)) < 1e-13 * max(1, N)


@pytest.mark.parametrize("N", range(1, 9))
def test_dtilde(orc, N):
    # the long double Dt agrees with 2 D - W^-1 B from the double basis, has a
    # zero diagonal to long double accuracy and W Dt is skew-symmetric
    xi, w = orc.lgl(N)
    D = orc.diff_matrix(N)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    Dt = orc.dtilde(N)
    assert np.max(np.abs(Dt - (2 * D - np.diag(1 / w) @ B))) < 1e-13 * max(1, N * N)
    assert np.max(np.abs(np.diag(Dt))) < 1e-17 * max(1, N * N)
    S = np.diag(w) @ Dt
    assert np.max(np.abs(S + S.T)) < 4e-15 * max(1, N)


def _golden_ck():
    A, B, c = [], [], []
    with open(os.path.join(GOLDEN, "carpenter_kennedy_1994.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            _, a, b, cc = (s.strip() for s in line.split(";"))
            A.append(Fraction(a))
            B.append(Fraction(b))
            c.append(Fraction(cc))
    return A, B, c


def test_lsrk_coefficients_match_publication(orc):
    A, B, c = orc.lsrk_coefficients()
    Ag, Bg, cg = _golden_ck()
    for x, g in zip(list(A) + list(B) + list(c), Ag + Bg + cg):
        assert x == float(g)


def _stability_polynomial(A, B):
    """Apply the 2N-storage scheme to y' = z y with exact rational arithmetic
    treating z as a formal variable: return the coefficients of R(z)."""
    # polynomials in z as lists of Fractions
    def add(p, q):
        n = max(len(p), len(q))
        return [(p[i] if i < len(p) else 0) + (q[i] if i < len(q) else 0) for i in range(n)]

    def scal(a, p):
        return [a * x for x in p]

    def mulz(p):
        return [Fraction(0)] + p

    u = [Fraction(1)]
    k = [Fraction(0)]
    for s in range(5):
        k = add(scal(A[s], k), mulz(u))  # dt = 1, rhs(u) = z u
        u = add(u, scal(B[s], k))
    return u


def test_lsrk_order_conditions(orc):
    # the published digits give R(z) = sum_{j<=4} z^j / j! + O(z^5): order 4
    A, B, _ = orc.lsrk_coefficients()
    R = _stability_polynomial([Fraction(a) for a in A], [Fraction(b) for b in B])
    for j in range(5):
        assert abs(float(R[j]) - 1.0 / math.factorial(j)) < 1e-12, (j, float(R[j]))
    assert abs(float(R[5]) - 1.0 / 120.0) > 1e-4  # genuinely a 4th-order method
    # the stage times are the partial sums implied by the scheme on y' = 1
    _, _, c = orc.lsrk_coefficients()
    t, kk = 0.0, 0.0
    for s in range(5):
        assert abs(t - c[s]) < 1e-12
        kk = A[s] * kk + 1.0
        t = t + B[s] * kk


def test_lsrk_observed_order_four(orc):
    # y' = -y + cos t, y(0) = 1: exact y = (e^-t + cos t + sin t)/2; run the
    # oracle's stage update with rhs values computed here
    A, B, c = orc.lsrk_coefficients()

    def solve(nsteps, T=2.0):
        dt = T / nsteps
        y = np.array([1.0])
        k = np.zeros(1)
        t = 0.0
        for _ in range(nsteps):
            for s in range(5):
                du = np.array([-y[0] + math.cos(t + c[s] * dt)])
                orc.rk_stage(y, k, du, A[s], B[s], dt)
            t += dt
        return y[0]

    exact = 0.5 * (math.exp(-2.0) + math.cos(2.0) + math.sin(2.0))
    e1 = abs(solve(10) - exact)
    e2 = abs(solve(20) - exact)
    e3 = abs(solve(40) - exact)
    for a, b in ((e1, e2), (e2, e3)):
        assert 3.7 < math.log2(a / b) < 4.4


def test_extended_precision_build_agrees(orc):
    # the long double build of the oracle evaluates the same operator: on a
    # well-conditioned random state it agrees with the double build to a few
    # ulps; on the smooth 8^3 density wave the double build's rounding shows
    from paper_2108_06476_gb300 import workloads as W
    for (d, N, n, vf, sf) in ((3, 2, (2, 2, 2), 1, 2), (2, 3, (3, 2), 0, 0), (3, 3, (2, 1, 2), 0, 1)):
        u = W.random_state(d, N, n, seed=3)
        a = orc.rhs(d, N, n, W.box(d), u, vflux=vf, sflux=sf)
        b = orc.rhs_extended(d, N, n, W.box(d), u, vflux=vf, sflux=sf)
        assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(b)
    xi, _ = orc.lgl(3)
    u = W.density_wave(3, 3, (8, 8, 8), W.box(3), xi)
    a = orc.rhs(3, 3, (8, 8, 8), W.box(3), u)
    b = orc.rhs_extended(3, 3, (8, 8, 8), W.box(3), u)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
