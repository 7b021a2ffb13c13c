"""Pins of the 3D ideal MHD oracle (the weak-form DGSEM with the Powell term
and the local Lax-Friedrichs flux used for the Alfven-wave runs of Sec. 3.1)
against what the physics and the mathematics fix: the hydrodynamic limit
(the pinned Euler oracle), rotational invariance, the characteristic speeds
of the flux Jacobian, free-stream preservation, conservation, the discrete
divergence theorem, the exact circularly polarised Alfven wave and the exact
solution of the Powell system that advects a divergence error. CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2108_06476_gb300 import workloads as W

G = 5.0 / 3.0
BOX = W.box(3)


def rand_state(rng, n=1):
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.uniform(-0.5, 0.5, (3, n))
    p = rng.uniform(0.5, 3.0, n)
    B = rng.uniform(-1.0, 1.0, (3, n))
    E = p / (G - 1) + 0.5 * rho * (v * v).sum(0) + 0.5 * (B * B).sum(0)
    return np.stack([rho, *(rho * v), E, *B], axis=1)


def jacobian(d, u, rel=1e-6):
    J = np.zeros((8, 8))
    for q in range(8):
        h = rel * max(1.0, abs(u[q]))
        up, um = u.copy(), u.copy()
        up[q] += h
        um[q] -= h
        J[:, q] = (orc.mhd_flux(d, up, G) - orc.mhd_flux(d, um, G)) / (2 * h)
    return J


def weights3(N):
    _, w = orc.lgl(N)
    return np.einsum("i,j,k->kji", w, w, w).reshape(-1)


def as_grid(u, N, n):
    """(nz, ny, nx, 8, k, j, i) view of a state in the element-major layout."""
    np1 = N + 1
    return u.reshape(n[2], n[1], n[0], 8, np1, np1, np1)


def swap_xy(u, N, n):
    g = as_grid(u, N, n).transpose(0, 2, 1, 3, 4, 6, 5)[:, :, :, [0, 2, 1, 3, 4, 6, 5, 7]]
    return np.ascontiguousarray(g).reshape(-1)


def swap_xz(u, N, n):
    g = as_grid(u, N, n).transpose(2, 1, 0, 3, 6, 5, 4)[:, :, :, [0, 3, 2, 1, 4, 7, 6, 5]]
    return np.ascontiguousarray(g).reshape(-1)


def test_flux_is_euler_flux_without_field():
    rng = np.random.default_rng(1)
    for u in rand_state(rng, 20):
        u[5:] = 0.0
        for d in range(3):
            f = orc.mhd_flux(d, u, G)
            e = orc.two_point(20, 3, d, u[:5], u[:5], G)
            assert np.allclose(f[:5], e, rtol=1e-14, atol=1e-14)
            assert np.all(f[5:] == 0.0)


def test_flux_is_rotation_invariant():
    """n . F(u) = R^T f_x(R u) for the rotation R taking n to e_x, with the
    vector parts (momentum, field) rotated: every direction's flux and the
    magnetic cross terms against one another."""
    rng = np.random.default_rng(2)
    for u in rand_state(rng, 10):
        R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        nvec = R[0]
        ur = u.copy()
        ur[1:4] = R @ u[1:4]
        ur[5:8] = R @ u[5:8]
        fx = orc.mhd_flux(0, ur, G)
        back = fx.copy()
        back[1:4] = R.T @ fx[1:4]
        back[5:8] = R.T @ fx[5:8]
        fn = sum(nvec[d] * orc.mhd_flux(d, u, G) for d in range(3))
        assert np.allclose(fn, back, rtol=1e-12, atol=1e-12)


def test_fast_speed_bounds_the_flux_jacobian_spectrum():
    """The spectrum of df_d/du holds v_d +- c_f, v_d +- c_a (c_a = |B_d| /
    sqrt(rho)), and nothing beyond |v_d| + c_f."""
    rng = np.random.default_rng(3)
    for u in rand_state(rng, 12):
        for d in range(3):
            lam = np.linalg.eigvals(jacobian(d, u))
            assert np.max(np.abs(lam.imag)) < 1e-5
            lam = np.sort(lam.real)
            vd = u[1 + d] / u[0]
            cf = orc.mhd_fast_speed(d, u, G)
            ca = abs(u[5 + d]) / math.sqrt(u[0])
            for s in (vd + cf, vd - cf, vd + ca, vd - ca):
                assert np.min(np.abs(lam - s)) < 1e-5
            assert abs(np.max(np.abs(lam)) - (abs(vd) + cf)) < 1e-5


def test_llf_is_consistent_and_dissipates_at_the_largest_speed():
    """Dissipation lambda/2 (u_R - u_L) with lambda = max|v_n| + max c_f over
    the two states, c_f read off the flux Jacobian's spectral radius."""
    rng = np.random.default_rng(4)
    us = rand_state(rng, 16)
    for uL, uR in zip(us[:8], us[8:]):
        for d in range(3):
            assert np.array_equal(orc.mhd_llf(d, uL, uL, G), orc.mhd_flux(d, uL, G))
            vn = [abs(x[1 + d] / x[0]) for x in (uL, uR)]
            cf = [np.max(np.abs(np.linalg.eigvals(jacobian(d, x)))) - a for x, a in
                  zip((uL, uR), vn)]
            rad = max(vn) + max(cf)
            assert rad >= max(a + c for a, c in zip(vn, cf))
            diss = 0.5 * (orc.mhd_flux(d, uL, G) + orc.mhd_flux(d, uR, G)) - orc.mhd_llf(
                d, uL, uR, G)
            assert np.allclose(diss, 0.5 * rad * (uR - uL), rtol=1e-5, atol=1e-6)


def test_hll_consistency_upwinding_and_llf_limit():
    """HLL: consistent; the upwind flux when every signal moves one way; and
    equal to LLF when both normal velocities vanish (then S_R = -S_L =
    max(c_f,L, c_f,R) = the LLF speed)."""
    rng = np.random.default_rng(11)
    us = rand_state(rng, 16)
    for uL, uR in zip(us[:8], us[8:]):
        for d in range(3):
            assert np.allclose(orc.mhd_hll(d, uL, uL, G), orc.mhd_flux(d, uL, G), rtol=1e-14,
                               atol=1e-14)
            for sgn, side in ((1.0, uL), (-1.0, uR)):
                a, b = uL.copy(), uR.copy()
                for x in (a, b):  # normal velocity 6, beyond every fast speed
                    e_kin = 0.5 * (x[1:4] ** 2).sum() / x[0]
                    x[1 + d] = sgn * 6.0 * x[0]
                    x[4] += 0.5 * (x[1:4] ** 2).sum() / x[0] - e_kin
                want = orc.mhd_flux(d, a if sgn > 0 else b, G)
                assert np.array_equal(orc.mhd_hll(d, a, b, G), want)
            a, b = uL.copy(), uR.copy()
            for x in (a, b):
                x[4] -= 0.5 * x[1 + d] ** 2 / x[0]
                x[1 + d] = 0.0
            assert np.allclose(orc.mhd_hll(d, a, b, G), orc.mhd_llf(d, a, b, G),
                               rtol=1e-13, atol=1e-13)


def test_surface_flux_enters_through_the_lifting():
    """Between the LLF and the HLL operator only the lifting of the face flux
    changes: at an x-face node off the y and z faces the rhs differs by
    -(2/h) (F_LLF - F_HLL)/w_N at i = N and +(2/h) (F_LLF - F_HLL)/w_0 at
    i = 0, F evaluated on the two traces."""
    N, n = 2, (3, 2, 2)
    u = W.mhd_random_state(N, n, seed=12, gamma=G)
    d = (orc.mhd_rhs(N, n, BOX, u, G, True, sflux="llf")
         - orc.mhd_rhs(N, n, BOX, u, G, True, sflux="hll"))
    g = as_grid(u, N, n)
    dg = as_grid(d, N, n)
    _, w = orc.lgl(N)
    h = 2.0 / n[0]
    for ex in range(n[0]):
        er = (ex + 1) % n[0]
        uL, uR = g[0, 0, ex, :, 1, 1, N], g[0, 0, er, :, 1, 1, 0]
        dF = orc.mhd_llf(0, uL, uR, G) - orc.mhd_hll(0, uL, uR, G)
        assert np.allclose(dg[0, 0, ex, :, 1, 1, N], -(2 / h) * dF / w[N], rtol=1e-10, atol=1e-11)
        assert np.allclose(dg[0, 0, er, :, 1, 1, 0], (2 / h) * dF / w[0], rtol=1e-10, atol=1e-11)
        assert np.max(np.abs(dF)) > 1e-3


@pytest.mark.parametrize("sflux", ["llf", "hll"])
@pytest.mark.parametrize("powell", [False, True])
def test_free_stream(powell, sflux):
    N, n = 3, (2, 3, 2)
    rng = np.random.default_rng(5)
    u0 = rand_state(rng, 1)[0]
    P = (N + 1) ** 3
    u = np.tile(np.repeat(u0, P), int(np.prod(n)))
    du = orc.mhd_rhs(N, n, BOX, u, G, powell, sflux=sflux)
    assert np.max(np.abs(du)) < 1e-12 * np.max(np.abs(u))


@pytest.mark.parametrize("sflux", ["llf", "hll"])
def test_conservation_without_powell_term(sflux):
    """The conservative part conserves all eight integrals; the Powell term
    leaves mass conserved and moves momentum when div B != 0."""
    N, n = 3, (2, 3, 2)
    u = W.mhd_random_state(N, n, seed=6, gamma=G)
    w = weights3(N)
    P = (N + 1) ** 3
    tot = lambda du: np.einsum("evp,p->v", du.reshape(-1, 8, P), w)
    c = tot(orc.mhd_rhs(N, n, BOX, u, G, powell=False, sflux=sflux))
    assert np.max(np.abs(c)) < 1e-11
    c = tot(orc.mhd_rhs(N, n, BOX, u, G, powell=True, sflux=sflux))
    assert abs(c[0]) < 1e-11
    assert np.max(np.abs(c[1:4])) > 1e-3


@pytest.mark.parametrize("which", ["xy", "xz"])
def test_axis_swap_equivariance(which):
    N, n = 3, (3, 2, 2)
    u = W.mhd_random_state(N, n, seed=7, gamma=G)
    f = swap_xy if which == "xy" else swap_xz
    m = (n[1], n[0], n[2]) if which == "xy" else (n[2], n[1], n[0])
    a = orc.mhd_rhs(N, m, BOX, f(u, N, n), G, True)
    b = f(orc.mhd_rhs(N, n, BOX, u, G, True), N, n)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-11 * np.max(np.abs(b)))


def divb_of(N, n, u):
    """The discrete div B the Powell term multiplies, read back from the
    difference of the two operators in the x-momentum component
    (Phi_1 = B_x)."""
    P = (N + 1) ** 3
    d = (orc.mhd_rhs(N, n, BOX, u, G, True) - orc.mhd_rhs(N, n, BOX, u, G, False))
    d = d.reshape(-1, 8, P)
    return -d[:, 1] / u.reshape(-1, 8, P)[:, 5]


def test_divergence_theorem_per_element():
    """Integrated over an element with the LGL quadrature, the discrete
    div B equals the flux through the element's faces of the averaged
    interface values of B_n (the SBP property of D)."""
    N, n = 3, (2, 2, 3)
    rng = np.random.default_rng(8)
    u = W.mhd_random_state(N, n, seed=8, gamma=G)
    g = as_grid(u, N, n).copy()
    g[:, :, :, 5] = 0.6 + 0.3 * rng.uniform(-1, 1, size=g[:, :, :, 5].shape)  # B_x away from 0
    u = g.reshape(-1)
    div = divb_of(N, n, u)
    _, w = orc.lgl(N)
    h = [(BOX[2 * k + 1] - BOX[2 * k]) / n[k] for k in range(3)]
    wv = weights3(N) * h[0] * h[1] * h[2] / 8
    B = as_grid(u, N, n)[:, :, :, 5:8]  # [ez, ey, ex, comp, k, j, i]
    for ez in range(n[2]):
        for ey in range(n[1]):
            for ex in range(n[0]):
                e = ex + n[0] * (ey + n[1] * ez)
                lhs = np.dot(wv, div[e])
                rhs = 0.0
                # x faces: weights over (k, j)
                wa = np.outer(w, w) * h[1] * h[2] / 4
                R = B[ez, ey, (ex + 1) % n[0], 0, :, :, 0]
                L = B[ez, ey, (ex - 1) % n[0], 0, :, :, N]
                me = B[ez, ey, ex, 0]
                rhs += np.sum(wa * 0.5 * (me[:, :, N] + R)) - np.sum(wa * 0.5 * (me[:, :, 0] + L))
                wa = np.outer(w, w) * h[0] * h[2] / 4
                R = B[ez, (ey + 1) % n[1], ex, 1, :, 0, :]
                L = B[ez, (ey - 1) % n[1], ex, 1, :, N, :]
                me = B[ez, ey, ex, 1]
                rhs += np.sum(wa * 0.5 * (me[:, N, :] + R)) - np.sum(wa * 0.5 * (me[:, 0, :] + L))
                wa = np.outer(w, w) * h[0] * h[1] / 4
                R = B[(ez + 1) % n[2], ey, ex, 2, 0, :, :]
                L = B[(ez - 1) % n[2], ey, ex, 2, N, :, :]
                me = B[ez, ey, ex, 2]
                rhs += np.sum(wa * 0.5 * (me[N] + R)) - np.sum(wa * 0.5 * (me[0] + L))
                assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


def test_divergence_is_exact_for_continuous_piecewise_quadratics():
    """B_x = (x - x_L)(x_R - x) in every element (continuous and periodic):
    the surface terms vanish and div B is the exact derivative x_L + x_R - 2x."""
    N, n = 3, (4, 2, 2)
    xi, _ = orc.lgl(N)
    X = W.node_coordinates(3, N, n, BOX, xi)
    h = 2.0 / n[0]
    ne = int(np.prod(n))
    ex = np.arange(ne) % n[0]
    xl = (-1.0 + ex * h)[:, None] * np.ones_like(X[0])
    xr = xl + h
    u = W.mhd_random_state(N, n, seed=9, gamma=G).reshape(ne, 8, -1)
    bx = 1.0 + (X[0] - xl) * (xr - X[0])
    u[:, 5] = bx
    u[:, 6] = 0.0
    u[:, 7] = 0.0
    rho = u[:, 0]
    v = u[:, 1:4] / rho[:, None]
    p = 1.0
    u[:, 4] = p / (G - 1) + 0.5 * rho * (v * v).sum(1) + 0.5 * bx * bx
    div = divb_of(N, n, u.reshape(-1))
    assert np.allclose(div, xl + xr - 2 * X[0], rtol=0, atol=1e-12)


def exact_time_derivative(N, n, t, delta=1e-5):
    xi, _ = orc.lgl(N)
    a = W.alfven_wave(N, n, xi, t + delta, gamma=G)
    b = W.alfven_wave(N, n, xi, t - delta, gamma=G)
    return (a - b) / (2 * delta)


@pytest.mark.parametrize("powell,sflux", [(False, "llf"), (True, "llf"), (True, "hll")])
def test_alfven_wave_rhs_converges(powell, sflux):
    """rhs(u) of the exact wave approaches du/dt, spectrally in N."""
    n = (2, 2, 2)
    errs = []
    for N in (3, 5, 7):
        xi, _ = orc.lgl(N)
        u = W.alfven_wave(N, n, xi, 0.3, gamma=G)
        du = orc.mhd_rhs(N, n, BOX, u, G, powell, sflux=sflux)
        errs.append(np.max(np.abs(du - exact_time_derivative(N, n, 0.3))))
    assert errs[0] < 0.2 and errs[1] < 1e-2 and errs[2] < 2e-4
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5


def test_alfven_wave_solution_converges():
    """Five-stage LSRK steps to t = 0.1 land on the exact wave, with the
    error falling spectrally in N."""
    n = (2, 2, 2)
    errs = []
    for N in (3, 5):
        xi, _ = orc.lgl(N)
        u = W.alfven_wave(N, n, xi, 0.0, gamma=G)
        T = 0.1
        dt0 = orc.mhd_max_dt(N, n, BOX, u, 0.5, G)
        steps = int(math.ceil(T / dt0))
        for _ in range(steps):
            u = orc.mhd_lsrk_step(N, n, BOX, u, T / steps, G, True)
        errs.append(np.max(np.abs(u - W.alfven_wave(N, n, xi, T, gamma=G))))
    assert errs[0] < 3e-2 and errs[1] < errs[0] / 10


def test_powell_system_advects_a_divergence_error():
    """rho, v = (V, 0, 0), p constant and B = (b(x), 0, 0): the Powell system
    moves b with the flow (db/dt = -V b') with no force on the fluid, and
    E carries b^2/2 along; the conservative system leaves b in place and
    pushes the fluid with d(b^2/2)/dx."""
    n = (3, 2, 2)
    V, p = 0.4, 1.0
    for N, tol in ((4, 2e-2), (7, 2e-4)):
        xi, _ = orc.lgl(N)
        X = W.node_coordinates(3, N, n, BOX, xi)
        b = 0.5 + 0.2 * np.sin(np.pi * X[0])
        db = 0.2 * np.pi * np.cos(np.pi * X[0])
        ne = X.shape[1]
        u = np.zeros((ne, 8, X.shape[2]))
        u[:, 0] = 1.0
        u[:, 1] = V
        u[:, 4] = p / (G - 1) + 0.5 * V * V + 0.5 * b * b
        u[:, 5] = b
        du = orc.mhd_rhs(N, n, BOX, u.reshape(-1), G, True).reshape(ne, 8, -1)
        want = np.zeros_like(du)
        want[:, 4] = -V * b * db
        want[:, 5] = -V * db
        assert np.max(np.abs(du - want)) < tol
        du = orc.mhd_rhs(N, n, BOX, u.reshape(-1), G, False).reshape(ne, 8, -1)
        want = np.zeros_like(du)
        want[:, 1] = b * db
        want[:, 4] = 0.0
        assert np.max(np.abs(du - want)) < tol


def test_max_dt_uses_the_fast_speed():
    """For a constant state the CFL step is cfl 2 / ((N+1) sum_r (2/h_r) rho_r),
    rho_r the spectral radius of the flux Jacobian in direction r."""
    N, n = 4, (2, 3, 4)
    rng = np.random.default_rng(10)
    u0 = rand_state(rng, 1)[0]
    P = (N + 1) ** 3
    u = np.tile(np.repeat(u0, P), int(np.prod(n)))
    rad = [np.max(np.abs(np.linalg.eigvals(jacobian(d, u0)))) for d in range(3)]
    want = 0.5 * 2 / ((N + 1) * sum(2.0 / (2.0 / n[d]) * rad[d] for d in range(3)))
    assert abs(orc.mhd_max_dt(N, n, BOX, u, 0.5, G) - want) < 1e-6 * want


def test_alfven_wave_is_an_exact_solution():
    """The wave of the inputs module solves ideal MHD exactly (symbolic
    residual of du/dt + div F with F written from the MHD equations)."""
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t", real=True)
    g, A, p0 = sp.Rational(5, 3), sp.Rational(1, 10), sp.Rational(1, 10)
    nv = sp.Matrix([1, 1, 1]) / sp.sqrt(3)
    e1 = sp.Matrix([1, -1, 0]) / sp.sqrt(2)
    e2 = nv.cross(e1)
    phi = sp.pi * (x + y + z) - sp.pi * sp.sqrt(3) * t
    B = nv + A * (sp.sin(phi) * e1 + sp.cos(phi) * e2)
    v = -A * (sp.sin(phi) * e1 + sp.cos(phi) * e2)
    b2 = B.dot(B)
    E = p0 / (g - 1) + v.dot(v) / 2 + b2 / 2
    U = [1] + list(v) + [E] + list(B)
    X = [x, y, z]
    res = [sp.diff(U[q], t) for q in range(8)]
    for d in range(3):
        pt = p0 + b2 / 2
        F = [v[d]] + [v[d] * v[k] - B[d] * B[k] + (pt if k == d else 0) for k in range(3)]
        F += [v[d] * (E + pt) - B[d] * v.dot(B)] + [v[d] * B[k] - B[d] * v[k] for k in range(3)]
        res = [res[q] + sp.diff(F[q], X[d]) for q in range(8)]
    assert all(sp.simplify(r) == 0 for r in res)
    # and the numeric generator matches the symbolic state at a few nodes
    xi, _ = orc.lgl(2)
    u = W.alfven_wave(2, (2, 1, 1), xi, 0.25, gamma=G).reshape(2, 8, -1)
    Xn = W.node_coordinates(3, 2, (2, 1, 1), BOX, xi)
    f = sp.lambdify((x, y, z, t), U, "math")
    for e in range(2):
        for node in (0, 7, 26):
            want = f(Xn[0, e, node], Xn[1, e, node], Xn[2, e, node], 0.25)
            assert np.allclose(u[e, :, node], want, rtol=1e-13, atol=1e-13)


# ---- entropy-conservative flux differencing (the paper's second MHD solver) ----

def entropy_parts(u, n):
    """Entropy variables w, theta = w . Phi and the potential psi_n =
    rho v_n + beta v_n |B|^2 of a state (beta = rho / (2p), s = ln p - gamma
    ln rho), from the entropy -rho s / (gamma - 1)."""
    rho, v, B = u[0], u[1:4] / u[0], u[5:8]
    p = (G - 1) * (u[4] - 0.5 * rho * v @ v - 0.5 * B @ B)
    beta = rho / (2 * p)
    s = np.log(p) - G * np.log(rho)
    w = np.array([(G - s) / (G - 1) - beta * v @ v, *(2 * beta * v), -2 * beta, *(2 * beta * B)])
    return w, 2 * beta * (v @ B), rho * v[n] + beta * v[n] * (B @ B)


def test_ec_flux_consistency_and_symmetry():
    rng = np.random.default_rng(21)
    us = rand_state(rng, 16)
    for uL, uR in zip(us[:8], us[8:]):
        for d in range(3):
            assert np.allclose(orc.mhd_flux_ec(d, uL, uL, G), orc.mhd_flux(d, uL, G), rtol=1e-14,
                               atol=1e-14)
            assert np.allclose(orc.mhd_flux_ec(d, uL, uR, G), orc.mhd_flux_ec(d, uR, uL, G),
                               rtol=1e-14, atol=1e-14)
            assert orc.mhd_flux_ec(d, uL, uR, G)[5 + d] == 0.0


def test_ec_flux_satisfies_the_discrete_entropy_condition():
    """[[w]] . f# + {B_n} [[theta]] = [[psi_n]] for random pairs (the
    condition under which flux differencing with the Powell term in split
    form conserves entropy); the central flux does not satisfy it."""
    rng = np.random.default_rng(22)
    us = rand_state(rng, 80)
    worst, central = 0.0, 0.0
    for uL, uR in zip(us[:40], us[40:]):
        for d in range(3):
            wL, tL, pL = entropy_parts(uL, d)
            wR, tR, pR = entropy_parts(uR, d)
            bn = 0.5 * (uL[5 + d] + uR[5 + d])
            scale = np.abs(wR - wL) @ np.abs(orc.mhd_flux_ec(d, uL, uR, G)) + abs(pR) + abs(pL)
            r = (wR - wL) @ orc.mhd_flux_ec(d, uL, uR, G) + bn * (tR - tL) - (pR - pL)
            worst = max(worst, abs(r) / scale)
            fc = 0.5 * (orc.mhd_flux(d, uL, G) + orc.mhd_flux(d, uR, G))
            central = max(central, abs((wR - wL) @ fc + bn * (tR - tL) - (pR - pL)) / scale)
    assert worst < 1e-14
    assert central > 1e-3


def entropy_rate(N, n, u, du):
    P = (N + 1) ** 3
    wq = weights3(N) * np.prod([(BOX[2 * k + 1] - BOX[2 * k]) / n[k] / 2 for k in range(3)])
    U, D = u.reshape(-1, 8, P), du.reshape(-1, 8, P)
    tot, mag = 0.0, 0.0
    for e in range(U.shape[0]):
        for i in range(P):
            w, _, _ = entropy_parts(U[e, :, i], 0)
            tot += wq[i] * (w @ D[e, :, i])
            mag += wq[i] * np.abs(w) @ np.abs(D[e, :, i])
    return tot, mag


def test_ec_rhs_conserves_entropy():
    """EC volume and surface fluxes with the Powell term: sum_nodes W w . du
    = 0; without the Powell term, or with the central volume flux, it is
    not; with LLF faces it decreases."""
    N, n = 3, (2, 2, 2)
    u = W.mhd_random_state(N, n, seed=23, gamma=G)
    tot, mag = entropy_rate(N, n, u, orc.mhd_rhs(N, n, BOX, u, G, True, vflux="ec", sflux="ec"))
    assert abs(tot) < 1e-13 * mag
    tot, mag = entropy_rate(N, n, u, orc.mhd_rhs(N, n, BOX, u, G, False, vflux="ec", sflux="ec"))
    assert abs(tot) > 1e-6 * mag
    tot, mag = entropy_rate(N, n, u, orc.mhd_rhs(N, n, BOX, u, G, True, vflux="central",
                                                 sflux="ec"))
    assert abs(tot) > 1e-6 * mag
    tot, mag = entropy_rate(N, n, u, orc.mhd_rhs(N, n, BOX, u, G, True, vflux="ec", sflux="llf"))
    assert tot < -1e-6 * mag


@pytest.mark.parametrize("sflux", ["ec", "llf"])
def test_ec_free_stream_and_conservation(sflux):
    N, n = 3, (2, 3, 2)
    rng = np.random.default_rng(24)
    u0 = rand_state(rng, 1)[0]
    P = (N + 1) ** 3
    uc = np.tile(np.repeat(u0, P), int(np.prod(n)))
    du = orc.mhd_rhs(N, n, BOX, uc, G, True, vflux="ec", sflux=sflux)
    assert np.max(np.abs(du)) < 1e-12 * np.max(np.abs(uc))
    u = W.mhd_random_state(N, n, seed=25, gamma=G)
    w = weights3(N)
    c = np.einsum("evp,p->v", orc.mhd_rhs(N, n, BOX, u, G, False, vflux="ec",
                                          sflux=sflux).reshape(-1, 8, P), w)
    assert np.max(np.abs(c)) < 1e-11


def test_ec_alfven_wave_rhs_converges():
    n = (2, 2, 2)
    errs = []
    for N in (3, 5, 7):
        xi, _ = orc.lgl(N)
        u = W.alfven_wave(N, n, xi, 0.3, gamma=G)
        du = orc.mhd_rhs(N, n, BOX, u, G, True, vflux="ec", sflux="ec")
        errs.append(np.max(np.abs(du - exact_time_derivative(N, n, 0.3))))
    assert errs[0] < 0.2 and errs[1] < 1e-2 and errs[2] < 2e-4
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5
