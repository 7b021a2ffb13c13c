"""Pins of the curvilinear-mesh oracle (the warped periodic box of the paper's
performance benchmark, Sec. 3.1) against what the mathematics fixes: the
Cartesian limit, the discrete metric identities, the box volume, free-stream
preservation, conservation, entropy conservation of the EC fluxes, the
manufactured solution's source term (derived symbolically here) and the
convergence order on the warped mesh. CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2108_06476_gb300 import workloads as W

GAMMA = 1.4


def weights3(N):
    _, w = orc.lgl(N)
    return np.einsum("i,j,k->kji", w, w, w).reshape(-1)  # node index i fastest


def divergence(N, g):
    """sum_r d/dxi^r (J a^r)_n per element and component, with the nodal D."""
    xi, _ = orc.lgl(N)
    D = orc.diff_matrix(N)
    np1 = N + 1
    Ja = g.Ja.reshape(g.Ja.shape[0], 3, 3, np1, np1, np1)  # [e][r][n][k][j][i]
    out = np.einsum("ia,enkja->enkji", D, Ja[:, 0])
    out += np.einsum("ja,enkai->enkji", D, Ja[:, 1])
    out += np.einsum("ka,enaji->enkji", D, Ja[:, 2])
    return out


def entropy_vars(u):
    rho, m, E = u[0], u[1:4], u[4]
    v = m / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * (v * v).sum(axis=0))
    s = np.log(p) - GAMMA * np.log(rho)
    return np.stack([(GAMMA - s) / (GAMMA - 1) - 0.5 * rho * (v * v).sum(axis=0) / p,
                     *(rho * v / p), -rho / p])


@pytest.mark.parametrize("N,n", [(2, (3, 2, 2)), (3, (2, 2, 3))])
def test_cartesian_limit_gives_the_cartesian_operator(N, n):
    g = orc.CurvedGeometry(N, n, warp=0.0)
    h = [2.0 / k for k in n]
    for r in range(3):
        scale = np.prod([h[k] / 2 for k in range(3) if k != r])
        assert np.allclose(g.Ja[:, r, r], scale, rtol=5e-14, atol=0)
        for c in range(3):
            if c != r:
                assert np.abs(g.Ja[:, r, c]).max() < 5e-14 * scale
    assert np.allclose(g.J, np.prod([x / 2 for x in h]), rtol=5e-14, atol=0)
    u = W.random_state(3, N, n, seed=5)
    for vf, sf in ((0, 0), (0, 1), (1, 3), (2, 2)):
        ref = orc.rhs(3, N, n, W.box(3), u, vflux=vf, sflux=sf)
        got = orc.curved_rhs(g, u, vflux=vf, sflux=sf)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), (vf, sf)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_metric_identities_and_volume(N):
    # the paper's mesh: 4^3 elements (coarser ones of low degree fold, J < 0)
    n = (4, 4, 4)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    scale = np.abs(g.Ja).max()
    # roundoff of the nodal derivatives grows like |D| ~ N^2, twice applied
    assert np.abs(divergence(N, g)).max() < 1e-15 * N ** 4 * scale
    assert g.J.min() > 0
    vol = (g.J * weights3(N)).sum()
    assert abs(vol - 8.0) < 1e-12  # the warping maps the box onto itself
    xi, _ = orc.lgl(N)
    X = W.warped_node_coordinates(N, n, xi, 0.15)
    assert np.abs(np.moveaxis(X, 0, 1) - g.X).max() < 1e-15


def jacobian_det(N, g):
    """det(dX/dxi) at every node from the nodal derivatives of X (numpy)."""
    D = orc.diff_matrix(N)
    np1 = N + 1
    X = g.X.reshape(-1, 3, np1, np1, np1)  # [e][k][zeta][eta][xi]
    d_xi = np.einsum("ia,ekcba->ekcbi", D, X)
    d_eta = np.einsum("jb,ekcba->ekcja", D, X)
    d_zeta = np.einsum("zc,ekcba->ekzba", D, X)
    A = np.stack([d_xi, d_eta, d_zeta], axis=-1)  # [e][k][zeta][eta][xi][r]
    return np.linalg.det(np.moveaxis(A, 1, -2)).reshape(g.J.shape)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_jacobian_is_the_determinant_of_the_mapping_derivative(N):
    g = orc.CurvedGeometry(N, (4, 3, 2), warp=0.15)
    ref = jacobian_det(N, g)
    assert np.abs(g.J - ref).max() < 1e-13 * np.abs(ref).max()


def test_face_metric_terms_agree_across_interior_faces():
    # the curl form builds (J a^r) at a face from the face's own nodes, so the
    # two elements sharing an interior face compute the same normal vector
    N, n = 3, (3, 3, 3)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    np1 = N + 1
    Ja = g.Ja.reshape(n[2], n[1], n[0], 3, 3, np1, np1, np1)
    left = Ja[:, :, 0, 0, :, :, :, N]   # element x = 0, its i = N face, r = 0
    right = Ja[:, :, 1, 0, :, :, :, 0]  # element x = 1, its i = 0 face
    assert np.abs(left - right).max() < 1e-15 * np.abs(Ja).max() * 10


@pytest.mark.parametrize("sf", [0, 1, 2, 3])
def test_free_stream_preservation_on_the_warped_mesh(sf):
    N, n = 3, (3, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.uniform_state(3, N, n)
    du = orc.curved_rhs(g, u, vflux=0, sflux=sf)
    # the flux terms are of size |f| |J a| / J ~ (p + rho v^2) (2/h)
    assert np.abs(du).max() < 1e-11 * 7.0 * 2.0


@pytest.mark.parametrize("vf,sf", [(0, 0), (0, 1), (1, 3), (2, 2)])
def test_conservation_on_the_warped_mesh(vf, sf):
    N, n = 3, (2, 3, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.random_state(3, N, n, seed=9)
    du = orc.curved_rhs(g, u, vflux=vf, sflux=sf).reshape(-1, 5, (N + 1) ** 3)
    wJ = g.J * weights3(N)
    tot = np.einsum("ep,evp->v", wJ, du)
    mag = np.einsum("ep,evp->v", wJ, np.abs(du))
    assert np.all(np.abs(tot) < 1e-13 * mag.max())


@pytest.mark.parametrize("vf,sf", [(0, 1), (1, 3)])
def test_entropy_conservation_of_ec_fluxes_on_the_warped_mesh(vf, sf):
    N, n = 3, (2, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.random_state(3, N, n, seed=11)
    du = orc.curved_rhs(g, u, vflux=vf, sflux=sf).reshape(-1, 5, (N + 1) ** 3)
    th = entropy_vars(np.moveaxis(u.reshape(-1, 5, (N + 1) ** 3), 1, 0))
    t = (g.J * weights3(N))[:, None, :] * np.moveaxis(th, 0, 1) * du
    assert abs(t.sum()) < 1e-12 * np.abs(t).sum()


def test_entropy_dissipation_with_llf_on_the_warped_mesh():
    N, n = 3, (2, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.random_state(3, N, n, seed=12)
    du = orc.curved_rhs(g, u, vflux=0, sflux=0).reshape(-1, 5, (N + 1) ** 3)
    th = entropy_vars(np.moveaxis(u.reshape(-1, 5, (N + 1) ** 3), 1, 0))
    t = (g.J * weights3(N))[:, None, :] * np.moveaxis(th, 0, 1) * du
    assert t.sum() < 0


def test_manufactured_source_is_dt_u_plus_div_f():
    sympy = pytest.importorskip("sympy")
    x, y, z, t = sympy.symbols("x y z t")
    A, g = sympy.Rational(1, 10), sympy.Rational(7, 5)
    rho = 2 + A * sympy.sin(sympy.pi * (x + y + z - t))
    v = (1, 1, 1)
    E = rho ** 2
    p = (g - 1) * (E - rho * sum(c * c for c in v) / 2)
    u = [rho, rho * v[0], rho * v[1], rho * v[2], E]
    F = [[rho * v[k], rho * v[0] * v[k] + (p if k == 0 else 0),
          rho * v[1] * v[k] + (p if k == 1 else 0), rho * v[2] * v[k] + (p if k == 2 else 0),
          (E + p) * v[k]] for k in range(3)]
    S = [sympy.diff(u[q], t) + sum(sympy.diff(F[k][q], c) for k, c in enumerate((x, y, z)))
         for q in range(5)]
    fn = sympy.lambdify((x, y, z, t), S, "math")
    rng = np.random.default_rng(3)
    for _ in range(20):
        X, tt = rng.uniform(-1, 1, 3), rng.uniform(0, 2)
        ref = np.array(fn(*X, tt), dtype=float)
        got = orc.manufactured_source_at(tt, X, GAMMA)
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-14)
        st = orc.manufactured_state_at(tt, X)
        r = 2 + 0.1 * math.sin(math.pi * (X.sum() - tt))
        assert np.allclose(st, [r, r, r, r, r * r], rtol=1e-15)


def _rhs_consistency_error(N, ne, t=0.3):
    """L2 (w J) norm of rhs_h(u_exact) + S - d_t u_exact on the warped mesh."""
    n = (ne,) * 3
    g = orc.CurvedGeometry(N, n, warp=0.15)
    xi, _ = orc.lgl(N)
    X = W.warped_node_coordinates(N, n, xi, 0.15)
    du = orc.curved_rhs(g, W.manufactured_state(X, t), vflux=0, sflux=0, source=True, t=t)
    phi = np.pi * (X[0] + X[1] + X[2] - t)
    rho, drho = 2 + 0.1 * np.sin(phi), 0.1 * np.pi * np.cos(phi)
    exact = np.stack([-drho, -drho, -drho, -drho, -2 * rho * drho], axis=1)
    wJ = g.J * weights3(N)
    return math.sqrt((wJ[:, None, :] * (du.reshape(exact.shape) - exact) ** 2).sum())


@pytest.mark.parametrize("N,rate", [(3, 2.6), (4, 3.5)])
def test_rhs_consistency_order_with_source_on_the_warped_mesh(N, rate):
    # the semidiscrete operator with the source term reproduces d_t u of the
    # manufactured solution to O(h^N) (measured: N = 3 rates 1.6, 2.6, 2.9;
    # N = 4 rates 2.8, 3.4, 3.8 over 2^3 .. 16^3 elements)
    errs = [_rhs_consistency_error(N, ne) for ne in (2, 4, 8, 16)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert rates[-1] > rate, (errs, rates)


def _l2_rho_error(N, ne, T=0.1):
    n = (ne,) * 3
    g = orc.CurvedGeometry(N, n, warp=0.15)
    xi, _ = orc.lgl(N)
    X = W.warped_node_coordinates(N, n, xi, 0.15)
    u = W.manufactured_state(X, 0.0)
    steps = math.ceil(T / orc.curved_max_dt(g, u, 0.5))
    dt = T / steps
    t = 0.0
    for _ in range(steps):
        u = orc.curved_lsrk_step(g, u, dt, t, vflux=0, sflux=0, source=True)
        t += dt
    ex = W.manufactured_state(X, T).reshape(-1, 5, (N + 1) ** 3)[:, 0]
    err = u.reshape(-1, 5, (N + 1) ** 3)[:, 0] - ex
    wJ = g.J * weights3(N)
    return math.sqrt((wJ * err * err).sum())


def test_time_integration_with_source_converges_on_the_warped_mesh():
    # stage times t + c_s dt for the source (measured errors at t = 0.1:
    # 3.3e-2, 1.0e-2, 1.8e-3 for 2^3, 4^3, 8^3 elements of degree 3)
    errs = [_l2_rho_error(3, ne) for ne in (4, 8)]
    assert errs[1] < 3e-3
    assert errs[0] / errs[1] > 4.0, errs
