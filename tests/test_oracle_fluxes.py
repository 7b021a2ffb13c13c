"""Pins of the oracle's logarithmic mean and two-point fluxes: high-precision
logarithmic mean, consistency with the Euler flux written here from the
equations, symmetry, Tadmor's entropy-conservation condition with entropy
variables written here, kinetic-energy preservation, and HLL upwinding."""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

GAMMA = 1.4


def prim2cons(rho, v, p):
    v = np.asarray(v, dtype=float)
    return np.array([rho, *(rho * v), p / (GAMMA - 1) + 0.5 * rho * v @ v])


def euler_flux(u, n):
    """Compressible Euler flux in direction n, from the equations."""
    d = len(u) - 2
    rho, m, E = u[0], u[1:1 + d], u[-1]
    v = m / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * v @ v)
    f = np.empty_like(u)
    f[0] = m[n]
    f[1:1 + d] = m[n] * v
    f[1 + n] += p
    f[-1] = (E + p) * v[n]
    return f


def entropy_vars(u):
    """theta = dS/du for S = -rho s/(gamma-1), s = ln p - gamma ln rho."""
    d = len(u) - 2
    rho, m, E = u[0], u[1:1 + d], u[-1]
    v = m / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * v @ v)
    s = np.log(p) - GAMMA * np.log(rho)
    b = rho / p
    return np.array([(GAMMA - s) / (GAMMA - 1) - 0.5 * b * v @ v, *(b * v), -b])


def rand_state(rng, d):
    return prim2cons(rng.uniform(0.3, 3.0), rng.uniform(-1, 1, size=d), rng.uniform(0.3, 5.0))


def test_ln_mean_high_precision(orc):
    mpmath.mp.dps = 40
    rng = np.random.default_rng(1)
    eps = np.finfo(float).eps
    xs = np.exp(rng.uniform(-3, 3, 4000))
    # ratios spanning both branches, concentrated near the switch f2 = 1e-4
    rs = np.exp(np.concatenate([rng.uniform(-2, 2, 1000), rng.uniform(-0.03, 0.03, 2000),
                                rng.uniform(-1e-6, 1e-6, 1000)]))
    for x, r in zip(xs, rs):
        y = x * r
        got = orc.ln_mean(x, y)
        X, Y = mpmath.mpf(x), mpmath.mpf(y)
        ref = X if X == Y else (Y - X) / mpmath.log(Y / X)
        rel = abs((mpmath.mpf(got) - ref) / ref)
        # a few ulps in both branches, independent of how close y is to x
        assert rel <= 6 * eps, (x, y, float(rel))


def test_ln_mean_special(orc):
    for x in (1e-3, 0.7, 1.0, 3.5, 1e4):
        assert orc.ln_mean(x, x) == pytest.approx(x, rel=2e-16)
        assert orc.ln_mean(x, 2 * x) == orc.ln_mean(2 * x, x) or \
            abs(orc.ln_mean(x, 2 * x) / orc.ln_mean(2 * x, x) - 1) < 4e-16
        # ln_mean(x, y) lies between the geometric and arithmetic means
        y = 3.0 * x
        assert np.sqrt(x * y) < orc.ln_mean(x, y) < 0.5 * (x + y)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1, 2, 10, 11, 12, 13])
def test_flux_consistency(orc, d, kind):
    rng = np.random.default_rng(2 + kind)
    for _ in range(50):
        u = rand_state(rng, d)
        for n in range(d):
            f = orc.two_point(kind, d, n, u, u)
            fe = euler_flux(u, n)
            assert np.max(np.abs(f - fe)) <= 8e-15 * np.max(np.abs(fe)), (kind, n)
            assert np.array_equal(orc.two_point(20, d, n, u, u), orc.two_point(20, d, n, u, u))
            np.testing.assert_allclose(orc.two_point(20, d, n, u, u), fe, rtol=4e-15, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1, 2, 11, 13])
def test_flux_symmetry(orc, d, kind):
    rng = np.random.default_rng(10 + kind)
    for _ in range(50):
        uL, uR = rand_state(rng, d), rand_state(rng, d)
        for n in range(d):
            a = orc.two_point(kind, d, n, uL, uR)
            b = orc.two_point(kind, d, n, uR, uL)
            assert np.max(np.abs(a - b)) <= 4e-15 * np.max(np.abs(a))


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1])
def test_tadmor_entropy_conservation(orc, d, kind):
    # (theta_R - theta_L) . f#(u_L, u_R) = psi_R - psi_L with psi_n = rho v_n
    rng = np.random.default_rng(20 + kind)
    worst = 0.0
    for _ in range(200):
        uL, uR = rand_state(rng, d), rand_state(rng, d)
        for n in range(d):
            f = orc.two_point(kind, d, n, uL, uR)
            tL, tR = entropy_vars(uL), entropy_vars(uR)
            lhs = (tR - tL) @ f
            rhs = uR[1 + n] - uL[1 + n]
            scale = np.abs(tR - tL) @ np.abs(f) + abs(uR[1 + n]) + abs(uL[1 + n])
            worst = max(worst, abs(lhs - rhs) / scale)
    assert worst < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_central_is_not_entropy_conservative(orc, d):
    # sensitivity check of the pin above: a plausible wrong flux fails it
    rng = np.random.default_rng(5)
    uL, uR = rand_state(rng, d), rand_state(rng, d)
    f = orc.two_point(2, d, 0, uL, uR)
    lhs = (entropy_vars(uR) - entropy_vars(uL)) @ f
    assert abs(lhs - (uR[1] - uL[1])) > 1e-3


@pytest.mark.parametrize("d", [2, 3])
def test_ranocha_kinetic_energy_preserving_form(orc, d):
    # momentum flux = mass flux * avg(v) + avg(p) e_n (Jameson's KEP condition)
    rng = np.random.default_rng(30)
    for _ in range(50):
        uL, uR = rand_state(rng, d), rand_state(rng, d)
        vL, vR = uL[1:1 + d] / uL[0], uR[1:1 + d] / uR[0]
        pL = (GAMMA - 1) * (uL[-1] - 0.5 * uL[0] * vL @ vL)
        pR = (GAMMA - 1) * (uR[-1] - 0.5 * uR[0] * vR @ vR)
        for n in range(d):
            f = orc.two_point(0, d, n, uL, uR)
            mom = f[0] * 0.5 * (vL + vR)
            mom[n] += 0.5 * (pL + pR)
            np.testing.assert_allclose(f[1:1 + d], mom, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_hll_upwinds_supersonic(orc, d):
    # all signal speeds positive: HLL returns f(u_L); all negative: f(u_R)
    v = np.zeros(d)
    v[0] = 5.0
    uL = prim2cons(1.0, v, 1.0)
    uR = prim2cons(1.2, v, 1.1)
    np.testing.assert_allclose(orc.two_point(12, d, 0, uL, uR), euler_flux(uL, 0), rtol=1e-15)
    uL2 = prim2cons(1.0, -v, 1.0)
    uR2 = prim2cons(1.2, -v, 1.1)
    np.testing.assert_allclose(orc.two_point(12, d, 0, uL2, uR2), euler_flux(uR2, 0), rtol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_llf_dissipation_sign(orc, d):
    # LLF = central - lambda/2 (u_R - u_L), lambda = max|v_n| + max c >= 0
    rng = np.random.default_rng(40)
    for _ in range(20):
        uL, uR = rand_state(rng, d), rand_state(rng, d)
        f = orc.two_point(10, d, 0, uL, uR)
        central = 0.5 * (euler_flux(uL, 0) + euler_flux(uR, 0))
        diff = central - f
        lam = diff / (0.5 * (uR - uL))
        assert np.allclose(lam, lam[0], rtol=1e-10)
        vL, vR = uL[1] / uL[0], uR[1] / uR[0]
        pL = (GAMMA - 1) * (uL[-1] - 0.5 * uL[1:1 + d] @ uL[1:1 + d] / uL[0])
        pR = (GAMMA - 1) * (uR[-1] - 0.5 * uR[1:1 + d] @ uR[1:1 + d] / uR[0])
        cL, cR = np.sqrt(GAMMA * pL / uL[0]), np.sqrt(GAMMA * pR / uR[0])
        assert lam[0] == pytest.approx(max(abs(vL), abs(vR)) + max(cL, cR), rel=1e-12)
