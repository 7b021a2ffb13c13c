"""Mutation check of the oracle's pins (CPU only): plausible mistakes are
planted in a copy of the oracle source, the copy is compiled, and a battery of
the pins (the same properties the pin tests check) must reject every mutant
while accepting the unmodified source."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2108_06476_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "dgsem_oracle.c")

import test_oracle_fluxes as TF  # noqa: E402
import test_oracle_rhs as TR  # noqa: E402
import test_oracle_basis as TB  # noqa: E402

# (name, text in the oracle source, replacement): each a mistake a careful
# reader could make when restating the cited formulas
MUTANTS = [
    ("series coefficient of the log mean", "f2 * (2.0 / 5.0 + f2", "f2 * (2.0 / 3.0 + f2"),
    ("dropped pressure in the Ranocha momentum flux",
     "  f[1 + n] += p_avg;\n  f[d + 1] = f[0] * (0.5 * v_dot", "  f[d + 1] = f[0] * (0.5 * v_dot"),
    ("swapped velocities in the Ranocha energy flux",
     "0.5 * (pL * vR[n] + pR * vL[n])", "0.5 * (pL * vL[n] + pR * vR[n])"),
    ("transposed split-form matrix", "vol[v] += Dt[i * m.np + a] * f[v];",
     "vol[v] += Dt[a * m.np + i] * f[v];"),
    ("sign of the left-face lifting", "vol[v] -= fs[v] / w[0];", "vol[v] += fs[v] / w[0];"),
    ("inverse Jacobian 1/h instead of 2/h", "acc[v] -= ((real)2.0 / (real)m.h[dir]) * vol[v];",
     "acc[v] -= ((real)1.0 / (real)m.h[dir]) * vol[v];"),
    ("LLF wave speed with min", "r_max(r_abs(vL[n]), r_abs(vR[n])) + r_max(cL, cR)",
     "r_max(r_abs(vL[n]), r_abs(vR[n])) + r_min(cL, cR)"),
    ("pressure with gamma instead of gamma - 1", "*p = (gamma - 1.0) * (u[d + 1]",
     "*p = (gamma) * (u[d + 1]"),
    ("mistyped Carpenter-Kennedy digit", "B[2] = 1720146321549.0 / 2090206949498.0;",
     "B[2] = 1720146321549.0 / 2090206949489.0;"),
    ("LGL weight formula", "w[j] = 2.0L / ((long double)N * (N + 1) * p * p);",
     "w[j] = 2.0L / ((long double)N * (N + 2) * p * p);"),
    ("Chandrashekar pressure average", "real p_mean = 0.5 * rho_avg / beta_avg;",
     "real p_mean = rho_avg / beta_avg;"),
]


def battery(orc):
    """Names of the failed pins."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    # basis: LGL closed forms
    for N, nodes, weights in TB._golden_lgl():
        xi, w = orc.lgl(N)
        check("lgl", np.allclose(xi, nodes, atol=1e-15) and np.allclose(w, weights, rtol=1e-14))
    # Runge-Kutta order conditions
    A, B, _ = orc.lsrk_coefficients()
    R = TB._stability_polynomial([Fraction(a) for a in A], [Fraction(b) for b in B])
    check("rk order", all(abs(float(R[j]) - 1 / math.factorial(j)) < 1e-12 for j in range(5)))
    # logarithmic mean against (y - x) / log1p((y - x)/x) near and away from x = y
    rng = np.random.default_rng(0)
    for x, r in zip(np.exp(rng.uniform(-2, 2, 50)), np.exp(rng.uniform(-0.02, 0.02, 50))):
        y = x * r
        ref = x if y == x else (y - x) / math.log1p((y - x) / x)
        check("ln mean", abs(orc.ln_mean(x, y) - ref) <= 1e-14 * ref)
    # fluxes: consistency, symmetry, Tadmor, LLF speed
    for d in (2, 3):
        for _ in range(5):
            uL, uR = TF.rand_state(rng, d), TF.rand_state(rng, d)
            for n in range(d):
                for kind in (0, 1, 2, 10, 11, 12):
                    f = orc.two_point(kind, d, n, uL, uL)
                    check(f"consistency {kind}",
                          np.allclose(f, TF.euler_flux(uL, n), rtol=1e-13, atol=1e-13))
                for kind in (0, 1):
                    f = orc.two_point(kind, d, n, uL, uR)
                    lhs = (TF.entropy_vars(uR) - TF.entropy_vars(uL)) @ f
                    check(f"tadmor {kind}", abs(lhs - (uR[1 + n] - uL[1 + n])) < 1e-10)
            f = orc.two_point(10, d, 0, uL, uR)
            lam = (0.5 * (TF.euler_flux(uL, 0) + TF.euler_flux(uR, 0)) - f)[0] / (0.5 * (uR - uL)[0])
            pL = 0.4 * (uL[-1] - 0.5 * uL[1:1 + d] @ uL[1:1 + d] / uL[0])
            pR = 0.4 * (uR[-1] - 0.5 * uR[1:1 + d] @ uR[1:1 + d] / uR[0])
            ref = max(abs(uL[1] / uL[0]), abs(uR[1] / uR[0])) + max(
                math.sqrt(1.4 * pL / uL[0]), math.sqrt(1.4 * pR / uR[0]))
            check("llf speed", abs(lam - ref) < 1e-10 * ref)
    # semidiscretisation: free stream, conservation, entropy, weak form
    d, N, n = 2, 3, (3, 2)
    dom = np.array([-1.0, 1.0, -0.5, 1.5])
    us = W.uniform_state(d, N, n)
    check("free stream", np.max(np.abs(orc.rhs(d, N, n, dom, us))) < 1e-11)
    u = W.random_state(d, N, n, seed=1)
    wq = TR.quad_weights(orc, d, N, n, dom)
    for vf, sf in ((0, 0), (1, 3)):
        du = orc.rhs(d, N, n, dom, u, vflux=vf, sflux=sf)
        tot = (wq * du).reshape(-1, d + 2, (N + 1) ** d).sum(axis=(0, 2))
        check("conservation", np.all(np.abs(tot) < 1e-12 * np.abs(wq * du).sum()))
    du = orc.rhs(d, N, n, W.box(d), u, vflux=0, sflux=1)
    t = TR.quad_weights(orc, d, N, n, W.box(d)) * TR.theta(u, d, 6) * du
    check("entropy", abs(t.sum()) < 1e-12 * np.abs(t).sum())
    du = orc.rhs(d, 2, (3, 2), dom, W.random_state(d, 2, (3, 2), seed=2), vflux=2, sflux=0)
    ref = TR._weak_form_rhs(orc, d, 2, (3, 2), dom, W.random_state(d, 2, (3, 2), seed=2), 0)
    check("weak form", np.max(np.abs(du - ref)) < 1e-11 * np.max(np.abs(ref)))
    # rhs converges to the exact time derivative of the density wave
    xi, _ = orc.lgl(3)
    errs = []
    for ne in (4, 8, 16):
        u = W.density_wave(2, 3, (ne, ne), W.box(2), xi, amplitude=0.5)
        du = orc.rhs(2, 3, (ne, ne), W.box(2), u).reshape(-1, 4, 16)
        X = W.node_coordinates(2, 3, (ne, ne), W.box(2), xi)
        ex = -np.pi * 0.5 * 0.3 * np.cos(np.pi * X.sum(axis=0))
        errs.append(np.max(np.abs(du[:, 0] - ex)))
    check("convergence", math.log2(errs[1] / errs[2]) > 2.3 and errs[2] < 1e-2)
    return failed


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


def test_battery_accepts_the_oracle(orc):
    assert battery(orc) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_battery_rejects_planted_mistake(orc, source, tmp_path, name, old, new):
    assert source.count(old) == 1, f"mutation site not found: {name}"
    so = orc.build_variant(source.replace(old, new), str(tmp_path))
    with orc.use_library(so):
        failed = battery(orc)
    assert failed, f"no pin rejects the mutant: {name}"
