"""Mutation check of the curvilinear oracle's pins (CPU only): plausible
mistakes are planted in a copy of dgsem_curved.c, and a battery of the pins
of test_oracle_curved must reject every one while accepting the source as
it is."""
import os

import numpy as np
import pytest

import oracle as orc
from paper_2108_06476_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "dgsem_oracle.c")
CURVED = os.path.join(ROOT, "oracle", "dgsem_curved.c")

import test_oracle_curved as TC  # noqa: E402

MUTANTS = [
    ("sign of the curl-form metric terms", "Ja[((e * 3 + i) * 3 + nc) * P + node] = -curl;",
     "Ja[((e * 3 + i) * 3 + nc) * P + node] = curl;"),
    ("cyclic order of the metric components", "const int mm = (nc + 1) % 3, l = (nc + 2) % 3;",
     "const int mm = (nc + 2) % 3, l = (nc + 1) % 3;"),
    ("sum instead of mean of the metric terms", "gavg[k] = 0.5 * (gi[k] + gm[k]);",
     "gavg[k] = (gi[k] + gm[k]);"),
    ("Jacobian cofactor sign", "a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +",
     "a[0][1] * (a[1][2] * a[2][0] - a[1][0] * a[2][2]) +"),
    ("LLF dissipation not scaled by |g|", "0.5 * lam * gn * (uR[v] - uL[v])",
     "0.5 * lam * (uR[v] - uL[v])"),
    ("pressure term of the energy source", "S[4] = 4.0 * rho * drho + 3.0 * dp;",
     "S[4] = 4.0 * rho * drho + 2.0 * dp;"),
    ("warping uses the box y in x", "cos(2.0 * kPi * y)", "cos(2.0 * kPi * c[1])"),
]


def battery(orc):
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    # Cartesian limit
    N, n = 2, (2, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.0)
    u = W.random_state(3, N, n, seed=5)
    for vf, sf in ((0, 0), (0, 1), (2, 2)):
        ref = orc.rhs(3, N, n, W.box(3), u, vflux=vf, sflux=sf)
        got = orc.curved_rhs(g, u, vflux=vf, sflux=sf)
        check("cartesian limit", np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref))
    # warped geometry: J > 0, volume, metric identities, mapping
    N = 3
    g = orc.CurvedGeometry(N, (4, 4, 4), warp=0.15)
    check("J > 0", g.J.min() > 0)
    check("volume", abs((g.J * TC.weights3(N)).sum() - 8.0) < 1e-12)
    check("metric identities", np.abs(TC.divergence(N, g)).max() < 1e-15 * N ** 4 * np.abs(g.Ja).max())
    xi, _ = orc.lgl(N)
    X = W.warped_node_coordinates(N, (4, 4, 4), xi, 0.15)
    check("mapping", np.abs(np.moveaxis(X, 0, 1) - g.X).max() < 1e-15)
    Jref = TC.jacobian_det(N, g)
    check("jacobian", np.abs(g.J - Jref).max() < 1e-13 * np.abs(Jref).max())
    # free stream and conservation on the warped mesh
    gs = orc.CurvedGeometry(3, (3, 2, 2), warp=0.15)
    du = orc.curved_rhs(gs, W.uniform_state(3, 3, (3, 2, 2)), vflux=0, sflux=0)
    check("free stream", np.abs(du).max() < 1.4e-10)
    # source against the closed form written independently here
    rng = np.random.default_rng(4)
    for _ in range(5):
        Xp, t = rng.uniform(-1, 1, 3), rng.uniform(0, 1)
        phi = np.pi * (Xp.sum() - t)
        rho, drho = 2 + 0.1 * np.sin(phi), 0.1 * np.pi * np.cos(phi)
        dp = 0.4 * (2 * rho - 1.5) * drho
        ref = np.array([2 * drho, 2 * drho + dp, 2 * drho + dp, 2 * drho + dp,
                        4 * rho * drho + 3 * dp])
        check("source", np.allclose(orc.manufactured_source_at(t, Xp), ref, rtol=1e-13,
                                    atol=1e-14))
    return failed


@pytest.fixture(scope="module")
def sources():
    with open(SRC) as fh:
        main = fh.read()
    with open(CURVED) as fh:
        curved = fh.read()
    return main, curved


def test_battery_accepts_the_curved_oracle():
    assert battery(orc) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_battery_rejects_planted_mistake(sources, tmp_path, name, old, new):
    main, curved = sources
    assert curved.count(old) == 1, f"mutation site not found: {name}"
    so = orc.build_variant(main, str(tmp_path), curved.replace(old, new))
    with orc.use_library(so):
        failed = battery(orc)
    assert failed, f"no pin rejects the mutant: {name}"
