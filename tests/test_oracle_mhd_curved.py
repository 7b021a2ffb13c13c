"""Pins of the MHD oracle on the warped periodic box of the paper's
performance runs (Sec. 3.1): the Cartesian limit (no warping) equal to the
Cartesian MHD operator, free-stream preservation with the Powell term,
conservation, entropy conservation of EC flux differencing with EC faces,
the CFL rule's Cartesian limit and the Alfven wave's rhs consistency on
the warped mesh. CPU only."""
import numpy as np
import pytest

import oracle as orc
from paper_2108_06476_gb300 import workloads as W

G = 5.0 / 3.0
COMBOS = [("central", "llf"), ("central", "hll"), ("ec", "ec"), ("ec", "llf")]


def weights3(N):
    _, w = orc.lgl(N)
    return np.einsum("i,j,k->kji", w, w, w).reshape(-1)


@pytest.mark.parametrize("vflux,sflux", COMBOS)
@pytest.mark.parametrize("powell", [True, False])
def test_cartesian_limit(vflux, sflux, powell):
    N, n = 3, (3, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.0)
    u = W.mhd_random_state(N, n, seed=51, gamma=G)
    ref = orc.mhd_rhs(N, n, W.box(3), u, G, powell, vflux=vflux, sflux=sflux)
    got = orc.mhd_curved_rhs(g, u, G, powell, vflux=vflux, sflux=sflux)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("vflux,sflux", COMBOS)
def test_free_stream_on_the_warped_box(vflux, sflux):
    N, n = 3, (3, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u0 = W.mhd_random_state(1, (1, 1, 1), seed=52, gamma=G).reshape(8, 8)[:, 0]
    P = (N + 1) ** 3
    u = np.tile(np.repeat(u0, P), int(np.prod(n)))
    du = orc.mhd_curved_rhs(g, u, G, True, vflux=vflux, sflux=sflux)
    assert np.max(np.abs(du)) < 1e-10 * np.max(np.abs(u))


@pytest.mark.parametrize("vflux,sflux", COMBOS)
def test_conservation_on_the_warped_box(vflux, sflux):
    N, n = 3, (2, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.mhd_random_state(N, n, seed=53, gamma=G)
    du = orc.mhd_curved_rhs(g, u, G, False, vflux=vflux, sflux=sflux)
    P = (N + 1) ** 3
    tot = np.einsum("evp,ep,p->v", du.reshape(-1, 8, P), g.J, weights3(N))
    scale = np.einsum("evp,ep,p->v", np.abs(du.reshape(-1, 8, P)), g.J, weights3(N))
    assert np.all(np.abs(tot) < 1e-12 * scale.max())


def entropy_vars(U):
    rho, v, B = U[:, 0], U[:, 1:4] / U[:, :1], U[:, 5:8]
    p = (G - 1) * (U[:, 4] - 0.5 * rho * (v * v).sum(1) - 0.5 * (B * B).sum(1))
    beta = rho / (2 * p)
    s = np.log(p) - G * np.log(rho)
    return np.concatenate([((G - s) / (G - 1) - beta * (v * v).sum(1))[:, None],
                           2 * beta[:, None] * v, -2 * beta[:, None], 2 * beta[:, None] * B], 1)


def test_ec_entropy_conservation_on_the_warped_box():
    N, n = 3, (2, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.mhd_random_state(N, n, seed=54, gamma=G)
    P = (N + 1) ** 3
    U = u.reshape(-1, 8, P)
    w = entropy_vars(U)
    for vflux, sflux, conserved in (("ec", "ec", True), ("ec", "llf", False)):
        D = orc.mhd_curved_rhs(g, u, G, True, vflux=vflux, sflux=sflux).reshape(-1, 8, P)
        rate = np.einsum("evp,evp,ep,p->", w, D, g.J, weights3(N))
        mag = np.einsum("evp,evp,ep,p->", np.abs(w), np.abs(D), g.J, weights3(N))
        if conserved:
            assert abs(rate) < 1e-12 * mag
        else:
            assert rate < -1e-6 * mag


def test_max_dt_cartesian_limit():
    N, n = 4, (2, 3, 2)
    g = orc.CurvedGeometry(N, n, warp=0.0)
    u = W.mhd_random_state(N, n, seed=55, gamma=G)
    assert orc.mhd_curved_max_dt(g, u, 0.5, G) == pytest.approx(
        orc.mhd_max_dt(N, n, W.box(3), u, 0.5, G), rel=1e-13)


def test_alfven_wave_rhs_converges_on_the_warped_box():
    """The rhs of the exact wave approaches its d_t u under mesh refinement of
    the warped box at about the order N (N = 3: 2.5, N = 4: 3.7 from 8^3 to
    16^3 elements; the warping's short wavelength keeps 4^3 pre-asymptotic)."""
    for N, min_order in ((3, 2.2), (4, 3.0)):
        errs = []
        for ne in (8, 16):
            n = (ne, ne, ne)
            xi, _ = orc.lgl(N)
            X = W.warped_node_coordinates(N, n, xi, 0.15)
            u = W.alfven_wave_at(X, 0.3, gamma=G)
            dudt = (W.alfven_wave_at(X, 0.3 + 1e-5, gamma=G)
                    - W.alfven_wave_at(X, 0.3 - 1e-5, gamma=G)) / 2e-5
            g = orc.CurvedGeometry(N, n, warp=0.15)
            du = orc.mhd_curved_rhs(g, u, G, True, vflux="central", sflux="hll")
            errs.append(np.max(np.abs(du - dudt)))
        assert np.log2(errs[0] / errs[1]) > min_order, errs


def test_reduces_to_the_curved_euler_operator_without_field():
    """B = 0: the first five components equal the pinned curvilinear Euler
    oracle (central volume flux with HLL or LLF faces)."""
    N, n = 3, (3, 2, 2)
    g = orc.CurvedGeometry(N, n, warp=0.15)
    u = W.mhd_random_state(N, n, seed=56, gamma=G).reshape(-1, 8, 64)
    u[:, 4] -= 0.5 * (u[:, 5:8] ** 2).sum(1)
    u[:, 5:8] = 0.0
    ue = np.ascontiguousarray(u[:, :5]).reshape(-1)
    for sflux, se in (("hll", orc.S_HLL), ("llf", orc.S_LLF)):
        a = orc.mhd_curved_rhs(g, u.reshape(-1), G, True, vflux="central",
                               sflux=sflux).reshape(-1, 8, 64)
        b = orc.curved_rhs(g, ue, vflux=orc.CENTRAL, sflux=se, gamma=G).reshape(-1, 5, 64)
        assert np.max(np.abs(a[:, :5] - b)) <= 1e-13 * np.max(np.abs(b))
        assert np.max(np.abs(a[:, 5:])) == 0.0


# ---- planted mistakes in the warped-box operators must fail a pin ----
import os  # noqa: E402

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MUTANTS = [
    ("volume flux along the node's own metric vector",
     "for (int k = 0; k < 3; ++k) g[k] = 0.5 * (gi[k] + gm[k]);",
     "for (int k = 0; k < 3; ++k) g[k] = gi[k];"),
    ("sign of the left face's div B term", "          db -= bg / w[0];",
     "          db += bg / w[0];"),
    ("LLF dissipation not scaled by |g|", "- 0.5 * lam * gn * (uR[v] - uL[v]);",
     "- 0.5 * lam * (uR[v] - uL[v]);"),
    ("fast speed along x instead of the face normal",
     "const double bn = B[0] * nh[0] + B[1] * nh[1] + B[2] * nh[2];", "const double bn = B[0];"),
    ("Powell term without 1/J", "du[(e * MV + v) * m.P + node] = -(acc[v] + phi[v] * db) / Jn;",
     "du[(e * MV + v) * m.P + node] = -acc[v] / Jn - phi[v] * db;"),
]


def _battery():
    failed = []
    for fn, args in ((test_cartesian_limit, ("central", "hll", True)),
                     (test_cartesian_limit, ("central", "llf", True)),
                     (test_free_stream_on_the_warped_box, ("central", "llf")),
                     (test_free_stream_on_the_warped_box, ("central", "hll")),
                     (test_ec_entropy_conservation_on_the_warped_box, ()),
                     (test_reduces_to_the_curved_euler_operator_without_field, ())):
        try:
            fn(*args)
        except (AssertionError, ValueError):
            failed.append(fn.__name__)
    return failed


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, name, old, new):
    texts = []
    for f in ("dgsem_oracle.c", "dgsem_curved.c", "dgsem_mhd.c"):
        with open(os.path.join(_ROOT, "oracle", f)) as fh:
            texts.append(fh.read())
    main, curved, mhd = texts
    assert mhd.count(old) == 1, f"mutation site not found: {name}"
    so = orc.build_variant(main, str(tmp_path), curved, mhd.replace(old, new))
    with orc.use_library(so):
        failed = _battery()
    assert failed, f"no pin rejects the mutant: {name}"
