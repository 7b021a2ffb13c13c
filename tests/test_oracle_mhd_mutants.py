"""Mutation check of the MHD oracle's pins (CPU only): plausible mistakes are
planted in a copy of dgsem_mhd.c, and the pins of test_oracle_mhd, run as a
battery, must reject every one while accepting the source as it is."""
import os

import pytest

import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "dgsem_oracle.c")
CURVED = os.path.join(ROOT, "oracle", "dgsem_curved.c")
MHD = os.path.join(ROOT, "oracle", "dgsem_mhd.c")

import test_oracle_mhd as TM  # noqa: E402

MUTANTS = [
    ("magnetic pressure dropped", "const double pt = p + 0.5 * b2;", "const double pt = p;"),
    ("Maxwell stress dropped", "f[1 + k] = rho * v[n] * v[k] - B[n] * B[k];",
     "f[1 + k] = rho * v[n] * v[k];"),
    ("sign of the induction flux", "f[5 + k] = v[n] * B[k] - B[n] * v[k];",
     "f[5 + k] = v[n] * B[k] + B[n] * v[k];"),
    ("energy flux without magnetic pressure", "f[4] = v[n] * (u[4] + pt) - B[n] * vb;",
     "f[4] = v[n] * (u[4] + p) - B[n] * vb;"),
    ("fast speed discriminant",
     "const double bn2 = B[n] * B[n] / rho;\n  const double s = a2 + b2;\n"
     "  return sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));",
     "const double bn2 = B[n] * B[n] / rho;\n  const double s = a2 + b2;\n"
     "  return sqrt(0.5 * (s + sqrt(s * s - 2.0 * a2 * bn2)));"),
    ("LLF speed from the mean velocity", "fmax(fabs(vL), fabs(vR)) +",
     "0.5 * (fabs(vL) + fabs(vR)) +"),
    ("transposed volume derivative",
     "vol[v] += Dt[i * m.np + a] * fp[v];", "vol[v] += Dt[a * m.np + i] * fp[v];"),
    ("sign of the left surface term", "for (int v = 0; v < MV; ++v) vol[v] -= fs[v] / w[0];",
     "for (int v = 0; v < MV; ++v) vol[v] += fs[v] / w[0];"),
    ("left neighbour taken on the right",
     "m_load(&m, u, m_neighbour(&m, e, r, -1), m_with(&m, node, r, N), uo);",
     "m_load(&m, u, m_neighbour(&m, e, r, +1), m_with(&m, node, r, N), uo);"),
    ("own trace instead of the interface mean in div B",
     "db += 0.5 * (ui[5 + r] + uo[5 + r]) / w[N];", "db += ui[5 + r] / w[N];"),
    ("div B without the mesh scaling", "divb += (2.0 / m.h[r]) * db;", "divb += db;"),
    ("Powell energy term drops a product", "v[0] * B[0] + v[1] * B[1] + v[2] * B[2],",
     "v[0] * B[0] + v[1] * B[1],"),
    ("Powell induction term permuted", "v[0], v[1], v[2]};", "v[1], v[0], v[2]};"),
    ("CFL step without the N+1 factor",
     "sum += (2.0 / m.h[r]) * lam[r];\n    if (sum > worst) worst = sum;\n  }\n"
     "  return cfl * 2.0 / ((N + 1) * worst);",
     "sum += (2.0 / m.h[r]) * lam[r];\n    if (sum > worst) worst = sum;\n  }\n"
     "  return cfl * 2.0 / (N * worst);"),
    ("HLL left speed takes the right state's fast wave the wrong way",
     "const double sL = fmin(vL - cL, vR - cR)", "const double sL = fmin(vL - cL, vR + cR)"),
    ("HLL jump term with the wrong sign", "sL * sR * (uR[v] - uL[v])", "sL * sR * (uL[v] - uR[v])"),
    ("HLL upwinds to the wrong side", "if (sL >= 0.0) f[v] = fL[v];",
     "if (sL >= 0.0) f[v] = fR[v];"),
    ("surface flux ids swapped", "if (sflux == 1) or_mhd_hll(n, gamma, uL, uR, f);",
     "if (sflux == 0) or_mhd_hll(n, gamma, uL, uR, f);"),
    ("EC magnetic pressure without the beta weighting", "f[1 + n] += (ra + bB2) / (2.0 * ba);",
     "f[1 + n] += ra / (2.0 * ba) + 0.5 * B2;"),
    ("EC energy flux drops the {B_n} {v.B} term", "- 0.5 * va[n] * B2 +\n         Ba[n] * vB;",
     "- 0.5 * va[n] * B2;"),
    ("EC flux with the arithmetic mean of beta", "beta_ln = or_ln_mean(bL, bR);",
     "beta_ln = 0.5 * (bL + bR);"),
    ("EC induction flux with the sign of {B_n} {v} flipped",
     "f[5 + k] = va[n] * Ba[k] - Ba[n] * va[k];", "f[5 + k] = va[n] * Ba[k] + Ba[n] * va[k];"),
    ("EC volume flux id ignored", "if (vflux == 1) {\n    or_mhd_flux_ec(n, gamma, ui, um, f);",
     "if (vflux == 7) {\n    or_mhd_flux_ec(n, gamma, ui, um, f);"),
]

PINS = [
    TM.test_flux_is_euler_flux_without_field,
    TM.test_flux_is_rotation_invariant,
    TM.test_fast_speed_bounds_the_flux_jacobian_spectrum,
    TM.test_llf_is_consistent_and_dissipates_at_the_largest_speed,
    lambda: TM.test_free_stream(True, "llf"),
    TM.test_hll_consistency_upwinding_and_llf_limit,
    TM.test_surface_flux_enters_through_the_lifting,
    lambda: TM.test_conservation_without_powell_term("llf"),
    lambda: TM.test_axis_swap_equivariance("xy"),
    lambda: TM.test_axis_swap_equivariance("xz"),
    TM.test_divergence_theorem_per_element,
    TM.test_divergence_is_exact_for_continuous_piecewise_quadratics,
    lambda: TM.test_alfven_wave_rhs_converges(True, "llf"),
    TM.test_powell_system_advects_a_divergence_error,
    TM.test_max_dt_uses_the_fast_speed,
    TM.test_ec_flux_consistency_and_symmetry,
    TM.test_ec_flux_satisfies_the_discrete_entropy_condition,
    TM.test_ec_rhs_conserves_entropy,
]


def battery():
    failed = []
    for i, pin in enumerate(PINS):
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(i)
    return failed


@pytest.fixture(scope="module")
def sources():
    out = []
    for path in (SRC, CURVED, MHD):
        with open(path) as fh:
            out.append(fh.read())
    return out


def test_battery_accepts_the_mhd_oracle():
    assert battery() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_battery_rejects_planted_mistake(sources, tmp_path, name, old, new):
    main, curved, mhd = sources
    old, new = old.replace("\\n", "\n"), new.replace("\\n", "\n")
    assert mhd.count(old) == 1, f"mutation site not found: {name}"
    so = orc.build_variant(main, str(tmp_path), curved, mhd.replace(old, new))
    with orc.use_library(so):
        failed = battery()
    assert failed, f"no pin rejects the mutant: {name}"
