"""The oracle's operation-counting build (every +, -, *, /, log1p and sqrt
of its formulas counts one operation), which gives the algorithmic work per
node used by the benchmark's roofline (CPU only).

Pins: hand counts of the primitive conversion and the physical and central
fluxes; the count of the whole rhs equals its composition from the counts
of the individual two-point and surface fluxes in the oracle's loop order
(both orders of every pair including m = i, the lifting, the scaling); the
stored tests/golden/op_counts.json equals a fresh computation."""
import json
import os
import sys

import numpy as np
import pytest

from paper_2108_06476_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_hand_counts(orc):
    u3 = np.array([1.0, 0.1, 0.2, 0.3, 50.0])
    u2 = np.array([1.0, 0.1, 0.2, 50.0])
    # v_k = m_k / rho (d divisions), |v|^2 (d products, d additions),
    # p = (gamma - 1)(E - rho |v|^2 / 2) (4, plus gamma - 1 formed in real)
    assert orc.ops_cons2prim(3, u3) == 3 * 3 + 5
    assert orc.ops_cons2prim(2, u2) == 3 * 2 + 5
    # f = (m_n, m_n v + p e_n, (E + p) v_n): primitives + d + 1 + 2
    assert orc.ops_two_point(20, 3, 0, u3, u3) == 14 + 3 + 1 + 2
    # central flux: two physical fluxes and (f_L + f_R) / 2 per variable
    assert orc.ops_two_point(2, 3, 1, u3, u3 * 1.01) == 2 * 20 + 2 * 5


def _line_node(N, d, node, direction, a):
    c = [(node // (N + 1) ** k) % (N + 1) for k in range(d)]
    c[direction] = a
    return sum(c[k] * (N + 1) ** k for k in range(d))


def test_rhs_count_is_the_sum_of_its_fluxes(orc):
    d, N, n = 3, 2, (2, 2, 1)
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=3)
    nv, P, ne = d + 2, (N + 1) ** d, int(np.prod(n))
    U = u.reshape(ne, nv, P)

    def neighbour(e, direction, s):
        c = [e % n[0], (e // n[0]) % n[1], e // (n[0] * n[1])]
        c[direction] = (c[direction] + s) % n[direction]
        return c[0] + n[0] * (c[1] + n[1] * c[2])

    total = 0
    for e in range(ne):
        for node in range(P):
            ui = U[e, :, node]
            for direction in range(d):
                i = (node // (N + 1) ** direction) % (N + 1)
                for a in range(N + 1):
                    um = U[e, :, _line_node(N, d, node, direction, a)]
                    total += orc.ops_two_point(0, d, direction, ui, um) + 2 * nv
                if i == N:
                    uo = U[neighbour(e, direction, +1), :, _line_node(N, d, node, direction, 0)]
                    total += orc.ops_two_point(10, d, direction, ui, uo) + 2 * nv
                if i == 0:
                    uo = U[neighbour(e, direction, -1), :, _line_node(N, d, node, direction, N)]
                    total += orc.ops_two_point(10, d, direction, uo, ui) + 2 * nv
                total += 3 * nv  # du -= (2/h) vol
    assert orc.ops_rhs(d, N, n, dom, u) == total


def test_stored_op_counts_are_current(orc):
    sys.path.insert(0, GOLDEN)
    try:
        import make_op_counts
    finally:
        sys.path.remove(GOLDEN)
    with open(os.path.join(GOLDEN, "op_counts.json")) as fh:
        stored = json.load(fh)["workloads"]
    fresh = make_op_counts.counts()
    assert set(stored) == set(fresh)
    for name in fresh:
        for key, value in fresh[name].items():
            assert stored[name][key] == pytest.approx(value, rel=1e-12), (name, key)
    # the pair flux of Ranocha's flux counts 66-72 operations (two log means,
    # the pressure and energy terms), the prologue 14
    for rec in stored.values():
        assert 60 < rec["pair_flux"] < 75 and rec["prim"] == 14.0
        N = round(2 * rec["pairs_per_node"] / 3)
        assert rec["lifting"] == 4 * 3 * 5 / (N + 1)
