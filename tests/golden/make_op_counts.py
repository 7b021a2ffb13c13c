"""Writes op_counts.json: the algorithmic operations per node of the fused
volume kernel (flux differencing, lifting and the Runge-Kutta stage update)
for the configured 3D Euler workloads, counted by the oracle's
operation-counting build (every +, -, *, /, log1p and sqrt of the oracle's
formulas counts one; a logarithm, a division or a square root is one
operation).

The method evaluates per node: one conserved -> primitive conversion, the
d N / 2 node pairs of its lines (each two-point flux once for both nodes,
since the flux is symmetric and the split-form matrix has a zero diagonal;
two multiply-adds per variable and pair accumulate it), the lifting of the
surface fluxes at the 2 of N+1 line nodes on a face (a multiply-add per
variable), and the 2N-storage stage update k <- A k + dt du, u <- u + B k
(five operations per variable). The pair flux is counted as the oracle's
two-point flux between the two nodes' conserved states minus its two
primitive conversions, averaged over the pairs of sampled elements of the
workload (the logarithmic mean's branch, and so the count, depends on the
pair).

Only the oracle and the seeded input generators are used. Run from the
repository root: python tests/golden/make_op_counts.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2108_06476_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "op_counts.json")

# the configured 3D workloads whose fused volume kernel bench.py times
WORKLOADS = {
    "euler3d_n3_64cubed_noisy_wave": dict(N=3, ne=64, noisy=True),
    "euler3d_n3_32cubed_wave": dict(N=3, ne=32, noisy=False),
    "euler3d_n7_24cubed_noisy_wave": dict(N=7, ne=24, noisy=True),
}
SAMPLE_ELEMENTS = 24
# the ensemble's degrees, each on a member-like density wave (8^3 elements,
# amplitude 0.5, velocity (0.1, 0.2, -0.1)): the work per node of a member
ENSEMBLE_DEGREES = (3, 4, 5)


def line_nodes(N, direction, line):
    NP = N + 1
    if direction == 0:
        return [a + NP * line for a in range(NP)]
    if direction == 1:
        return [(line % NP) + NP * a + NP * NP * (line // NP) for a in range(NP)]
    return [line + NP * NP * a for a in range(NP)]


def volume_counts(N, u, nelem, elems, d=3, vflux=0, gamma=1.4):
    nv, P = d + 2, (N + 1) ** d
    U = u.reshape(nelem, nv, P)
    prims, fluxes = [], []
    for e in elems:
        for node in range(P):
            prims.append(oracle.ops_cons2prim(d, U[e, :, node], gamma))
        for direction in range(d):
            for line in range(P // (N + 1)):
                nodes = line_nodes(N, direction, line)
                for a in range(N + 1):
                    for b in range(a + 1, N + 1):
                        fluxes.append(oracle.ops_two_point(vflux, d, direction, U[e, :, nodes[a]],
                                                           U[e, :, nodes[b]], gamma))
    prim = float(np.mean(prims))
    flux = float(np.mean(fluxes)) - 2.0 * prim
    pairs = d * N / 2.0
    accumulate = 4.0 * nv
    lifting = 4.0 * d * nv / (N + 1)
    stage = 5.0 * nv
    return {"prim": prim, "pair_flux": flux, "pairs_per_node": pairs,
            "accumulate_per_pair": accumulate, "lifting": lifting, "stage_update": stage,
            "volume_rhs_per_node": prim + pairs * (flux + accumulate) + lifting,
            "volume_fused_per_node": prim + pairs * (flux + accumulate) + lifting + stage,
            "pairs_counted": len(fluxes)}


def counts():
    out = {}
    for name, spec in WORKLOADS.items():
        N, ne = spec["N"], spec["ne"]
        n = (ne, ne, ne)
        xi, _ = oracle.lgl(N)
        gen = W.noisy_density_wave if spec["noisy"] else W.density_wave
        u = gen(3, N, n, W.box(3), xi)
        nelem = ne ** 3
        elems = np.random.default_rng(ne).choice(nelem, size=SAMPLE_ELEMENTS, replace=False)
        out[name] = volume_counts(N, u, nelem, sorted(int(e) for e in elems))
    for N in ENSEMBLE_DEGREES:
        n = (8, 8, 8)
        xi, _ = oracle.lgl(N)
        u = W.density_wave(3, N, n, W.box(3), xi, amplitude=0.5, velocity=(0.1, 0.2, -0.1))
        out[f"ensemble_member_n{N}"] = volume_counts(N, u, 512, list(range(0, 512, 37)))
    return out


if __name__ == "__main__":
    data = {"note": "algorithmic operations per node of the fused volume kernel, counted by "
                    "the oracle's operation-counting build (tests/golden/make_op_counts.py)",
            "workloads": counts()}
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    print(json.dumps(data, indent=1, sort_keys=True))
