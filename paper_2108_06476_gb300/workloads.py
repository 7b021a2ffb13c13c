"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module holds no arithmetic of the method itself: it evaluates initial
states (density waves, seeded noise, cotangents) at node coordinates that the
caller supplies from the 1D node positions of whichever side it is testing,
and it draws the seeded ensemble descriptions. All states are float64 in the
layout u[e][v][k][j][i] (element-major; within an element, variable, then
nodes with x fastest; elements lexicographic with x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np


def node_coordinates(d, N, n, dom, xi):
    """Physical coordinates of every node, shape (d, n_elem, (N+1)^d).

    Element (ex, ey[, ez]) covers [lo + ex h, lo + (ex+1) h] per direction;
    reference node xi in [-1, 1] maps to lo + (ex + (xi + 1)/2) h."""
    xi = np.asarray(xi, dtype=np.float64)
    np1 = N + 1
    n = list(n)
    h = [(dom[2 * k + 1] - dom[2 * k]) / n[k] for k in range(d)]
    # element coordinate grids, x fastest
    eidx = np.indices(n[::-1]).reshape(d, -1)[::-1]  # eidx[k] = element index along k
    nidx = np.indices([np1] * d).reshape(d, -1)[::-1]  # node index along k, x fastest
    X = np.empty((d, eidx.shape[1], nidx.shape[1]))
    for k in range(d):
        X[k] = dom[2 * k] + (eidx[k][:, None] + 0.5 * (xi[nidx[k]][None, :] + 1.0)) * h[k]
    return X


def prim_to_cons(rho, v, p, gamma=1.4):
    """Conserved state (rho, rho v, E) from primitives; the ideal-gas energy
    E = p/(gamma-1) + rho |v|^2 / 2 defines the initial condition."""
    d = len(v)
    v2 = sum(vk * vk for vk in v)
    out = [rho] + [rho * vk for vk in v] + [p / (gamma - 1.0) + 0.5 * rho * v2]
    return np.stack(out, axis=1).reshape(rho.shape[0], d + 2, -1)


def density_wave(d, N, n, dom, xi, amplitude=0.98, velocity=None, pressure=20.0, gamma=1.4,
                 t=0.0):
    """rho = 1 + A sin(pi (sum_k x_k - t sum_k v_k)), constant v and p: an exact
    solution of the Euler equations on a periodic [-1, 1]^d box."""
    if velocity is None:
        velocity = (0.1, 0.2, 0.3)[:d]
    X = node_coordinates(d, N, n, dom, xi)
    phase = X.sum(axis=0) - t * float(np.sum(velocity))
    rho = 1.0 + amplitude * np.sin(np.pi * phase)
    v = [np.full_like(rho, velocity[k]) for k in range(d)]
    p = np.full_like(rho, pressure)
    return np.ascontiguousarray(prim_to_cons(rho, v, p, gamma).reshape(-1))


def noisy_density_wave(d, N, n, dom, xi, seed=0, noise=1.0e-2, amplitude=0.98, velocity=None,
                       pressure=20.0, gamma=1.4):
    """Density wave plus independent uniform noise of the given amplitude on
    rho, every v_k and p at every node (drawn in layout order from
    numpy default_rng(seed))."""
    if velocity is None:
        velocity = (0.1, 0.2, 0.3)[:d]
    X = node_coordinates(d, N, n, dom, xi)
    rho = 1.0 + amplitude * np.sin(np.pi * X.sum(axis=0))
    rng = np.random.default_rng(seed)
    r = rng.uniform(-1.0, 1.0, size=(rho.shape[0], d + 2, rho.shape[1])) * noise
    rho = rho + r[:, 0]
    v = [velocity[k] + r[:, 1 + k] for k in range(d)]
    p = pressure + r[:, d + 1]
    return np.ascontiguousarray(prim_to_cons(rho, v, p, gamma).reshape(-1))


def uniform_state(d, N, n, rho=1.3, velocity=None, pressure=7.0, gamma=1.4):
    """A constant state (free stream)."""
    if velocity is None:
        velocity = (0.3, -0.2, 0.1)[:d]
    ne = int(np.prod(n))
    P = (N + 1) ** d
    r = np.full((ne, P), rho)
    v = [np.full((ne, P), velocity[k]) for k in range(d)]
    p = np.full((ne, P), pressure)
    return np.ascontiguousarray(prim_to_cons(r, v, p, gamma).reshape(-1))


def random_state(d, N, n, seed=0, gamma=1.4):
    """Seeded random but physical state: rho in [0.5, 2], v in [-0.5, 0.5]^d,
    p in [0.5, 3], independent per node."""
    rng = np.random.default_rng(seed)
    ne = int(np.prod(n))
    P = (N + 1) ** d
    rho = rng.uniform(0.5, 2.0, size=(ne, P))
    v = [rng.uniform(-0.5, 0.5, size=(ne, P)) for _ in range(d)]
    p = rng.uniform(0.5, 3.0, size=(ne, P))
    return np.ascontiguousarray(prim_to_cons(rho, v, p, gamma).reshape(-1))


def gaussian(size, seed=0):
    """i.i.d. N(0, 1) entries (cotangents, random directions)."""
    return np.random.default_rng(seed).standard_normal(size)


@dataclass
class EnsembleMember:
    d: int
    N: int
    n: tuple
    amplitude: float
    velocity: tuple
    pressure: float


def ensemble(n_sims=48, seed=0, n_range=(8, 24), degrees=(3, 4, 5), pressure=20.0):
    """Seeded ensemble of independent periodic 3D density-wave simulations on
    [-1, 1]^3: per member (generator default_rng([seed, member])) elements per
    dimension uniform in n_range, N from degrees, amplitude in [0.1, 0.98],
    velocity in [-0.3, 0.3]^3."""
    out = []
    for s in range(n_sims):
        rng = np.random.default_rng([seed, s])
        ne = int(rng.integers(n_range[0], n_range[1] + 1))
        N = int(rng.choice(degrees))
        A = float(rng.uniform(0.1, 0.98))
        v = tuple(float(x) for x in rng.uniform(-0.3, 0.3, size=3))
        out.append(EnsembleMember(3, N, (ne, ne, ne), A, v, pressure))
    return out


def ensemble_state(members, nodes_of_degree):
    """Concatenated initial states of ensemble members (density waves with
    each member's amplitude, velocity and pressure on [-1, 1]^3);
    nodes_of_degree(N) gives the 1D node positions."""
    parts = []
    for m in members:
        parts.append(density_wave(3, m.N, m.n, box(3), nodes_of_degree(m.N),
                                  amplitude=m.amplitude, velocity=m.velocity,
                                  pressure=m.pressure))
    return np.ascontiguousarray(np.concatenate(parts))


def warped_node_coordinates(N, n, xi, warp=0.15):
    """Physical node coordinates, shape (3, n_elem, (N+1)^3), of the periodic
    box [-1,1]^3 of n[0] x n[1] x n[2] elements warped by the mapping of the
    paper's curvilinear benchmark: Cartesian reference coordinates c of the
    box go to y = c1 + a cos(1.5 pi c0) cos(0.5 pi c1) cos(0.5 pi c2), then
    x = c0 + a cos(0.5 pi c0) cos(2 pi y) cos(0.5 pi c2), then
    z = c2 + a cos(0.5 pi x) cos(pi y) cos(0.5 pi c2), with a = warp."""
    c0, c1, c2 = node_coordinates(3, N, n, box(3), xi)
    pi = np.pi
    y = c1 + warp * np.cos(1.5 * pi * c0) * np.cos(0.5 * pi * c1) * np.cos(0.5 * pi * c2)
    x = c0 + warp * np.cos(0.5 * pi * c0) * np.cos(2.0 * pi * y) * np.cos(0.5 * pi * c2)
    z = c2 + warp * np.cos(0.5 * pi * x) * np.cos(pi * y) * np.cos(0.5 * pi * c2)
    return np.stack([x, y, z])


def manufactured_state(X, t=0.0, amplitude=0.1):
    """The manufactured solution used with source terms: rho = 2 +
    A sin(pi (x + y + z - t)), v = (1, 1, 1), E = rho^2, at the node
    coordinates X (3, n_elem, P); flat state in the usual layout."""
    rho = 2.0 + amplitude * np.sin(np.pi * (X[0] + X[1] + X[2] - t))
    u = np.stack([rho, rho, rho, rho, rho * rho], axis=1)
    return np.ascontiguousarray(u.reshape(-1))


def alfven_wave(N, n, xi, t=0.0, amplitude=0.1, gamma=5.0 / 3.0, pressure=0.1):
    """Circularly polarised Alfven wave on the periodic box [-1,1]^3 (3D ideal
    MHD state (rho, rho v, E, B), E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2):
    rho = 1, p = pressure, B = n + A (sin phi e1 + cos phi e2),
    v = -A (sin phi e1 + cos phi e2), phi = pi (x + y + z) - pi sqrt(3) t,
    n = (1,1,1)/sqrt(3), e1 = (1,-1,0)/sqrt(2), e2 = n x e1: a wave moving
    along n at the Alfven speed |B.n|/sqrt(rho) = 1, an exact solution."""
    return alfven_wave_at(node_coordinates(3, N, n, box(3), xi), t, amplitude, gamma, pressure)


def alfven_wave_at(X, t=0.0, amplitude=0.1, gamma=5.0 / 3.0, pressure=0.1):
    """The Alfven wave of alfven_wave at given node coordinates X (3, n_elem,
    nodes per element), e.g. those of the warped box."""
    phi = np.pi * (X[0] + X[1] + X[2]) - np.pi * np.sqrt(3.0) * t
    nv = np.ones(3) / np.sqrt(3.0)
    e1 = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    e2 = np.cross(nv, e1)
    s, c = np.sin(phi), np.cos(phi)
    B = [nv[k] + amplitude * (s * e1[k] + c * e2[k]) for k in range(3)]
    v = [-amplitude * (s * e1[k] + c * e2[k]) for k in range(3)]
    rho = np.ones_like(phi)
    v2 = sum(vk * vk for vk in v)
    b2 = sum(bk * bk for bk in B)
    E = pressure / (gamma - 1.0) + 0.5 * rho * v2 + 0.5 * b2
    u = np.stack([rho, *(rho * vk for vk in v), E, *B], axis=1)
    return np.ascontiguousarray(u.reshape(-1))


def mhd_random_state(N, n, seed=0, gamma=5.0 / 3.0):
    """Seeded random physical MHD state: rho U[0.5, 2], v U[-0.5, 0.5]^3,
    p U[0.5, 3], B U[-1, 1]^3 per node."""
    rng = np.random.default_rng(seed)
    ne = int(np.prod(n))
    P = (N + 1) ** 3
    rho = rng.uniform(0.5, 2.0, size=(ne, P))
    v = [rng.uniform(-0.5, 0.5, size=(ne, P)) for _ in range(3)]
    p = rng.uniform(0.5, 3.0, size=(ne, P))
    B = [rng.uniform(-1.0, 1.0, size=(ne, P)) for _ in range(3)]
    v2 = sum(vk * vk for vk in v)
    b2 = sum(bk * bk for bk in B)
    E = p / (gamma - 1.0) + 0.5 * rho * v2 + 0.5 * b2
    u = np.stack([rho, *(rho * vk for vk in v), E, *B], axis=1)
    return np.ascontiguousarray(u.reshape(-1))


def box(d, lo=-1.0, hi=1.0):
    """Domain [lo, hi]^d as [lo0, hi0, lo1, hi1, ...]."""
    return np.array([lo, hi] * d, dtype=np.float64)
