"""ctypes front end of the plain FP64 CPU oracle (``dgsem_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is imported by ``tests/``,
``__graft_entry__.smoke()`` and the cpu_baseline / reference legs of
``bench.py``, never by the product package. It shares no code with the CUDA
library. Every function here only marshals numpy arrays to the C routines;
the arithmetic (and its citations) lives in ``dgsem_oracle.c``.

All arrays use the state layout u[e][v][k][j][i] (element-major, variable,
then nodes with x fastest), float64, C-contiguous.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgsem_oracle.c")
_SRC_CURVED = os.path.join(_HERE, "dgsem_curved.c")
_SRC_MHD = os.path.join(_HERE, "dgsem_mhd.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP): with
    double, with double complex (complex-step JVP), with long double (the
    extended-precision evaluation used to measure FP64 rounding errors) and,
    as C++, with an operation-counting scalar (the algorithmic work of the
    method's pieces), plus the curvilinear-mesh operator and the MHD operator
    (double)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_CURVED),
                 os.path.getmtime(_SRC_MHD), os.path.getmtime(os.path.join(_HERE, "op_count.hpp")))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    bdir = os.path.join(_HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp", "-std=c11"]
    o1 = os.path.join(bdir, "or_real.o")
    o2 = os.path.join(bdir, "or_cstep.o")
    o3 = os.path.join(bdir, "or_ld.o")
    o4 = os.path.join(bdir, "or_curved.o")
    o5 = os.path.join(bdir, "or_mhd.o")
    o6 = os.path.join(bdir, "or_count.o")
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *flags, "-c", _SRC, "-o", o1])
    # the operation-counting build: the same source as C++ with a counting
    # scalar (op_count.hpp), single-threaded
    subprocess.check_call(["g++", "-x", "c++", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-DOR_COUNT", "-c", _SRC, "-o", o6])
    subprocess.check_call(["gcc", *flags, "-DOR_CSTEP", "-c", _SRC, "-o", o2])
    subprocess.check_call(["gcc", *flags, "-DOR_LONGDOUBLE", "-c", _SRC, "-o", o3])
    subprocess.check_call(["gcc", *flags, "-c", _SRC_CURVED, "-o", o4])
    subprocess.check_call(["gcc", *flags, "-c", _SRC_MHD, "-o", o5])
    subprocess.check_call(["g++", "-shared", "-fopenmp", o1, o2, o3, o4, o5, o6, "-o", tmp,
                           "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _declare(L):
    """Argument types of the oracle's C entry points on a loaded library."""
    L.or_lgl.argtypes = [ctypes.c_int, _dp, _dp]
    L.or_diff_matrix.argtypes = [ctypes.c_int, _dp, _dp]
    L.or_dtilde.argtypes = [ctypes.c_int, _dp, _dp]
    L.or_lsrk_coefficients.argtypes = [_dp, _dp, _dp]
    L.or_ln_mean.argtypes = [ctypes.c_double, ctypes.c_double]
    L.or_ln_mean.restype = ctypes.c_double
    L.or_two_point.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               _dp, _dp, _dp]
    rhs_args = [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_double, ctypes.c_int,
                ctypes.c_int]
    L.or_rhs.argtypes = rhs_args + [_dp, _dp, _llp, ctypes.c_longlong, ctypes.c_int]
    L.or_set_direction_mask.argtypes = [ctypes.c_int]
    if hasattr(L, "orn_ops_two_point"):  # the counting build (not in planted-mistake variants)
        L.orn_ops_two_point.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _dp, _dp]
        L.orn_ops_two_point.restype = ctypes.c_longlong
        L.orn_ops_cons2prim.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.orn_ops_cons2prim.restype = ctypes.c_longlong
        L.orn_ops_rhs.argtypes = rhs_args + [_dp, _llp, ctypes.c_longlong]
        L.orn_ops_rhs.restype = ctypes.c_longlong
    L.or_rhs_jvp.argtypes = rhs_args + [_dp, _dp, _dp, _llp, ctypes.c_longlong,
                                        ctypes.c_int]
    L.orl_rhs.argtypes = rhs_args + [ctypes.c_void_p, ctypes.c_void_p, _llp,
                                     ctypes.c_longlong, ctypes.c_int]
    L.or_rk_stage.argtypes = [ctypes.c_longlong, _dp, _dp, _dp, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double]
    L.or_max_dt.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_double,
                            ctypes.c_double, _dp]
    L.or_max_dt.restype = ctypes.c_double
    L.or_integrals.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, ctypes.c_double, _dp,
                               _dp]
    if hasattr(L, "or_curved_rhs"):  # variant builds of dgsem_oracle.c alone lack these
        L.or_curved_geometry.argtypes = [ctypes.c_int, _ip, ctypes.c_double, _dp, _dp, _dp]
        L.or_curved_rhs.argtypes = [ctypes.c_int, _ip, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                    _dp, _dp, _llp, ctypes.c_longlong, ctypes.c_int]
        L.or_curved_max_dt.argtypes = [ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double,
                                       _dp, _dp, _dp]
        L.or_curved_max_dt.restype = ctypes.c_double
        L.or_manufactured_state.argtypes = [ctypes.c_double, _dp, _dp]
        L.or_manufactured_source.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
    if hasattr(L, "or_mhd_rhs"):
        L.or_mhd_flux.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
        L.or_mhd_fast_speed.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        L.or_mhd_fast_speed.restype = ctypes.c_double
        L.or_mhd_llf.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        L.or_mhd_hll.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        L.or_mhd_flux_ec.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        L.or_mhd_rhs.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, _dp, _dp, _llp, ctypes.c_longlong,
                                 ctypes.c_int]
        L.or_mhd_max_dt.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.or_mhd_max_dt.restype = ctypes.c_double
        L.or_mhd_curved_rhs.argtypes = [ctypes.c_int, _ip, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _llp,
                                        ctypes.c_longlong, ctypes.c_int]
        L.or_mhd_curved_max_dt.argtypes = [ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double,
                                           _dp, _dp, _dp]
        L.or_mhd_curved_max_dt.restype = ctypes.c_double
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _declare(ctypes.CDLL(_SO))
    return _lib


def build_variant(src_text: str, out_dir: str, curved_text: str | None = None,
                  mhd_text: str | None = None) -> str:
    """Compile a (modified) copy of the oracle source into out_dir, for tests
    that plant mistakes and check that the pins catch them; curved_text and
    mhd_text, when given, replace the curvilinear and the MHD sources too."""
    src = os.path.join(out_dir, "variant.c")
    with open(src, "w") as fh:
        fh.write(src_text)
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp", "-std=c11"]
    objs = []
    for tag, defs in (("r", []), ("c", ["-DOR_CSTEP"]), ("l", ["-DOR_LONGDOUBLE"])):
        o = os.path.join(out_dir, f"v_{tag}.o")
        subprocess.check_call(["gcc", *flags, *defs, "-c", src, "-o", o])
        objs.append(o)
    if curved_text is not None:
        csrc = os.path.join(out_dir, "variant_curved.c")
        with open(csrc, "w") as fh:
            fh.write(curved_text)
        o = os.path.join(out_dir, "v_curved.o")
        subprocess.check_call(["gcc", *flags, "-c", csrc, "-o", o])
        objs.append(o)
    if mhd_text is not None:
        msrc = os.path.join(out_dir, "variant_mhd.c")
        with open(msrc, "w") as fh:
            fh.write(mhd_text)
        o = os.path.join(out_dir, "v_mhd.o")
        subprocess.check_call(["gcc", *flags, "-c", msrc, "-o", o])
        objs.append(o)
    so = os.path.join(out_dir, "libvariant.so")
    subprocess.check_call(["gcc", "-shared", "-fopenmp", *objs, "-o", so, "-lm"])
    return so


class use_library:
    """Context manager: route this module's functions to another build."""

    def __init__(self, so_path):
        self.so_path = so_path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _declare(ctypes.CDLL(self.so_path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lgl(N: int):
    """LGL nodes and weights (xi, w), each of length N+1."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().or_lgl(N, _d(xi), _d(w)) != 0:
        raise ValueError("bad N")
    return xi, w


def diff_matrix(N: int, xi=None):
    """Nodal differentiation matrix D[i, j] = l_j'(xi_i)."""
    if xi is None:
        xi, _ = lgl(N)
    xi = _f64(xi)
    D = np.zeros((N + 1, N + 1))
    lib().or_diff_matrix(N, _d(xi), _d(D))
    return D


def dtilde(N: int):
    """Split-form volume matrix Dt = 2 D - W^-1 B (long double, rounded once)."""
    Dt = np.zeros((N + 1, N + 1))
    w = np.zeros(N + 1)
    if lib().or_dtilde(N, _d(Dt), _d(w)) != 0:
        raise ValueError("bad N")
    return Dt


def lsrk_coefficients():
    """Carpenter-Kennedy 5-stage 4th-order 2N-storage coefficients (A, B, c)."""
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().or_lsrk_coefficients(_d(A), _d(B), _d(c))
    return A, B, c


def ln_mean(x: float, y: float) -> float:
    return lib().or_ln_mean(float(x), float(y))


# two_point kinds: volume fluxes 0 Ranocha, 1 Chandrashekar, 2 central;
# surface fluxes 10 LLF, 11 Ranocha, 12 HLL, 13 Chandrashekar; 20 physical f(u_L)
RANOCHA, CHANDRASHEKAR, CENTRAL = 0, 1, 2
S_LLF, S_RANOCHA, S_HLL, S_CHANDRASHEKAR = 0, 1, 2, 3
PHYSICAL = 20


def two_point(kind: int, d: int, n: int, uL, uR, gamma: float = 1.4):
    uL, uR = _f64(uL), _f64(uR)
    f = np.zeros(d + 2)
    if lib().or_two_point(kind, d, n, gamma, _d(uL), _d(uR), _d(f)) != 0:
        raise ValueError("bad flux kind")
    return f


def ops_two_point(kind: int, d: int, n: int, uL, uR, gamma: float = 1.4) -> int:
    """Operations (+, -, *, /, log1p, sqrt) of one two-point flux of the
    oracle between conserved states, including its two primitive conversions
    (kind as two_point)."""
    r = lib().orn_ops_two_point(kind, d, n, gamma, _d(_f64(uL)), _d(_f64(uR)))
    if r < 0:
        raise ValueError("orn_ops_two_point: bad arguments")
    return int(r)


def ops_cons2prim(d: int, u, gamma: float = 1.4) -> int:
    """Operations of one conserved -> primitive conversion of the oracle."""
    return int(lib().orn_ops_cons2prim(d, gamma, _d(_f64(u))))


def ops_rhs(d, N, n, dom, u, gamma=1.4, vflux=RANOCHA, sflux=S_LLF, elems=None) -> int:
    """Operations of the oracle's whole rhs (both orders of every pair,
    primitives inside every flux) on the listed elements."""
    n_arr, dom = _mesh_args(d, n, dom)
    ep, ne, keep = _elems(elems)
    r = lib().orn_ops_rhs(d, N, n_arr, _d(dom), gamma, vflux, sflux, _d(_f64(u)), ep, ne)
    if r < 0:
        raise ValueError("orn_ops_rhs: bad arguments")
    return int(r)


def _mesh_args(d, n, dom):
    n_arr = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    dom = _f64(dom)
    return n_arr, dom


def _elems(elems):
    if elems is None:
        return None, 0, None
    e = np.ascontiguousarray(elems, dtype=np.int64)
    return e.ctypes.data_as(_llp), len(e), e


def rhs(d, N, n, dom, u, gamma=1.4, vflux=RANOCHA, sflux=S_LLF, elems=None, nthreads=0,
        out=None, directions=None):
    """du = rhs(u) (all elements, or only `elems`; other entries of du are 0,
    or left as they are in `out` when an output buffer is given).
    directions: evaluate only the volume and surface terms of these
    coordinate directions (their parts sum to the full rhs)."""
    n_arr, dom = _mesh_args(d, n, dom)
    u = _f64(u)
    if out is not None:
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == u.shape
        du = out
    else:
        du = np.zeros_like(u)
    ep, ne, keep = _elems(elems)
    L = lib()
    if directions is not None:
        L.or_set_direction_mask(sum(1 << int(k) for k in directions))
    try:
        rc = L.or_rhs(d, N, n_arr, _d(dom), gamma, vflux, sflux, _d(u), _d(du), ep, ne,
                      nthreads)
    finally:
        if directions is not None:
            L.or_set_direction_mask(7)
    if rc != 0:
        raise ValueError("or_rhs: bad arguments")
    return du


def rhs_extended(d, N, n, dom, u, gamma=1.4, vflux=RANOCHA, sflux=S_LLF, elems=None,
                 nthreads=0):
    """The same rhs evaluated in long double (returned as float64): a
    reference for the rounding error of FP64 evaluations."""
    n_arr, dom = _mesh_args(d, n, dom)
    ul = np.ascontiguousarray(u, dtype=np.longdouble)
    dul = np.zeros_like(ul)
    ep, ne, keep = _elems(elems)
    rc = lib().orl_rhs(d, N, n_arr, _d(dom), gamma, vflux, sflux,
                       ul.ctypes.data_as(ctypes.c_void_p), dul.ctypes.data_as(ctypes.c_void_p),
                       ep, ne, nthreads)
    if rc != 0:
        raise ValueError("orl_rhs: bad arguments")
    return dul.astype(np.float64)


def rhs_jvp(d, N, n, dom, u, v, gamma=1.4, vflux=RANOCHA, sflux=S_LLF, elems=None, nthreads=0):
    """J(u) v of the rhs by complex-step differentiation."""
    n_arr, dom = _mesh_args(d, n, dom)
    u, v = _f64(u), _f64(v)
    jv = np.zeros_like(u)
    ep, ne, keep = _elems(elems)
    rc = lib().or_rhs_jvp(d, N, n_arr, _d(dom), gamma, vflux, sflux, _d(u), _d(v), _d(jv), ep,
                          ne, nthreads)
    if rc != 0:
        raise ValueError("or_rhs_jvp failed")
    return jv


def rk_stage(u, k, du, a, b, dt):
    """In place: k <- a k + dt du; u <- u + b k (float64 contiguous arrays)."""
    for x in (u, k, du):
        assert x.dtype == np.float64 and x.flags.c_contiguous
    lib().or_rk_stage(u.size, _d(u), _d(k), _d(du), a, b, dt)


def max_dt(d, N, n, dom, u, cfl=0.5, gamma=1.4):
    n_arr, dom = _mesh_args(d, n, dom)
    u = _f64(u)
    return lib().or_max_dt(d, N, n_arr, _d(dom), gamma, cfl, _d(u))


def integrals(d, N, n, dom, u, gamma=1.4):
    """[rho, rho v_1..rho v_d, E, entropy S, kinetic energy] integrated."""
    n_arr, dom = _mesh_args(d, n, dom)
    u = _f64(u)
    out = np.zeros(d + 4)
    if lib().or_integrals(d, N, n_arr, _d(dom), gamma, _d(u), _d(out)) != 0:
        raise ValueError("bad mesh")
    return out


def lsrk_step(d, N, n, dom, u, dt, gamma=1.4, vflux=RANOCHA, sflux=S_LLF, nthreads=0):
    """One full Carpenter-Kennedy step (5 stages) on a copy of u."""
    A, B, _ = lsrk_coefficients()
    u = _f64(u).copy()
    k = np.zeros_like(u)
    for s in range(5):
        du = rhs(d, N, n, dom, u, gamma, vflux, sflux, nthreads=nthreads)
        rk_stage(u, k, du, A[s], B[s], dt)
    return u


# ---- curvilinear (warped) periodic box, 3D Euler (dgsem_curved.c) ----

class CurvedGeometry:
    """Node coordinates X[e][3][P], metric terms Ja[e][r][n][P] = (J a^r)_n
    and Jacobians J[e][P] of the warped periodic box [-1,1]^3."""

    def __init__(self, N, n, warp=0.15):
        self.N, self.n, self.warp = N, tuple(int(x) for x in n), float(warp)
        ne = int(np.prod(self.n))
        P = (N + 1) ** 3
        self.X = np.zeros((ne, 3, P))
        self.Ja = np.zeros((ne, 3, 3, P))
        self.J = np.zeros((ne, P))
        rc = lib().or_curved_geometry(N, _n3(self.n), self.warp, _d(self.X), _d(self.Ja),
                                      _d(self.J))
        if rc != 0:
            raise ValueError(f"or_curved_geometry failed ({rc})")


def _n3(n):
    return (ctypes.c_int * 3)(*[int(x) for x in n])


def curved_rhs(geom, u, vflux=RANOCHA, sflux=S_LLF, source=False, t=0.0, gamma=1.4,
               elems=None, out=None, nthreads=0):
    """du on the curved mesh (plus the manufactured source at time t)."""
    u = _f64(u)
    du = np.zeros_like(u) if out is None else out
    if elems is None:
        ep, ne = None, 0
    else:
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        ep, ne = elems.ctypes.data_as(_llp), len(elems)
    rc = lib().or_curved_rhs(geom.N, _n3(geom.n), gamma, vflux, sflux, int(bool(source)),
                             float(t), _d(geom.Ja), _d(geom.J), _d(geom.X), _d(u), _d(du), ep,
                             ne, nthreads)
    if rc != 0:
        raise ValueError("bad curved rhs arguments")
    return du


def curved_max_dt(geom, u, cfl=0.5, gamma=1.4):
    return lib().or_curved_max_dt(geom.N, _n3(geom.n), gamma, cfl, _d(geom.Ja), _d(geom.J),
                                  _d(_f64(u)))


def curved_lsrk_step(geom, u, dt, t=0.0, vflux=RANOCHA, sflux=S_LLF, source=False, gamma=1.4,
                     nthreads=0):
    """One Carpenter-Kennedy step on a copy of u; stage s evaluates the source
    at t + c_s dt."""
    A, B, C = lsrk_coefficients()
    u = _f64(u).copy()
    k = np.zeros_like(u)
    for s in range(5):
        du = curved_rhs(geom, u, vflux, sflux, source, t + C[s] * dt, gamma, nthreads=nthreads)
        rk_stage(u, k, du, A[s], B[s], dt)
    return u


def manufactured_state_at(t, X):
    """The manufactured state at one point X (3,)."""
    x = np.ascontiguousarray(X, dtype=np.float64)
    u = np.zeros(5)
    lib().or_manufactured_state(float(t), _d(x), _d(u))
    return u


def manufactured_source_at(t, X, gamma=1.4):
    x = np.ascontiguousarray(X, dtype=np.float64)
    S = np.zeros(5)
    lib().or_manufactured_source(float(gamma), float(t), _d(x), _d(S))
    return S


# ---- 3D ideal MHD on the Cartesian periodic mesh (dgsem_mhd.c) ----

def mhd_flux(n, u, gamma=5.0 / 3.0):
    f = np.zeros(8)
    lib().or_mhd_flux(n, gamma, _d(_f64(u)), _d(f))
    return f


def mhd_fast_speed(n, u, gamma=5.0 / 3.0):
    return lib().or_mhd_fast_speed(n, gamma, _d(_f64(u)))


def mhd_llf(n, uL, uR, gamma=5.0 / 3.0):
    f = np.zeros(8)
    lib().or_mhd_llf(n, gamma, _d(_f64(uL)), _d(_f64(uR)), _d(f))
    return f


MHD_SFLUX = {"llf": 0, "hll": 1, "ec": 2}
MHD_VFLUX = {"central": 0, "ec": 1}


def mhd_flux_ec(n, uL, uR, gamma=5.0 / 3.0):
    f = np.zeros(8)
    lib().or_mhd_flux_ec(n, gamma, _d(_f64(uL)), _d(_f64(uR)), _d(f))
    return f


def mhd_hll(n, uL, uR, gamma=5.0 / 3.0):
    f = np.zeros(8)
    lib().or_mhd_hll(n, gamma, _d(_f64(uL)), _d(_f64(uR)), _d(f))
    return f


def mhd_rhs(N, n, dom, u, gamma=5.0 / 3.0, powell=True, elems=None, out=None, nthreads=0,
            sflux="llf", vflux="central"):
    """du of the MHD operator (+ the Powell term): volume flux "central" (the
    weak form) or "ec"; surface flux "llf", "hll" or "ec"."""
    u = _f64(u)
    du = np.zeros_like(u) if out is None else out
    if elems is None:
        ep, ne = None, 0
    else:
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        ep, ne = elems.ctypes.data_as(_llp), len(elems)
    rc = lib().or_mhd_rhs(N, _n3(n), _d(_f64(dom)), gamma, int(bool(powell)),
                          MHD_VFLUX[vflux], MHD_SFLUX[sflux], _d(u), _d(du), ep, ne, nthreads)
    if rc != 0:
        raise ValueError("bad MHD rhs arguments")
    return du


def mhd_max_dt(N, n, dom, u, cfl=0.5, gamma=5.0 / 3.0):
    return lib().or_mhd_max_dt(N, _n3(n), _d(_f64(dom)), gamma, cfl, _d(_f64(u)))


def mhd_lsrk_step(N, n, dom, u, dt, gamma=5.0 / 3.0, powell=True, nthreads=0, sflux="llf",
                  vflux="central"):
    A, B, _ = lsrk_coefficients()
    u = _f64(u).copy()
    k = np.zeros_like(u)
    for s in range(5):
        du = mhd_rhs(N, n, dom, u, gamma, powell, nthreads=nthreads, sflux=sflux, vflux=vflux)
        rk_stage(u, k, du, A[s], B[s], dt)
    return u


def mhd_curved_rhs(geom, u, gamma=5.0 / 3.0, powell=True, vflux="central", sflux="llf",
                   elems=None, nthreads=0):
    """du of the MHD operator on the warped box (geometry from CurvedGeometry)."""
    u = _f64(u)
    du = np.zeros_like(u)
    if elems is None:
        ep, ne = None, 0
    else:
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        ep, ne = elems.ctypes.data_as(_llp), len(elems)
    rc = lib().or_mhd_curved_rhs(geom.N, _n3(geom.n), gamma, int(bool(powell)), MHD_VFLUX[vflux],
                                 MHD_SFLUX[sflux], _d(geom.Ja), _d(geom.J), _d(u), _d(du), ep,
                                 ne, nthreads)
    if rc != 0:
        raise ValueError("bad curved MHD rhs arguments")
    return du


def mhd_curved_max_dt(geom, u, cfl=0.5, gamma=5.0 / 3.0):
    return lib().or_mhd_curved_max_dt(geom.N, _n3(geom.n), gamma, cfl, _d(geom.Ja), _d(geom.J),
                                      _d(_f64(u)))
