"""Python binding of libdgsem.so: argument marshalling only.

Every step of the rhs, the RK stage, the time step and the integrals runs in
the library's CUDA kernels; torch provides device memory and streams. There
is no CPU fallback: if the shared library is missing or cannot be loaded,
every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libdgsem.so")

VFLUX = {"ranocha": 0, "chandrashekar": 1, "central": 2, "ec": 3}
SFLUX = {"llf": 0, "ranocha": 1, "hll": 2, "chandrashekar": 3, "ec": 4}
PRECISION = {"fp64": 0, "fp32": 1}

# Carpenter-Kennedy (1994) five-stage fourth-order 2N-storage coefficients
RK_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
RK_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
        2277821191437.0 / 14882151754819.0)

EXPORTS = ("dg_mesh_create", "dg_mesh_create_curved", "dg_mesh_create_mhd",
           "dg_mesh_create_mhd_curved", "dg_set_source", "dg_set_time",
           "dg_get_time", "dg_mesh_destroy", "dg_mesh_info", "dg_mesh_set_stream",
           "dg_lgl_nodes", "dg_rhs", "dg_rhs_part", "dg_rhs_vjp", "dg_rk_stage", "dg_rk_reset", "dg_step", "dg_step_cfl", "dg_step_graph",
           "dg_step_dt", "dg_step_cfl_host", "dg_last_dt", "dg_max_dt",
           "dg_integrals", "dg_mesh_check", "dg_last_error", "dg_rhs_noalloc",
           "dg_ensemble_create", "dg_ensemble_destroy", "dg_ensemble_info",
           "dg_ensemble_set_dt", "dg_ensemble_get_dt", "dg_ensemble_compute_dt",
           "dg_ensemble_stage", "dg_ensemble_step", "dg_ensemble_step_graph",
           "dg_ensemble_rk_reset", "dg_ensemble_check", "dg_ensemble_set_block",
           "dg_ensemble_get_block", "dg_ensemble_tune", "dg_measure_peaks",
           "dg_selftest_arith", "dg_mesh_set_nodes", "dg_mesh_set_metric",
           "dg_ensemble_set_pair_parallel", "dg_ensemble_get_pair_parallel",
           "dg_measure_fp64_issue")


class DGError(RuntimeError):
    pass


class _Options(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("volume_flux", ctypes.c_int),
                ("surface_flux", ctypes.c_int), ("precision", ctypes.c_int)]


_lib = None


def load(path: str = SO_PATH):
    """Load the shared library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise DGError(f"libdgsem.so not built ({path}); run paper_2108_06476_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, dp, ip, llp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), \
        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)
    L.dg_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp, ctypes.POINTER(_Options), vp,
                                 ctypes.POINTER(vp)]
    L.dg_mesh_destroy.argtypes = [vp]
    L.dg_mesh_info.argtypes = [vp, llp, ip, llp]
    L.dg_mesh_set_stream.argtypes = [vp, vp]
    L.dg_lgl_nodes.argtypes = [ctypes.c_int, dp, dp]
    L.dg_rhs.argtypes = [vp, vp, vp]
    L.dg_rhs_part.argtypes = [vp, vp, vp, ctypes.c_int]
    L.dg_rhs_vjp.argtypes = [vp, vp, vp, vp]
    L.dg_rk_stage.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.dg_rk_reset.argtypes = [vp]
    L.dg_step.argtypes = [vp, vp, vp, ctypes.c_double]
    L.dg_step_cfl.argtypes = [vp, vp, ctypes.c_double]
    L.dg_step_graph.argtypes = [vp, vp, ctypes.c_double]
    L.dg_step_cfl_host.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int]
    L.dg_step_dt.argtypes = [vp, vp, ctypes.c_double]
    L.dg_mesh_create_curved.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_double, vp, vp, vp]
    L.dg_mesh_create_mhd.argtypes = [ctypes.c_int, ip, dp, ctypes.POINTER(_Options), ctypes.c_int,
                                     vp, ctypes.POINTER(vp)]
    L.dg_mesh_create_mhd_curved.argtypes = [ctypes.c_int, ip, ctypes.c_double,
                                            ctypes.POINTER(_Options), ctypes.c_int, vp,
                                            ctypes.POINTER(vp)]
    L.dg_set_source.argtypes = [vp, ctypes.c_int]
    L.dg_set_time.argtypes = [vp, ctypes.c_double]
    L.dg_get_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.dg_last_dt.argtypes = [vp, dp]
    L.dg_max_dt.argtypes = [vp, vp, ctypes.c_double, dp]
    L.dg_integrals.argtypes = [vp, vp, dp]
    L.dg_mesh_check.argtypes = [vp, ip]
    L.dg_rhs_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ip, dp, vp, vp, vp, vp]
    L.dg_ensemble_create.argtypes = [ctypes.c_int, ip, ip, ip, dp, ctypes.POINTER(_Options), vp,
                                     ctypes.POINTER(vp)]
    L.dg_ensemble_destroy.argtypes = [vp]
    L.dg_ensemble_info.argtypes = [vp, llp, llp, llp]
    L.dg_ensemble_set_dt.argtypes = [vp, dp]
    L.dg_ensemble_get_dt.argtypes = [vp, dp]
    L.dg_ensemble_compute_dt.argtypes = [vp, vp, ctypes.c_double]
    L.dg_ensemble_stage.argtypes = [vp, vp, vp, ctypes.c_int]
    L.dg_ensemble_step.argtypes = [vp, vp, ctypes.c_double]
    L.dg_ensemble_step_graph.argtypes = [vp, vp, ctypes.c_double]
    L.dg_ensemble_rk_reset.argtypes = [vp]
    L.dg_ensemble_check.argtypes = [vp, ip]
    L.dg_ensemble_set_block.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.dg_ensemble_get_block.argtypes = [vp, ip, ip, ip]
    L.dg_ensemble_set_pair_parallel.argtypes = [vp, ctypes.c_int]
    L.dg_ensemble_get_pair_parallel.argtypes = [vp, ip]
    L.dg_measure_peaks.argtypes = [dp, dp, ip, vp]
    L.dg_measure_fp64_issue.argtypes = [dp, dp, vp]
    L.dg_selftest_arith.argtypes = [ctypes.c_int, vp, vp, ctypes.c_longlong, vp]
    L.dg_mesh_set_nodes.argtypes = [vp, vp]
    L.dg_mesh_set_metric.argtypes = [vp, vp, vp]
    L.dg_ensemble_tune.argtypes = [vp, vp, vp, ip, ip, ctypes.POINTER(ctypes.c_float)]
    L.dg_last_error.restype = ctypes.c_char_p
    L.dg_last_error.argtypes = []
    for name in EXPORTS:
        getattr(L, name).restype = ctypes.c_char_p if name == "dg_last_error" else ctypes.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().dg_last_error().decode(errors="replace")
        raise DGError(f"{what} failed ({rc}): {msg}")


def measure_peaks(fp64=True, fp32=True, stream=None):
    """Measured FP64/FP32 vector FMA throughput (TFLOP/s) and SM count of the
    current device (dg_measure_peaks)."""
    import torch
    L = load()
    a, b, n = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int(0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(L.dg_measure_peaks(ctypes.byref(a) if fp64 else None, ctypes.byref(b) if fp32 else None,
                              ctypes.byref(n), ctypes.c_void_p(st.cuda_stream)),
           "dg_measure_peaks")
    return {"fp64_tflops": a.value if fp64 else None, "fp32_tflops": b.value if fp32 else None,
            "sm_count": n.value}


def measure_fp64_issue(stream=None):
    """SM cycles per dependent FP64 FMA of one warp per SM with 32 active
    lanes and with one (dg_measure_fp64_issue)."""
    import torch
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load().dg_measure_fp64_issue(ctypes.byref(a), ctypes.byref(b),
                                        ctypes.c_void_p(st.cuda_stream)), "dg_measure_fp64_issue")
    return {"cycles_full_warp": a.value, "cycles_one_lane": b.value}


def lgl_nodes(N: int):
    """The library's LGL nodes and weights (host numpy arrays)."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().dg_lgl_nodes(N, xi.ctypes.data_as(dp), w.ctypes.data_as(dp)), "dg_lgl_nodes")
    return xi, w


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class MeshSpec:
    d: int
    N: int
    n: tuple
    domain: tuple
    gamma: float = 1.4
    volume_flux: str = "ranocha"
    surface_flux: str = "llf"
    precision: str = "fp64"


SOURCE = {"none": 0, "manufactured": 1}


class Mesh:
    """A periodic DGSEM mesh on the current CUDA device: uniform Cartesian, or
    with warp given, the warped box [-1,1]^3 of the paper's curvilinear
    benchmark (3D, FP64; warp = 0.15 is the paper's amplitude). With
    equations="mhd": the 3D ideal MHD equations (eight variables; the weak
    form, or EC flux differencing with volume_flux="ec"; LLF, HLL or EC
    faces (surface_flux); the Powell term unless powell=False; FP64; gamma
    defaults to 5/3), on the Cartesian mesh or, with warp, the warped box.

    State tensors are float64 CUDA tensors of n_values entries in the layout
    u[e][v][k][j][i]; rhs outputs are float64 (fp64) or float32 (fp32)."""

    def __init__(self, d, N, n, domain=None, gamma=None, volume_flux="ranocha",
                 surface_flux="llf", precision="fp64", stream=None, warp=None,
                 equations="euler", powell=True):
        import torch
        self._torch = torch
        L = load()
        if domain is None:
            domain = (-1.0, 1.0) * d
        self.d, self.N, self.n = int(d), int(N), tuple(int(x) for x in n)
        self.domain = tuple(float(x) for x in domain)
        self.precision = precision
        self.equations = equations
        if equations not in ("euler", "mhd"):
            raise DGError(f"unknown equations {equations!r}")
        if gamma is None:
            gamma = 5.0 / 3.0 if equations == "mhd" else 1.4
        self.rhs_dtype = torch.float64 if precision == "fp64" else torch.float32
        opt = _Options(gamma, VFLUX[volume_flux], SFLUX[surface_flux], PRECISION[precision])
        n_arr = (ctypes.c_int * 3)(*(list(self.n) + [1] * (3 - len(self.n))))
        dom = (ctypes.c_double * 6)(*(list(self.domain) + [0.0] * (6 - len(self.domain))))
        h = ctypes.c_void_p()
        st = stream if stream is not None else torch.cuda.current_stream()
        self._stream = st
        self.warp = warp
        if equations == "mhd":
            if self.d != 3 or precision != "fp64":
                raise DGError("MHD meshes are 3D and FP64")
            vf = volume_flux if volume_flux in ("central", "ec") else "central"
            mopt = _Options(gamma, VFLUX[vf], SFLUX[surface_flux], PRECISION["fp64"])
            if warp is None:
                _check(L.dg_mesh_create_mhd(self.N, n_arr, dom, ctypes.byref(mopt),
                                            int(bool(powell)), ctypes.c_void_p(st.cuda_stream),
                                            ctypes.byref(h)), "dg_mesh_create_mhd")
            else:
                if tuple(self.domain) != (-1.0, 1.0) * 3:
                    raise DGError("curved meshes are the 3D box [-1,1]^3")
                _check(L.dg_mesh_create_mhd_curved(self.N, n_arr, float(warp), ctypes.byref(mopt),
                                                   int(bool(powell)),
                                                   ctypes.c_void_p(st.cuda_stream),
                                                   ctypes.byref(h)), "dg_mesh_create_mhd_curved")
        elif warp is None:
            _check(L.dg_mesh_create(self.d, self.N, n_arr, dom, ctypes.byref(opt),
                                    ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)),
                   "dg_mesh_create")
        else:
            if self.d != 3 or tuple(self.domain) != (-1.0, 1.0) * 3:
                raise DGError("curved meshes are the 3D box [-1,1]^3")
            _check(L.dg_mesh_create_curved(self.N, n_arr, float(warp), ctypes.byref(opt),
                                           ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)),
                   "dg_mesh_create_curved")
        self._h = h
        nn, nv, nvals = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong()
        _check(L.dg_mesh_info(h, ctypes.byref(nn), ctypes.byref(nv), ctypes.byref(nvals)),
               "dg_mesh_info")
        self.n_nodes, self.n_vars, self.n_values = nn.value, nv.value, nvals.value

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _sync_stream(self):
        st = self._torch.cuda.current_stream()
        if st.cuda_stream != self._stream.cuda_stream:
            _check(load().dg_mesh_set_stream(self._h, ctypes.c_void_p(st.cuda_stream)),
                   "dg_mesh_set_stream")
            self._stream = st

    def _check_state(self, u):
        t = self._torch
        if not (u.is_cuda and u.dtype == t.float64 and u.is_contiguous()
                and u.numel() == self.n_values):
            raise DGError("u must be a contiguous float64 CUDA tensor of n_values entries")

    def empty_rhs(self):
        return self._torch.empty(self.n_values, dtype=self.rhs_dtype, device="cuda")

    # -- compute --
    def rhs(self, u, du=None):
        self._check_state(u)
        if du is None:
            du = self.empty_rhs()
        if not (du.is_cuda and du.dtype == self.rhs_dtype and du.is_contiguous()
                and du.numel() == self.n_values):
            raise DGError("du has the wrong dtype, size or layout")
        self._sync_stream()
        _check(load().dg_rhs(self._h, _ptr(u), _ptr(du)), "dg_rhs")
        return du

    def rhs_vjp(self, u, w, ubar=None):
        """ubar = (d rhs / d u)^T w (float64 CUDA tensors of n_values)."""
        self._check_state(u)
        self._check_state(w)
        if ubar is None:
            ubar = self._torch.empty_like(u)
        self._check_state(ubar)
        self._sync_stream()
        _check(load().dg_rhs_vjp(self._h, _ptr(u), _ptr(w), _ptr(ubar)), "dg_rhs_vjp")
        return ubar

    def rhs_part(self, u, du, parts):
        """Launch only the surface kernel (parts=1), only the volume kernel
        (parts=2), both (3), or the volume kernel of the fused step with stage
        coefficients A = 1, B = 0 (6: k <- k + dt du, u unchanged); used to
        time the kernels separately."""
        self._sync_stream()
        _check(load().dg_rhs_part(self._h, _ptr(u), _ptr(du), int(parts)), "dg_rhs_part")

    def rk_stage(self, u, du, a, b, dt):
        self._check_state(u)
        self._sync_stream()
        _check(load().dg_rk_stage(self._h, _ptr(u), _ptr(du), float(a), float(b), float(dt)),
               "dg_rk_stage")

    def rk_reset(self):
        self._sync_stream()
        _check(load().dg_rk_reset(self._h), "dg_rk_reset")

    def step(self, u, dt, du=None):
        self._check_state(u)
        if du is None:
            du = self.empty_rhs()
        self._sync_stream()
        _check(load().dg_step(self._h, _ptr(u), _ptr(du), float(dt)), "dg_step")
        return du

    def step_cfl(self, u, cfl=0.5, graph=False):
        """One LSRK step with the CFL time step computed on the device and the
        stage updates fused into the volume kernel (optionally as a replayed
        CUDA graph)."""
        self._check_state(u)
        self._sync_stream()
        fn = load().dg_step_graph if graph else load().dg_step_cfl
        _check(fn(self._h, _ptr(u), float(cfl)), "dg_step_cfl")

    def set_nodes(self, X):
        """Curved meshes: take the node coordinates X (float64 CUDA tensor of
        n_elem x 3 x (N+1)^3, contiguous) and rebuild the metric terms."""
        t = self._torch
        P = (self.N + 1) ** 3
        if not (X.is_cuda and X.dtype == t.float64 and X.is_contiguous()
                and X.numel() == 3 * P * (self.n_nodes // P)):
            raise DGError("node coordinates must be a contiguous float64 CUDA tensor "
                          "of n_elem x 3 x (N+1)^3")
        self._sync_stream()
        _check(load().dg_mesh_set_nodes(self._h, _ptr(X)), "dg_mesh_set_nodes")

    def set_metric(self, Ja, J):
        """Curved meshes: take the metric terms Ja (n_elem x 3 x 3 x (N+1)^3)
        and Jacobians J (n_elem x (N+1)^3), float64 CUDA tensors."""
        t = self._torch
        for a, k in ((Ja, 9), (J, 1)):
            if not (a.is_cuda and a.dtype == t.float64 and a.is_contiguous()
                    and a.numel() == k * self.n_nodes):
                raise DGError("metric terms must be contiguous float64 CUDA tensors")
        self._sync_stream()
        _check(load().dg_mesh_set_metric(self._h, _ptr(Ja), _ptr(J)), "dg_mesh_set_metric")

    def set_source(self, kind):
        """Source terms on a curved mesh: "none" or "manufactured"."""
        _check(load().dg_set_source(self._h, SOURCE[kind]), "dg_set_source")

    def set_time(self, t):
        self._sync_stream()
        _check(load().dg_set_time(self._h, float(t)), "dg_set_time")

    @property
    def time(self):
        out = ctypes.c_double()
        _check(load().dg_get_time(self._h, ctypes.byref(out)), "dg_get_time")
        return out.value

    def step_dt(self, u, dt):
        """One LSRK step with the given time step, the stage updates fused
        into the volume kernel."""
        self._check_state(u)
        self._sync_stream()
        _check(load().dg_step_dt(self._h, _ptr(u), float(dt)), "dg_step_dt")

    def step_cfl_host(self, u, cfl=0.5, n_steps=1):
        """n_steps CFL steps on a state in host memory: a contiguous float64
        CPU tensor or numpy array of n_values entries, overwritten with the
        new state. Pinned tensors (pin_memory=True) are read and written by
        the kernels directly; other host memory is copied in and out."""
        t = self._torch
        if isinstance(u, t.Tensor):
            if u.is_cuda or u.dtype != t.float64 or not u.is_contiguous() \
                    or u.numel() != self.n_values:
                raise DGError("u must be a contiguous float64 CPU tensor of n_values entries")
            ptr = ctypes.c_void_p(u.data_ptr())
        else:
            import numpy as np
            if not (isinstance(u, np.ndarray) and u.dtype == np.float64
                    and u.flags["C_CONTIGUOUS"] and u.size == self.n_values):
                raise DGError("u must be a contiguous float64 array of n_values entries")
            ptr = ctypes.c_void_p(u.ctypes.data)
        self._sync_stream()
        _check(load().dg_step_cfl_host(self._h, ptr, float(cfl), int(n_steps)),
               "dg_step_cfl_host")

    def last_dt(self):
        out = ctypes.c_double()
        _check(load().dg_last_dt(self._h, ctypes.byref(out)), "dg_last_dt")
        return out.value

    def max_dt(self, u, cfl=0.5):
        self._check_state(u)
        self._sync_stream()
        out = ctypes.c_double()
        _check(load().dg_max_dt(self._h, _ptr(u), float(cfl), ctypes.byref(out)), "dg_max_dt")
        return out.value

    def integrals(self, u):
        self._check_state(u)
        self._sync_stream()
        out = np.zeros(self.d + 4)
        _check(load().dg_integrals(self._h, _ptr(u),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "dg_integrals")
        return out

    def check(self):
        """Synchronise and raise DGError if a non-physical state was met."""
        self._sync_stream()
        flags = ctypes.c_int()
        rc = load().dg_mesh_check(self._h, ctypes.byref(flags))
        if rc != 0:
            _check(rc, "dg_mesh_check")
        return flags.value


class Ensemble:
    """A batch of independent 3D periodic Euler meshes with degrees N[s] in
    {3, 4, 5} and n[s]^3 elements on the boxes domains[s] ((lo, hi) per
    direction; default [-1, 1]^3), advanced together (one kernel launch per
    Runge-Kutta stage). The state of all members is one float64 CUDA tensor;
    member s is the slice offsets[s]:offsets[s+1]."""

    def __init__(self, N, n, gamma=1.4, surface_flux="llf", precision="fp64", stream=None,
                 domains=None, d=None):
        import torch
        self._torch = torch
        L = load()
        self.N = [int(x) for x in N]
        self.n = [int(x) for x in n]
        self.n_sims = len(self.N)
        opt = _Options(gamma, VFLUX["ranocha"], SFLUX[surface_flux], PRECISION[precision])
        Na = (ctypes.c_int * self.n_sims)(*self.N)
        na = (ctypes.c_int * self.n_sims)(*self.n)
        da = (ctypes.c_int * self.n_sims)(*([3] * self.n_sims if d is None else d))
        doms = None
        if domains is not None:
            flat = np.ascontiguousarray(domains, dtype=np.float64).reshape(-1)
            doms = (ctypes.c_double * flat.size)(*flat)
        st = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(L.dg_ensemble_create(self.n_sims, da, Na, na, doms, ctypes.byref(opt),
                                    ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)),
               "dg_ensemble_create")
        self._h = h
        nv, nn = ctypes.c_longlong(), ctypes.c_longlong()
        offs = (ctypes.c_longlong * (self.n_sims + 1))()
        _check(L.dg_ensemble_info(h, ctypes.byref(nv), ctypes.byref(nn), offs),
               "dg_ensemble_info")
        self.n_values, self.n_nodes = nv.value, nn.value
        self.offsets = [offs[i] for i in range(self.n_sims + 1)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dg_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, u):
        t = self._torch
        if not (u.is_cuda and u.dtype == t.float64 and u.is_contiguous()
                and u.numel() == self.n_values):
            raise DGError("ensemble state must be a contiguous float64 CUDA tensor")

    def set_dt(self, dt):
        a = np.ascontiguousarray(dt, dtype=np.float64)
        _check(load().dg_ensemble_set_dt(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "dg_ensemble_set_dt")

    def get_dt(self):
        a = np.zeros(self.n_sims)
        _check(load().dg_ensemble_get_dt(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "dg_ensemble_get_dt")
        return a

    def compute_dt(self, u, cfl=0.5):
        self._chk(u)
        _check(load().dg_ensemble_compute_dt(self._h, _ptr(u), float(cfl)), "dg_ensemble_compute_dt")

    def stage(self, u_in, u_out, s):
        """u_out = u_in + B_s k with k = A_s k + dt du(u_in); u_out may be u_in."""
        self._chk(u_in)
        self._chk(u_out)
        _check(load().dg_ensemble_stage(self._h, _ptr(u_in), _ptr(u_out), int(s)), "dg_ensemble_stage")

    def step(self, u, cfl=0.0, graph=False):
        """One LSRK step in place on u (device CFL steps first when cfl > 0)."""
        self._chk(u)
        fn = load().dg_ensemble_step_graph if graph else load().dg_ensemble_step
        _check(fn(self._h, _ptr(u), float(cfl)), "dg_ensemble_step")

    def rk_reset(self):
        _check(load().dg_ensemble_rk_reset(self._h), "dg_ensemble_rk_reset")

    def check(self):
        f = ctypes.c_int()
        _check(load().dg_ensemble_check(self._h, ctypes.byref(f)), "dg_ensemble_check")
        return f.value

    def set_block(self, threads, blocks_per_sm):
        _check(load().dg_ensemble_set_block(self._h, int(threads), int(blocks_per_sm)),
               "dg_ensemble_set_block")

    def get_block(self):
        """(threads per CTA, requested CTAs per SM, CTAs launched)."""
        t, b, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().dg_ensemble_get_block(self._h, ctypes.byref(t), ctypes.byref(b),
                                            ctypes.byref(g)), "dg_ensemble_get_block")
        return t.value, b.value, g.value

    @property
    def pair_parallel(self):
        """Threads per line of the volume phase: False, one thread per line;
        True (FP64 only), one thread per node pair (the same result)."""
        on = ctypes.c_int()
        _check(load().dg_ensemble_get_pair_parallel(self._h, ctypes.byref(on)),
               "dg_ensemble_get_pair_parallel")
        return bool(on.value)

    @pair_parallel.setter
    def pair_parallel(self, on):
        _check(load().dg_ensemble_set_pair_parallel(self._h, int(bool(on))),
               "dg_ensemble_set_pair_parallel")

    def tune(self, u, u_tmp):
        """Autotune the CTA shape and (FP64) the threads per line; returns
        (threads, ctas_per_sm, ms_per_stage); the chosen threads per line:
        pair_parallel."""
        self._chk(u)
        self._chk(u_tmp)
        t, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(load().dg_ensemble_tune(self._h, _ptr(u), _ptr(u_tmp), ctypes.byref(t),
                                       ctypes.byref(b), ctypes.byref(ms)), "dg_ensemble_tune")
        return t.value, b.value, ms.value
