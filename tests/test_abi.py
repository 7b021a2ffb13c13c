"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point that include/dgsem.h declares, and validates its host-side
arguments (no device compute here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_06476_gb300 import build, dgsem
    build.build()
    return dgsem.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(dg_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dg_mesh_create", "dg_rhs", "dg_rk_stage", "dg_integrals", "dg_max_dt"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2108_06476_gb300 import dgsem
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(dgsem.EXPORTS) <= set(declared_functions())


def test_library_lgl_nodes_match_oracle(lib, orc):
    from paper_2108_06476_gb300 import lgl_nodes
    for N in range(1, 8):
        xi, w = lgl_nodes(N)
        xo, wo = orc.lgl(N)
        np.testing.assert_allclose(xi, xo, rtol=0, atol=3e-16)
        np.testing.assert_allclose(w, wo, rtol=3e-16, atol=0)


def test_mesh_create_rejects_bad_arguments(lib):
    from paper_2108_06476_gb300 import dgsem
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(4, 4, 4)
    dom = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    for d, N in ((1, 3), (4, 3), (3, 0), (3, 8)):
        rc = lib.dg_mesh_create(d, N, n, dom, None, None, ctypes.byref(h))
        assert rc == -1 and not h.value
        assert lib.dg_last_error()
    bad_n = (ctypes.c_int * 3)(4, 0, 4)
    assert lib.dg_mesh_create(3, 3, bad_n, dom, None, None, ctypes.byref(h)) == -1
    bad_dom = (ctypes.c_double * 6)(-1, 1, 1, 1, -1, 1)
    assert lib.dg_mesh_create(3, 3, n, bad_dom, None, None, ctypes.byref(h)) == -1
    opt = dgsem._Options(0.9, 0, 0, 0)
    assert lib.dg_mesh_create(3, 3, n, dom, ctypes.byref(opt), None, ctypes.byref(h)) == -1
    opt = dgsem._Options(1.4, 7, 0, 0)
    assert lib.dg_mesh_create(3, 3, n, dom, ctypes.byref(opt), None, ctypes.byref(h)) == -1
    for vf, sf in ((3, 0), (0, 4)):  # the MHD-only EC fluxes
        opt = dgsem._Options(1.4, vf, sf, 0)
        assert lib.dg_mesh_create(3, 3, n, dom, ctypes.byref(opt), None, ctypes.byref(h)) == -1
    assert lib.dg_rhs(None, None, None) == -1
    assert lib.dg_mesh_destroy(None) == 0


def test_curved_and_step_entry_points_reject_bad_arguments(lib):
    # checked before any CUDA call, so this runs without a GPU
    from paper_2108_06476_gb300 import dgsem
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(4, 4, 4)
    for N, warp in ((0, 0.15), (8, 0.15), (3, 0.6), (3, float("nan"))):
        rc = lib.dg_mesh_create_curved(N, n, warp, None, None, ctypes.byref(h))
        assert rc == -1 and not h.value, (N, warp)
        assert lib.dg_last_error()
    assert lib.dg_mesh_create_curved(3, None, 0.15, None, None, ctypes.byref(h)) == -1
    bad_n = (ctypes.c_int * 3)(4, 4, 0)
    assert lib.dg_mesh_create_curved(3, bad_n, 0.15, None, None, ctypes.byref(h)) == -1
    fp32 = dgsem._Options(1.4, 0, 0, 1)
    assert lib.dg_mesh_create_curved(3, n, 0.15, ctypes.byref(fp32), None, ctypes.byref(h)) == -1
    assert b"FP64" in lib.dg_last_error()
    # a null mesh is rejected by every mesh call
    t = ctypes.c_double()
    assert lib.dg_set_source(None, 1) == -1
    assert lib.dg_set_time(None, 0.0) == -1
    assert lib.dg_get_time(None, ctypes.byref(t)) == -1
    assert lib.dg_step_dt(None, None, 1e-3) == -1
    assert lib.dg_step_cfl_host(None, None, 0.5, 1) == -1


def test_mhd_mesh_create_rejects_bad_arguments(lib):
    # checked before any CUDA call, so this runs without a GPU
    from paper_2108_06476_gb300 import dgsem
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(4, 4, 4)
    dom = (ctypes.c_double * 6)(-1, 1, -1, 1, -1, 1)
    good = dgsem._Options(5 / 3, 2, 2, 0)  # central volume flux, HLL, FP64
    for N, powell in ((0, 1), (8, 1), (3, 2), (3, -1)):
        rc = lib.dg_mesh_create_mhd(N, n, dom, ctypes.byref(good), powell, None, ctypes.byref(h))
        assert rc == -1 and not h.value, (N, powell)
        assert lib.dg_last_error()
    for opt in (dgsem._Options(1.0, 2, 0, 0), dgsem._Options(float("nan"), 2, 0, 0),
                dgsem._Options(5 / 3, 0, 0, 0), dgsem._Options(5 / 3, 2, 1, 0),
                dgsem._Options(5 / 3, 2, 3, 0), dgsem._Options(5 / 3, 2, 0, 1)):
        rc = lib.dg_mesh_create_mhd(3, n, dom, ctypes.byref(opt), 1, None, ctypes.byref(h))
        assert rc == -1 and not h.value
    assert lib.dg_mesh_create_mhd(3, None, dom, None, 1, None, ctypes.byref(h)) == -1
    bad_n = (ctypes.c_int * 3)(4, 0, 4)
    assert lib.dg_mesh_create_mhd(3, bad_n, dom, None, 1, None, ctypes.byref(h)) == -1
    bad_dom = (ctypes.c_double * 6)(-1, 1, -1, 1, 2, 1)
    assert lib.dg_mesh_create_mhd(3, n, bad_dom, None, 1, None, ctypes.byref(h)) == -1
    # the warped-box MHD creator: the same option checks, the curved mesh's own
    for N, warp, powell in ((0, 0.15, 1), (8, 0.15, 1), (3, 0.6, 1), (3, float("nan"), 1),
                            (3, 0.15, 2)):
        rc = lib.dg_mesh_create_mhd_curved(N, n, warp, None, powell, None, ctypes.byref(h))
        assert rc == -1 and not h.value, (N, warp, powell)
    bad = dgsem._Options(5 / 3, 0, 0, 0)
    assert lib.dg_mesh_create_mhd_curved(3, n, 0.15, ctypes.byref(bad), 1, None,
                                         ctypes.byref(h)) == -1
    assert lib.dg_mesh_create_mhd_curved(3, None, 0.15, None, 1, None, ctypes.byref(h)) == -1


def test_built_for_sm_103a():
    from paper_2108_06476_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
