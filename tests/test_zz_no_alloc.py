"""dg_rhs_noalloc: the rhs entry point for callers that cannot allocate
device memory (embedders whose runtime owns every allocation, or which may
not allocate after setup). Its scratch is a static device array, so it is
checked against the ordinary dg_rhs through the C ABI, on two calls in a row
(the second call sees the first call's leftovers in the shared scratch).

This file is collected last so that a stop-at-first-failure run has already
run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_06476_gb300 import Mesh, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_2108_06476_gb300 import build, dgsem
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = dgsem.load()
    vp = ctypes.c_void_p
    L.dg_rhs_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double), vp, vp, vp, vp]
    L.dg_rhs_noalloc.restype = ctypes.c_int
    return L


def _noalloc_rhs(L, d, N, n, dom, ut, dut):
    n_arr = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    dom_arr = (ctypes.c_double * 6)(*(list(dom) + [0.0] * (6 - len(dom))))
    st = torch.cuda.current_stream().cuda_stream
    return L.dg_rhs_noalloc(d, N, n_arr, dom_arr, None, ctypes.c_void_p(ut.data_ptr()),
                            ctypes.c_void_p(dut.data_ptr()), ctypes.c_void_p(st))


@pytest.mark.parametrize("d,N,n", [(3, 3, (6, 5, 4)), (2, 3, (16, 16))])
def test_noalloc_matches_dg_rhs_twice(lib, d, N, n):
    dom = tuple(W.box(d))
    xi, _ = W_nodes(N)
    states = [W.noisy_density_wave(d, N, n, W.box(d), xi, seed=1),
              W.random_state(d, N, n, seed=2)]
    mesh = Mesh(d, N, n, dom)
    for u in states:
        ut = torch.from_numpy(u).cuda()
        ref = mesh.rhs(ut)
        got = torch.full_like(ut, float("nan"))
        assert _noalloc_rhs(lib, d, N, n, dom, ut, got) == 0, lib.dg_last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        assert err <= TOL64, err


def test_noalloc_rejects_meshes_beyond_the_static_scratch(lib):
    d, N, n = 3, 3, (64, 64, 64)
    ut = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _noalloc_rhs(lib, d, N, n, tuple(W.box(3)), ut, ut) == -1
    assert b"static scratch" in lib.dg_last_error()


def W_nodes(N):
    from paper_2108_06476_gb300 import lgl_nodes
    return lgl_nodes(N)
