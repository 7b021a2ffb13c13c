"""dg_rhs_noalloc: the rhs entry point for callers that cannot allocate
device memory (embedders whose runtime owns every allocation, or which may
not allocate after setup). Its scratch is a static device array, so it is
checked against the ordinary dg_rhs through the C ABI: on two calls in a row
(the second call sees the first call's leftovers in the shared scratch), on
a sequence of meshes of different sizes, dimensions and degrees (a smaller
mesh after a larger one), at the largest mesh the scratch accepts and the
smallest it rejects, without any change of the device's free memory, and
across a device reset in a child process (no address cached from the
context that ended).

This file is collected last so that a stop-at-first-failure run has already
run every other test."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_06476_gb300 import Mesh, lgl_nodes, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _check_against_dg_rhs(L, d, N, n, u):
    dom = tuple(W.box(d))
    ut = torch.from_numpy(u).cuda()
    ref = Mesh(d, N, n, dom).rhs(ut)
    got = torch.full_like(ut, float("nan"))
    assert _noalloc_rhs(L, d, N, n, dom, ut, got) == 0, L.dg_last_error()
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
    assert err <= TOL64, (d, N, n, err)


def _face_values(d, N, n):
    return d * (d + 2) * int(np.prod(n)) * (N + 1) ** (d - 1)


@pytest.mark.parametrize("d,N,n", [(3, 3, (6, 5, 4)), (2, 3, (16, 16))])
def test_noalloc_matches_dg_rhs_twice(lib, d, N, n):
    xi, _ = lgl_nodes(N)
    states = [W.noisy_density_wave(d, N, n, W.box(d), xi, seed=1),
              W.random_state(d, N, n, seed=2)]
    for u in states:
        _check_against_dg_rhs(lib, d, N, n, u)


def test_noalloc_sequence_of_meshes(lib):
    # a large 3D mesh, then a small 2D one and a 3D one of another degree:
    # leftovers of the larger call in the shared scratch must not leak in
    for d, N, n in [(3, 3, (20, 20, 20)), (2, 3, (16, 16)), (3, 2, (3, 4, 5)),
                    (3, 7, (2, 2, 1)), (2, 1, (1, 1))]:
        _check_against_dg_rhs(lib, d, N, n, W.random_state(d, N, n, seed=sum(n) + N))


def test_noalloc_size_limit_at_the_boundary(lib):
    limit = (1 << 21) - 32
    # 3D N=3: 240 face values per element, so 8738 elements fit and 8739 do not
    ok, too_big = (2, 17, 257), (3, 3, 971)
    assert _face_values(3, 3, ok) <= limit < _face_values(3, 3, too_big)
    _check_against_dg_rhs(lib, 3, 3, ok, W.random_state(3, 3, ok, seed=5))
    ut = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert _noalloc_rhs(lib, 3, 3, too_big, tuple(W.box(3)), ut, ut) == -1
    assert b"static scratch" in lib.dg_last_error()
    assert _noalloc_rhs(lib, 3, 3, (64, 64, 64), tuple(W.box(3)), ut, ut) == -1


def test_noalloc_allocates_no_device_memory(lib):
    d, N, n = 3, 3, (8, 8, 8)
    dom = tuple(W.box(d))
    ut = torch.from_numpy(W.random_state(d, N, n, seed=9)).cuda()
    out = torch.empty_like(ut)
    assert _noalloc_rhs(lib, d, N, n, dom, ut, out) == 0  # warm-up: module loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert _noalloc_rhs(lib, d, N, n, dom, ut, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the 16 MiB scratch (or any other allocation) would show up here
    assert abs(free0 - free1) < (1 << 20), (free0, free1)


_CHILD = r'''
import ctypes, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2108_06476_gb300 import workloads as W
L = ctypes.CDLL(os.path.join(sys.argv[1], "paper_2108_06476_gb300", "libdgsem.so"))
cudart = None
for line in open("/proc/self/maps"):
    if "libcudart.so" in line:
        cudart = ctypes.CDLL(line.split()[-1])
        break
assert cudart is not None, "libcudart not mapped"
vp = ctypes.c_void_p
L.dg_last_error.restype = ctypes.c_char_p
L.dg_rhs_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_double), vp, vp, vp, vp]
L.dg_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_double), vp, vp, ctypes.POINTER(vp)]
L.dg_rhs.argtypes = [vp, vp, vp]
L.dg_mesh_destroy.argtypes = [vp]
d, N, n = 3, 3, (5, 4, 3)
u = W.random_state(d, N, n, seed=31)
n_arr = (ctypes.c_int * 3)(*n)
dom = (ctypes.c_double * 6)(*W.box(3))
nb = u.nbytes

def dev(nbytes):
    p = vp()
    assert cudart.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(nbytes)) == 0
    return p

def h2d(p, a):
    assert cudart.cudaMemcpy(p, a.ctypes.data_as(vp), ctypes.c_size_t(a.nbytes), 1) == 0

def d2h(p):
    a = np.empty_like(u)
    assert cudart.cudaMemcpy(a.ctypes.data_as(vp), p, ctypes.c_size_t(a.nbytes), 2) == 0
    return a

def noalloc_once():
    du_, dd_ = dev(nb), dev(nb)
    h2d(du_, u)
    rc = L.dg_rhs_noalloc(d, N, n_arr, dom, None, du_, dd_, None)
    assert rc == 0, L.dg_last_error()
    assert cudart.cudaDeviceSynchronize() == 0
    out = d2h(dd_)
    cudart.cudaFree(du_)
    cudart.cudaFree(dd_)
    return out

pu, pd = dev(nb), dev(nb)
h2d(pu, u)
mesh = vp()
assert L.dg_mesh_create(d, N, n_arr, dom, None, None, ctypes.byref(mesh)) == 0
assert L.dg_rhs(mesh, pu, pd) == 0
assert cudart.cudaDeviceSynchronize() == 0
ref = d2h(pd)
L.dg_mesh_destroy(mesh)
cudart.cudaFree(pu)
cudart.cudaFree(pd)
first = noalloc_once()
assert cudart.cudaDeviceReset() == 0
second = noalloc_once()
e1 = np.linalg.norm(first - ref) / np.linalg.norm(ref)
e2 = np.linalg.norm(second - ref) / np.linalg.norm(ref)
print(f"before reset {e1:.3e} after reset {e2:.3e}")
assert e1 <= 1e-12 and e2 <= 1e-12
'''


def _compute_mode():
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=compute_mode", "--format=csv,noheader",
                            "-i", "0"], capture_output=True, text=True, timeout=60)
        return r.stdout.strip()
    except (OSError, subprocess.SubprocessError):
        return ""


def test_noalloc_after_device_reset_in_child_process(lib):
    # a child process (its own CUDA context, no torch) calls the entry point,
    # resets the device and calls it again with new buffers
    if "Exclusive" in _compute_mode():
        pytest.skip("GPU in an exclusive compute mode: a second process cannot open it")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "after reset" in r.stdout
