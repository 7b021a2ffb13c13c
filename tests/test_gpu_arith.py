"""Device arithmetic helpers of the kernels, through dg_selftest_arith, and
the logarithmic mean's branch switches, element by element.

* The FP64 reciprocal (hardware approximation refined by a cubic Newton
  step) against IEEE 1/x: within one ulp over random operands of every
  magnitude whose reciprocal is a normal number, powers of two and operands
  next to the subnormal range; the FP32 reciprocal within one FP32 ulp.
* The FP32 kernels' double <-> float conversions (integer bit manipulation)
  against IEEE round-to-nearest-even conversion: bitwise, including exact
  halfway cases, zeros, and values that take the hardware path (subnormal
  floats, overflow).
* Two-element states whose node pairs sit just below and just above every
  switch of the log mean's ranges (FP64 kernels: 1e-2 and 0.25; FP32
  kernels: 1e-4, the FP64 small-difference branch, and 0.25; the oracle's
  1e-4), for the density and for rho/p, compared with the oracle per node
  and variable (largest error over the mesh relative to the variable's
  largest value), not as one global norm.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_06476_gb300 import Mesh, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2108_06476_gb300 import build, dgsem
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dgsem.load()


def arith(L, op, x):
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yt = torch.empty_like(xt)
    st = torch.cuda.current_stream().cuda_stream
    assert L.dg_selftest_arith(op, ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()),
                               xt.numel(), ctypes.c_void_p(st)) == 0, L.dg_last_error()
    torch.cuda.synchronize()
    return yt.cpu().numpy()


def ulp_distance64(a, b):
    ia = a.view(np.int64).astype(object)
    ib = b.view(np.int64).astype(object)
    return np.array([abs(int(x) - int(y)) for x, y in zip(ia, ib)])


def operands64(rng, count=200000):
    # |x| in [2^-1021, 2^1021] (reciprocal normal), both signs, log-uniform
    e = rng.uniform(-1021.0, 1021.0, count)
    x = np.exp2(e) * rng.choice([-1.0, 1.0], count)
    pow2 = np.exp2(np.arange(-1021, 1022, dtype=np.float64))
    edge = np.array([2.0 ** -1021 * (1 + k * 2.0 ** -52) for k in range(64)]
                    + [2.0 ** 1021 * (2 - k * 2.0 ** -52) for k in range(1, 64)]
                    + [np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 3.0, 0.1, 1e300, 1e-300])
    return np.concatenate([x, pow2, -pow2, edge, -edge])


def test_fp64_reciprocal_within_one_ulp(lib):
    x = operands64(np.random.default_rng(0))
    y = arith(lib, 0, x)
    ref = 1.0 / x
    d = ulp_distance64(y, ref)
    assert d.max() <= 1, (x[np.argmax(d)], d.max())
    # and on the state values the kernels meet (densities, sums of two)
    x = np.random.default_rng(1).uniform(1e-3, 1e3, 100000)
    assert ulp_distance64(arith(lib, 0, x), 1.0 / x).max() <= 1


def test_fp32_reciprocal_within_one_ulp(lib):
    rng = np.random.default_rng(2)
    xf = (np.exp2(rng.uniform(-125.0, 125.0, 100000)) * rng.choice([-1.0, 1.0], 100000)
          ).astype(np.float32)
    y = arith(lib, 1, xf.astype(np.float64)).astype(np.float32)
    ref = np.float32(1.0) / xf
    d = np.abs(y.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert d.max() <= 1


def test_fp64_square_root_within_one_ulp(lib):
    # positive normal operands of every magnitude, powers of two (exact
    # roots), the ends of the normal range and perfect squares: within one
    # ulp of the correctly rounded IEEE root
    rng = np.random.default_rng(5)
    x = np.exp2(rng.uniform(-1022.0, 1023.9, 200000))
    pow2 = np.exp2(np.arange(-1022, 1024, dtype=np.float64))
    k = rng.integers(1, 2 ** 26, 20000).astype(np.float64)
    edge = np.array([2.0 ** -1022 * (1 + j * 2.0 ** -52) for j in range(64)]
                    + [np.finfo(np.float64).max * (1 - j * 2.0 ** -53) for j in range(64)]
                    + [np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0, 3.0, 0.1, 28.0])
    x = np.concatenate([x, pow2, k * k, edge])
    y = arith(lib, 4, x)
    d = ulp_distance64(y, np.sqrt(x))
    assert d.max() <= 1, (x[np.argmax(d)], d.max())
    # even powers of two and perfect squares have exact roots
    sq = np.concatenate([np.exp2(np.arange(-1022, 1024, 2, dtype=np.float64)), k * k])
    assert np.array_equal(arith(lib, 4, sq), np.sqrt(sq))
    # squared sound speeds of the kernels' states (gamma p / rho)
    c2 = 1.4 * rng.uniform(1e-2, 1e2, 100000) / rng.uniform(1e-2, 2.0, 100000)
    assert ulp_distance64(arith(lib, 4, c2), np.sqrt(c2)).max() <= 1
    # everything else takes the library root: zeros, negative, subnormal,
    # infinite and NaN arguments give the IEEE results
    special = np.array([0.0, -0.0, -1.0, -np.inf, 5e-324, 1e-310, np.inf, np.nan])
    with np.errstate(invalid="ignore"):
        ref = np.sqrt(special)
    got = arith(lib, 4, special)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.array_equal(got[ok].view(np.int64), ref[ok].view(np.int64))


def test_double_to_float_is_ieee_round_to_nearest_even(lib):
    rng = np.random.default_rng(3)
    x = np.exp2(rng.uniform(-130.0, 130.0, 200000)) * rng.choice([-1.0, 1.0], 200000)
    # exact halfway cases between neighbouring floats (ties to even), and
    # one ulp (of the double) either side of them
    f = (np.exp2(rng.uniform(-120.0, 120.0, 20000))).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    half = (f.astype(np.float64) + g.astype(np.float64)) / 2.0
    special = np.array([0.0, -0.0, 1e-40, -1e-40, 1.4e-45, 3.4e38, 3.5e38, 1e39, -1e39,
                        np.float64(np.finfo(np.float32).max) * (1 + 2.0 ** -25),
                        np.float64(np.finfo(np.float32).tiny), np.inf, -np.inf])
    x = np.concatenate([x, half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf),
                        -half, special])
    y = arith(lib, 2, x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(y.view(np.int64), ref.view(np.int64))


def test_float_to_double_is_exact(lib):
    rng = np.random.default_rng(4)
    xf = (np.exp2(rng.uniform(-149.0, 127.0, 200000)) * rng.choice([-1.0, 1.0], 200000)
          ).astype(np.float32)
    xf = np.concatenate([xf, np.array([0.0, -0.0, 1e-45, np.inf, -np.inf], dtype=np.float32)])
    y = arith(lib, 3, xf.astype(np.float64))
    assert np.array_equal(y.view(np.int64), xf.astype(np.float64).view(np.int64))


def ratio_for(f2):
    """y/x with ((y - x)/(y + x))^2 = f2."""
    t = np.sqrt(f2)
    return (1.0 + t) / (1.0 - t)


def branch_state(N, cases, v=(0.1, 0.2, 0.3)):
    """n = (2, 1, 1) elements of degree N = 1: every x-line of each element
    is one node pair; line k of element e gets the case (f2_rho, f2_sig) of
    cases[4 e + k]: node 0 (rho, p) = (1, 20), node 1 (r, 20 r / s) with
    r = ratio_for(f2_rho), s = ratio_for(f2_sig)."""
    P = 8
    u = np.zeros((2, 5, P))
    for e in range(2):
        for k in range(4):
            f2r, f2s = cases[4 * e + k]
            r, s = ratio_for(f2r), ratio_for(f2s)
            for i, (rho, p) in enumerate(((1.0, 20.0), (r, 20.0 * r / s))):
                node = i + 2 * k
                m = rho * np.array(v)
                u[e, 0, node] = rho
                u[e, 1:4, node] = m
                u[e, 4, node] = p / 0.4 + 0.5 * rho * float(np.dot(v, v))
    return u.reshape(-1)


def per_variable_error(got, ref):
    g, r = got.reshape(-1, 5, 8), ref.reshape(-1, 5, 8)
    return max(float(np.abs(g[:, v] - r[:, v]).max() / np.abs(r[:, v]).max()) for v in range(5))


SWITCHES64 = (1e-2, 0.25, 1e-4)  # FP64 kernel ranges, and the oracle's switch
SWITCHES32 = (1e-4, 0.25)


def cases_around(T, rel):
    lo, hi = T * (1 - rel), T * (1 + rel)
    return [(lo, lo), (hi, hi), (lo, hi), (hi, lo), (lo, 0.0), (hi, 0.0), (0.0, lo), (0.0, hi)]


@pytest.mark.parametrize("sf", ["llf", "ranocha"])
@pytest.mark.parametrize("T", SWITCHES64)
def test_fp64_log_mean_switches_element_by_element(orc, T, sf):
    u = branch_state(1, cases_around(T, 1e-12))
    n, dom = (2, 1, 1), W.box(3)
    ref = orc.rhs(3, 1, n, dom, u, vflux=0, sflux={"llf": 0, "ranocha": 1}[sf])
    m = Mesh(3, 1, n, tuple(dom), surface_flux=sf)
    got = m.rhs(torch.from_numpy(u).cuda()).cpu().numpy()
    assert m.check() == 0
    err = per_variable_error(got, ref)
    print(f"FP64 f2 around {T}: largest per-variable error {err:.2e}")
    assert err <= 1e-12


@pytest.mark.parametrize("sf", ["llf", "ranocha"])
@pytest.mark.parametrize("T", SWITCHES32 + (1e-2,))
def test_fp32_log_mean_switches_element_by_element(orc, T, sf):
    u = branch_state(1, cases_around(T, 1e-6))
    n, dom = (2, 1, 1), W.box(3)
    ref = orc.rhs(3, 1, n, dom, u, vflux=0, sflux={"llf": 0, "ranocha": 1}[sf])
    m = Mesh(3, 1, n, tuple(dom), surface_flux=sf, precision="fp32")
    got = m.rhs(torch.from_numpy(u).cuda()).double().cpu().numpy()
    assert m.check() == 0
    err = per_variable_error(got, ref)
    print(f"FP32 f2 around {T}: largest per-variable error {err:.2e}")
    assert err <= 1e-5
