"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 bar: relative L2 error ||du_gpu - du_oracle|| / ||du_oracle|| <= 1e-12
(the tolerance the method's FP64 target states). The two sides differ only in
rounding order (pair halving with the symmetric flux, FMA contraction, scaled
tables), so the error is a few ulps of the flux-sized terms, amplified by the
cancellation in sum_m Dt_im f#(u_i,u_m) (terms ~ (2/h)|Dt||f|, result ~|du|).
"""
import ctypes
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_06476_gb300 import Mesh, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
VF = {0: "ranocha", 1: "chandrashekar", 2: "central"}
SF = {0: "llf", 1: "ranocha", 2: "hll", 3: "chandrashekar"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_06476_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_rhs(d, N, n, dom, u, vf=0, sf=0, precision="fp64"):
    m = Mesh(d, N, n, tuple(dom), volume_flux=VF[vf], surface_flux=SF[sf], precision=precision)
    ut = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    du = m.rhs(ut)
    assert m.check() == 0
    return du.double().cpu().numpy()


def oracle_rhs(orc, d, N, n, dom, u, vf=0, sf=0, elems=None):
    return orc.rhs(d, N, n, dom, u, vflux=vf, sflux=sf, elems=elems)


@pytest.mark.parametrize("d,N,n", [(2, 3, (16, 16)), (3, 3, (4, 4, 4)), (3, 2, (3, 4, 5)),
                                   (2, 4, (5, 3)), (3, 3, (1, 2, 3)), (2, 1, (1, 1)),
                                   (3, 1, (1, 1, 1))])
def test_rhs_fp64_density_wave_and_random(orc, d, N, n):
    dom = np.array([-1.0, 1.0, -0.5, 1.5, 0.0, 3.0][:2 * d]) if n[0] != n[-1] else W.box(d)
    xi, _ = orc.lgl(N)
    states = [W.random_state(d, N, n, seed=21)]
    if max(n) > 1:  # one element per direction: the wave's rhs is roundoff-sized
        states.append(W.density_wave(d, N, n, dom, xi))
    for u in states:
        ref = oracle_rhs(orc, d, N, n, dom, u)
        got = gpu_rhs(d, N, n, dom, u)
        assert rel_l2(got, ref) <= TOL64, rel_l2(got, ref)


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("d", [2, 3])
def test_rhs_fp64_every_degree(orc, d, N):
    n = (3, 2, 2)[:d] if N < 6 else (2, 2, 1)[:d]
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=100 + N)
    ref = oracle_rhs(orc, d, N, n, dom, u)
    got = gpu_rhs(d, N, n, dom, u)
    assert rel_l2(got, ref) <= TOL64, rel_l2(got, ref)


@pytest.mark.parametrize("vf", [0, 1, 2])
@pytest.mark.parametrize("sf", [0, 1, 2, 3])
@pytest.mark.parametrize("d,N,n", [(3, 3, (3, 2, 2)), (2, 2, (4, 3))])
def test_rhs_fp64_every_flux(orc, d, N, n, vf, sf):
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=7 * vf + sf)
    ref = oracle_rhs(orc, d, N, n, dom, u, vf, sf)
    got = gpu_rhs(d, N, n, dom, u, vf, sf)
    assert rel_l2(got, ref) <= TOL64, rel_l2(got, ref)


def test_rhs_fp64_3d_32cubed_full(orc):
    # 3D N=3 on 32^3 elements, density wave with v = (0.1, 0.2, 0.3), p = 20
    d, N, n = 3, 3, (32, 32, 32)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u = W.density_wave(d, N, n, dom, xi)
    ref = oracle_rhs(orc, d, N, n, dom, u)
    got = gpu_rhs(d, N, n, dom, u)
    err = rel_l2(got, ref)
    print(f"32^3 N=3 FP64 rel L2 = {err:.3e}")
    assert err <= TOL64


def _sample_elements(n, count, seed):
    rng = np.random.default_rng(seed)
    ne = int(np.prod(n))
    corners = [0, ne - 1, n[0] - 1, ne - n[0]]
    return np.unique(np.concatenate([corners, rng.choice(ne, size=count, replace=False)]))


@pytest.mark.parametrize("N,ne,count", [(3, 64, 400), (7, 24, 60)])
def test_rhs_fp64_full_size_sampled(orc, N, ne, count):
    # full-size noisy density waves: GPU rhs over the whole mesh, oracle on a
    # sample of elements (including the domain's corners)
    d, n = 3, (ne, ne, ne)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u = W.noisy_density_wave(d, N, n, dom, xi, seed=0)
    elems = _sample_elements(n, count, seed=N)
    ref = oracle_rhs(orc, d, N, n, dom, u, elems=elems).reshape(-1, d + 2, (N + 1) ** d)[elems]
    got = gpu_rhs(d, N, n, dom, u).reshape(-1, d + 2, (N + 1) ** d)[elems]
    err = rel_l2(got, ref)
    print(f"{ne}^3 N={N} FP64 sampled rel L2 = {err:.3e}")
    assert err <= TOL64


def test_entropy_conservation_ec_32cubed(orc):
    # EC volume + EC surface flux on a periodic mesh: sum_e J sum_i w_i theta(u_i) . du_i
    # vanishes to roundoff (relative to the sum of magnitudes)
    d, N, n = 3, 3, (32, 32, 32)
    dom = W.box(d)
    xi, w = orc.lgl(N)
    u = W.noisy_density_wave(d, N, n, dom, xi, seed=1)
    du = gpu_rhs(d, N, n, dom, u, vf=0, sf=1)
    U = u.reshape(-1, d + 2, (N + 1) ** d)
    rho, m, E = U[:, 0], U[:, 1:4], U[:, 4]
    v = m / rho[:, None]
    v2 = (v * v).sum(axis=1)
    p = 0.4 * (E - 0.5 * rho * v2)
    s = np.log(p) - 1.4 * np.log(rho)
    b = rho / p
    th = np.concatenate([((1.4 - s) / 0.4 - 0.5 * b * v2)[:, None], b[:, None, :] * v,
                         -b[:, None]], axis=1)
    wq = np.multiply.outer(w, np.multiply.outer(w, w)).reshape(-1) * (1 / 32) ** 3
    t = wq[None, None, :] * th * du.reshape(U.shape)
    assert abs(t.sum()) <= 1e-12 * np.abs(t).sum(), abs(t.sum()) / np.abs(t).sum()


def test_rk_stage_matches_oracle(orc):
    d, N, n = 3, 3, (4, 3, 2)
    m = Mesh(d, N, n)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(m.n_values)
    du = rng.standard_normal(m.n_values)
    ut = torch.from_numpy(u0.copy()).cuda()
    dut = torch.from_numpy(du).cuda()
    uo, ko = u0.copy(), np.zeros_like(u0)
    from paper_2108_06476_gb300 import RK_A, RK_B
    for s in range(5):
        m.rk_stage(ut, dut, RK_A[s], RK_B[s], 1e-3)
        orc.rk_stage(uo, ko, du, RK_A[s], RK_B[s], 1e-3)
    np.testing.assert_allclose(ut.cpu().numpy(), uo, rtol=1e-15, atol=1e-15)


def test_odd_value_count_rk_tail(orc):
    # 3D N=2 on 1x1x1: 5 * 27 values (odd count exercises the scalar tail)
    m = Mesh(3, 2, (1, 1, 1))
    assert m.n_values % 2 == 1
    rng = np.random.default_rng(4)
    u0, du = rng.standard_normal(m.n_values), rng.standard_normal(m.n_values)
    ut, dut = torch.from_numpy(u0.copy()).cuda(), torch.from_numpy(du).cuda()
    m.rk_stage(ut, dut, 0.0, 0.5, 0.1)
    uo, ko = u0.copy(), np.zeros_like(u0)
    orc.rk_stage(uo, ko, du, 0.0, 0.5, 0.1)
    np.testing.assert_allclose(ut.cpu().numpy(), uo, rtol=1e-15, atol=1e-16)


def test_20_steps_2d_config_trajectory(orc):
    # 2D 16^2 N=3 density wave, one rhs plus 20 LSRK steps at CFL 0.5 (fixed dt)
    d, N, n = 2, 3, (16, 16)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u0 = W.density_wave(d, N, n, dom, xi, velocity=(0.1, 0.2))
    dt = orc.max_dt(d, N, n, dom, u0, cfl=0.5)
    m = Mesh(d, N, n, tuple(dom))
    ut = torch.from_numpy(u0.copy()).cuda()
    assert m.max_dt(ut, cfl=0.5) == pytest.approx(dt, rel=1e-14)
    du = m.empty_rhs()
    uo = u0.copy()
    for _ in range(20):
        m.step(ut, dt, du)
        uo = orc.lsrk_step(d, N, n, dom, uo, dt)
    assert m.check() == 0
    err = rel_l2(ut.cpu().numpy() - u0, uo - u0)
    assert err <= 1e-11, err


def test_max_dt_and_integrals_3d(orc):
    d, N, n = 3, 4, (5, 4, 3)
    dom = np.array([-1.0, 1.0, -0.5, 1.5, 0.0, 3.0])
    xi, _ = orc.lgl(N)
    u = W.noisy_density_wave(d, N, n, dom, xi, seed=5)
    m = Mesh(d, N, n, tuple(dom))
    ut = torch.from_numpy(u).cuda()
    assert m.max_dt(ut, cfl=0.5) == pytest.approx(orc.max_dt(d, N, n, dom, u, cfl=0.5), rel=1e-14)
    np.testing.assert_allclose(m.integrals(ut), orc.integrals(d, N, n, dom, u), rtol=1e-14,
                               atol=1e-14)


def test_integrals_32cubed(orc):
    d, N, n = 3, 3, (32, 32, 32)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u = W.noisy_density_wave(d, N, n, dom, xi, seed=6)
    got = Mesh(d, N, n).integrals(torch.from_numpy(u).cuda())
    np.testing.assert_allclose(got, orc.integrals(d, N, n, dom, u), rtol=1e-14, atol=1e-13)


def test_nonphysical_state_is_reported():
    from paper_2108_06476_gb300 import DGError
    d, N, n = 3, 2, (2, 2, 2)
    u = W.uniform_state(d, N, n).reshape(-1, 5, 27)
    u[3, 0, 5] = -1.0  # negative density at one node
    m = Mesh(d, N, n)
    ut = torch.from_numpy(u.reshape(-1).copy()).cuda()
    m.rhs(ut)
    with pytest.raises(DGError):
        m.check()
    assert m.check() == 0  # the word was cleared
    with pytest.raises(DGError):
        m.max_dt(ut)


# ---- FP32 kernels (FP64 state, FP32 volume/surface arithmetic) ----
TOL32 = 1e-5  # the FP32 target's relative L2 rhs error


@pytest.mark.parametrize("N,ne,count", [(3, 64, 400), (7, 24, 60)])
def test_rhs_fp32_full_size_sampled(orc, N, ne, count):
    d, n = 3, (ne, ne, ne)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u = W.noisy_density_wave(d, N, n, dom, xi, seed=0)
    elems = _sample_elements(n, count, seed=N + 10)
    ref = oracle_rhs(orc, d, N, n, dom, u, elems=elems).reshape(-1, d + 2, (N + 1) ** d)[elems]
    got = gpu_rhs(d, N, n, dom, u, precision="fp32").reshape(-1, d + 2, (N + 1) ** d)[elems]
    err = rel_l2(got, ref)
    print(f"{ne}^3 N={N} FP32 sampled rel L2 = {err:.3e}")
    assert err <= TOL32


@pytest.mark.parametrize("d,N,n", [(3, 3, (4, 3, 2)), (2, 4, (5, 3)), (3, 5, (2, 2, 2))])
@pytest.mark.parametrize("vf,sf", [(0, 0), (1, 1), (2, 2), (0, 3)])
def test_rhs_fp32_small(orc, d, N, n, vf, sf):
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=40 + N)
    ref = oracle_rhs(orc, d, N, n, dom, u, vf, sf)
    got = gpu_rhs(d, N, n, dom, u, vf, sf, precision="fp32")
    assert rel_l2(got, ref) <= TOL32, rel_l2(got, ref)


# Meshes of 608 elements or more run the line-owning volume kernel, whose
# direction phase is the row loop from N = 6 in FP64 and from N = 4 in FP32
# (smaller FP64 meshes run the pair-parallel kernel, so the every-degree test
# above does not reach it). Every volume flux through the row loop, 2D and
# 3D, on anisotropic meshes; FP64 against the oracle on sampled elements
# and FP32 on whole small meshes (FP32 meshes have no pair-parallel path),
# random states.
@pytest.mark.parametrize("vf,sf", [(0, 0), (1, 1), (2, 2), (0, 3)])
@pytest.mark.parametrize("d,N,n", [(3, 6, (9, 9, 8)), (3, 7, (8, 8, 10)), (2, 7, (25, 26))])
def test_rhs_fp64_row_loop_every_flux(orc, d, N, n, vf, sf):
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=200 + 10 * N + vf)
    elems = _sample_elements(n, 40, seed=N + vf)
    P = (N + 1) ** d
    ref = oracle_rhs(orc, d, N, n, dom, u, vf, sf, elems=elems).reshape(-1, d + 2, P)[elems]
    got = gpu_rhs(d, N, n, dom, u, vf, sf).reshape(-1, d + 2, P)[elems]
    assert rel_l2(got, ref) <= TOL64, rel_l2(got, ref)


@pytest.mark.parametrize("vf,sf", [(0, 0), (1, 1), (2, 2), (0, 3)])
@pytest.mark.parametrize("d,N,n", [(3, 4, (3, 2, 2)), (3, 6, (2, 2, 3)), (3, 7, (2, 1, 2)),
                                   (2, 7, (4, 3))])
def test_rhs_fp32_row_loop_every_flux(orc, d, N, n, vf, sf):
    dom = W.box(d)
    u = W.random_state(d, N, n, seed=300 + N)
    ref = oracle_rhs(orc, d, N, n, dom, u, vf, sf)
    got = gpu_rhs(d, N, n, dom, u, vf, sf, precision="fp32")
    assert rel_l2(got, ref) <= TOL32, rel_l2(got, ref)


# ---- fused step: device CFL time step, stage update inside the volume kernel ----
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_step_matches_unfused(orc, precision):
    d, N, n = 3, 3, (6, 5, 4)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, dom, xi, seed=8)
    m1 = Mesh(d, N, n, precision=precision)
    m2 = Mesh(d, N, n, precision=precision)
    a = torch.from_numpy(u0.copy()).cuda()
    b = torch.from_numpy(u0.copy()).cuda()
    du = m1.empty_rhs()
    for _ in range(3):
        dt = m1.max_dt(a, cfl=0.5)
        m1.step(a, dt, du)
        m2.step_cfl(b, cfl=0.5)
        assert m2.last_dt() == pytest.approx(dt, rel=1e-15)
    inc_a = (a.cpu().numpy() - u0)
    inc_b = (b.cpu().numpy() - u0)
    bound = 1e-13 + 1e-15 * np.linalg.norm(u0) / np.linalg.norm(inc_a)
    assert rel_l2(inc_b, inc_a) <= bound


def test_graph_step_equals_fused_step(orc):
    d, N, n = 3, 3, (4, 4, 4)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, W.box(d), xi, seed=9)
    m1, m2 = Mesh(d, N, n), Mesh(d, N, n)
    a = torch.from_numpy(u0.copy()).cuda()
    b = torch.from_numpy(u0.copy()).cuda()
    for _ in range(3):
        m1.step_cfl(a, cfl=0.5)
        m2.step_cfl(b, cfl=0.5, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_rhs_part_fused_volume_leaves_state_unchanged(orc):
    # parts=6 (the fused step's volume kernel with B = 0) must not move u and
    # must leave the face-buffer/volume pair consistent with a plain rhs
    d, N, n = 3, 3, (4, 3, 2)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, W.box(d), xi, seed=4)
    m = Mesh(d, N, n)
    u = torch.from_numpy(u0.copy()).cuda()
    m.step_cfl(u, cfl=0.5)  # sets the device time step
    before = u.clone()
    du = m.empty_rhs()
    m.rhs_part(u, du, 1)
    for _ in range(3):
        m.rhs_part(u, du, 6)
    torch.cuda.synchronize()
    assert torch.equal(u, before)
    assert m.check() == 0
    ref = oracle_rhs(orc, d, N, n, W.box(d), before.cpu().numpy())
    assert rel_l2(m.rhs(u).cpu().numpy(), ref) <= TOL64


@pytest.mark.parametrize("memory", ["pinned", "pageable"])
@pytest.mark.parametrize("n_steps", [1, 3])
def test_host_state_step_equals_device_step(orc, memory, n_steps):
    # dg_step_cfl_host: pinned buffers are read by the wave-speed pass and
    # written by the last stage, pageable ones copied; both must give the
    # device step's state bitwise
    d, N, n = 3, 3, (4, 3, 5)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, W.box(d), xi, seed=13)
    m1, m2 = Mesh(d, N, n), Mesh(d, N, n)
    ud = torch.from_numpy(u0.copy()).cuda()
    for _ in range(n_steps):
        m1.step_cfl(ud, cfl=0.5)
    if memory == "pinned":
        uh = torch.from_numpy(u0.copy()).pin_memory()
        m2.step_cfl_host(uh, cfl=0.5, n_steps=n_steps)
        got = uh.numpy()
    else:
        got = u0.copy()
        m2.step_cfl_host(got, cfl=0.5, n_steps=n_steps)
    assert np.array_equal(got, ud.cpu().numpy())
    assert m2.last_dt() == m1.last_dt()
    assert m2.check() == 0


def test_step_with_given_dt_equals_cfl_step(orc):
    d, N, n = 2, 4, (5, 3)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, W.box(d), xi, seed=6)
    m1, m2 = Mesh(d, N, n), Mesh(d, N, n)
    a = torch.from_numpy(u0.copy()).cuda()
    b = torch.from_numpy(u0.copy()).cuda()
    for _ in range(3):
        m1.step_cfl(a, cfl=0.5)
        m2.step_dt(b, m1.last_dt())
        assert m2.last_dt() == m1.last_dt()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_host_state_step_rejects_device_memory():
    from paper_2108_06476_gb300 import load
    m = Mesh(2, 2, (2, 2))
    u = torch.zeros(m.n_values, dtype=torch.float64, device="cuda")
    rc = load().dg_step_cfl_host(m._h, ctypes.c_void_p(u.data_ptr()), 0.5, 1)
    assert rc == -1
    rc = load().dg_step_cfl_host(m._h, ctypes.c_void_p(u.data_ptr()), 0.5, 0)
    assert rc == -1


def test_fused_20_steps_2d_against_oracle(orc):
    # 2D 16^2 N=3 density wave, 20 steps at CFL 0.5 with the time step taken
    # from each side's own state every step
    d, N, n = 2, 3, (16, 16)
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u0 = W.density_wave(d, N, n, dom, xi, velocity=(0.1, 0.2))
    m = Mesh(d, N, n, tuple(dom))
    ut = torch.from_numpy(u0.copy()).cuda()
    uo = u0.copy()
    for _ in range(20):
        m.step_cfl(ut, cfl=0.5)
        uo = orc.lsrk_step(d, N, n, dom, uo, orc.max_dt(d, N, n, dom, uo, cfl=0.5))
    assert m.check() == 0
    assert rel_l2(ut.cpu().numpy() - u0, uo - u0) <= 1e-11


# Meshes under 608 elements (about four per SM) evaluate a whole FP64 rhs in
# one launch (the pair-parallel volume kernel with its element's face fluxes
# in shared memory), and a stage from one buffer into another; the separate
# face and volume launches (parts 1 and 2) stay available. Both orders of
# work give the same result bitwise, and the size boundary changes nothing
# but the kernels.
@pytest.mark.parametrize("vf,sf", [(0, 0), (1, 1), (2, 2), (0, 3)])
@pytest.mark.parametrize("d,N,n", [(2, 3, (16, 16)), (3, 3, (4, 3, 5)), (3, 7, (2, 2, 1)),
                                   (2, 1, (1, 1)), (3, 5, (3, 2, 2))])
def test_one_launch_small_rhs_equals_face_and_volume_launches(orc, d, N, n, vf, sf):
    dom = W.box(d)
    u = torch.from_numpy(W.random_state(d, N, n, seed=5)).cuda()
    m = Mesh(d, N, n, tuple(dom), volume_flux=VF[vf], surface_flux=SF[sf])
    one = m.rhs(u).cpu().numpy()
    du = m.empty_rhs()
    m.rhs_part(u, du, 1)
    m.rhs_part(u, du, 2)
    torch.cuda.synchronize()
    assert m.check() == 0
    assert np.array_equal(one, du.cpu().numpy())
    ref = oracle_rhs(orc, d, N, n, dom, u.cpu().numpy(), vf=vf, sf=sf)
    assert rel_l2(one, ref) <= TOL64


@pytest.mark.parametrize("n", [(607, 1), (19, 32), (607, 1, 1), (8, 8, 9), (2, 16, 19)])
def test_small_mesh_boundary(orc, n):
    # 607 or 576 elements (one launch per rhs or stage) and 608 (face and
    # volume kernels, stages in place)
    d = len(n)
    N = 2
    dom = W.box(d)
    xi, _ = orc.lgl(N)
    u0 = W.noisy_density_wave(d, N, n, dom, xi, seed=3)
    ref = oracle_rhs(orc, d, N, n, dom, u0)
    got = gpu_rhs(d, N, n, dom, u0)
    assert rel_l2(got, ref) <= TOL64
    # steps: the small path runs its stages through two other buffers
    m = Mesh(d, N, n, tuple(dom))
    a = torch.from_numpy(u0.copy()).cuda()
    dt = 0.5 * m.max_dt(a, cfl=1.0)
    m.step_dt(a, dt)
    b = orc.lsrk_step(d, N, n, dom, u0.copy(), dt)
    torch.cuda.synchronize()
    assert m.check() == 0
    inc = a.cpu().numpy() - u0
    assert rel_l2(inc, b - u0) <= 1e-11
