"""GPU batched ensemble (one kernel launch per RK stage over all members)
against the FP64 oracle member by member: one stage, one full step with the
device-computed CFL time steps, the CUDA-graph step, the autotuner, and the
seeded 48-member configuration (FP64 sampled against the oracle, FP32 against
FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_06476_gb300 import Ensemble, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_06476_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small_members():
    M = W.EnsembleMember
    return [M(3, 3, (2, 2, 2), 0.5, (0.1, -0.2, 0.3), 20.0),
            M(3, 4, (3, 3, 3), 0.9, (-0.3, 0.1, 0.05), 20.0),
            M(3, 5, (2, 2, 2), 0.3, (0.2, 0.2, -0.1), 20.0),
            M(3, 3, (4, 4, 4), 0.98, (0.0, 0.25, 0.1), 20.0)]


def split(E, x):
    return [x[E.offsets[s]:E.offsets[s + 1]] for s in range(E.n_sims)]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_ensemble_step_matches_oracle(orc):
    mem = small_members()
    u0 = W.ensemble_state(mem, lambda N: orc.lgl(N)[0])
    E = Ensemble([m.N for m in mem], [m.n[0] for m in mem])
    assert E.n_values == u0.size
    ut = torch.from_numpy(u0.copy()).cuda()
    tmp = torch.empty_like(ut)
    # device CFL steps equal the oracle's per member
    E.compute_dt(ut, cfl=0.5)
    dts = E.get_dt()
    parts0 = split(E, u0)
    for s, m in enumerate(mem):
        assert dts[s] == pytest.approx(orc.max_dt(3, m.N, m.n, W.box(3), parts0[s], cfl=0.5),
                                       rel=1e-14)
    # one stage: u1 = u0 + B_0 dt rhs(u0)
    from paper_2108_06476_gb300 import RK_A, RK_B
    E.stage(ut, tmp, 0)
    got = split(E, tmp.cpu().numpy())
    for s, m in enumerate(mem):
        du = orc.rhs(3, m.N, m.n, W.box(3), parts0[s])
        ref = parts0[s] + RK_B[0] * dts[s] * du
        assert rel(got[s] - parts0[s], ref - parts0[s]) <= 1e-12
    # a full step from u0 (k reset) against the oracle's five stages
    E.rk_reset()
    ut.copy_(torch.from_numpy(u0))
    E.step(ut, tmp, cfl=0.0)  # uses the dt computed above
    assert E.check() == 0
    got = split(E, ut.cpu().numpy())
    for s, m in enumerate(mem):
        ref = orc.lsrk_step(3, m.N, m.n, W.box(3), parts0[s], dts[s])
        assert rel(got[s] - parts0[s], ref - parts0[s]) <= 1e-11


def test_graph_step_and_tuner_are_bitwise_consistent(orc):
    mem = small_members()
    u0 = W.ensemble_state(mem, lambda N: orc.lgl(N)[0])
    E = Ensemble([m.N for m in mem], [m.n[0] for m in mem])
    a = torch.from_numpy(u0.copy()).cuda()
    b = torch.from_numpy(u0.copy()).cuda()
    tmp = torch.empty_like(a)
    for _ in range(2):
        E.step(a, tmp, cfl=0.5)
    E.rk_reset()
    for _ in range(2):
        E.step(b, tmp, cfl=0.5, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # every element is computed the same way whatever the CTA shape
    threads, per_sm, ms = E.tune(a, tmp)
    assert threads in (64, 128, 192, 256) and per_sm in (2, 4, 8) and ms > 0
    E.rk_reset()
    c = torch.from_numpy(u0.copy()).cuda()
    for _ in range(2):
        E.step(c, tmp, cfl=0.5)
    torch.cuda.synchronize()
    assert torch.equal(a, c)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_48_member_configuration(orc, precision):
    mem = W.ensemble(n_sims=48, seed=0)
    u0 = W.ensemble_state(mem, lambda N: orc.lgl(N)[0])
    E = Ensemble([m.N for m in mem], [m.n[0] for m in mem], precision=precision)
    ut = torch.from_numpy(u0.copy()).cuda()
    tmp = torch.empty_like(ut)
    E.compute_dt(ut, cfl=0.5)
    dts = E.get_dt()
    E.stage(ut, tmp, 0)
    torch.cuda.synchronize()
    got = split(E, tmp.cpu().numpy())
    parts0 = split(E, u0)
    from paper_2108_06476_gb300 import RK_B
    # the two smallest members against the oracle
    order = np.argsort([m.n[0] ** 3 * (m.N + 1) ** 3 for m in mem])[:2]
    tol = 1e-12 if precision == "fp64" else 1e-5
    for s in order:
        m = mem[s]
        du = orc.rhs(3, m.N, m.n, W.box(3), parts0[s])
        ref = RK_B[0] * dts[s] * du
        err = rel(got[s] - parts0[s], ref)
        print(f"ensemble member {s} (N={m.N}, n={m.n[0]}) {precision} stage rel err {err:.3e}")
        assert err <= tol
