"""GPU parity of the forward Euler and DOPRI5 steppers (Sec. 3) against the
oracle's steppers on the same inputs, and of the adaptive DOPRI5 driver
against a fixed-step oracle replay of the steps it accepted."""

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from oracle.system import FRSystem
from tests.libutil import ensure_built, oracle_state, rel_l2_per_var

pytestmark = pytest.mark.gpu

NS_PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


def _vortex():
    m = periodic_box("quad", 16, -5.0, 5.0)
    o = FRSystem(m, 2, "euler")
    U = oracle_state(o, lambda X: fields.isentropic_vortex(X, S=5.0, M=0.4, R=1.5))
    return m, o, U


def _tgv():
    m = periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.1, seed=2)
    o = FRSystem(m, 3, "ns", **NS_PRM)
    U = oracle_state(o, lambda X: fields.taylor_green(X, M=0.3))
    return m, o, U


def _run(torch, s, U, fn):
    u = [torch.from_numpy(s.pack(b, U[b])).cuda() for b in range(len(U))]
    out = fn(u)
    torch.cuda.synchronize()
    return [u[b].cpu().numpy()[:, :, :U[b].shape[2]].astype(np.float64) for b in range(len(U))], out


def test_euler_matches_oracle(torch):
    from paper_1312_1638_b300 import fr
    m, o, U = _vortex()
    ref = o.euler(U, 1e-3, 10)
    s = fr.Solver(m, 2, "euler", "fp64", device=0)
    g, _ = _run(torch, s, U, lambda u: s.euler(u, 1e-3, 10))
    assert rel_l2_per_var(g[0], ref[0]) < 1e-13
    assert np.abs(g[0] - ref[0]).max() < 1e-12


@pytest.mark.parametrize("case", ["vortex", "tgv"])
def test_dopri5_fp64_matches_oracle(torch, case):
    from paper_1312_1638_b300 import fr
    m, o, U = _vortex() if case == "vortex" else _tgv()
    p, system, prm = (2, "euler", {}) if case == "vortex" else (3, "ns", NS_PRM)
    dt = 2e-2 if case == "vortex" else 5e-3
    ref, err_ref = o.dopri5(U, dt, 3, atol=1e-6, rtol=1e-6)
    s = fr.Solver(m, p, system, "fp64", device=0, **prm)
    g, err = _run(torch, s, U, lambda u: s.dopri5(u, dt, 3, 1e-6, 1e-6, error=True))
    # the RHS matches to rel-L2 1e-12 (FP64 parity bound); the state after 3 steps of 7 stages
    assert rel_l2_per_var(g[0], ref[0]) < 1e-12
    # E is a difference of nearly equal 4th/5th-order solutions: relative accuracy of
    # its norm ~ eps |u| / |E|
    assert err == pytest.approx(err_ref, rel=1e-6)
    assert err > 0


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_dopri5_single_precision_close_to_oracle(torch, prec):
    from paper_1312_1638_b300 import fr
    m, o, U = _tgv()
    U = [u.astype(np.float32).astype(np.float64) for u in U]
    dt, n = 5e-3, 2
    ref, _ = o.dopri5(U, dt, n)
    _, S = o.rhs(U, scale=True)
    s = fr.Solver(m, 3, "ns", prec, device=0, **NS_PRM, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))
    g, _ = _run(torch, s, U, lambda u: s.dopri5(u, dt, n))
    # componentwise: the RHS bound tol * S integrated over the interval (S at the
    # initial state, doubled for its variation) plus the FP32 rounding of every
    # stage state (7 stages per step, a few ulps of |u| each)
    tol = {"fp32": 2e-6, "tf32x3": 4e-6}[prec]
    bound = tol * 2 * S[0] * n * dt + 16 * np.finfo(np.float32).eps * np.abs(ref[0]) * n
    assert np.all(np.abs(g[0] - ref[0]) <= bound), float(np.max(np.abs(g[0] - ref[0]) / bound))


def test_dopri5_adaptive_matches_fixed_step_replay(torch):
    from paper_1312_1638_b300 import fr
    m, o, U = _vortex()
    s = fr.Solver(m, 2, "euler", "fp64", device=0)
    g, rec = _run(torch, s, U, lambda u: s.dopri5_adaptive(u, t_end=0.3, dt0=0.2, atol=1e-7, rtol=1e-7))
    assert rec["t"] == pytest.approx(0.3, rel=1e-12)
    assert rec["rejected"] >= 1 and len(rec["accepted"]) >= 3
    ref = [u.copy() for u in U]
    for h in rec["accepted"]:
        ref, _ = o.dopri5(ref, h, 1)
    # FP64 RHS parity (rel-L2 ~1e-13 per evaluation) accumulated over the accepted steps
    assert rel_l2_per_var(g[0], ref[0]) < 1e-11


def test_stepper_argument_errors(torch):
    from paper_1312_1638_b300 import fr
    m, o, U = _vortex()
    s = fr.Solver(m, 2, "euler", "fp64", device=0)
    u = [torch.from_numpy(s.pack(0, U[0])).cuda()]
    with pytest.raises(fr.FRError):
        s.euler(u, 1e-3, -1)
    with pytest.raises(fr.FRError):
        s.dopri5(u, 1e-3, 1, atol=0.0, error=True)
    assert s.sync_status() == fr.OK
