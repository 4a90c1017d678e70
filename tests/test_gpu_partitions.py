"""Partitioned right-hand side (Sec. 3.6 int/mpi split) on one GPU: 2-4
partitions exchanging flux-point values give the whole-mesh right-hand side
bit for bit (every pair is evaluated with the same inputs in the same
order of operations), and match the FP64 oracle's whole-mesh right-hand side
element by element within the componentwise bound of the parity tests."""

import numpy as np
import pytest

from fr_inputs import periodic_box, annulus_mixed, fields
from oracle.system import FRSystem
from tests.libutil import ensure_built, m0_spread, oracle_state
from tests.test_gpu_parity import TOL_C, mean_ref
from tests.test_part_host import _partition

pytestmark = pytest.mark.gpu

NS_PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)
MIXED_PRM = dict(NS_PRM, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0), bc_p=1 / (1.4 * 0.04), outflow_p=1 / (1.4 * 0.04),
                 wall_cpTw=1.4 / 0.4 * (1 / (1.4 * 0.04)))


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


def _case(name):
    if name == "hex_ns":
        m = periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.1, seed=2)
        return m, 3, "ns", NS_PRM, lambda X: fields.taylor_green(X, M=0.3)
    if name == "quad_euler":
        m = periodic_box("quad", 8, -5.0, 5.0, jitter=0.1, seed=4)
        return m, 2, "euler", {}, lambda X: fields.isentropic_vortex(X, S=5.0, M=0.4, R=1.5)
    m = annulus_mixed(ntheta=16, nr_quad=2, nr_tri=2, r0=0.5, r1=4.0, jitter=0.05, seed=7)
    m.bfaces[(m.bfaces[:, 0] == 1) & (m.bfaces[:, 1] % 2 == 0), 3] = 1
    return m, 3, "ns", MIXED_PRM, lambda X: fields.smooth_random(X, seed=3, amp=0.1, vel0=(1.0, 0.0),
                                                                 p0=1 / (1.4 * 0.04))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("name,nparts", [("hex_ns", 2), ("hex_ns", 4), ("quad_euler", 3), ("mixed_ns", 2),
                                         ("mixed_ns", 3)])
def test_partitioned_rhs_is_bit_identical(torch, name, nparts, prec):
    from paper_1312_1638_b300 import fr
    m, p, system, prm, st = _case(name)
    whole = fr.Solver(m, p, system, prec, device=0, **prm)
    dt = torch.float64 if prec == "fp64" else torch.float32
    U, u, r = [], [], []
    for b in range(len(m.blocks)):
        X = whole.solution_points(b)
        Ub = st(X).transpose(1, 0, 2)                             # [nupts, V, nelem]
        U.append(Ub)
        u.append(torch.from_numpy(whole.pack(b, Ub)).to(dt).cuda())
        r.append(torch.full_like(u[-1], float("nan")))
    whole.rhs(u, r)
    part = _partition(m, nparts, seed=11 * nparts)
    ps = fr.PartitionedSolver(m, part, nparts, p, system, prec, device=0, **prm)
    up, rp = [], []
    for k in range(nparts):
        s = ps.ranks[k]
        uk, rk = [], []
        for b in range(len(m.blocks)):
            loc = ps.local_elements(k, b)
            x = torch.from_numpy(s.pack(b, U[b][:, :, loc])).to(dt).cuda()
            uk.append(x)
            rk.append(torch.full_like(x, float("nan")))
        up.append(uk)
        rp.append(rk)
    ps.rhs(up, rp)
    torch.cuda.synchronize()
    for b in range(len(m.blocks)):
        ref = r[b][:, :, :m.blocks[b].nodes.shape[0]].cpu().numpy()
        got = np.full_like(ref, np.nan)
        for k in range(nparts):
            loc = ps.local_elements(k, b)
            got[:, :, loc] = rp[k][b][:, :, :len(loc)].cpu().numpy()
        assert np.isfinite(got).all()
        assert np.array_equal(got, ref), float(np.nanmax(np.abs(got - ref)))
    for s in ps.ranks:
        assert s.sync_status() == fr.OK
    with pytest.raises(fr.FRError) as e:                           # a partition alone has no whole RHS
        ps.ranks[0].rhs(up[0], rp[0])
    assert e.value.status == fr.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name,nparts", [("hex_ns", 2), ("hex_ns", 4), ("quad_euler", 3), ("mixed_ns", 2),
                                         ("mixed_ns", 3)])
def test_partitioned_rhs_matches_oracle(torch, name, nparts, prec):
    from paper_1312_1638_b300 import fr
    m, p, system, prm, st = _case(name)
    o = FRSystem(m, p, system, **prm)
    U = oracle_state(o, st)
    if prec != "fp64":
        U = [u.astype(np.float32).astype(np.float64) for u in U]
    R, S = o.rhs(U, scale=True)
    # FP64: 1e-13 S plus twice the oracle's own spread under 8-ulp perturbations of M0
    # (the library builds M0 by another exact-equivalent construction)
    extra = m0_spread(o, U) if prec == "fp64" else [np.zeros(r.shape[1]) for r in R]
    part = _partition(m, nparts, seed=11 * nparts)
    ps = fr.PartitionedSolver(m, part, nparts, p, system, prec, device=0, **prm, **mean_ref(U))
    dt = torch.float64 if prec == "fp64" else torch.float32
    up, rp = [], []
    for k in range(nparts):
        s = ps.ranks[k]
        uk, rk = [], []
        for b in range(len(m.blocks)):
            loc = ps.local_elements(k, b)
            x = torch.from_numpy(s.pack(b, U[b][:, :, loc])).to(dt).cuda()
            uk.append(x)
            rk.append(torch.full_like(x, float("nan")))
        up.append(uk)
        rp.append(rk)
    ps.rhs(up, rp)
    torch.cuda.synchronize()
    for b in range(len(m.blocks)):
        got = np.full_like(R[b], np.nan)
        for k in range(nparts):
            loc = ps.local_elements(k, b)
            got[:, :, loc] = rp[k][b][:, :, :len(loc)].double().cpu().numpy()
        assert np.isfinite(got).all()
        bound = TOL_C[prec] * S[b] + 2 * extra[b][None, :, None]
        assert np.all(np.abs(got - R[b]) <= bound), (b, float(np.max(np.abs(got - R[b]) / bound)))
    for s in ps.ranks:
        assert s.sync_status() == fr.OK
    ps.close()
