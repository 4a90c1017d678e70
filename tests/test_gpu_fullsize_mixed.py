"""Full-size parity on the mixed-mesh workload: 2D Navier-Stokes on the
annulus r in [0.5, 20] with 100,000 quadratic-wall quads and 60,000
triangles (shuffled numbering, jittered nodes), p = 4, Re 100 (D = 1,
V = 1, mu = 0.01), Mach 0.2, Pr 0.72; isothermal wall at free-stream
temperature on r = 0.5 and free-stream ghosts on r = 20.  The oracle
evaluates the whole mesh once (about half a minute); every element of the
GPU result is compared with it under the componentwise bound of the small
cases, in FP64, FP32 and TF32x3 (perturbation form about the free stream)."""

import numpy as np
import pytest

from fr_inputs import annulus_mixed, fields
from oracle.system import FRSystem
from tests.libutil import ensure_built, kappa_per_var, record_parity, rel_l2_vars
from tests.test_gpu_parity import KAPPA_WELL, TOL_C, TOL_L2

pytestmark = pytest.mark.gpu

P_INF = 1.0 / (1.4 * 0.2 ** 2)
PRM = dict(gamma=1.4, mu=0.01, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0),
           bc_p=P_INF, outflow_p=P_INF, wall_cpTw=1.4 / 0.4 * P_INF)


@pytest.fixture(scope="module")
def case():
    m = annulus_mixed()                                   # 100k quads + 60k triangles
    o = FRSystem(m, 4, "ns", **PRM)
    U = [fields.smooth_random(o.solution_coords(b), seed=3, amp=0.1, vel0=(1.0, 0.0), p0=P_INF)
         .transpose(1, 0, 2).copy() for b in range(len(m.blocks))]
    U32 = [u.astype(np.float32).astype(np.float64) for u in U]
    return m, o, U, o.rhs(U, scale=True), U32, o.rhs(U32, scale=True)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_full_size_mixed_annulus(case, prec):
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_1312_1638_b300 import fr
    m, o, U64, (R64, S64), U32, (R32, S32) = case
    U, R, S = (U64, R64, S64) if prec == "fp64" else (U32, R32, S32)
    assert [b.nodes.shape[0] for b in m.blocks] == [100000, 60000]
    s = fr.Solver(m, 4, "ns", prec, device=0, **PRM, ref_rho=1.0, ref_p=P_INF)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = [torch.from_numpy(s.pack(b, U[b])).to(dt).cuda() for b in range(2)]
    r = [torch.full_like(x, float("nan")) for x in u]
    s.rhs(u, r)
    torch.cuda.synchronize()
    for b in range(2):
        g = r[b][:, :, :U[b].shape[2]].double().cpu().numpy()
        err = float(np.max(np.abs(g - R[b]) / np.maximum(S[b], 1e-300)))
        assert err <= TOL_C[prec], (b, err)
        rel, kap = rel_l2_vars(g, R[b]), kappa_per_var(S[b], R[b])
        record_parity(f"c3_annulus_p4_ns_block{b}", prec, rel_l2=rel, kappa=kap, componentwise=err)
        if prec != "fp64":
            ok = kap <= KAPPA_WELL
            assert np.all(rel[ok] <= TOL_L2[prec]), (b, rel, kap)
    assert s.sync_status() == fr.OK
    s.close()
