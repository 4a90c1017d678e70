"""RK4 on the tensor-core paths runs each stage combination inside the
divergence GEMM's epilogue.  It must equal RK4 assembled from separate
right-hand-side calls up to FP32 rounding, and leave the padding columns of
the state untouched."""

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from oracle.system import FRSystem
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

NS_PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("graphs", [0, 1])
def test_fused_rk4_equals_composed_rk4(torch, prec, graphs):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.1, seed=5)       # 27 elements: ld = 128 > nelem
    s = fr.Solver(m, 3, "ns", prec, device=0, **NS_PRM)
    s.set_option("graphs", graphs)
    X = s.solution_points(0)
    U = fields.taylor_green(X, M=0.3).transpose(1, 0, 2)
    ne = U.shape[2]
    u0 = torch.from_numpy(s.pack(0, U)).cuda()
    u0[:, :, ne:] = 12345.0                                              # padding sentinel
    dt, nsteps = 2e-3, 3
    a = [u0.clone()]
    s.rk4(a, dt, nsteps)
    # the same RK4 from separate right-hand sides
    u = u0.clone()
    k = [torch.empty_like(u) for _ in range(4)]
    for _ in range(nsteps):
        s.rhs([u], [k[0]])
        y = u + 0.5 * dt * k[0]
        s.rhs([y], [k[1]])
        y = u + 0.5 * dt * k[1]
        s.rhs([y], [k[2]])
        y = u + dt * k[2]
        s.rhs([y], [k[3]])
        u = u + dt / 6 * (k[0] + 2 * k[1] + 2 * k[2] + k[3])
    torch.cuda.synchronize()
    A, B = a[0][:, :, :ne].double().cpu().numpy(), u[:, :, :ne].double().cpu().numpy()
    # The two RK4 compositions round their stage states differently; the
    # split-precision RHS reproduces a 1-ulp change of its input only to its
    # componentwise bound tol * S.  Bound: tol * 2 S(u0) * T plus FP32 rounding.
    prm = {k: v for k, v in NS_PRM.items() if not k.startswith("ref_")}
    _, S = FRSystem(m, 3, "ns", **prm).rhs([U], scale=True)
    tol = {"tf32x3": 4e-6, "bf16x3": 1e-4}[prec]
    bound = tol * 2 * S[0] * nsteps * dt + 16 * np.finfo(np.float32).eps * np.abs(B) * nsteps
    assert np.all(np.abs(A - B) <= bound), float(np.max(np.abs(A - B) / bound))
    assert torch.all(a[0][:, :, ne:] == 12345.0)                         # padding untouched
    assert s.sync_status() == fr.OK
