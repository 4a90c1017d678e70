"""fr_rk4 runs each stage combination inside the divergence kernel: the
structured kernel on tensor elements (every precision) or the tensor-core
GEMM's epilogue (split precisions, dense operator).  It must equal RK4
assembled from separate right-hand-side calls up to FP32 rounding, and leave
the padding columns of the state untouched; and fr_rk4 in every single
precision (CUDA-graph replay on and off) must match the FP64 oracle's RK4
(end of Sec. 2) from the same FP32-rounded state within the RHS bound
integrated over the interval."""

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from oracle.system import FRSystem
from tests.libutil import ensure_built, kappa_per_var, record_parity, rel_l2_vars

pytestmark = pytest.mark.gpu

NS_PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("structured", [0, 1])
def test_fused_rk4_equals_composed_rk4(torch, prec, graphs, structured):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.1, seed=5)       # 27 elements: ld = 128 > nelem
    s = fr.Solver(m, 3, "ns", prec, device=0, **NS_PRM)
    s.set_option("graphs", graphs)
    s.set_option("structured_div", structured)
    s.set_option("structured_grad", structured)
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
    tol = {"fp32": 2e-6, "tf32x3": 4e-6, "bf16x3": 1e-4}[prec]
    bound = tol * 2 * S[0] * nsteps * dt + 16 * np.finfo(np.float32).eps * np.abs(B) * nsteps
    assert np.all(np.abs(A - B) <= bound), float(np.max(np.abs(A - B) / bound))
    assert torch.all(a[0][:, :, ne:] == 12345.0)                         # padding untouched
    assert s.sync_status() == fr.OK


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("graphs", [0, 1])
def test_rk4_single_precision_matches_oracle(torch, prec, graphs):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.1, seed=5)
    prm = {k: v for k, v in NS_PRM.items() if not k.startswith("ref_")}
    o = FRSystem(m, 3, "ns", **prm)
    U = fields.taylor_green(o.solution_coords(0), M=0.3).transpose(1, 0, 2)
    U = U.astype(np.float32).astype(np.float64)
    dt, nsteps = 2e-3, 3
    ref = o.rk4([U], dt, nsteps)[0]
    R, S = o.rhs([U], scale=True)
    s = fr.Solver(m, 3, "ns", prec, device=0, **NS_PRM)
    s.set_option("graphs", graphs)
    u = [torch.from_numpy(s.pack(0, U)).cuda()]
    s.rk4(u, dt, nsteps)
    torch.cuda.synchronize()
    G = u[0][:, :, :U.shape[2]].double().cpu().numpy()
    # the RHS bound tol * S integrated over the interval (S at the initial state,
    # doubled for its variation) plus the FP32 rounding of every stage state
    tol = {"fp32": 2e-6, "tf32x3": 4e-6, "bf16x3": 1e-4}[prec]
    bound = tol * 2 * S[0] * nsteps * dt + 16 * np.finfo(np.float32).eps * np.abs(ref) * nsteps
    assert np.all(np.abs(G - ref) <= bound), float(np.max(np.abs(G - ref) / bound))
    # stated, not bounded: the state's and the increment's error per variable (the
    # increment's is dominated by the FP32 rounding of the stored stage states)
    record_parity("rk4_hex3_p3_ns_tgv_m03", prec, graphs=graphs, rel_l2_state=rel_l2_vars(G, ref),
                  rel_l2_increment=rel_l2_vars(G - U, ref - U), kappa_rhs=kappa_per_var(S[0], R[0]))
    assert s.sync_status() == fr.OK
