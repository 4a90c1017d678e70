"""Structured operator kernels on tensor elements (quadrilaterals, hexahedra).

With tensor Gauss-Legendre solution and flux points, a row (i, s) of the
corrected-gradient operator [M6 | M4 - M6 M0] (Eq. tquptsm) has nonzeros only
at the p+1 solution points on the line through s in direction i and at the
two flux points that end that line, and a row s of the divergence operator
[M3 | M1 - M3 M2] (Eq. tdivflux) only, per direction, at the p+1 flux values
on the line through s and the two common fluxes ending it.  The structured
kernels keep those entries (dropping the rounding of vanishing Lagrange
factors, below 1e-15 of their row's largest), sum them in the dense
product's order and apply the transform Q = J^-T Q~ (Eq. gradufpts) or the
-1/J scaling (Eq. negdivconf) with the arithmetic of the dense path.  Both
forms must meet the precision's parity bound against the FP64 oracle, and
differ from each other by a small fraction of it."""
import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))
TOL_C = {"fp64": 1e-13, "fp32": 2e-6, "tf32x3": 4e-6, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    ensure_built()
    return t


def _rhs(torch, s, u):
    r = [torch.full_like(x, float("nan")) for x in u]
    s.rhs(u, r)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("etype,n,p,system", [("quad", 12, 3, "ns"), ("quad", 9, 4, "ns"), ("hex", 4, 4, "ns"),
                                              ("hex", 3, 2, "ns"), ("hex", 4, 4, "euler")])
@pytest.mark.parametrize("op", ["grad", "div"])
@pytest.mark.parametrize("form", [1, 2])
def test_structured_operator_matches_the_dense_product(torch, etype, n, p, system, prec, op, form):
    """op = grad: the corrected gradient (Eq. tquptsm, gradufpts); op = div: the
    divergence (Eq. tdivflux, negdivconf); form 1: the tensor-line kernel, 2:
    the row-wise kernel.  Each structured kernel against the dense product of
    the same context, both against the oracle."""
    from oracle.system import FRSystem
    from paper_1312_1638_b300 import fr
    if op == "grad" and system == "euler":
        pytest.skip("the Euler right-hand side has no gradient")
    m = periodic_box(etype, n, 0.0, 2 * np.pi, jitter=0.1, seed=4)
    s = fr.Solver(m, p, system, prec, device=0, **PRM)
    t = fr.Solver(m, p, system, prec, device=0, **PRM)
    s.set_option("structured_" + op, form)
    t.set_option("structured_" + op, 0)
    U = fields.smooth_random(s.solution_points(0), seed=3, amp=0.1, vel0=(0.3, 0.1, 0.0)[:m.ndims],
                             p0=1.0 / (1.4 * 0.09)).transpose(1, 0, 2).copy()
    if prec != "fp64":
        U = U.astype(np.float32).astype(np.float64)
    prm = {k: v for k, v in PRM.items() if not k.startswith("ref_")}
    R, S = FRSystem(m, p, system, **prm).rhs([U], scale=True)
    u = [torch.from_numpy(s.pack(0, U)).cuda()]
    s.profile_enable(True)
    t.profile_enable(True)
    a, b = _rhs(torch, s, u), _rhs(torch, t, u)
    ps, pt = s.profile_read(), t.profile_read()
    if op == "grad":
        # the structured kernel carries the transform: no separate transform launch
        assert ps["tgradu_gemm"][0] == 1 and ps["gradcoru"][0] == 0
        if prec in ("fp64", "fp32"):
            assert pt["gradcoru"][0] == 1
        # the tensor-line kernel also forms the gradient at flux points (when its
        # tiles fit: FP64 hexahedra at p = 4 take the row-wise kernel)
        line = form == 1 and not (prec == "fp64" and etype == "hex" and p == 4)
        assert ps["gradfpts_gemm"][0] == (0 if line else m.ndims), ps["gradfpts_gemm"]
    else:
        assert ps["tdivf_gemm"][0] == 1 and pt["tdivf_gemm"][0] == 1
    ne = m.blocks[0].nodes.shape[0]
    ga, gb = (x[0].cpu().numpy()[:, :, :ne].astype(np.float64) for x in (a, b))
    tol = TOL_C[prec]
    ea, eb, ed = (np.max(np.abs(x) / S[0]) for x in (ga - R[0], gb - R[0], ga - gb))
    print(f"structured {op} form {form} {etype} p{p} {system} {prec}: {ea:.2e} dense {eb:.2e} difference {ed:.2e} "
          f"(bound {tol:.0e})")
    assert ea <= tol and eb <= tol
    # FP64 / FP32: the same sums (the row-wise form in the same order, the line
    # form grouped by line); split precisions: the dense product carries the
    # split's error
    assert ed <= (tol / 4 if prec in ("fp64", "fp32") else tol)
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK


def test_structured_gradient_rk4_graph_equals_direct_launches(torch):
    """The structured gradient inside the captured RK4 step (graph replay) gives
    the same bits as the same steps launched directly."""
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 5, 0.0, 2 * np.pi, jitter=0.05, seed=2)
    s = fr.Solver(m, 4, "ns", "tf32x3", device=0, **PRM)
    t = fr.Solver(m, 4, "ns", "tf32x3", device=0, **PRM)
    t.set_option("graphs", 0)
    U = fields.smooth_random(s.solution_points(0), seed=5, amp=0.1, vel0=(0.3, 0.1, 0.0),
                             p0=1.0 / (1.4 * 0.09)).transpose(1, 0, 2).copy()
    a = [torch.from_numpy(s.pack(0, U)).cuda()]
    b = [a[0].clone()]
    s.rk4(a, 1e-3, 4)
    t.rk4(b, 1e-3, 4)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0])
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mixed_mesh_structured_gradient_grouped_and_per_block(torch, prec):
    """On a mixed mesh the quadrilaterals' gradient takes the structured kernel
    and the triangles' the tensor-core product, grouped or not: the same bits
    either way, two gradient launches per right-hand side."""
    from fr_inputs import annulus_mixed
    from paper_1312_1638_b300 import fr
    m = annulus_mixed(ntheta=24, nr_quad=3, nr_tri=3, r0=0.5, r1=4.0, jitter=0.05, seed=7)
    p_inf = 1 / (1.4 * 0.04)
    kw = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0),
              bc_p=p_inf, outflow_p=p_inf, wall_cpTw=1.4 / 0.4 * p_inf, ref_rho=1.0, ref_p=p_inf)
    s = fr.Solver(m, 4, "ns", prec, device=0, **kw)
    t = fr.Solver(m, 4, "ns", prec, device=0, **kw)
    t.set_option("group_blocks", 0)
    u = []
    for b in range(len(m.blocks)):
        U = fields.smooth_random(s.solution_points(b), seed=3 + b, amp=0.1, vel0=(0.3, 0.1),
                                 p0=p_inf).transpose(1, 0, 2)
        u.append(torch.from_numpy(s.pack(b, U)).cuda())
    s.profile_enable(True)
    t.profile_enable(True)
    a, b = _rhs(torch, s, u), _rhs(torch, t, u)
    ps, pt = s.profile_read(), t.profile_read()
    assert ps["tgradu_gemm"][0] == 2 and pt["tgradu_gemm"][0] == 2
    for x, y, blk in zip(a, b, m.blocks):
        ne = blk.nodes.shape[0]
        assert torch.equal(x[:, :, :ne], y[:, :, :ne])
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("system", ["euler", "ns"])
def test_structured_adjoint_matches_the_dense_products(torch, prec, system):
    """The adjoint's transposed operators in structured form (M3^T,
    (M1 - M3 M2)^T, M0^T, M6^T: p+1 or 2D nonzeros per row; [M0^T |
    (M4 - M6 M0)^T] over two stacked sources) give the adjoint RHS of the
    dense products to the precision's rounding (tests/test_gpu_adjoint.py
    holds both against the oracle's transpose)."""
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.1, seed=4)
    s = fr.Solver(m, 3, system, prec, device=0, **PRM)
    t = fr.Solver(m, 3, system, prec, device=0, **PRM)
    t.set_option("structured_adjoint", 0)
    U = fields.smooth_random(s.solution_points(0), seed=3, amp=0.1, vel0=(0.3, 0.1, 0.0),
                             p0=1.0 / (1.4 * 0.09)).transpose(1, 0, 2).copy()
    rng = np.random.default_rng(11)
    L = rng.standard_normal(U.shape)
    u = [torch.from_numpy(s.pack(0, U)).cuda()]
    lam = [torch.from_numpy(s.pack(0, L)).cuda()]
    a = [torch.zeros_like(u[0])]
    b = [torch.zeros_like(u[0])]
    s.adjoint_rhs(u, lam, a)
    t.adjoint_rhs(u, lam, b)
    torch.cuda.synchronize()
    ne = m.blocks[0].nodes.shape[0]
    ga, gb = (x[0][:, :, :ne].double().cpu().numpy() for x in (a, b))
    rel = np.linalg.norm(ga - gb) / np.linalg.norm(gb)
    bound = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 2e-5}[prec]
    print(f"structured adjoint {system} {prec}: rel-L2 difference {rel:.2e}")
    assert rel <= bound
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK
