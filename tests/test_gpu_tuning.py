"""Kernel-variant tuning of the tensor-core operator products (fr_autotune,
fr_get_tuning, fr_set_tuning).  The variants differ only in how the work of a
CTA is split between warps (subtiles per work item, converter warps,
epilogue warp groups), not in the order of any arithmetic, so every variant
that fits a product must give the right-hand side bit for bit; the autotuner
must return choices from that set and leave the state untouched."""
import numpy as np
import pytest

from fr_inputs import periodic_box, annulus_mixed, fields
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

PLAIN = ["1.8.3", "2.8.2", "1.8.2", "1.12.2", "2.4.3", "1.4.3"]       # plain / -1/J / RK-stage epilogue
GRAD = ["1.4.4", "2.4.4", "1.8.3", "1.8.4", "2.8.3"]                  # gradient-transform epilogue
PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    ensure_built()
    return t


def _solver(fr, case, prec):
    if case == "hex":
        m = periodic_box("hex", 6, 0.0, 2 * np.pi, jitter=0.05, seed=2)       # 216 elements: 2 tiles per variable
        s = fr.Solver(m, 4, "ns", prec, device=0, **PRM)
    else:
        m = annulus_mixed(ntheta=24, nr_quad=3, nr_tri=3, r0=0.5, r1=4.0, jitter=0.05, seed=7)
        p_inf = 1 / (1.4 * 0.04)
        s = fr.Solver(m, 4, "ns", prec, device=0, gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1,
                      bc_rho=1.0, bc_v=(1.0, 0.0, 0.0), bc_p=p_inf, outflow_p=p_inf, wall_cpTw=1.4 / 0.4 * p_inf,
                      ref_rho=1.0, ref_p=p_inf)
    # these tests are about the tensor-core products: the corrected gradient and
    # the divergence of the tensor elements run there too (not on their
    # structured kernels)
    s.set_option("structured_grad", 0)
    s.set_option("structured_div", 0)
    return m, s


def _state(torch, s, m):
    u = []
    for b in range(len(m.blocks)):
        X = s.solution_points(b)
        U = fields.smooth_random(X, seed=3 + b, amp=0.1, vel0=(0.3, 0.1, 0.0)[:m.ndims],
                                 p0=1.0 / (1.4 * 0.09)).transpose(1, 0, 2)
        u.append(torch.from_numpy(s.pack(b, U)).cuda())
    return u


def _rhs(torch, s, u):
    r = [torch.full_like(x, float("nan")) for x in u]
    s.rhs(u, r)
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("case", ["hex", "mixed"])
def test_every_variant_gives_the_same_bits(torch, case, prec):
    from paper_1312_1638_b300 import fr
    m, s = _solver(fr, case, prec)
    u = _state(torch, s, m)
    ref = _rhs(torch, s, u)
    tried = 0
    for prod, table in (("disu", PLAIN), ("tgradu", GRAD), ("gradfpts", PLAIN), ("tdivf", PLAIN)):
        for v in table:
            text = ";".join(f"b{b}:{prod}={v}" for b in range(len(m.blocks)))
            try:
                s.set_tuning(text)
            except fr.FRError as e:                     # the variant does not fit this operator
                assert e.status == fr.ERR_ARG
                continue
            tried += 1
            got = _rhs(torch, s, u)
            for b in range(len(m.blocks)):
                ne = m.blocks[b].nodes.shape[0]
                assert torch.equal(got[b][:, :, :ne], ref[b][:, :, :ne]), (prod, v, b)
            s.set_tuning(";".join(f"b{b}:{prod}=default" for b in range(len(m.blocks))))
    assert tried >= 10
    assert s.sync_status() == fr.OK


def test_autotune_chooses_fitting_variants_and_keeps_the_state(torch):
    from paper_1312_1638_b300 import fr
    m, s = _solver(fr, "mixed", "tf32x3")
    u = _state(torch, s, m)
    before = [x.clone() for x in u]
    ref = _rhs(torch, s, u)
    text = s.autotune(u, reps=1)
    assert [torch.equal(a, b) for a, b in zip(u, before)] == [True] * len(u)
    parts = dict(p.split(":", 1) for p in text.split(";"))
    assert sorted(parts) == ["b0", "b1"]
    for b, body in parts.items():
        kv = dict(x.split("=") for x in body.split(","))
        assert kv["tgradu"] in GRAD + ["default"]
        for k in ("disu", "gradfpts", "tdivf"):
            assert kv[k] in PLAIN + ["default"]
        assert kv["tdivf"] == "default" or kv["tdivf"].startswith("2.")     # the RK stage stays fused
    got = _rhs(torch, s, u)
    for b in range(len(m.blocks)):
        ne = m.blocks[b].nodes.shape[0]
        assert torch.equal(got[b][:, :, :ne], ref[b][:, :, :ne])
    # the text round-trips and malformed or unfit entries change nothing
    s.set_tuning(text)
    assert s.tuning() == text
    for bad in ("b0:disu=3.3.3", "b9:disu=1.8.3", "b0:nosuch=1.8.3", "b0:disu", "x"):
        with pytest.raises(fr.FRError):
            s.set_tuning(bad)
        assert s.tuning() == text
    assert s.sync_status() == fr.OK


def test_tuned_rk4_equals_default_rk4(torch):
    """A tuned context advances RK4 (graph replay, fused RK stage) exactly as
    the default one."""
    from paper_1312_1638_b300 import fr
    m, s = _solver(fr, "hex", "tf32x3")
    _, t = _solver(fr, "hex", "tf32x3")
    t.set_tuning("b0:disu=1.12.2,tgradu=1.8.3,gradfpts=1.4.3,tdivf=2.4.3")
    a = _state(torch, s, m)
    b = [x.clone() for x in a]
    s.rk4(a, 1e-3, 3)
    t.rk4(b, 1e-3, 3)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0])
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK


@pytest.mark.parametrize("structured", [0, 1])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_grouped_launches_match_per_block_launches(torch, prec, structured):
    """On a mixed mesh (quadrilaterals and triangles) each tensor-core product
    runs as one launch over both blocks' work items: the same bits as one
    launch per block, for the right-hand side and for graph-replayed RK4, with
    one launch per product and stage (the gradient interpolations of both
    blocks included) instead of one per block.  With the structured
    interpolation on, the quadrilaterals' M0 products take it in both."""
    from paper_1312_1638_b300 import fr
    m, s = _solver(fr, "mixed", prec)
    _, t = _solver(fr, "mixed", prec)
    t.set_option("group_blocks", 0)
    for x in (s, t):
        x.set_option("structured_interp", structured)
    u = _state(torch, s, m)
    s.profile_enable(True)
    t.profile_enable(True)
    a, b = _rhs(torch, s, u), _rhs(torch, t, u)
    ps, pt = s.profile_read(), t.profile_read()
    for k in ("tgradu_gemm", "tdivf_gemm") + (() if structured else ("disu_gemm", "gradfpts_gemm")):
        assert ps[k][0] == 1, (k, ps[k])
        assert pt[k][0] == (4 if k == "gradfpts_gemm" else 2), (k, pt[k])    # per block (and direction)
    for x, y, blk in zip(a, b, m.blocks):
        ne = blk.nodes.shape[0]
        assert torch.equal(x[:, :, :ne], y[:, :, :ne])
    s.profile_enable(False)
    t.profile_enable(False)
    ua, ub = [x.clone() for x in u], [x.clone() for x in u]
    s.rk4(ua, 1e-6, 3)
    t.rk4(ub, 1e-6, 3)
    torch.cuda.synchronize()
    for x, y, blk in zip(ua, ub, m.blocks):
        ne = blk.nodes.shape[0]
        assert torch.equal(x[:, :, :ne], y[:, :, :ne])
    assert s.sync_status() == fr.OK and t.sync_status() == fr.OK


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("etype,n,p", [("quad", 12, 3), ("hex", 4, 4), ("hex", 3, 2)])
def test_structured_interpolation_matches_the_dense_product(torch, etype, n, p, prec):
    """On tensor elements M0 has p+1 nonzeros per row; the structured kernel
    keeps those (entries below 1e-15 of their row's largest, the rounding of
    a vanishing Lagrange factor, are dropped) and adds them in the order the
    dense CUDA-core product does.  Both right-hand sides meet the precision's
    parity bound against the oracle (|R_gpu - R| <= tol S), and they differ
    from each other by a small fraction of it."""
    from oracle.system import FRSystem
    from paper_1312_1638_b300 import fr
    m = periodic_box(etype, n, 0.0, 2 * np.pi, jitter=0.1, seed=4)
    s = fr.Solver(m, p, "ns", prec, device=0, **PRM)
    t = fr.Solver(m, p, "ns", prec, device=0, **PRM)
    t.set_option("structured_interp", 0)
    U = fields.smooth_random(s.solution_points(0), seed=3, amp=0.1, vel0=(0.3, 0.1, 0.0)[:m.ndims],
                             p0=1.0 / (1.4 * 0.09)).transpose(1, 0, 2).copy()
    if prec == "fp32":
        U = U.astype(np.float32).astype(np.float64)
    prm = {k: v for k, v in PRM.items() if not k.startswith("ref_")}
    R, S = FRSystem(m, p, "ns", **prm).rhs([U], scale=True)
    u = [torch.from_numpy(s.pack(0, U)).cuda()]
    a, b = _rhs(torch, s, u), _rhs(torch, t, u)
    ne = m.blocks[0].nodes.shape[0]
    ga, gb = (x[0].cpu().numpy()[:, :, :ne].astype(np.float64) for x in (a, b))
    tol = {"fp64": 1e-13, "fp32": 2e-6}[prec]
    ea, eb, ed = (np.max(np.abs(x) / S[0]) for x in (ga - R[0], gb - R[0], ga - gb))
    print(f"structured {etype} p{p} {prec}: {ea:.2e} dense {eb:.2e} difference {ed:.2e} (bound {tol:.0e})")
    assert ea <= tol and eb <= tol
    assert ed <= tol / 4
    assert s.sync_status() == fr.OK


def test_structured_kernel_limits_do_not_shrink_between_contexts(torch):
    """The structured kernel's shared-memory limit belongs to the kernel, not
    to a context or block: a context with a large tile (hexahedra, p = 4,
    FP64) still runs after contexts with smaller ones are set up, as does a
    mesh whose two structured blocks need different tiles (quadrilaterals and
    triangles at p = 1), through an RK4 graph."""
    from paper_1312_1638_b300 import fr
    from fr_inputs.meshes import channel_mixed
    m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.1, seed=4)
    big = fr.Solver(m, 4, "ns", "fp64", device=0, **PRM)
    u = _state(torch, big, m)
    before = _rhs(torch, big, u)
    mc = channel_mixed(4, 4, jitter=0.1, seed=1)
    small = fr.Solver(mc, 1, "ns", "fp64", device=0, **PRM)
    uc = _state(torch, small, mc)
    small.rk4(uc, 1e-5, 2)
    torch.cuda.synchronize()
    assert small.sync_status() == fr.OK
    after = _rhs(torch, big, u)
    assert torch.equal(before[0], after[0])
    assert big.sync_status() == fr.OK
