"""Couette flow (Sec. 5.2) on the GPU: RHS parity on the mixed channel with
both wall types against the oracle, and the steady-state energy error
converging at order ~p+1 (the paper's expected order) for p = 1."""

import numpy as np
import pytest

from fr_inputs import fields
from fr_inputs.meshes import channel_mixed
from oracle.system import FRSystem
from tests import couette_study as C
from tests.libutil import ensure_built, oracle_state
from tests.test_gpu_parity import check, gpu_rhs, mean_ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_rhs_channel_with_moving_wall_matches_oracle(torch, prec):
    from paper_1312_1638_b300 import fr
    m = channel_mixed(6, 6, jitter=0.1, seed=2)
    o = FRSystem(m, 3, "ns", **C.PRM)
    rng = np.random.default_rng(3)
    U = oracle_state(o, lambda X: fields.couette(X, C.G, C.PR, C.CPTW, C.VW, C.PC))
    U = [u * (1 + 0.01 * rng.standard_normal(u.shape)) for u in U]       # off the steady state
    if prec != "fp64":
        U = [u.astype(np.float32).astype(np.float64) for u in U]
    R, S = o.rhs(U, scale=True)
    s = fr.Solver(m, 3, "ns", prec, device=0, **C.PRM, **mean_ref(U))
    check(gpu_rhs(torch, s, U), R, S, prec)
    assert s.sync_status() == fr.OK


@pytest.mark.parametrize("p,meshes", [(1, (4, 6, 8))])
def test_couette_steady_energy_error_order(torch, p, meshes):
    # analytic start integrated to t = 1.2 (the p = 2..4 table comes from the study driver)
    hs, sg = [], []
    for n in meshes:
        r = C.run(p, n, start="exact")
        hs.append(r["h"])
        sg.append(r["sigma"])
    o, se = C.order(hs, sg)
    assert o > p + 1 - 0.5, (o, se, sg)
