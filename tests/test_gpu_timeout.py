"""Failure detection without a GPU fault: the tensor-core GEMMs' bounded
waits.  A wait limit of a few cycles makes the waits give up; the kernels
then drain their own copies and MMAs and return, fr_sync_status reports
FR_ERR_TIMEOUT, and the same context computes the exact RHS again once the
default limit is restored."""

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

NS_PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU test without a GPU"
    ensure_built()
    return t


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_forced_wait_timeout_is_reported_and_context_recovers(torch, prec):
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.1, seed=3)
    s = fr.Solver(m, 3, "ns", prec, device=0, **NS_PRM, ref_rho=1.0, ref_p=1.0 / (1.4 * 0.09))
    # every operator product on the tensor cores (on hexahedra the structured
    # kernels would otherwise take them, and they have no waits to give up)
    for opt in ("structured_interp", "structured_grad", "structured_div"):
        s.set_option(opt, 0)
    U = fields.taylor_green(s.solution_points(0), M=0.3).transpose(1, 0, 2)
    u = torch.from_numpy(s.pack(0, U)).float().cuda()
    r = torch.empty_like(u)
    s.rhs([u], [r])
    torch.cuda.synchronize()
    assert s.sync_status() == fr.OK
    ref = r.clone()
    s.set_option("tc_wait_limit", 4)                     # a few cycles: the waits give up
    r.zero_()
    s.rhs([u], [r])
    assert s.sync_status() == fr.ERR_TIMEOUT
    u2 = u.clone()
    s.rk4([u2], 1e-4, 1)                                 # the graph is captured with the short limit too
    assert s.sync_status() == fr.ERR_TIMEOUT
    s.set_option("tc_wait_limit", 0)
    s.rhs([u], [r])
    torch.cuda.synchronize()
    assert s.sync_status() == fr.OK
    assert torch.equal(r, ref)                           # same context, same bits
    u3 = u.clone()
    s.rk4([u3], 1e-4, 1)
    torch.cuda.synchronize()
    assert s.sync_status() == fr.OK
    assert torch.isfinite(u3).all()
