"""fr_rk4's CUDA-graph replay of one RK4 step gives exactly the bits of the
direct launches, and is re-captured when the state pointers or dt change."""
import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_graph_replay_bit_identical(prec):
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.05, seed=2)
    prm = dict(gamma=1.4, mu=0.01, prandtl=0.71)
    sg = fr.Solver(m, 3, "ns", prec, device=0, **prm, ref_rho=1.0, ref_p=10.0)
    sd = fr.Solver(m, 3, "ns", prec, device=0, **prm, ref_rho=1.0, ref_p=10.0)
    sd.set_option("graphs", 0)
    X = sg.solution_points(0)
    U = fields.smooth_random(X, period=2 * np.pi, seed=4, amp=0.1, p0=10.0).transpose(1, 0, 2)
    a = torch.from_numpy(sg.pack(0, U)).cuda()
    b = a.clone()
    for dt, steps in ((1e-3, 3), (1e-3, 2), (5e-4, 2)):           # dt change forces a new capture
        sg.rk4([a], dt, steps)
        sd.rk4([b], dt, steps)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    a2 = a.clone()                                              # new pointer: new capture
    b2 = b.clone()
    sg.rk4([a2], 5e-4, 2)
    sd.rk4([b2], 5e-4, 2)
    torch.cuda.synchronize()
    assert torch.equal(a2, b2)
    assert sg.sync_status() == fr.OK


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_rk4_host_buffers_and_rk_step_name(prec):
    """fr_rk4_host (host buffers, copies inside) and fr_rk_step (the generic
    name) give exactly fr_rk4's bits, call after call."""
    import ctypes as C
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_1312_1638_b300 import fr
    m = periodic_box("hex", 3, 0.0, 2 * np.pi, jitter=0.05, seed=3)
    prm = dict(gamma=1.4, mu=0.01, prandtl=0.71, ref_rho=1.0, ref_p=10.0)
    s = fr.Solver(m, 3, "ns", prec, device=0, **prm)
    X = s.solution_points(0)
    U = s.pack(0, fields.smooth_random(X, period=2 * np.pi, seed=6, amp=0.1, p0=10.0).transpose(1, 0, 2))
    a = torch.from_numpy(U.copy()).cuda()
    b = a.clone()
    h = torch.from_numpy(U.copy()).pin_memory()
    for _ in range(2):
        s.rk4([a], 1e-3, 2)
        st = s.lib.fr_rk_step(s.ctx, (C.c_void_p * 1)(b.data_ptr()), C.c_double(1e-3), 2, None)
        assert st == fr.OK
        s.rk4_host([h], 1e-3, 2)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert torch.equal(a.cpu(), h)
    assert s.sync_status() == fr.OK
