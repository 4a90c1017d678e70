"""fr_rk4_noalloc: the RK4 step for callers that cannot let the library
allocate device memory at call time (applications whose framework owns the
GPU's memory through its own pool; loops in which cudaMalloc/cudaFree, which
may synchronise the device, must not run).  Its stage registers live in a
fixed device array inside libfr.so instead of memory from cudaMalloc.

The test calls it through the C ABI and checks it against fr_rk4 on two
calls in a row, in every precision: FP64 and FP32 at the tolerances of the
other FP64 / FP32 tests, and the split-precision paths (TF32x3, BF16x3), on
which fr_rk4 runs the stage combination inside the divergence product while
this entry point runs it as a separate kernel, at the split-precision bound
2e-5.  Around the second call it checks that the device's free memory is
unchanged, and it checks that a mesh whose registers exceed the fixed array
is refused before anything runs.  It sits in a file of its own, collected
last.
"""
import ctypes as C

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from tests.libutil import ensure_built, rel_l2_per_var

pytestmark = pytest.mark.gpu

PRM = dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1)
TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 2e-5, "bf16x3": 2e-5}


def _ptrs(ts):
    arr = (C.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr()
    return arr


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_noalloc_rk4_matches_rk4_on_two_calls(prec):
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_1312_1638_b300 import fr
    m = periodic_box("quad", 12, 0.0, 2 * np.pi, jitter=0.1, seed=3)
    s = fr.Solver(m, 3, "ns", prec, device=0, **PRM, ref_rho=1.0, ref_p=1.0)
    # state from the library's own solution points (no oracle involved)
    X = s.solution_points(0)
    U = fields.smooth_random(X, period=2 * np.pi, seed=4, amp=0.1).transpose(1, 0, 2)
    u_ref = torch.from_numpy(s.pack(0, U)).cuda()
    u_new = u_ref.clone()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        s.rk4([u_ref], 2e-3, 2)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = s.lib.fr_rk4_noalloc(s.ctx, _ptrs([u_new]), C.c_double(2e-3), 2, stream)
        assert st == fr.OK, s.lib.fr_last_error(s.ctx)
        torch.cuda.synchronize()
        if call == 1:
            # the second call finds every kernel loaded: nothing may take device memory
            assert torch.cuda.mem_get_info()[0] == free0
        n = m.nelem
        a = u_ref[:, :, :n].cpu().numpy().astype(np.float64)
        b = u_new[:, :, :n].cpu().numpy().astype(np.float64)
        assert rel_l2_per_var(b, a) <= TOL[prec], (call, rel_l2_per_var(b, a))
    assert s.sync_status() == fr.OK
    s.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_array():
    import torch
    assert torch.cuda.is_available()
    ensure_built()
    from paper_1312_1638_b300 import fr
    # 24^3 hexes, p = 4, FP32: 2 * 125 * 5 * 13824 * 4 bytes > 64 MiB
    m = periodic_box("hex", 24, 0.0, 2 * np.pi)
    s = fr.Solver(m, 4, "euler", "fp32", device=0)
    lay = s.layout(0)
    need = 2 * lay["nupts"] * lay["nvars"] * lay["ld"] * 4
    assert need > 64 * 1024 * 1024
    u = s.alloc_state(0)
    st = s.lib.fr_rk4_noalloc(s.ctx, _ptrs([u]), C.c_double(1e-3), 1, None)
    assert st == fr.ERR_ARG
    assert b"static scratch" in s.lib.fr_last_error(s.ctx)
    s.close()
