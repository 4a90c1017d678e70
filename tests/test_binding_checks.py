"""The Python binding checks every state-shaped buffer against the context's
layout before it hands the pointers to the C ABI (which cannot see a size or
a dtype): a wrong shape, dtype, memory space, count or a strided view is a
ValueError on the host, never a launch."""
import types

import numpy as np
import pytest
import torch

from paper_1312_1638_b300 import fr


def _stub(precision):
    s = fr.Solver.__new__(fr.Solver)             # no context: the checks are host logic
    s.mesh = types.SimpleNamespace(blocks=[None, None])
    s.precision, s.device = precision, 0
    s._shapes = [(8, 4, 128), (6, 4, 256)]
    return s


def _host(s, dt):
    return [np.zeros(sh, dt) for sh in s._shapes]


@pytest.mark.parametrize("precision,dt", [(fr.FP64, np.float64), (fr.FP32, np.float32), (fr.TF32X3, np.float32)])
def test_matching_host_buffers_pass(precision, dt):
    s = _stub(precision)
    bufs = _host(s, dt)
    arr = s._bufs(bufs, host=True)
    assert [arr[i] for i in range(2)] == [b.ctypes.data for b in bufs]
    tb = [torch.zeros(sh, dtype=torch.float64 if dt == np.float64 else torch.float32) for sh in s._shapes]
    arr = s._bufs(tb, host=True)
    assert [arr[i] for i in range(2)] == [t.data_ptr() for t in tb]


def test_raw_addresses_pass_unchecked():
    s = _stub(fr.FP64)
    arr = s._bufs([4096, 8192])
    assert (arr[0], arr[1]) == (4096, 8192)


@pytest.mark.parametrize("bad", ["dtype", "shape", "count", "strided", "space"])
def test_mismatched_buffers_are_rejected(bad):
    s = _stub(fr.FP64)
    bufs = _host(s, np.float64)
    host = True
    if bad == "dtype":
        bufs[1] = bufs[1].astype(np.float32)           # an FP32 state handed to an FP64 context
    elif bad == "shape":
        bufs[0] = np.zeros((8, 4, 100))
    elif bad == "count":
        bufs = bufs[:1]
    elif bad == "strided":
        bufs[0] = np.zeros((8, 4, 256))[:, :, ::2]
    else:
        host = False                                   # host memory for a device entry point
    with pytest.raises(ValueError):
        s._bufs(bufs, host=host)
