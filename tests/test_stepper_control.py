"""Host logic of the adaptive DOPRI5 driver (fr.adaptive_dopri5), run on CPU
with the oracle's DOPRI5 step as the stepper: rejected steps leave no trace,
accepted steps reproduce a fixed-step replay, and the global error follows
the tolerance."""

import numpy as np
import pytest

from oracle import steppers as S
from paper_1312_1638_b300 import fr


class _Fake:
    """u' = -u^2 on a few entries, stepped by the oracle's DOPRI5."""

    def __init__(self, u0, atol, rtol):
        self.u = [u0.copy()]
        self.saved = None
        self.atol, self.rtol = atol, rtol
        self.calls = 0

    @staticmethod
    def rhs(U):
        return [-u * u for u in U]

    def step(self, dt):
        self.calls += 1
        U1, E, _ = S.dopri5_step(self.rhs, self.u, dt)
        err = S.error_norm(self.u, U1, E, self.atol, self.rtol)
        self.u = U1
        return err

    def save(self):
        self.saved = [x.copy() for x in self.u]

    def restore(self):
        self.u = [x.copy() for x in self.saved]


@pytest.mark.parametrize("tol", [1e-4, 1e-7])
def test_adaptive_dopri5_tracks_tolerance_and_replays(tol):
    u0 = np.array([0.5, 1.0, 4.0]).reshape(3, 1, 1)
    f = _Fake(u0, tol, tol)
    rec = fr.adaptive_dopri5(f.step, f.save, f.restore, t_end=3.0, dt0=1.0)
    assert rec["t"] == pytest.approx(3.0, rel=1e-12)
    assert rec["rejected"] >= 1                               # dt0 = 1 is far too large at u0 = 4
    assert f.calls == len(rec["accepted"]) + rec["rejected"]
    assert sum(rec["accepted"]) == pytest.approx(3.0, rel=1e-12)
    exact = u0 / (1 + 3.0 * u0)
    err = np.abs(f.u[0] - exact).max()
    assert err < 50 * tol                                     # global error follows the local tolerance
    # replaying the accepted steps with fixed DOPRI5 steps gives the same state bit for bit
    U = [u0.copy()]
    for h in rec["accepted"]:
        U, _, _ = S.dopri5_step(_Fake.rhs, U, h)
    assert np.array_equal(U[0], f.u[0])


def test_adaptive_dopri5_gives_up_after_max_steps():
    f = _Fake(np.ones((2, 1, 1)), 1e-12, 1e-12)
    with pytest.raises(RuntimeError):
        fr.adaptive_dopri5(f.step, f.save, f.restore, t_end=1.0, dt0=1e-3, max_steps=5)
