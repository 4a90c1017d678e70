"""Error budget of storing the metric terms in the compute precision.

The library computes every geometric term in FP64 on the host (adj(J),
1/J, |J n|, n; Sec. 2, reading 5) and hands the single-precision kernels
their FP32 roundings, while the conservation sums use FP64 w J.  This CPU
test measures, with the oracle alone, what that rounding costs: the oracle's
RHS with only its metric terms rounded to FP32, against the exact one, in the
perturbation form the kernels run (R is linear in the fluxes, so the part
due to the constant flux of the reference state at rest, which the kernels
never multiply by the metric terms, is the rest state's own residual and is
removed).  On a curved mixed mesh with walls and on jittered hexahedra the
rounding moves R by at most a few 1e-8 of the terms' magnitude S: a small
fraction of the FP32 path's own bound (2e-6 S) and of its measured error
(2e-7 .. 1e-6 S)."""
import numpy as np
import pytest

from fr_inputs import periodic_box, annulus_mixed, fields
from oracle.system import FRSystem

P_INF = 1.0 / (1.4 * 0.2 ** 2)
CASES = {
    "annulus_curved_walls_p3": (
        lambda: annulus_mixed(ntheta=24, nr_quad=3, nr_tri=3, r0=0.5, r1=4.0, jitter=0.05, seed=7), 3,
        dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1, bc_rho=1.0, bc_v=(1.0, 0.0, 0.0),
             bc_p=P_INF, outflow_p=P_INF, wall_cpTw=1.4 / 0.4 * P_INF),
        lambda X: fields.smooth_random(X, seed=3, amp=0.1, vel0=(1.0, 0.0), p0=P_INF)),
    "hex_jittered_tgv_m01_p3": (
        lambda: periodic_box("hex", 4, 0.0, 2 * np.pi, jitter=0.15, seed=2), 3,
        dict(gamma=1.4, mu=0.02, prandtl=0.72, ldg_beta=0.5, ldg_tau=0.1),
        lambda X: fields.taylor_green(X, M=0.1)),
}


def _r32(a):
    return a.astype(np.float32).astype(np.float64)


def _round_metric_terms(o):
    for g in o.geo:
        g["adj"] = _r32(g["adj"])
        g["det"] = 1.0 / _r32(1.0 / g["det"])          # the kernels store 1/J
    for k in ("nrm", "magL", "magR"):
        o.pairs[k] = _r32(o.pairs[k])
    for k in ("nrm", "mag"):
        o.bpairs[k] = _r32(o.bpairs[k])


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_metric_terms_cost_a_small_fraction_of_the_fp32_bound(name):
    mk, p, prm, fn = CASES[name]
    m = mk()
    o = FRSystem(m, p, "ns", **prm)
    U = [_r32(fn(o.solution_coords(b)).transpose(1, 0, 2).copy()) for b in range(len(o.eles))]
    rho = np.concatenate([u[:, 0].ravel() for u in U])
    pr = np.concatenate([(0.4 * (u[:, -1] - 0.5 * (u[:, 1:-1] ** 2).sum(1) / u[:, 0])).ravel() for u in U])
    rest = [fields.uniform(o.solution_coords(b), rho.mean(), (0.0,) * m.ndims, pr.mean(), 1.4)
            .transpose(1, 0, 2).copy() for b in range(len(o.eles))]
    R, S = o.rhs(U, scale=True)
    R0 = o.rhs(rest)
    _round_metric_terms(o)
    Rr, R0r = o.rhs(U), o.rhs(rest)
    for b in range(len(R)):
        E = (Rr[b] - R[b]) - (R0r[b] - R0[b])
        assert np.max(np.abs(E) / S[b]) <= 5e-8            # 1/40 of the FP32 bound 2e-6 S
        # the rounding does act: the metric terms are not exactly representable
        assert np.max(np.abs(Rr[b] - R[b])) > 0.0
