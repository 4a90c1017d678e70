"""Pins of the SD and HU correction functions (the VCJH family named in
Sec. 5.1) in the oracle: closed forms and defining properties in 1D, the DG
member against the independent exact-mass lift, and the system-level
invariants (face-weight, freestream, conservation, order of accuracy)."""

from math import factorial

import numpy as np
import pytest

from fr_inputs import periodic_box, fields
from oracle.elements import RefElement, vcjh_right, VCJH_ETA
from oracle.polys import gauss_legendre, legendre
from oracle.system import FRSystem
from tests.libutil import oracle_state


@pytest.mark.parametrize("p", range(1, 7))
def test_eta_from_published_c(p):
    ap = factorial(2 * p) / (2 ** p * factorial(p) ** 2)
    k = (ap * factorial(p)) ** 2
    c_sd = 2 * p / ((2 * p + 1) * (p + 1) * k)
    c_hu = 2 * (p + 1) / ((2 * p + 1) * p * k)
    eta = lambda c: c * (2 * p + 1) * k / 2
    assert eta(c_sd) == pytest.approx(VCJH_ETA["sd"](p), rel=1e-12)
    assert eta(c_hu) == pytest.approx(VCJH_ETA["hu"](p), rel=1e-12)
    assert VCJH_ETA["dg"](p) == 0.0


@pytest.mark.parametrize("p", range(1, 7))
def test_sd_is_gauss_point_correction(p):
    # SD: g_R = (1 + x) P_p(x) / 2, zero at x = -1 and at the p Gauss points
    x = np.linspace(-1, 1, 41)
    g, _ = vcjh_right(p, "sd", x)
    lp, _ = legendre(p, x)
    assert np.allclose(g, 0.5 * (1 + x) * lp, atol=1e-14)
    xg, _ = gauss_legendre(p)
    assert np.allclose(vcjh_right(p, "sd", xg)[0], 0.0, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 7))
@pytest.mark.parametrize("corr", ["dg", "sd", "hu"])
def test_vcjh_endpoint_values_and_orthogonality(p, corr):
    g, _ = vcjh_right(p, corr, np.array([-1.0, 1.0]))
    assert np.allclose(g, [0.0, 1.0], atol=1e-14)
    xq, wq = gauss_legendre(p + 3)
    gq, _ = vcjh_right(p, corr, xq)
    for k in range(p - 1):                       # orthogonal to P_{p-2}
        assert abs(np.sum(wq * gq * legendre(k, xq)[0])) < 1e-14


@pytest.mark.parametrize("p", range(1, 7))
def test_hu_has_zero_slope_at_the_far_end(p):
    # HU is the member of the family with g_R'(-1) = 0 (no correction slope at the opposite end)
    _, dg = vcjh_right(p, "hu", np.array([-1.0]))
    assert abs(dg[0]) < 1e-13
    _, dsd = vcjh_right(p, "sd", np.array([-1.0]))
    assert abs(dsd[0]) > 1e-3                    # ... which SD does not have


@pytest.mark.parametrize("etype", ["quad", "hex"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_vcjh_dg_member_equals_exact_mass_lift(etype, p):
    el = RefElement(etype, p)                    # DG by the exact-mass lift
    assert np.allclose(el._vcjh_M3(), el.M3, atol=1e-12)


@pytest.mark.parametrize("corr", ["sd", "hu"])
@pytest.mark.parametrize("etype", ["quad", "hex"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_correction_integrates_to_face_weight(etype, p, corr):
    el = RefElement(etype, p, corr)
    _, w1 = gauss_legendre(p + 1)
    w = w1
    for _ in range(el.ndims - 1):
        w = np.outer(w1, w).ravel()
    integral = w @ el.M3                         # exact: degree p per direction
    fw = np.empty(el.nfpts)
    for f, ids in enumerate(el.face_fpts):
        fw[ids] = w1 if el.ndims == 2 else np.outer(w1, w1).ravel()
    assert np.allclose(integral, fw, atol=1e-13)
    assert not np.allclose(el.M3, RefElement(etype, p).M3)


def test_triangle_rejects_sd_hu():
    with pytest.raises(ValueError):
        RefElement("tri", 2, "sd")


@pytest.mark.parametrize("corr", ["sd", "hu"])
@pytest.mark.parametrize("system", ["euler", "ns"])
def test_freestream_and_conservation(corr, system):
    m = periodic_box("hex", 2, 0.0, 1.0, jitter=0.1, seed=3)
    prm = dict(mu=0.05) if system == "ns" else {}
    s = FRSystem(m, 2, system, correction=corr, **prm)
    U = oracle_state(s, lambda X: fields.uniform(X, 1.2, (0.3, -0.2, 0.1), 1.0, 1.4))
    R = s.rhs(U)
    assert np.abs(R[0]).max() < 1e-12
    U = oracle_state(s, lambda X: fields.smooth_random(X, period=1.0, seed=4, amp=0.2))
    R = s.rhs(U)
    tot = np.einsum("un,uvn->v", s.quadrature_weights(0), R[0])
    scale = np.einsum("un,uvn->v", s.quadrature_weights(0), np.abs(R[0]))
    assert np.all(np.abs(tot) < 1e-12 * scale.max())


@pytest.mark.slow
@pytest.mark.parametrize("corr", ["sd", "hu"])
@pytest.mark.parametrize("p", [2, 3])
def test_vortex_order_p_plus_one(corr, p):
    # same meshes and bound as the DG test of the isentropic vortex
    from tests.test_oracle_system import _vortex_error
    ns = [14, 20, 28]
    errs = [_vortex_error(n, p, correction=corr) for n in ns]
    slope = np.polyfit(np.log(20.0 / np.array(ns)), np.log(errs), 1)[0]
    assert slope > p + 1 - 0.4, (errs, slope)
