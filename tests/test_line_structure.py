"""The line structure of the tensor-element operators, on the oracle's matrices.

The structured kernels rely on a property of the FR operators on
quadrilaterals and hexahedra with tensor Gauss-Legendre solution points and
Gauss-Legendre face points (Sec. 2, App. A): along a line of solution points
in direction i, the corrected gradient [M6 | M4 - M6 M0] (Eq. tquptsm) and
the divergence [M3 | M1 - M3 M2] (Eq. tdivflux) involve only the line's p+1
points and the two flux points that end it, with ONE (p+1) x (p+3) matrix for
every line and every direction; the interpolation M0 at a line's end points
involves only the line's points.  The library checks this on its own
operators at set-up; here it is checked on the oracle's, which are built
independently (mass-matrix lift, its own point ordering), with the lines
found from the points' coordinates alone.  Triangles have no such form.
"""
import numpy as np
import pytest

from oracle.elements import RefElement


def _lines(el):
    """(direction, solution points ordered along it, [flux point at -1, at +1])
    for every line of a tensor element, found from coordinates."""
    d, tol = el.ndims, 1e-12
    out = []
    for i in range(d):
        other = [j for j in range(d) if j != i]
        keys = {}
        for s, x in enumerate(el.upts):
            keys.setdefault(tuple(np.round(x[other], 12)), []).append(s)
        for key, pts in keys.items():
            pts = sorted(pts, key=lambda s: el.upts[s, i])
            ends = [None, None]
            for f, x in enumerate(el.fpts):
                if np.all(np.abs(x[other] - np.array(key)) < tol):
                    if abs(x[i] + 1) < tol:
                        ends[0] = f
                    elif abs(x[i] - 1) < tol:
                        ends[1] = f
            assert None not in ends, (i, key)
            out.append((i, pts, ends))
    return out


@pytest.mark.parametrize("correction", ["dg", "sd", "hu"])
@pytest.mark.parametrize("etype,p", [("quad", 1), ("quad", 2), ("quad", 4), ("hex", 1), ("hex", 2), ("hex", 4)])
def test_gradient_and_divergence_act_along_lines(etype, p, correction):
    el = RefElement(etype, p, correction)
    nu, nf, d, n = el.nupts, el.nfpts, el.ndims, p + 1
    lines = _lines(el)
    assert len(lines) == d * n ** (d - 1)
    M46 = el.M4 - el.M6 @ el.M0
    M132 = el.M1 - el.M3 @ el.M2
    G = np.hstack([el.M6, M46])                     # rows (i, s), columns [flux | solution]
    Dv = np.hstack([el.M3, M132])                   # rows s, columns [flux | (i, solution)]
    # the line matrices, from the first line of direction 0
    i0, pts0, ends0 = lines[0]
    A = np.array([[M46[i0 * nu + s, k] for k in pts0] + [el.M6[i0 * nu + s, f] for f in ends0] for s in pts0])
    B = np.array([[M132[s, i0 * nu + k] for k in pts0] + [el.M3[s, f] for f in ends0] for s in pts0])
    assert A.shape == B.shape == (n, n + 2)

    # gradient: every row (i, s) is A's row for s's position on its line
    worst = 0.0
    for i, pts, ends in lines:
        for q, s in enumerate(pts):
            rec = np.zeros(nf + nu)
            rec[[nf + k for k in pts]] = A[q, :n]
            rec[ends] = A[q, n:]
            row = G[i * nu + s]
            worst = max(worst, np.max(np.abs(rec - row)) / np.max(np.abs(row)))
    assert worst < 1e-10, worst

    # divergence: every row s is the sum of B's rows over the d lines through s
    rec = np.zeros((nu, nf + d * nu))
    for i, pts, ends in lines:
        for q, s in enumerate(pts):
            rec[s, [nf + i * nu + k for k in pts]] += B[q, :n]
            rec[s, ends] += B[q, n:]
    err = np.max(np.abs(rec - Dv), axis=1) / np.max(np.abs(Dv), axis=1)
    assert np.max(err) < 1e-10, np.max(err)

    # interpolation: a line's end flux points from the line's points only, with
    # the same two rows on every line; every flux point ends exactly one line
    I0 = np.array([[el.M0[f, k] for k in pts0] for f in ends0])
    ends_all = []
    for i, pts, ends in lines:
        for e, f in enumerate(ends):
            rec = np.zeros(nu)
            rec[pts] = I0[e]
            assert np.max(np.abs(rec - el.M0[f])) < 1e-10 * np.max(np.abs(el.M0[f]))
            ends_all.append(f)
    assert sorted(ends_all) == list(range(nf))


@pytest.mark.parametrize("p", [2, 4])
def test_triangle_operators_are_dense(p):
    """No line form on triangles: every row of the corrected-gradient operator
    [M6 | M4 - M6 M0] has more than the p+3 nonzeros of a line (8 to 12 of 15
    at p = 2, 22 to 25 of 30 at p = 4), so the structured kernels do not
    apply and triangles take the dense products."""
    el = RefElement("tri", p)
    G = np.hstack([el.M6, el.M4 - el.M6 @ el.M0])
    nz = np.sum(np.abs(G) > 1e-12 * np.max(np.abs(G), axis=1, keepdims=True), axis=1)
    assert np.min(nz) > p + 3, nz.min()
