"""Element mappings M_en and their metric terms (Sec. 2).

The mapping of each element is the Lagrange shape-function interpolant of its
nodes (node orderings as in ``fr_inputs``).  The paper does not say how the
metric terms are evaluated; they are taken analytically from this mapping at
every point, in FP64:

* J_ij = d x_i / d xi_j, det J, and adj(J) = det(J) J^{-1} (so that
  J J^{-1} = adj(J) in the transformed flux of Sec. 2);
* at flux points the transformed normal magnitude J^(f) n^(f) =
  |adj(J)^T n_ref| and the physical unit normal adj(J)^T n_ref / |...|
  (n^(f) = J^{-T} n_ref, Sec. 2).
"""

from __future__ import annotations

import numpy as np

from .polys import lagrange


def shape_functions(etype: str, nnodes: int, x):
    """Values N[k, npts] and derivatives dN[d, k, npts] at reference points x."""
    x = np.asarray(x, np.float64)
    if etype in ("quad", "hex"):
        nd = 2 if etype == "quad" else 3
        m = round(nnodes ** (1.0 / nd))
        if m ** nd != nnodes or m not in (2, 3):
            raise ValueError(f"{etype} with {nnodes} nodes")
        nodes1d = np.linspace(-1.0, 1.0, m)
        L = [lagrange(nodes1d, x[d]) for d in range(nd)]
        N, dN = [], []
        for idx in np.ndindex(*(m,) * nd):
            idx = idx[::-1]                       # tensor order, xi fastest
            v = np.ones(x.shape[1:])
            for d in range(nd):
                v = v * L[d][0][idx[d]]
            g = []
            for dd in range(nd):
                gd = np.ones(x.shape[1:])
                for d in range(nd):
                    gd = gd * (L[d][1][idx[d]] if d == dd else L[d][0][idx[d]])
                g.append(gd)
            N.append(v); dN.append(g)
        return np.asarray(N), np.asarray(dN).transpose(1, 0, *range(2, x.ndim + 1))
    if etype == "tri":
        r, s = x[0], x[1]
        l0, l1, l2 = -(r + s) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0
        dl = np.array([[-0.5, 0.5, 0.0], [-0.5, 0.0, 0.5]])   # [d, lambda]
        lam = [l0, l1, l2]
        if nnodes == 3:
            N = np.stack(lam)
            dN = np.stack([np.stack([np.full_like(r, dl[d, k]) for k in range(3)]) for d in range(2)])
            return N, dN
        if nnodes == 6:
            pairs = [(0, 1), (1, 2), (2, 0)]
            N = [lam[k] * (2.0 * lam[k] - 1.0) for k in range(3)]
            N += [4.0 * lam[a] * lam[b] for a, b in pairs]
            dN = []
            for d in range(2):
                g = [dl[d, k] * (4.0 * lam[k] - 1.0) for k in range(3)]
                g += [4.0 * (dl[d, a] * lam[b] + lam[a] * dl[d, b]) for a, b in pairs]
                dN.append(g)
            return np.stack(N), np.asarray(dN)
        raise ValueError(f"tri with {nnodes} nodes")
    raise ValueError(etype)


def _adjugate(J):
    """adj(J) for J of shape [..., d, d] (d = 2 or 3)."""
    d = J.shape[-1]
    if d == 2:
        A = np.empty_like(J)
        A[..., 0, 0] = J[..., 1, 1]
        A[..., 0, 1] = -J[..., 0, 1]
        A[..., 1, 0] = -J[..., 1, 0]
        A[..., 1, 1] = J[..., 0, 0]
        return A
    A = np.empty_like(J)
    for i in range(3):
        for j in range(3):
            # adj(J)_{ij} = cofactor C_{ji}
            r = [k for k in range(3) if k != j]
            c = [k for k in range(3) if k != i]
            minor = J[..., r[0], c[0]] * J[..., r[1], c[1]] - J[..., r[0], c[1]] * J[..., r[1], c[0]]
            A[..., i, j] = (-1) ** (i + j) * minor
    return A


def map_points(etype, nodes, x):
    """Physical coordinates and Jacobians at reference points x.

    nodes: [nelem, nnodes, d]; returns X [nelem, npts, d], J [nelem, npts, d, d]
    with J[..., i, j] = d x_i / d xi_j.
    """
    N, dN = shape_functions(etype, nodes.shape[1], x)
    X = np.einsum("kp,nki->npi", N, nodes)
    J = np.einsum("jkp,nki->npij", dN, nodes)
    return X, J


def solution_point_metrics(etype, nodes, upts):
    """det J, adj(J) and physical coordinates at the solution points."""
    X, J = map_points(etype, nodes, upts.T)
    det = np.linalg.det(J)
    return X, det, _adjugate(J)


def flux_point_metrics(etype, nodes, fpts, fnorm):
    """Physical coords, J^(f) n^(f) and unit physical normals at flux points."""
    X, J = map_points(etype, nodes, fpts.T)
    adj = _adjugate(J)
    # adj(J)^T n_ref for every point
    v = np.einsum("npji,pj->npi", adj, fnorm)
    mag = np.linalg.norm(v, axis=-1)
    return X, mag, v / mag[..., None], np.linalg.det(J)
