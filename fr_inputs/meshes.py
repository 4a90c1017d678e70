"""Seeded synthetic meshes shaped like the workloads of the FR paper.

The paper benchmarks on fully periodic hexahedral boxes (Sec. 6, Sec. 7) and
validates on vortex / Couette / cylinder cases (Sec. 5) whose meshes are not
published; these generators stand in for them.  Nothing here evaluates the FR
method: only node coordinates, boundary tags and periodic shifts.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ETYPES = ("quad", "tri", "hex")


@dataclass
class Block:
    etype: str                 # "quad" | "tri" | "hex"
    nodes: np.ndarray          # float64 [nelem, nnodes, ndims]

    @property
    def nelem(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def nnodes(self) -> int:
        return int(self.nodes.shape[1])


@dataclass
class Mesh:
    ndims: int
    blocks: list
    # [nbfaces, 4] int64 rows (block, element, face, bctype)
    bfaces: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int64))
    # [nperiodic, ndims] translation vectors of the periodic identifications
    periodic: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))

    @property
    def nelem(self) -> int:
        return sum(b.nelem for b in self.blocks)


def _periodic_lattice(n, lo, hi, ndims, jitter, rng):
    """Node lattice of an n^d periodic box; jitter is periodic-consistent."""
    h = (hi - lo) / n
    axes = [lo + h * np.arange(n + 1) for _ in range(ndims)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)  # [n+1]^d x d
    if jitter > 0.0:
        shape = (n,) * ndims + (ndims,)
        d = rng.uniform(-jitter * h, jitter * h, size=shape)
        # node index n is the periodic image of node index 0
        d = np.pad(d, [(0, 1)] * ndims + [(0, 0)], mode="wrap")
        grid = grid + d
    return grid, h


def periodic_box(etype: str, n: int, lo: float = 0.0, hi: float = 2 * np.pi,
                 jitter: float = 0.0, seed: int = 0, shuffle: bool = False) -> Mesh:
    """Fully periodic [lo, hi]^d box of n^d quads (2D) or hexes (3D).

    ``jitter`` moves every lattice node by U(-jitter*h, jitter*h) per axis,
    consistently across the periodic identification.  ``shuffle`` permutes the
    element numbering with the same seed (unstructured-looking indirection).
    """
    if etype not in ("quad", "hex"):
        raise ValueError("periodic_box builds quads or hexes")
    ndims = 2 if etype == "quad" else 3
    rng = np.random.default_rng(seed)
    grid, h = _periodic_lattice(n, lo, hi, ndims, jitter, rng)
    idx = np.arange(n)
    if ndims == 2:
        i, j = np.meshgrid(idx, idx, indexing="ij")
        i, j = i.ravel(order="F"), j.ravel(order="F")   # i fastest
        corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
        nodes = np.stack([grid[i + a, j + b] for a, b in corners], axis=1)
    else:
        i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
        i, j, k = (v.ravel(order="F") for v in (i, j, k))
        corners = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
        nodes = np.stack([grid[i + a, j + b, k + c] for a, b, c in corners], axis=1)
    if shuffle:
        nodes = nodes[rng.permutation(nodes.shape[0])]
    L = hi - lo
    periodic = L * np.eye(ndims)
    return Mesh(ndims, [Block(etype, np.ascontiguousarray(nodes))],
                np.zeros((0, 4), np.int64), periodic)


def _tri_edges():
    return [(0, 1), (1, 2), (2, 0)]


def _quad_edges():
    # tensor corner order: 0=(-1,-1) 1=(1,-1) 2=(-1,1) 3=(1,1)
    return [(0, 1), (1, 3), (3, 2), (2, 0)]


def annulus_mixed(ntheta: int = 500, nr_quad: int = 200, nr_tri: int = 60,
                  r0: float = 0.5, r1: float = 20.0, jitter: float = 0.05,
                  seed: int = 1638, shuffle: bool = True) -> Mesh:
    """Annulus r in [r0, r1] meshed with quads (inner rings) and triangles.

    Radial spacing is geometric over nr_quad + nr_tri rings.  The inner
    ``nr_quad`` rings are 9-node quads (xi radial, eta angular); the wall ring's
    inner edge carries its mid-side node on the circle r = r0, every other edge
    is straight.  The outer rings are cells split into two 3-node triangles on
    a seeded random diagonal.  Interior nodes are jittered by
    U(-jitter, jitter) * local spacing.  Faces on r0 are no-slip walls
    (bctype 2); faces on r1 are free-stream (bctype 0).
    """
    rng = np.random.default_rng(seed)
    nr = nr_quad + nr_tri
    ratio = (r1 / r0) ** (1.0 / nr)
    radii = r0 * ratio ** np.arange(nr + 1)
    radii[-1] = r1
    theta = 2 * np.pi * np.arange(ntheta) / ntheta
    rr, tt = np.meshgrid(radii, theta, indexing="ij")        # [nr+1, ntheta]
    dr = np.diff(radii)
    # local spacing per ring of nodes (min of adjacent radial steps, arc step)
    hr = np.minimum(np.r_[dr[0], dr], np.r_[dr, dr[-1]])
    hloc = np.minimum(hr, radii * 2 * np.pi / ntheta)[:, None]
    jr = rng.uniform(-jitter, jitter, size=rr.shape) * hloc
    jt = rng.uniform(-jitter, jitter, size=rr.shape) * hloc
    jr[0], jt[0], jr[-1], jt[-1] = 0.0, 0.0, 0.0, 0.0       # boundary rings exact
    x = rr * np.cos(tt) - jt * np.sin(tt) + jr * np.cos(tt)
    y = rr * np.sin(tt) + jt * np.cos(tt) + jr * np.sin(tt)
    P = np.stack([x, y], axis=-1)                             # [nr+1, ntheta, 2]

    def node(i, j):
        return P[i, j % ntheta]

    quads, qwall = [], []
    for i in range(nr_quad):
        for j in range(ntheta):
            c00, c10 = node(i, j), node(i + 1, j)
            c01, c11 = node(i, j + 1), node(i + 1, j + 1)
            # xi radial (from ring i to i+1), eta angular (j to j+1)
            m_eta_lo = 0.5 * (c00 + c10)           # edge eta=-1
            m_eta_hi = 0.5 * (c01 + c11)           # edge eta=+1
            m_xi_hi = 0.5 * (c10 + c11)            # edge xi=+1
            if i == 0:
                tm = 0.5 * (theta[j] + (theta[(j + 1) % ntheta] if j + 1 < ntheta else 2 * np.pi))
                m_xi_lo = r0 * np.array([np.cos(tm), np.sin(tm)])   # curved wall edge
            else:
                m_xi_lo = 0.5 * (c00 + c01)
            ctr = 0.5 * (m_xi_lo + m_xi_hi)
            # 9-node tensor order, xi fastest: rows eta=-1,0,1
            quads.append([c00, m_eta_lo, c10,
                          m_xi_lo, ctr, m_xi_hi,
                          c01, m_eta_hi, c11])
            qwall.append(i == 0)
    tris, tout = [], []
    for i in range(nr_quad, nr):
        for j in range(ntheta):
            A, B = node(i, j), node(i + 1, j)
            C, D = node(i + 1, j + 1), node(i, j + 1)
            last = i == nr - 1
            if rng.integers(2) == 0:        # diagonal A-C
                tris.append([A, B, C]); tout.append(1 if last else -1)   # B-C is edge v1-v2
                tris.append([A, C, D]); tout.append(-1)
            else:                           # diagonal B-D
                tris.append([A, B, D]); tout.append(-1)
                tris.append([B, C, D]); tout.append(0 if last else -1)   # B-C is edge v0-v1
    qn = np.asarray(quads, np.float64)
    tn = np.asarray(tris, np.float64)
    qwall = np.asarray(qwall)
    tout = np.asarray(tout)
    qperm = rng.permutation(len(qn)) if shuffle else np.arange(len(qn))
    tperm = rng.permutation(len(tn)) if shuffle else np.arange(len(tn))
    qn, qwall = qn[qperm], qwall[qperm]
    tn, tout = tn[tperm], tout[tperm]
    bf = []
    for e in np.nonzero(qwall)[0]:
        bf.append((0, e, 3, 2))             # xi=-1 face lies on r0: wall
    for e in np.nonzero(tout >= 0)[0]:
        bf.append((1, e, int(tout[e]), 0))  # outer circle: free-stream
    bfaces = np.asarray(bf, np.int64).reshape(-1, 4)
    return Mesh(2, [Block("quad", qn), Block("tri", tn)], bfaces, np.zeros((0, 2)))


def single_element(etype: str, nodes: np.ndarray) -> Mesh:
    """One element with every face tagged free-stream (tiny edge cases)."""
    ndims = 3 if etype == "hex" else 2
    nf = {"quad": 4, "tri": 3, "hex": 6}[etype]
    bfaces = np.asarray([(0, 0, f, 0) for f in range(nf)], np.int64)
    return Mesh(ndims, [Block(etype, np.asarray(nodes, np.float64)[None])], bfaces,
                np.zeros((0, ndims)))


def channel_mixed(nx: int, ny: int, lx: float = 1.0, h: float = 1.0, tri_rows: int = -1,
                  jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Channel [0, lx] x [0, h], periodic in x, walls at y = 0 and y = h.

    nx x ny cells; the lower rows are 4-node quads and the upper ``tri_rows``
    rows (default: half of them) are cells split into two 3-node triangles on a
    seeded random diagonal, a mixed mesh like the paper's Couette meshes
    (Sec. 5.2; those meshes are not published).  Interior nodes move by
    U(-jitter, jitter) times the cell size (periodic-consistently in x; wall
    rows only along x).  Bottom faces are no-slip isothermal walls (bctype 2),
    top faces the second wall type (bctype 3, the moving plate).
    """
    rng = np.random.default_rng(seed)
    if tri_rows < 0:
        tri_rows = ny // 2
    dx, dy = lx / nx, h / ny
    X, Y = np.meshgrid(dx * np.arange(nx + 1), dy * np.arange(ny + 1), indexing="ij")
    jx = rng.uniform(-jitter, jitter, size=(nx, ny + 1)) * dx
    jy = rng.uniform(-jitter, jitter, size=(nx, ny + 1)) * dy
    jy[:, 0] = jy[:, -1] = 0.0
    jx = np.concatenate([jx, jx[:1]], axis=0)                 # node nx is the image of node 0
    jy = np.concatenate([jy, jy[:1]], axis=0)
    P = np.stack([X + jx, Y + jy], axis=-1)                   # [nx+1, ny+1, 2]
    P[nx, :, 0] = P[0, :, 0] + lx
    quads, tris, bq, bt = [], [], [], []
    for j in range(ny):
        for i in range(nx):
            c00, c10, c01, c11 = P[i, j], P[i + 1, j], P[i, j + 1], P[i + 1, j + 1]
            if j < ny - tri_rows:
                if j == 0:
                    bq.append((len(quads), 0, 2))             # eta = -1 face on y = 0
                if j == ny - 1:
                    bq.append((len(quads), 2, 3))             # eta = +1 face on y = h
                quads.append([c00, c10, c01, c11])
            else:
                if rng.random() < 0.5:
                    t1, t2 = [c00, c10, c11], [c00, c11, c01]
                else:
                    t1, t2 = [c00, c10, c01], [c10, c11, c01]
                if j == 0:
                    bt.append((len(tris), 0, 2))              # edge v0 v1 of t1 on y = 0
                tris.append(t1)
                if j == ny - 1:
                    bt.append((len(tris), 1, 3))              # edge v1 v2 of t2 on y = h
                tris.append(t2)
    blocks, bf = [], []
    if quads:
        blocks.append(Block("quad", np.asarray(quads, np.float64)))
        bf += [(0, e, f, t) for e, f, t in bq]
    if tris:
        blocks.append(Block("tri", np.asarray(tris, np.float64)))
        bf += [(len(blocks) - 1, e, f, t) for e, f, t in bt]
    return Mesh(2, blocks, np.asarray(bf, np.int64).reshape(-1, 4), np.array([[lx, 0.0]]))
