"""The adjoint workload c4 (not in the paper): gradient of the volume-integrated
kinetic energy after 50 RK4 steps (dt = 1e-3, checkpoints every 10) with
respect to the initial state, 3D Euler on a periodic n^3 hex box, p = 4,
Taylor-Green + seeded perturbation, computed by fr_rk4_adjoint in FP32 (or
TF32x3) and checked against FP64 central finite differences along seeded
directions d ~ N(0, I) scaled per variable by its RMS (default_rng(4242)):
|g.d - FD| <= 1e-4 (|FD| + 1e-3 |g| |d|).  The FP64 trajectories run
`batch` directions at a time on disjoint copies of the box.

    python -m tests.adjoint_fd_study [n] [ndir] [euler|ns]   # default: the full c4 (16, 200, euler)
"""

from __future__ import annotations

import sys
import time

import numpy as np

from fr_inputs import Mesh, Block, periodic_box, fields


def kinetic_energy(w, u, nelem):
    u = u[:, :, :nelem]
    m2 = (u[:, 1:4] ** 2).sum(1)
    return float((w * 0.5 * m2 / u[:, 0]).sum())


def kinetic_energy_grad(w, u, nelem):
    g = np.zeros_like(u)
    uu = u[:, :, :nelem]
    m2 = (uu[:, 1:4] ** 2).sum(1)
    g[:, 0, :nelem] = -0.5 * w * m2 / uu[:, 0] ** 2
    for i in range(3):
        g[:, 1 + i, :nelem] = w * uu[:, 1 + i] / uu[:, 0]
    return g


def replicated(box, copies, L):
    """`copies` disjoint copies of a periodic box in one element block, spaced
    10 L apart along x; the box's own translations keep each copy periodic in
    itself, so one RHS evaluates `copies` independent states."""
    nodes = box.blocks[0].nodes
    allnodes = np.concatenate([nodes + np.array([10.0 * L * c, 0.0, 0.0]) for c in range(copies)])
    return Mesh(3, [Block("hex", allnodes)], box.bfaces, box.periodic)


# Navier-Stokes variant: the Taylor-Green constants (mu = 1/1600, Pr = 0.71,
# LDG beta = 1/2, tau = 0.1), single precision in perturbation form about the
# mean state (rho 1, p 1/(gamma M^2), M = 0.1)
NS_PRM = dict(mu=1.0 / 1600.0, prandtl=0.71, ldg_beta=0.5, ldg_tau=0.1)
NS_REF = dict(ref_rho=1.0, ref_p=1.0 / (1.4 * 0.01))


def fd_check(n_box, ndir, prec="fp32", batch=8, nsteps=50, dt=1e-3, every=10, system="euler"):
    """Returns dict(bad=[(k, g.d, FD)], worst relative deviation, directions)."""
    import torch
    from oracle.system import FRSystem
    from paper_1312_1638_b300 import fr
    L = 2 * np.pi
    m = periodic_box("hex", n_box, 0.0, L)
    prm = NS_PRM if system == "ns" else {}
    o = FRSystem(m, 4, system, **prm)
    w = o.quadrature_weights(0)
    U = fields.perturbed_taylor_green(o.solution_coords(0), M=0.1).transpose(1, 0, 2).copy()
    U = U.astype(np.float32).astype(np.float64)
    s1 = fr.Solver(m, 4, system, prec, device=0, **prm, **(NS_REF if system == "ns" else {}))
    ne = m.nelem
    u0 = torch.from_numpy(s1.pack(0, U)).cuda()
    uN = u0.clone()
    s1.rk4([uN], dt, nsteps)
    lam = torch.from_numpy(kinetic_energy_grad(w, uN.cpu().numpy().astype(np.float64), ne)
                           .astype(np.float32)).cuda()
    s1.rk4_adjoint([u0], [lam], dt, nsteps, every)
    g = lam.cpu().numpy().astype(np.float64)[:, :, :ne]
    s1.close()
    rng = np.random.default_rng(4242)
    rms = np.sqrt((U ** 2).mean(axis=(0, 2)))
    dirs = [rng.standard_normal(U.shape) * rms[None, :, None] for _ in range(ndir)]
    s64 = fr.Solver(replicated(m, batch, L), 4, system, "fp64", device=0, **prm)
    bad, worst = [], 0.0
    for k0 in range(0, ndir, batch):
        ds = dirs[k0:k0 + batch]
        eps = [1e-6 * np.sqrt((U ** 2).mean()) / np.sqrt((d ** 2).mean()) for d in ds]
        res = []
        for sign in (1.0, -1.0):
            parts = [U + sign * e * d for e, d in zip(eps, ds)]
            parts += [U] * (batch - len(ds))
            ub = torch.from_numpy(s64.pack(0, np.concatenate(parts, axis=2))).cuda()
            s64.rk4([ub], dt, nsteps)
            uh = ub.cpu().numpy()
            res.append([kinetic_energy(w, uh[:, :, c * ne:(c + 1) * ne], ne) for c in range(len(ds))])
        for c, (d, e) in enumerate(zip(ds, eps)):
            fd = (res[0][c] - res[1][c]) / (2 * e)
            gd = float(np.sum(g * d))
            tol = 1e-4 * (abs(fd) + 1e-3 * np.linalg.norm(g) * np.linalg.norm(d))
            worst = max(worst, abs(gd - fd) / tol * 1e-4)
            if abs(gd - fd) > tol:
                bad.append((k0 + c, gd, fd))
    s64.close()
    return dict(bad=bad, worst=worst, ndir=ndir, n_box=n_box, prec=prec, system=system)


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 16
    nd = int(sys.argv[2]) if len(sys.argv) > 2 else 200
    sysname = sys.argv[3] if len(sys.argv) > 3 else "euler"
    t0 = time.time()
    r = fd_check(n, nd, system=sysname)
    print(f"{sysname} adjoint vs FP64 central FD: {n}^3 hexes, p=4, {nd} directions, FP32 adjoint: "
          f"{len(r['bad'])} outside the bound; largest |g.d - FD| / (|FD| + 1e-3 |g||d|) = {r['worst']:.2e} "
          f"(bound 1e-4); {time.time() - t0:.0f} s")
