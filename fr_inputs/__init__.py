"""Seeded synthetic inputs for the FR right-hand side: meshes and initial fields.

This package is the one piece shared by the CUDA library's tests/benchmark and
the CPU oracle.  It holds no arithmetic of the FR method itself (no point sets,
bases, operators, metric terms, fluxes or interface pairing): only element
node coordinates, boundary tags, periodic translation vectors and analytic
initial fields evaluated at caller-supplied physical coordinates.

Element node orderings (the input format both sides read):

* ``quad`` 4 nodes: tensor product of {-1, 1}^2, xi fastest; 9 nodes: tensor
  product of {-1, 0, 1}^2, xi fastest.
* ``hex`` 8 nodes: tensor product of {-1, 1}^3, xi fastest then eta then zeta;
  27 nodes: tensor product of {-1, 0, 1}^3.
* ``tri`` 3 nodes: (-1,-1), (1,-1), (-1,1); 6 nodes: those three then the
  mid-points of edges 0-1, 1-2, 2-0.

Face numbering (used by boundary tags):

* quad: 0 eta=-1, 1 xi=+1, 2 eta=+1, 3 xi=-1
* tri: 0 edge v0-v1 (eta=-1), 1 edge v1-v2 (xi+eta=0), 2 edge v2-v0 (xi=-1)
* hex: 0 zeta=-1, 1 eta=-1, 2 xi=+1, 3 eta=+1, 4 xi=-1, 5 zeta=+1

Boundary types: 0 free-stream (supersonic inflow) ghost, 1 subsonic outflow,
2 no-slip isothermal wall.
"""

from .meshes import Mesh, Block, periodic_box, annulus_mixed  # noqa: F401
from . import fields  # noqa: F401
