"""B300 (sm_103a) Flux Reconstruction right-hand side behind a C ABI.

``fr.Solver`` wraps ``libfr.so`` (include/fr.h); ``build.build()`` compiles it
in-tree with nvcc.  The library evaluates R(U) of the FR method (arXiv
1312.1638, Sec. 2, App. A) for Euler / Navier-Stokes on quads, triangles and
hexahedra, and advances it with classical RK4.
"""

from .fr import Solver, FRError, load  # noqa: F401
