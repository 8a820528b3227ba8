"""Plain FP64 CPU oracle of the explicit divergence-free DG method (Fu, arXiv:1808.04669).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only the tests, the smoke check and the benchmark's CPU-baseline
leg do. It shares no code with the CUDA path; both only consume the seeded
inputs of ``synth``.

It computes everything by its plain definition, in float64, with its own
choices wherever a choice does not change the result:

* a monomial basis (centred, scaled by the element diameter) instead of an
  orthonormal one, with the mass matrix assembled by quadrature;
* a collapsed Gauss-Legendre x Gauss-Legendre volume rule with extra points;
* the hybrid-mixed system of Sec. 2.4, eq. (12), assembled globally, condensed
  element by element and solved by a sparse direct factorisation computed once
  (the paper's own solver, Sec. 4), plus independent routes for checking:
  the uncondensed saddle system, an explicit SVD null-space basis of the
  divergence-free space, and the locally divergence-free variant eq. (13).

The facet rule is the one place both sides must agree: the upwind flux of
eq. (7) switches with the sign of u.n inside a facet, so it is evaluated at the
q = ceil((3k+1)/2) Gauss-Legendre points of each facet on both sides.

Parity pins (see tests/test_oracle_*.py): Taylor-Green closed forms and their
convergence orders, the energy identity of Sec. 2.2, symmetry of the SIPG form
eq. (18), zero divergence and normal jump, agreement of the four solve routes,
dimension counts of the divergence-free space and of Table 3, and the third
order of the SSP-RK3 scheme eq. (8).

``dg3`` is the same method on closed tetrahedral meshes (d = 3), pinned in
tests/test_oracle3_pins.py.
"""
from .mesh import Topology
from .dg import Discretization
from .dg3 import Discretization3, Topology3

__all__ = ["Topology", "Discretization", "Topology3", "Discretization3"]
