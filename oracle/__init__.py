"""Plain FP64 CPU oracle of the CFF / Yn-filter pseudospectral shell method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, tables or helpers); the only module both
sides consume is the seeded input generator ``paper_1104_3408_gb300.inputs``,
which holds none of the method's arithmetic.

Every routine follows the paper (Brügmann, "A pseudospectral matrix method for
time-dependent tensor fields on a spherical shell", arXiv:1104.3408) step by
step, in the paper's notation, with numpy matmul / einsum / SVD as the only
library primitives.  No blocking, fusion or reordering beyond the paper's
definitions.

Modules
-------
cff      grid (eqs. rk, thetai, phij), 1-d differentiation matrices (Sec. 2.3),
         3-d derivatives with the theta double cover (Secs. 2.1, 2.4) and the
         Cartesian chain rule (eq. dvdx).
dft      real DFT as matrices (Sec. 3.1, eqs. Fsynthesis, Fanalysis).
swsh     normalised associated Legendre functions, spin-weighted recursion
         (eqs. Yninc, Yncoeffs, Ynnegative), synthesis matrices P^n_m, SVD
         pseudo-inverse (eq. forwardL) and filter matrices F = P f P^+
         (eq. FasPfQ).
ynfilter triad decomposition of Cartesian tensors (Sec. 3.4, eqs. tetrad,
         tensorexpansion), the Yn tensor filter (Sec. 3.5), and the
         component-wise Y and graded Yg filters (Sec. 3.5, eq. nfofmu).
ghg      first-order GHG right-hand side (App. A.1, eqs. gdot, Phidot, Pidot),
         freeze-incoming outer boundary condition (App. A.2), gauge source
         initialisation (eq. gauge) and constraint norms.
evolve   method of lines with classical RK4 (Sec. 2.5) and the two filter
         placements.

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints, closed forms, invariants or brute force.  Parity status per
function is listed in each module's docstring.
"""

from . import cff, dft, swsh, ynfilter, ghg, evolve  # noqa: F401
from .evolve import OracleShell  # noqa: F401
