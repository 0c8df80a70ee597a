"""FP64 CPU oracle for the preconditioned Richardson iteration of
Dölz, Palii and Schlottbom (arXiv 2102.09038) for the even-parity anisotropic
radiative transfer equation.

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of the paper's discretisation (Section 4) and iteration
(Section 5, Algorithms 1-3) used to check the CUDA library.  Only the test
suite, the smoke entry point and the CPU-baseline leg of the benchmark may
import it.  It shares no code with the CUDA path; the two meet only in the
seeded input generators of the ``workloads`` package.

Parity status of each function is pinned by the ``-m "not gpu"`` tests
(tests/test_oracle_*.py): closed forms, invariants, special cases and brute
force on tiny meshes.
"""
from .geometry import square_mesh, sphere_reps, spherical_area, quad_rule
from .assemble import Discretisation, hg_kernel
from .operators import Operators
from .richardson import Coarse, richardson, d_of
from .h2 import H2Scattering
