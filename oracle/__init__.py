"""FP64 CPU oracle for PGCP (arXiv 1903.12359) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, readable restatement of what the paper computes: partition
(Section 4.1), cotangent Laplacian and DNCP (Section 4.2), the intermediate-form
and partial-welding algorithms (Algorithms 1 and 2, Section 4.3), the disk and
sphere constraints (Section 4.4), the final Laplace solves and stereographic
projection (Section 4.5, Algorithm 3), the fold-over fix by quasi-conformal
composition (Section 4.5 and Algorithm 3's last step, Section 3.5), the
angle-distortion statistics (Section 5) and the Mobius area step (Section 6.2).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it; the product path must not route through it.

Linear solves use SciPy's sparse direct solver (a library primitive), the
partition's connected components use ``scipy.sparse.csgraph``; everything else
is written out here.  Every function cites the passage it follows.
"""

from .common import OracleError  # noqa: F401
