"""CPU oracle for the pTEBD layer (arXiv:2312.02667).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA library; the
two meet only through the seeded inputs of ``paper_2312_02667_gb300.inputs``.

Everything here is plain numpy in complex128 / float64.  The one library
primitive used as a step is LAPACK's SVD (``numpy.linalg.svd``), for the SVD the
TEBD procedure calls for (Sec. II C); every other step is written out in the
paper's order and notation.
"""
from .mps import *  # noqa: F401,F403
from . import statevector  # noqa: F401
