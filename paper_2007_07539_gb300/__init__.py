"""GB300-native mixed-precision multigrid-preconditioned iterative refinement.

The solver library is ``libmgfp.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/mg.h``).  ``paper_2007_07539_gb300.mg`` is its
ctypes binding; ``paper_2007_07539_gb300.inputs`` holds the seeded synthetic
input recipes.  Importing the package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
__all__ = ["inputs", "mg"]
