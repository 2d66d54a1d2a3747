"""MatExPre on GB300: the matrix-exponential preconditioner for the FD Helmholtz
operator with PML and complex shift (arXiv 2506.03617), as sm_103a CUDA behind a
C ABI (``include/matexpre.h``).

Importing the package loads nothing native; ``paper_2506_03617_gb300.native``
loads the CUDA library and fails loudly when it is missing.
"""
__all__ = ["inputs"]
