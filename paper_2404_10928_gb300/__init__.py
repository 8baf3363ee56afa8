"""GB300 (sm_103a) library for iterative photoacoustic reconstruction with a
matrix-free time-of-flight operator (forward A, adjoint A^T, projected Landweber
and CGLS), exposed through the C ABI in ``include/pa.h``.

``Plan`` (in ``api``) wraps that ABI for PyTorch users; ``phantoms`` holds the
seeded synthetic inputs.  Importing ``api`` requires the built ``libpa.so``.
"""

__all__ = ["api", "phantoms", "build"]


def __getattr__(name):
    if name == "Plan":
        from .api import Plan
        return Plan
    raise AttributeError(name)
