"""GB300 (sm_103a) implementation of the reduced basis warm-start iterative method
(arXiv 2311.13862): a CUDA library with a C ABI (include/rbws.h) and a thin
Python binding (rbws.py).  The CPU oracle under oracle/ is test infrastructure
and is never imported from here."""
from . import inputs  # noqa: F401
