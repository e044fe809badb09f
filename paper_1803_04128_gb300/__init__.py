"""GB300 butterfly-factorisation (IBF-MAT) apply library: Python binding.

See include/bf.h for the C ABI.  ``api.Plan`` wraps a plan; ``build.build()``
compiles the library in tree.
"""
from .api import BF16X3, F32, F64, Plan, grid_indices, version  # noqa: F401
