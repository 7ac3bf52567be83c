"""GB300-native view-independent adjoint light tracing (arXiv 2310.02043).

The compute path is a C-ABI CUDA library (``include/lt.h``); ``lighttrace``
is its Python binding and ``scenes`` the seeded synthetic input generators.
"""
