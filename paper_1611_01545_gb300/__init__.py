"""GB300-native two-species particle-mesh step (CUBEP3M-with-neutrinos method).

The compute lives in libpm.so (CUDA kernels for sm_103a behind the C ABI of
include/pm.h); this package is its Python binding.  Build the library with
``python -m paper_1611_01545_gb300.build``.
"""
from .pm import PM, Codes, PMError, config_struct, deserialize, serialize  # noqa: F401
