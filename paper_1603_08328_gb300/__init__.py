"""Local-expansion-move stereo (arXiv 1603.08328) on GB300 (sm_103a).

The computation lives in the CUDA library ``liblem.so`` behind the C ABI of
``include/lem.h``; ``lem`` is its ctypes binding.  Importing the package does
not load the library; ``lem.lib()`` does, and raises if it has not been built.
"""
from . import lem  # noqa: F401
