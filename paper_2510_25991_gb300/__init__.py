"""GB300 (sm_103a) overlapping solution-transfer domain decomposition (arXiv 2510.25991).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/ddst.h``);
``ddst`` is its Python binding.  Importing the package does not load the library; the first
call does, and fails loudly if it has not been built.
"""
from .ddst import *  # noqa: F401,F403
