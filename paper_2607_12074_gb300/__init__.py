"""GB300-native exact induced 4-vertex motif counting (HARP-ME, arXiv 2607.12074).

The counting path is the CUDA library ``libharp.so`` (sources in ``csrc/``, C ABI in
``include/harp.h``); ``harp`` is its ctypes binding.  Importing this package does not load the
library; the first call does, and raises ``HarpUnavailable`` if it has not been built.
"""
from .harp import *  # noqa: F401,F403
from .harp import HarpError, HarpUnavailable, Csr, harp_plan, lib  # noqa: F401
