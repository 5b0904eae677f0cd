"""GB300-native tensor power flow (dense fixed-point iteration of arXiv 2403.04578).

* ``inputs``  -- seeded synthetic feeders and load tensors (no power-flow arithmetic).
* ``tpf``     -- ctypes binding of libtpf.so, the CUDA library that does every step of a solve.
* ``build``   -- in-tree nvcc build of libtpf.so for sm_103a.
"""
from . import inputs  # noqa: F401
from .tpf import Feeder, TpfError, precompute_host  # noqa: F401
