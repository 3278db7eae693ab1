"""GB300-native ASSE: sliding-window super-point detection and cardinality
estimation with asynchronous timestamps (arXiv 1807.01527).

The hot path lives in hand-written CUDA kernels for sm_103a behind the C ABI
of include/asse.h (libasse.so, built in-tree by ``build.build()``);
``asse.Pool`` is its Python binding.
"""
from . import asse  # noqa: F401  (the binding loads libasse.so lazily)
from .asse import AsseError, Pool  # noqa: F401
