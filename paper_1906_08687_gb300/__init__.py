"""GB300 engine for batches of group-by aggregates over acyclic joins.

The engine is liblmf.so (C ABI, include/lmf.h; CUDA kernels for sm_103a);
`lmf` is its thin ctypes binding.
"""
from . import build  # noqa: F401
from .lmf import Engine, LmfError, load, register_schema  # noqa: F401
