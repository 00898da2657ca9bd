"""GB300-native compressed cluster neighbor lists over an SFC particle layout.

The compute path lives in a native CUDA library (``libnlgb.so``, sm_103a)
behind a C ABI declared in ``include/nl.h``; ``nl`` re-exports its Python
binding.  Importing this package does not load the library: the first call
into ``nl`` does, and raises if it is missing or has no usable GPU.
"""
__all__ = ["nl", "workloads"]
