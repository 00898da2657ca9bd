"""CPU oracle for the compressed cluster neighbor list (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product library never does,
and this package never imports the product.  ``nl_oracle.c`` holds every
definition (FP32 canonical predicate, FP64 sums); this module compiles it with
gcc and marshals numpy arrays through ctypes.  Parity-unpinned items are listed
in the header of ``nl_oracle.c``.
"""
from .api import *  # noqa: F401,F403
from .api import build, lib  # noqa: F401
