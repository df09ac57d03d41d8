"""fmap: transient F-statistic maps (Keitel & Ashton, arXiv:1805.05652) on one
GB300, as hand-written sm_103a CUDA behind the C ABI of ``include/fmap.h``.

The Python layer is a thin ctypes binding (``binding``) with the C names;
``build`` compiles ``_lib/libfmap.so`` in-tree with nvcc.
"""

from .binding import *  # noqa: F401,F403
from .binding import Plan, Server, Batch, FmapError, SUMMARY_DTYPE, summary_to_numpy, lib  # noqa: F401
from .build import build, lib_path  # noqa: F401
