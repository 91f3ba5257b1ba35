"""GB300-native D2Q9 lattice Boltzmann library with learned outflow boundaries
(arXiv 2506.05293).  The compute path is the CUDA library behind the C ABI in
include/lbm.h; this package is its Python binding."""
from . import _lib
from .api import *  # noqa: F401,F403
from .api import LbmError, Sim, make_mlp, unflatten, use_torch_allocator

__all__ = [n for n in dir() if n.startswith("lbm_")] + ["LbmError", "Sim", "make_mlp", "unflatten",
                                                        "use_torch_allocator"]
