"""Device memory of the library from PyTorch's caching allocator.

The library allocates through an ``lbm_allocator`` (include/lbm.h).  This
module installs one backed by ``torch.cuda.caching_allocator_alloc`` /
``caching_allocator_delete`` as the library's process-wide default, so every
population buffer, geometry table, force ring and scratch block the library
takes is memory of torch's pool: it shows in ``torch.cuda.memory_allocated()``
and is returned to the pool, not to the driver, when the library frees it.

It is installed when the binding loads the library, unless the environment
variable ``LBM_TORCH_ALLOCATOR`` is ``0``; ``use_torch_allocator(False)``
restores cudaMalloc / cudaFree for sims created afterwards.  A failed torch
allocation returns NULL, which the library reports as LBM_ERR_OOM.

At interpreter exit every live sim and batch of the binding is destroyed
while torch is still intact (an ``atexit`` hook), and frees that would come
later are dropped.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref
from ctypes import c_size_t, c_void_p

try:   # imported before the exit hook is registered, so the hook runs first
    import torch  # noqa: F401
except Exception:   # pragma: no cover - torch is a dependency of the package
    torch = None

_ALLOC_T = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)

_closing = False
_handles = weakref.WeakSet()     # live Sim and Batch objects of the binding


def _alloc(nbytes, ctx):
    try:
        import torch
        return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
    except Exception:            # out of memory, or no device: NULL
        return None


def _free(ptr, ctx):
    if _closing or not ptr:
        return
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


# the callbacks and the struct live as long as the module
_alloc_cb = _ALLOC_T(_alloc)
_free_cb = _FREE_T(_free)
_struct = None


def _allocator_struct(lbm_allocator_type):
    global _struct
    if _struct is None:
        _struct = lbm_allocator_type(_alloc_cb, _free_cb, None)
    return _struct


def track(handle):
    """Register a Sim or Batch so the exit hook destroys it while torch lives."""
    _handles.add(handle)


def use_torch_allocator(enable=True):
    """Make torch's caching allocator the library's default (or, with False,
    cudaMalloc / cudaFree) for sims and scratch allocated from now on."""
    from . import _lib
    lib = _lib.load()
    st = lib.lbm_set_default_allocator(
        ctypes.byref(_allocator_struct(_lib.LbmAllocator)) if enable else None)
    if st != 0:
        raise RuntimeError(lib.lbm_last_error().decode(errors="replace"))


def install_default(lib, lbm_allocator_type):
    """Called once by the loader: install the torch allocator unless disabled."""
    if os.environ.get("LBM_TORCH_ALLOCATOR", "1") == "0":
        return
    lib.lbm_set_default_allocator(ctypes.byref(_allocator_struct(lbm_allocator_type)))


@atexit.register
def _shutdown():
    global _closing
    # batches before their member sims
    live = list(_handles)
    for h in sorted(live, key=lambda o: 0 if type(o).__name__ == "Batch" else 1):
        try:
            h.close()
        except Exception:
            pass
    _closing = True
