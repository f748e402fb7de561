"""B300-native batched ABD-IPC step (Taccel, arXiv 2504.12908).

The compute path is the CUDA library ``libipc_b300.so`` (sources in
``csrc/``, C-ABI in ``include/ipc_b300.h``); ``ipc`` is its ctypes binding.
"""
from . import ipc  # noqa: F401
from .ipc import Envs, IpcError, lib  # noqa: F401

__all__ = ["ipc", "Envs", "IpcError", "lib"]
