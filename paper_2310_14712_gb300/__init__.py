"""GB300-native immersed Newmark IMEX time stepping (arXiv 2310.14712).

The compute path is a C-ABI shared library (``libimex``: host setup in C++,
time stepping in hand-written CUDA for sm_103a) declared in ``include/imex.h``.
``paper_2310_14712_gb300.imex`` is the thin ctypes binding; it is imported
lazily so that ``workloads`` (seeded inputs only) can be used without it.
"""
import importlib

__all__ = ["workloads", "imex"]


def __getattr__(name):
    if name in ("imex", "workloads"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
