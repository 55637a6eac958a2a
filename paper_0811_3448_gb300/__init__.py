"""libbinar: binar sort for GB300 (sm_103a).

The compute path is the C-ABI shared library built from ``csrc/`` (declared in
``include/binar.h``); :mod:`.binding` marshals torch tensors into it.  Nothing
is loaded at import time: the library is opened on the first call, and a
missing library raises instead of falling back to any other implementation.
"""
from __future__ import annotations

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in ("binding",):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
