"""GB300-native hot path of the electrostatic PIC step of arXiv 2205.11052.

The compute lives in the CUDA library ``libpic_gb300.so`` (C ABI in
``include/pic.h``); this package only builds and binds it.  ``capi`` holds
ctypes wrappers with the C names, ``sim.Simulation`` a torch-backed handle.
"""
from . import build, capi  # noqa: F401
from .capi import PicError, load_library  # noqa: F401

__all__ = ["build", "capi", "PicError", "load_library", "Simulation"]


def __getattr__(name):
    if name == "Simulation":
        from .sim import Simulation
        return Simulation
    raise AttributeError(name)
