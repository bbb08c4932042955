"""GB300 (sm_103a) library of xorgens pseudo-random number generators.

The generator is that of arXiv:1108.0486 (xorgensGP): the Sec. 2 recurrence
over a 128-word ring, combined with a Weyl sequence (Sec. 1.5, Eq. 1), run
over many independent streams at once in hand-written CUDA kernels behind the
C ABI of ``include/xorgens_gb300.h``; a 64-bit-word member of the family
with FP64 uniforms sits behind ``include/xorgens_w64.h``.

Submodules load lazily so that ``workloads`` (seeded synthetic inputs) can be
imported without torch or the CUDA library.
"""
import importlib

__all__ = ["Streams", "Streams64", "XGError", "as_u32", "build", "workloads"]


def __getattr__(name):
    if name in ("Streams", "Streams64", "as_u32"):
        return getattr(importlib.import_module(".api", __name__), name)
    if name == "XGError":
        return importlib.import_module("._lib", __name__).XGError
    if name == "build":
        return importlib.import_module(".build", __name__).build
    if name in ("workloads", "api", "_lib", "server"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
