"""GB300-native distribute-probe-gather (DPG) record retrieval.

The compute path is the CUDA library libdpg.so (C ABI in include/dpg.h);
``paper_cs_0308004_gb300.dpg`` is its Python binding.  The binding is loaded
lazily so that the build step (``paper_cs_0308004_gb300._build``) can run
before the library exists.
"""
import importlib

__all__ = ["dpg", "Context"]


def __getattr__(name):
    if name in ("dpg", "Context", "DpgError", "DpgRangeError"):
        mod = importlib.import_module(__name__ + ".dpg")
        return mod if name == "dpg" else getattr(mod, name)
    raise AttributeError(name)
