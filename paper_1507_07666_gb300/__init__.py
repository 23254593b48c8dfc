"""GB300-native lattice-kinetic Kohn-Sham solver (liblbks + ctypes binding).

    from paper_1507_07666_gb300 import lbks     # loads _lib/liblbks.so
    from paper_1507_07666_gb300.build import build

The binding is imported lazily so that `build` works before the library exists.
"""
import importlib

__all__ = ["lbks", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
