"""GB300-native batched low-rank updates of determinants and Pfaffians.

``paper_2602_05255_gb300.lrugb`` is the Python binding of the C-ABI library
(``include/lrugb.h``); importing it loads the CUDA library and raises if the
library has not been built.  ``paper_2602_05255_gb300.workloads`` holds the
seeded synthetic input generators and nothing of the method's arithmetic.
"""
import importlib

__all__ = ["lrugb", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
