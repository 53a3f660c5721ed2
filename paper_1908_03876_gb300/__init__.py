"""GB300-native MRT / AMRT lattice Boltzmann optimal control for the
two-species chemotaxis system (Belmiloudi, arXiv 1908.03876).

The compute path is the CUDA library ``libcxlbm.so`` (C ABI in
``include/cxlbm.h``); this package holds its Python binding, the autograd
wrapper and the seeded workload generators.  Importing the package does not
load the library; ``Problem`` does, and fails loudly if it is missing.
"""
import importlib

__all__ = ["Problem", "workloads", "build_library"]


def __getattr__(name):
    if name == "Problem":
        return importlib.import_module(".problem", __name__).Problem
    if name == "build_library":
        return importlib.import_module(".build", __name__).build
    if name == "workloads":
        return importlib.import_module(".workloads", __name__)
    raise AttributeError(name)
