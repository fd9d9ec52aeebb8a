"""GB300-native per-timestep fluid-particle step of the Metaball-Imaging
Discrete Element Lattice Boltzmann Method (arXiv 2209.10411).

The compute path is the C-ABI library libmi_delbm.so (CUDA for sm_103a,
declared in include/mi_delbm.h); `paper_2209_10411_gb300.binding` is its thin
ctypes binding.  Importing this package does not load the library; importing
the binding does, and fails loudly if it is not built.
"""
import importlib

__all__ = ["binding", "scenes", "build"]


def __getattr__(name):
    if name == "binding":
        return importlib.import_module("._binding", __name__)
    if name in ("scenes", "build"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
