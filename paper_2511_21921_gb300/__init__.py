"""GB300-native CRKSPH neighbor-sum path (CRK-HACC hydrodynamics, arXiv 2511.21921).

The computation lives in ``libcrk`` (CUDA C++ for sm_103a, C ABI in
``include/crk.h``); :mod:`._lib` is its same-name ctypes binding and
:mod:`.solver` a torch-tensor wrapper with an autograd function.
:mod:`.synth` generates the seeded synthetic workloads.
"""
__all__ = ["Solver", "CRKRates", "rates", "make_params", "copy_"]


def __getattr__(name):
    if name in __all__:
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
