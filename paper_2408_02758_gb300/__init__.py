"""GB300-native FTLE hot path: RK4 flowmap advection and the least-squares flowmap-gradient /
Cauchy-Green / lambda_max / FTLE kernel, as hand-written sm_103a CUDA behind a C-ABI
(``include/ftle.h``, ``libftle.so``).

Submodules are imported on demand so that importing the seeded input generator
(``paper_2408_02758_gb300.inputs``) never loads the CUDA library.
"""
__all__ = ["ftle", "inputs"]


def __getattr__(name):
    if name in ("ftle", "inputs", "autotune", "autograd"):
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
