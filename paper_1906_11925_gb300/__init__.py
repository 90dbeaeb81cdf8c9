"""GB300-native sparse lattice-Boltzmann (LBGK) collide-and-stream for HemeLB
vessel geometries (arXiv 1906.11925).

The compute path is the CUDA library ``libhemelb_gb300.so`` (built for sm_103a
from ``csrc/``) behind the C ABI of ``include/lbm.h``; ``lbm`` is its thin
ctypes binding, ``geometry`` the seeded synthetic vessel inputs and
``metrics`` the throughput arithmetic.
"""
from . import geometry, metrics  # noqa: F401


def __getattr__(name):
    if name in ("lbm",):
        import importlib
        return importlib.import_module(".lbm", __name__)
    raise AttributeError(name)
