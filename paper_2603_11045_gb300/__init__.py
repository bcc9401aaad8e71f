"""GB300 (sm_103a) hot path of NeFTY: the differentiable implicit-Euler heat
solve, its discrete adjoint and the diffusivity gradient, behind the C ABI of
libnefty (include/nefty.h).

``synthetic`` draws seeded inputs; ``solver`` is the ctypes binding and the
autograd Function; ``field`` the neural diffusivity field; ``serve`` the
serving queue.  Importing the package does not load the CUDA library;
the first call into ``Solver`` does, and fails loudly if it is missing.
"""
__all__ = ["Problem", "Solver", "HeatLoss", "heat_loss", "Server", "synthetic"]


def __getattr__(name):
    import importlib
    if name in ("Problem", "Solver", "HeatLoss", "heat_loss"):
        return getattr(importlib.import_module(__name__ + ".solver"), name)
    if name == "Server":
        return importlib.import_module(__name__ + ".serve").Server
    if name in ("synthetic", "solver", "build", "field", "serve"):
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
