"""GB300-native timestep-splitting Euler-Maruyama on metric graphs.

The compute path is the CUDA library ``libmetricgraph.so`` (C ABI declared in
``include/mg.h``); ``binding`` marshals Python arguments into it and nothing
else.  The library is loaded on first use and a missing or unloadable library
raises: there is no CPU fallback.
"""
__all__ = ["binding", "workloads"]
