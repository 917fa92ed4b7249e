"""B300-native rollout-step library for VisFly-style quadrotor simulation.

Submodules:
  workloads  seeded synthetic inputs (scenes, spawn states, commands)
  build      nvcc build of libvisfly_b300.so (sm_103a)
  binding    ctypes declarations of the C ABI (include/visfly_b300.h)
  sim        Sim context wrapper and the differentiable Rollout function
  serve      continuous-batching step server
"""
__all__ = ["workloads", "build", "binding", "sim"]


def __getattr__(name):
    import importlib
    if name in ("workloads", "build", "binding", "sim", "serve"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("Sim", "Rollout", "rollout"):
        return getattr(importlib.import_module(f"{__name__}.sim"), name)
    raise AttributeError(name)
