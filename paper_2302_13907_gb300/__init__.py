"""GB300-native cased-well acoustic simulator (arXiv 2302.13907).

Explicit velocity-stress time stepping in cylindrical coordinates on a
staggered grid with PML, over a fluid / steel casing / cement / rock medium,
behind a small C-ABI library of hand-written sm_103a CUDA kernels.

`workloads` builds seeded synthetic media; `binding` is the thin ctypes layer
over the C-ABI (imported lazily: it needs the built CUDA library).
"""
__all__ = ["workloads", "binding"]


def __getattr__(name):
    if name in ("binding",):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
