"""GB300-native spectral domain-decomposition path tracer (arXiv:1912.06474).

The compute path lives in ``libsddm.so`` (hand-written sm_103a CUDA behind a
C ABI declared in ``include/sddm.h``); ``paper_1912_06474_gb300.sddm`` is the
thin ctypes binding with the same call names. ``scenes`` produces seeded
synthetic inputs and imports nothing else from the package.
"""
__all__ = ["scenes", "sddm"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
