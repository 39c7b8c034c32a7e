"""GB300-native Newton-Schulz polar factorisation A = U H (arXiv 2112.09017, Sec. III.D).

The compute path is the CUDA library ``libpolar.so`` built from ``csrc/``;
``polar`` is its thin ctypes binding. Importing this package does not load the
library: ``synth`` (seeded inputs) can be used without a GPU.
"""
__all__ = ["synth", "polar", "build"]


def __getattr__(name):
    if name in ("polar", "build", "synth"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
