"""Flood complex filtration on NVIDIA B300 (sm_103a).

The compute path is libflood.so (hand-written CUDA, C ABI in include/flood.h);
this package holds its thin Python binding (ops), the host Delaunay complex
builder (complex) and the seeded synthetic workloads (data). Importing the
package does not load the library; the first call does, and raises if it is
missing. There is no CPU fallback.
"""
__version__ = "0.1.0"

from .complex import SimplexLists, delaunay_complex, complex_from_simplices  # noqa: F401


def __getattr__(name):
    # Lazy access to the torch/CUDA binding so that CPU-only users of the
    # complex/data modules do not need a GPU.
    if name in ("ops", "serve"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
