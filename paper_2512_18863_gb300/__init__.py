"""GB300-native (sm_103a) differentiable pencil-beam VMAT dose engine.

Hot path of arXiv 2512.18863 ("PyDoseRT"): fluence rasterisation from MLC
leaves and jaws, central-ray radiological depth, depth-dependent lateral
kernel convolution and MU-weighted dose accumulation, plus the hand-written
adjoint for leaves, jaws and MUs.  The compute runs in hand-written CUDA
kernels behind the C ABI of include/pdrt.h; this package is the Python
binding (_lib), the torch autograd wrapper (engine) and seeded synthetic
workloads (synth).
"""
from . import synth  # noqa: F401

__all__ = ["synth", "DoseEngine", "DoseFn", "build_library"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def __getattr__(name):
    if name in ("DoseEngine", "DoseFn"):
        from . import engine
        return getattr(engine, name)
    raise AttributeError(name)
