"""GB300-native engine for the data-parallel hot path of single-event-upset
injection into 3D Gaussian splatting models (arXiv 2606.21791): batched
bit-flip injection, forward tile rasterisation of each corrupted model, the
per-pixel comparison against the clean frame, and the per-primitive support
guard.  The compute lives in libgs.so (hand-written sm_103a CUDA behind the C
ABI of include/gs.h); ``gs`` is its thin binding and ``synth`` the seeded input
generators."""
from . import synth  # noqa: F401

__all__ = ["synth", "gs", "build"]


def build(force: bool = False) -> str:
    from .buildlib import build as _b
    return _b(force=force)
