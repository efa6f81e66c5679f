"""GB300-native pressure recovery and surface forces for penalised 2-D vortex flows.

The compute path is the CUDA library ``libpp.so`` (C ABI in ``include/pp.h``);
``api`` is its thin ctypes binding and ``synth`` builds seeded synthetic inputs.
Nothing here falls back to the CPU: without ``libpp.so`` every call raises.
"""
from . import api  # noqa: F401  (ctypes binding; loads libpp.so on first use)
from . import synth  # noqa: F401  (input generators only; no method arithmetic)

__all__ = ["api", "synth", "build"]


def build(force: bool = False) -> str:
    """Compile libpp.so in-tree for sm_103a (see ``_build.py``)."""
    from . import _build
    return _build.build(force=force)
