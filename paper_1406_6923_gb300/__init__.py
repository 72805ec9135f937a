"""GB300-native S-fraction multiscale finite-volume wave propagation.

The compute path is ``libsfm.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/sfm.h``); :mod:`.sfm` is its thin ctypes binding.  Build it with
``python -m paper_1406_6923_gb300._build``."""
from . import sfm  # noqa: F401

__all__ = ["sfm"]
