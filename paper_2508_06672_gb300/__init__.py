"""GB300 (sm_103a) direct geolocation of GNSS interference.

The compute path is libdg.so (CUDA, built from ``csrc/``, C ABI in
``include/dg.h``); :mod:`paper_2508_06672_gb300.dg` is its thin Python binding.
"""
from .dg import *  # noqa: F401,F403
