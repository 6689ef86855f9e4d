"""GB300-native (sm_103a) seam carving: the hot path of arXiv 2410.21207 behind a C ABI.

``binding`` wraps libsc_gb300.so (include/sc.h); ``synth`` makes the seeded synthetic inputs;
``build`` compiles the CUDA library.
"""
from . import binding, synth  # noqa: F401
from .binding import carve, carve_batch, carve_host, check, energy, find_seam, version  # noqa: F401
