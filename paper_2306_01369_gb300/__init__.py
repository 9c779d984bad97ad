"""GB300-native granular contact step (GranularGym, arxiv 2306.01369).

The compute path is libgg.so (hand-written sm_103a CUDA behind the C ABI of
include/gg.h); `paper_2306_01369_gb300.gg` is its Python binding and `scenes`
the seeded input generators.  Nothing here falls back to the CPU.
"""
from . import scenes  # noqa: F401
