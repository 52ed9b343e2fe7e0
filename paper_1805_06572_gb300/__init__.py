"""GB300-native EM for two-source full-rank spatial covariance analysis (FCA).

Conventional frame-wise EM and FastFCA (Ito, Araki, Nakatani, arXiv 1805.06572) as
hand-written sm_103a CUDA kernels behind the C ABI in include/fca.h; ``fca`` is the thin
Python binding. Build the library with ``paper_1805_06572_gb300.build.build()``.
"""
from .build import build, LIB as LIB_PATH  # noqa: F401
