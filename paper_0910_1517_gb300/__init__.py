"""GB300-native FX correlator and beamformer (Roy et al., arXiv:0910.1517).

The compute path is the sm_103a CUDA library ``libgb300corr.so`` (csrc/),
reached through the C ABI of include/corr.h; ``corr`` is its thin Python
binding and ``build`` compiles it in-tree.
"""
from . import corr  # noqa: F401
from .corr import (  # noqa: F401
    CORR_F16,
    CORR_FP32,
    CORR_FP32TC,
    CORR_I8,
    CorrError,
)
