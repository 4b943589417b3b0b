"""GridShift mode seeking (Kumar et al., arXiv 2206.02200) on GB300 (sm_103a).

The hot path (binning, neighbour-weighted centroid update, re-keying, merging,
label propagation) runs in the CUDA library libgridshift.so behind the C ABI of
include/gridshift.h; ``gridshift`` is its Python binding and ``synth`` holds the
seeded synthetic inputs.
"""
from . import gridshift  # noqa: F401
from .gridshift import GridShift, fit  # noqa: F401
