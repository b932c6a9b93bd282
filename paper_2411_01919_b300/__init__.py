"""B300 (sm_103a) implementation of the per-frame hot path of arXiv 2411.01919:
anisotropic diffusion of the depth image, back-projection + normal image, and
sequential multi-plane RANSAC, behind the C ABI of libpm (include/pm.h)."""
from ._ffi import PmError, load as load_library  # noqa: F401
from .pipeline import (Params, Pipeline, Planes, RegionPlanes, measure_peaks,  # noqa: F401
                       scratch_bytes)
