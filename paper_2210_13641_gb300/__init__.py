"""GB300-native mapping hot path of NeRF-SLAM (arXiv 2210.13641).

The library `libnerfmap.so` (CUDA kernels for sm_103a behind the C ABI of
include/nerfmap.h) fits a multiresolution hash-grid radiance field to posed
keyframes with dense depth and per-pixel depth variance, minimising the paper's
mapping loss (colour L2 plus Sigma_D-weighted depth), and renders views of it.
`binding` is the ctypes layer; `build` compiles the library in-tree.
"""

from .binding import (  # noqa: F401
    MapError,
    NerfMap,
    level_resolutions,
    load,
    make_config,
    pack_params,
    unpack_params,
)
