"""FP64 CPU oracle of the NeRF-SLAM mapping step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only
the tests, the smoke check of the graft entry point and the CPU-baseline / reference
legs of the benchmark may import or run it.  It shares no code with the CUDA path;
both consume the seeded inputs of the separate `synth` package.

Every function states the passage of the paper (arXiv 2210.13641, "NeRF-SLAM") or of
the definition it follows.  Parity status per function is listed in the module
docstring of `nerf_oracle`.
"""

from .nerf_oracle import *  # noqa: F401,F403
