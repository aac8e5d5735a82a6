"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package generates configurations, parameters, keyframes, occupancy bitfields
and procedural scenes.  It contains none of the mapping method's arithmetic: no
hash indexing, no encoding, no MLP, no compositing, no loss and no optimiser.  Both
the CUDA path (through the Python binding) and the FP64 oracle consume what it
produces, so the two never share method code.
"""

from .workloads import (  # noqa: F401
    FieldConfig,
    Keyframe,
    config_small,
    config_c1,
    config_c2,
    config_c5,
    random_params,
    c1_keyframe,
    random_pose,
    look_at_pose,
)
from .room import (  # noqa: F401
    Room,
    make_room,
    render_room,
    room_keyframes,
    room_occupancy_bits,
    room_spline_poses,
)
from .multiroom import (  # noqa: F401
    make_multiroom,
    multiroom_poses,
    render_keyframes_torch,
    occupancy_bits_torch,
)
