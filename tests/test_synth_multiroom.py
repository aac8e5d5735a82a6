"""The multi-room generator: its tensor renderer and occupancy agree with the host
(numpy, FP64) renderer and occupancy of the same scene, walls have doorways, and the
poses keep clear of the geometry.  CPU only (the tensor paths run on the CPU here)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
from synth.multiroom import make_multiroom, multiroom_poses, occupancy_bits_torch, render_keyframes_torch
from synth.room import _inside_prims, render_room, room_occupancy_bits


def test_tensor_render_matches_host_render():
    room = make_multiroom(0)
    poses = multiroom_poses(room, 3, seed=1)
    K = np.array([60.0, 60.0, 60.0, 34.0], np.float32)
    outs = list(render_keyframes_torch(room, poses, 120, 68, K, seed=3, device="cpu", noise_k=0.0))
    for (kf, rgb, depth, var), c2w in zip(outs, poses):
        z, rgb_ref = render_room(room, c2w, K, 120, 68)
        assert np.abs(depth.numpy() - z).max() < 1e-4 * max(1.0, z.max())
        assert np.abs(rgb.numpy() - rgb_ref).max() < 1e-3
        assert kf.depth_is_z and kf.W == 120 and kf.H == 68


def test_tensor_occupancy_matches_host_occupancy():
    room = make_multiroom(0)
    cfg = synth.config_c5("fp32")
    a = occupancy_bits_torch(room, 32, cfg.grid_origin, cfg.grid_inv_size, device="cpu")
    b = room_occupancy_bits(room, 32, cfg.grid_origin, cfg.grid_inv_size)
    assert np.array_equal(a, b)
    assert 0.05 < np.unpackbits(a).mean() < 0.5


def test_walls_doorways_and_poses():
    room = make_multiroom(0)
    assert room.n_walls == 72                      # 6 wall lines x 4 segments x (2 sides + lintel)
    # every wall segment has a doorway with a lintel from 2.2 m to the ceiling
    walls_lo = room.box_c[:room.n_walls] - room.box_h[:room.n_walls]
    lintels = walls_lo[:, 2] > 2.0
    assert lintels.sum() == 24 and np.allclose(walls_lo[lintels, 2], 2.2)
    poses = multiroom_poses(room, 50, seed=4)
    eyes = np.array([p[:, 3] for p in poses])
    assert not np.any(_inside_prims(room, eyes, 0.1))
    assert np.all((eyes > 0) & (eyes < room.extent))
