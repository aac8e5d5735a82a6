"""The room generator's depth-outlier injection (used by the depth-weighting
ablation): the requested fraction of pixels carries a gross error within the stated
range and reports sigma_d = outlier_sigma; the other pixels keep their noise model."""

import numpy as np

import synth
from synth.room import render_room


def test_outlier_injection():
    room = synth.make_room(0)
    K = (52.5, 52.5, 32.0, 24.0)
    poses = synth.room_spline_poses(room, 2, seed=5)
    kfs = synth.room_keyframes(room, 2, seed=1, W=64, H=48, K=K, poses=poses, sigma_floor=0.05,
                               outlier_frac=0.25, outlier_range=2.0, outlier_sigma=1.0)
    for kf, c2w in zip(kfs, poses):
        z, _ = render_room(room, c2w, np.asarray(K, np.float32), 64, 48)
        bad = kf.var == 1.0
        assert abs(bad.mean() - 0.25) < 0.05
        err = kf.depth - z
        assert np.all(np.abs(err[bad]) <= 2.0 + 1e-5) and np.abs(err[bad]).mean() > 0.5
        good = ~bad
        assert np.all(kf.var[good] >= 0.05 ** 2 - 1e-7) and np.all(kf.var[good] < 1.0)
        assert np.abs(err[good] / np.sqrt(kf.var[good])).max() < 6.0
