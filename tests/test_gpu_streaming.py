"""Keyframe streaming (the paper's memory mitigation: inactive parts of the map live
on the host, a window on the GPU): a streamed-out keyframe frees its device memory
and leaves the ray draw - the step then equals the oracle's step over the resident
keyframes (FP32 form, 1e-5, bit-exact sample lists) - and comes back bit-identical
(the same step's loss, bit for bit, as before the eviction)."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def test_evict_restore_keyframes():
    from paper_2210_13641_gb300 import MapError, NerfMap, pack_params
    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 6, table_scale=0.3, mlp_std=0.2)
    kfs = []
    for j, (W, H) in enumerate([(40, 30), (23, 17), (31, 19), (16, 12)]):
        kf = synth.c1_keyframe(60 + j, W=W, H=H, kf_id=j)
        kf.depth_is_z = True
        kfs.append(kf)
    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    for kf in kfs:
        m.add_keyframe(kf)
    n, seed = 1500, 4
    l_full = m.step(n, seed=seed, no_update=True)
    b0 = m.stats().device_bytes
    m.evict_keyframe(1)
    m.evict_keyframe(3)
    m.evict_keyframe(3)                              # already out: no-op
    assert not m.keyframe_resident(1) and m.keyframe_resident(2)
    freed = (23 * 17 + 16 * 12) * 32                 # 32 bytes per pixel; the draw's active list is small
    assert freed - 4096 <= b0 - m.stats().device_bytes <= freed
    l_part = m.step(n, seed=seed, no_update=True, pose_grad=True)
    b2 = m.stats().device_bytes                      # (the pose gradient's buffers are allocated now)
    ref = oracle.forward_backward(cfg, P, [kfs[0], kfs[2]], n, seed, 0)
    rid, t = m.samples()
    assert np.array_equal(rid, ref["ray_id"].astype(np.uint32)) and np.array_equal(t, ref["t"])
    assert l_part == pytest.approx(ref["loss"], rel=1e-5)
    g = m.pose_grads()
    assert np.all(g[[1, 3]] == 0) and np.all(np.abs(g[[0, 2]]).sum(axis=1) > 0)
    m.restore_keyframe(1)
    m.restore_keyframe(3)
    assert m.stats().device_bytes - b2 == freed
    assert m.step(n, seed=seed, no_update=True) == l_full
    for j in range(4):
        m.evict_keyframe(j)
    with pytest.raises(MapError) as e:
        m.step(n, seed=seed, no_update=True)
    assert e.value.code == -3
    m.add_keyframe(kfs[2])                           # a streamed-out id replaced by new images
    assert m.keyframe_resident(2)
    assert np.isfinite(m.step(n, seed=seed, no_update=True))
    m.close()
