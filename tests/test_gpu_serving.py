"""The multi-scene serving loop: each scene's results are the same alone and in the
mix with other scenes' continuous mapping and renders, keyframes complete after the
first step that covers them, and admission follows free device memory.

Tolerance of "the same": a render before any step is bit-identical (its inputs are
identical); step losses within 1e-5 relative (the FP32 tolerance: the table-gradient
atomics add in a different order when other streams share the GPU); a render after
three Adam steps within 1e-3 relative in L2 over the image (Adam's first steps move
an entry by +-lr whatever the size of its gradient, so an entry whose gradient
cancels to the FP32 rounding level can flip its step when the summation order
changes; the same happens between two runs of the scene alone)."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


def _scene_a(server, P):
    from paper_2210_13641_gb300 import pack_params
    cfg = synth.config_c1()
    sid = server.add_scene(cfg, continuous_mapping=False)
    server.scene_map(sid, cfg).set_params(pack_params(P))
    return cfg, sid


def _script_a(server, sid, kfs, view):
    ids = [server.submit_keyframe(sid, k) for k in kfs]
    r0, rgb0, d0 = server.submit_render(sid, view.c2w, view.K, 64, 48)
    steps = [server.submit_step(sid, 4096, want_loss=True) for _ in range(3)]
    r1, rgb1, d1 = server.submit_render(sid, view.c2w, view.K, 64, 48)
    done = server.wait(ids + [r0, r1] + steps)
    assert all(done[i]["status"] == 0 for i in done)
    losses = [done[i]["loss"] for i in steps]
    assert [done[i]["step_index"] for i in steps] == [0, 1, 2]
    return rgb0, d0, losses, rgb1, d1


def test_results_same_alone_and_in_the_mix():
    from paper_2210_13641_gb300 import pack_params
    from paper_2210_13641_gb300.binding import MapServer
    cfg = synth.config_c1()
    P = synth.random_params(cfg, 3)
    kfs = [synth.c1_keyframe(40 + i, kf_id=i) for i in range(2)]
    view = synth.c1_keyframe(50)

    alone = MapServer(max_scenes=4, max_inflight=2, step_rays=4096)
    _, sa = _scene_a(alone, P)
    ref = _script_a(alone, sa, kfs, view)
    alone.close()

    mix = MapServer(max_scenes=4, max_inflight=2, step_rays=8192)
    others = []
    for j in range(2):                                   # two busy scenes: continuous mapping
        c = synth.config_small(occ_res=0, log2_table=12 + j)
        sid = mix.add_scene(c, continuous_mapping=True)
        mix.scene_map(sid, c).set_params(pack_params(synth.random_params(c, 10 + j)))
        others.append(sid)
        mix.submit_keyframe(sid, synth.c1_keyframe(60 + j, W=48, H=32))
    _, sa = _scene_a(mix, P)
    busy = [mix.submit_render(o, view.c2w, view.K, 160, 120)[0] for o in others]
    got = _script_a(mix, sa, kfs, view)
    busy += [mix.submit_render(o, view.c2w, view.K, 320, 240)[0] for o in others]
    mix.wait(busy)
    assert mix.stats()["steps_done"] > 3                 # the other scenes really ran
    mix.close()

    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    assert np.allclose(got[2], ref[2], rtol=1e-5)
    for a, b in ((got[3], ref[3]), (got[4], ref[4])):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


def test_keyframe_completes_after_a_covering_step_and_admission():
    from paper_2210_13641_gb300 import MapError, pack_params
    from paper_2210_13641_gb300.binding import MapServer
    s = MapServer(max_scenes=2, max_inflight=2, step_rays=4096)
    cfg = synth.config_c1()
    sid = s.add_scene(cfg, continuous_mapping=True)
    s.scene_map(sid, cfg).set_params(pack_params(synth.random_params(cfg, 0)))
    first = s.submit_keyframe(sid, synth.c1_keyframe(1, kf_id=0))
    d = s.wait([first])[first]
    assert d["status"] == 0 and d["t_submit"] <= d["t_start"] <= d["t_done"]
    later = [s.submit_keyframe(sid, synth.c1_keyframe(2 + i, kf_id=1 + i)) for i in range(3)]
    recs = s.wait(later)
    st = s.stats()
    for i in later:
        assert recs[i]["status"] == 0
        assert recs[i]["step_index"] >= 1                # inserted while steps were running
        assert st["steps_done"] > recs[i]["step_index"]  # the covering step has completed
    # admission by free device memory: a reserve larger than the GPU refuses the scene
    s2 = MapServer(max_scenes=1, step_rays=4096, hbm_reserve=1 << 50)
    with pytest.raises(MapError) as e:
        s2.add_scene(cfg)
    assert e.value.code == -2
    s2.close()
    s.close()
