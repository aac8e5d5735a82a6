"""The multi-scene serving loop: each scene's results are the same alone and in the
mix with other scenes' continuous mapping and renders (plain FP32 and FP16 scenes,
render queries of 64x48 up to 1280x720), grouped renders of several scenes and
resolutions equal the single-view renders of the mapping library, keyframes complete
after the first step that covers them, and admission follows free device memory.

Tolerance of "the same": a render before any step is bit-identical (its inputs are
identical, and a grouped render evaluates every pixel with the arithmetic of a
single-view render); step losses within 1e-5 relative for FP32 and 2e-3 for FP16
(the table-gradient atomics add in a different order when other streams share the
GPU, and in FP16 the order of a step's FP32 sums also moves the power-of-two
gradient scales' inputs); a render after three Adam steps within 1e-3 relative in L2
over the image (Adam's first steps move an entry by +-lr whatever the size of its
gradient, so an entry whose gradient cancels to the FP32 rounding level can flip its
step when the summation order changes; the same happens between two runs of the
scene alone)."""

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


SIZES = ((64, 48), (640, 480), (1280, 720))


def _scaled(view, W, H):
    """The intrinsics of a view scaled to a W x H image of the same field of view."""
    return np.array([view.K[0] * W / view.W, view.K[1] * H / view.H, W / 2.0, H / 2.0], np.float32)


def _scene_a(server, P, prec):
    from paper_2210_13641_gb300 import pack_params
    cfg = synth.config_c1(precision=prec)
    sid = server.add_scene(cfg, continuous_mapping=False)
    server.scene_map(sid, cfg).set_params(pack_params(P))
    return cfg, sid


def _script_a(server, sid, kfs, view):
    ids = [server.submit_keyframe(sid, k) for k in kfs]
    before = [server.submit_render(sid, view.c2w, _scaled(view, W, H), W, H) for W, H in SIZES]
    steps = [server.submit_step(sid, 4096, want_loss=True) for _ in range(3)]
    after = [server.submit_render(sid, view.c2w, _scaled(view, W, H), W, H) for W, H in SIZES]
    done = server.wait(ids + [r[0] for r in before + after] + steps)
    assert all(done[i]["status"] == 0 for i in done)
    losses = [done[i]["loss"] for i in steps]
    assert [done[i]["step_index"] for i in steps] == [0, 1, 2]
    return [(r[1], r[2]) for r in before], losses, [(r[1], r[2]) for r in after]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_results_same_alone_and_in_the_mix(prec):
    from paper_2210_13641_gb300 import pack_params
    from paper_2210_13641_gb300.binding import MapServer
    cfg = synth.config_c1(precision=prec)
    P = synth.random_params(cfg, 3)
    kfs = [synth.c1_keyframe(40 + i, kf_id=i) for i in range(2)]
    view = synth.c1_keyframe(50)

    alone = MapServer(max_scenes=4, max_inflight=2, step_rays=4096)
    _, sa = _scene_a(alone, P, prec)
    ref = _script_a(alone, sa, kfs, view)
    alone.close()

    mix = MapServer(max_scenes=4, max_inflight=2, step_rays=8192)
    others = []
    for j in range(2):                                   # two busy scenes: continuous mapping
        c = synth.config_small(precision=prec, occ_res=0, log2_table=12 + j)
        sid = mix.add_scene(c, continuous_mapping=True)
        mix.scene_map(sid, c).set_params(pack_params(synth.random_params(c, 10 + j)))
        others.append(sid)
        mix.submit_keyframe(sid, synth.c1_keyframe(60 + j, W=48, H=32))
    _, sa = _scene_a(mix, P, prec)
    busy = [mix.submit_render(o, view.c2w, _scaled(view, 160, 120), 160, 120)[0] for o in others]
    got = _script_a(mix, sa, kfs, view)
    busy += [mix.submit_render(o, view.c2w, _scaled(view, 1280, 720), 1280, 720)[0] for o in others]
    mix.wait(busy)
    st = mix.stats()
    assert st["steps_done"] > 3                          # the other scenes really ran
    if prec == "fp16":
        assert st["grouped_renders"] >= 8                # the FP16 renders went through grouped launches
    mix.close()

    for (rgb, d), (rgb0, d0) in zip(got[0], ref[0]):
        assert np.array_equal(rgb, rgb0) and np.array_equal(d, d0)
    assert np.allclose(got[1], ref[1], rtol=1e-5 if prec == "fp32" else 2e-3)
    for (rgb, d), (rgb0, d0) in zip(got[2], ref[2]):
        for a, b in ((rgb, rgb0), (d, d0)):
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_grouped_renders_equal_single_view_renders(prec):
    """Twelve views of four maps (different table sizes, grids, bitfields and
    weights, one of them dense enough that most rays stop within their first 32
    samples) at 160x120, 640x480 and 1280x720 in one map_render_group call (batches
    of 2^18 rays that mix views, scenes and resolutions, views split across batches,
    both render passes): every image equals, bit for bit, the mapping library's own
    render of that view (map_render, parity-tested against the oracle).  The same
    queries through the serving loop go through grouped renders and give the same
    images."""
    import torch
    from paper_2210_13641_gb300 import NerfMap, pack_params
    from paper_2210_13641_gb300.binding import MapServer, render_group
    cfgs = [synth.config_c1(precision=prec),
            synth.config_small(precision=prec, occ_res=16, step=np.float32(0.02), n_steps=150),
            synth.config_small(precision=prec, occ_res=0, log2_table=12),
            synth.config_small(precision=prec, occ_res=0, step=np.float32(0.01), n_steps=300, max_samples=256)]
    Ps = [synth.random_params(c, 20 + j, table_scale=0.5, mlp_std=0.15) for j, c in enumerate(cfgs)]
    Ps[3]["W2"][0] += 2.6      # a dense field: most rays stop early, the passes matter
    bits = np.packbits(np.random.default_rng(5).uniform(size=16 ** 3) < 0.6, bitorder="little")
    view = synth.c1_keyframe(51)
    sizes = ((160, 120), (640, 480), (1280, 720))
    maps = []
    for c, P in zip(cfgs, Ps):
        m = NerfMap(c, occ_every=0)
        m.set_params(pack_params(P))
        if c.occ_res:
            m.set_occupancy(bits)
        maps.append(m)
    order = [(j, W, H) for W, H in sizes for j in range(len(cfgs))]  # resolutions and scenes interleaved
    outs = [(torch.full((H, W, 3), -1.0, device="cuda"), torch.full((H, W), -1.0, device="cuda"))
            for _, W, H in order]
    render_group([maps[j] for j, _, _ in order], [(view.c2w, _scaled(view, W, H), W, H) for _, W, H in order],
                 outs)
    torch.cuda.synchronize()
    single = {}
    for (j, W, H), (rgb, d) in zip(order, outs):
        rgb0, d0, _ = maps[j].render(view.c2w, _scaled(view, W, H), W, H)
        single[(j, W, H)] = (rgb0, d0)
        assert np.array_equal(rgb.cpu().numpy(), rgb0), (j, W, H)
        assert np.array_equal(d.cpu().numpy(), d0), (j, W, H)
    for m in maps:
        m.close()

    server = MapServer(max_scenes=4, max_inflight=3, step_rays=4096)
    sids = []
    for c, P in zip(cfgs, Ps):
        sid = server.add_scene(c, continuous_mapping=False)
        sm = server.scene_map(sid, c)
        sm.set_params(pack_params(P))
        if c.occ_res:
            sm.set_occupancy(bits)
        sids.append(sid)
    reqs = [(j, W, H, server.submit_render(sids[j], view.c2w, _scaled(view, W, H), W, H)) for j, W, H in order]
    done = server.wait([r[3][0] for r in reqs])
    st = server.stats()
    server.close()
    assert all(d["status"] == 0 for d in done.values())
    assert st["grouped_renders"] == len(reqs) and st["group_batches"] <= len(reqs)
    for j, W, H, (_, rgb, d) in reqs:
        assert np.array_equal(rgb, single[(j, W, H)][0]) and np.array_equal(d, single[(j, W, H)][1])


def test_render_group_refuses_plain_fp32_maps_and_bad_sizes():
    """map_render_group takes tensor-core maps only (a plain FP32 map renders with
    map_render) and refuses empty views, with MAP_EINVAL and a message on maps[0],
    before anything is launched."""
    import torch
    from paper_2210_13641_gb300 import MapError, NerfMap, pack_params
    from paper_2210_13641_gb300.binding import MAP_EINVAL, render_group
    c16, c32 = synth.config_c1(precision="fp16"), synth.config_c1(precision="fp32")
    m16, m32 = NerfMap(c16, occ_every=0), NerfMap(c32, occ_every=0)
    m16.set_params(pack_params(synth.random_params(c16, 1)))
    view = synth.c1_keyframe(52)
    out = (torch.zeros((12, 16, 3), device="cuda"), torch.zeros((12, 16), device="cuda"))
    with pytest.raises(MapError) as e:
        render_group([m16, m32], [(view.c2w, view.K, 16, 12)] * 2, [out, out])
    assert e.value.code == MAP_EINVAL and "FP32" in str(e.value)
    with pytest.raises(MapError) as e:
        render_group([m16], [(view.c2w, view.K, 0, 12)], [out])
    assert e.value.code == MAP_EINVAL
    render_group([m16], [(view.c2w, view.K, 16, 12)], [out])      # the valid call still works
    torch.cuda.synchronize()
    rgb0, d0, _ = m16.render(view.c2w, view.K, 16, 12)
    assert np.array_equal(out[0].cpu().numpy(), rgb0) and np.array_equal(out[1].cpu().numpy(), d0)
    m16.close()
    m32.close()


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
