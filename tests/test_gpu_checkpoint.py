"""Checkpoint and resume (map_save / map_load; the paper describes none): a map saved
after three Adam steps, one occupancy refresh and with one keyframe streamed out is
loaded into a new map, whose state equals the saved one bit for bit (parameters,
Adam moments, step count, occupancy bits and density, keyframe ids and residency)
and whose next step draws the same rays and samples and gives the same loss bit for
bit; its gradients agree with the original's up to the order of the FP32 atomics.
A checkpoint without keyframes loads into a map with none (a step then returns
MAP_ENOKF until they are added again)."""

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


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_saved_map_resumes(tmp_path, prec):
    from paper_2210_13641_gb300 import MapError, NerfMap, pack_params
    from paper_2210_13641_gb300.binding import MAP_ENOKF
    cfg = synth.config_small(precision=prec)
    m = NerfMap(cfg, occ_every=2)
    m.set_params(pack_params(synth.random_params(cfg, 5, table_scale=0.5, mlp_std=0.3)))
    kfs = [synth.c1_keyframe(40 + i, kf_id=10 + i) for i in range(3)]
    for kf in kfs:
        m.add_keyframe(kf)
    for i in range(3):
        m.step(1024, seed=i)
    m.evict_keyframe(11)
    path = tmp_path / "map.ckpt"
    m.save(path)
    r = NerfMap.load(path, cfg)

    assert np.array_equal(r.get_params(), m.get_params())
    for a, b in zip(r.get_adam(), m.get_adam()):
        assert np.array_equal(a, b)
    for a, b in zip(r.get_occupancy(), m.get_occupancy()):
        assert np.array_equal(a, b)
    assert r.stats().step == m.stats().step == 3
    assert r.keyframe_ids() == m.keyframe_ids() == [10, 11, 12]
    assert [r.keyframe_resident(k) for k in (10, 11, 12)] == [True, False, True]

    loss_m = m.step(1024, seed=7, no_update=True)
    loss_r = r.step(1024, seed=7, no_update=True)
    assert loss_m == loss_r
    (rid_m, t_m), (rid_r, t_r) = m.samples(), r.samples()
    assert np.array_equal(rid_m, rid_r) and np.array_equal(t_m, t_r)
    assert _rel(r.get_grads(), m.get_grads()) < 1e-5

    # the streamed-out keyframe comes back in both; the next Adam step starts from
    # the same parameters (its loss is the forward's: bit for bit)
    m.restore_keyframe(11)
    r.restore_keyframe(11)
    assert m.step(1024, seed=8) == r.step(1024, seed=8)
    assert r.stats().step == 4
    assert _rel(r.get_params(), m.get_params()) < 1e-6

    nokf = tmp_path / "nokf.ckpt"
    m.save(nokf, keyframes=False)
    e = NerfMap.load(nokf, cfg)
    assert e.keyframe_ids() == []
    assert np.array_equal(e.get_params(), m.get_params())
    with pytest.raises(MapError) as err:
        e.step(256, seed=1)
    assert err.value.code == MAP_ENOKF
    for kf in kfs:
        e.add_keyframe(kf)
    assert np.isfinite(e.step(256, seed=1))
    for x in (m, r, e):
        x.close()
