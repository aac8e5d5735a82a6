"""Parity of the CUDA mapping path (through the C ABI) with the FP64 oracle.

Tolerances (plain FP32 form): sample lists and occupancy bits bit-exact; loss and
per-ray renders within 1e-5 relative; each gradient tensor within 1e-5 relative in
L2 norm, and each entry within 1e-5 of the sum of the absolute values of the
products that form it (the oracle's `grads_abs`).  An entry is a sum of thousands
of products accumulated in FP32 in an arbitrary (atomic) order, so its rounding
error scales with that absolute sum, not with the entry itself when terms cancel.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    torch.cuda.init()
    yield


def _map(cfg, P, kfs, occ_bits=None):
    from paper_2210_13641_gb300 import NerfMap, pack_params
    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    for kf in kfs:
        m.add_keyframe(kf)
    if occ_bits is not None:
        m.set_occupancy(occ_bits)
    return m


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _check_grads(g_gpu, ref, rel=REL, elem=REL):
    """Per-tensor relative L2, and element-wise against grads_abs except for the table
    entries touched by samples with a ReLU pre-activation within 1e-5 of zero relative
    to its terms (oracle.near_kink_samples): there FP32 and FP64 may take different
    branches, and both results are correct; those entries stay under the L2 bound."""
    for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
        a = np.asarray(g_gpu[k], np.float64)
        b = ref["grads"][k]
        assert _rel(a, b) <= rel, (k, _rel(a, b))
        tol = elem * ref["grads_abs"][k] + 1e-30
        bad = np.abs(a - b) > tol
        if k == "tables":
            bad &= ~ref["near_kink_entries"][:, :, None]
        assert not bad.any(), (k, int(bad.sum()), float((np.abs(a - b)[bad] / tol[bad]).max()))


def _check_step(m, ref, n_rays, loss):
    rid, t = m.samples()
    assert np.array_equal(rid, ref["ray_id"].astype(np.uint32))
    assert np.array_equal(t.view(np.uint32), ref["t"].astype(np.float32).view(np.uint32))
    assert loss == pytest.approx(ref["loss"], rel=REL)
    rgb, D, acc = m.ray_outputs(n_rays)
    assert np.allclose(rgb, ref["I_hat"], rtol=REL, atol=1e-6)
    assert np.allclose(D, ref["D_hat"], rtol=REL, atol=1e-6)
    assert np.allclose(acc, ref["acc"], rtol=REL, atol=1e-6)


def test_c1_step_parity_fp32():
    cfg = synth.config_c1()
    P = synth.random_params(cfg, 0)
    kf = synth.c1_keyframe(0)
    m = _map(cfg, P, [kf])
    loss = m.step(4096, seed=7, no_update=True)
    ref = oracle.forward_backward(cfg, P, [kf], 4096, 7, 0, magnitudes=True)
    _check_step(m, ref, 4096, loss)
    _check_grads(m.unpack(m.get_grads()), ref)


def test_small_multi_keyframe_occupancy_truncation_ragged():
    """Two dense and two hashed levels, a random 16^3 bitfield, at most 16 samples
    per ray (truncation), three keyframes of different sizes with z-depth, and a
    ray count that is not a multiple of any tile."""
    cfg = synth.config_small(occ_res=16, step=np.float32(0.02), n_steps=150)
    P = synth.random_params(cfg, 3, table_scale=0.05, mlp_std=0.2)
    rng = np.random.default_rng(4)
    kfs = []
    for j, (W, H) in enumerate([(40, 30), (23, 17), (64, 9)]):
        kf = synth.c1_keyframe(10 + j, W=W, H=H, kf_id=100 + j)
        kf.depth_is_z = True
        kfs.append(kf)
    bits = np.packbits(rng.uniform(size=16 ** 3) < 0.6, bitorder="little")
    m = _map(cfg, P, kfs, bits)
    n = 3001
    loss = m.step(n, seed=11, no_update=True)
    ref = oracle.forward_backward(cfg, P, kfs, n, 11, 0, occ_bits=bits, magnitudes=True)
    assert np.bincount(ref["ray_id"], minlength=n).max() == cfg.max_samples
    _check_step(m, ref, n, loss)
    _check_grads(m.unpack(m.get_grads()), ref)


def test_adam_update_and_step_counter():
    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 5, table_scale=0.05, mlp_std=0.2)
    kf = synth.c1_keyframe(6, W=32, H=24)
    m = _map(cfg, P, [kf])
    m.step(1000, seed=3, no_update=True)
    G = m.unpack(m.get_grads().copy())
    m.step(1000, seed=3)                      # same draw (step index 0), now with Adam
    newP = m.unpack(m.get_params())
    mm, vv = m.get_adam()
    z = {k: np.zeros_like(v, dtype=np.float64) for k, v in P.items()}
    refP, refM, refV = oracle.adam_update(P, G, z, z, 1, cfg)
    lr = float(cfg.lr)
    for k in P:
        # the update step recomputes the gradient: entries whose terms cancel to the
        # FP32 rounding level may change sign, and the first Adam step is +-lr there
        firm = np.abs(G[k]) > 1e-3 * np.abs(G[k]).max()
        # FP32 update: the lr-sized step carries ~1e-7 relative rounding
        assert np.allclose(newP[k][firm], refP[k][firm], rtol=1e-6, atol=1e-5 * lr), k
        assert np.all(np.abs(newP[k] - P[k]) <= lr * (1 + 1e-5)), k
    for k, tol in (("W4", 1e-5), ("tables", 1e-5)):
        firm = np.abs(G[k]) > 1e-3 * np.abs(G[k]).max()
        assert np.allclose(m.unpack(mm)[k][firm], refM[k][firm], rtol=tol, atol=0), k
        assert np.allclose(m.unpack(vv)[k][firm], refV[k][firm], rtol=2 * tol, atol=0), k
    assert m.stats().step == 1
    # the next draw uses step index 1
    m.step(1000, seed=3, no_update=True)
    rid, t = m.samples()
    kfi, u, v = oracle.draw_rays(3, 1, 1000, [(kf.W, kf.H)])
    o, d = oracle.cast_rays_f32(np.broadcast_to(kf.c2w, (1000, 3, 4)), np.broadcast_to(kf.K, (1000, 4)), u, v)
    r_ref, _, t_ref, _ = oracle.march(cfg, o, d)
    assert np.array_equal(rid, r_ref) and np.array_equal(t, t_ref)


def test_render_parity_with_early_termination():
    cfg = synth.config_small(occ_res=0, render_t_min=np.float32(1e-2))
    P = synth.random_params(cfg, 8, table_scale=0.5, mlp_std=0.3)
    P["W2"][0] += 1.0                          # denser field: rays terminate early
    m = _map(cfg, P, [synth.c1_keyframe(0, W=8, H=8)])
    kf = synth.c1_keyframe(9, W=48, H=36)
    rgb, D, acc = m.render(kf.c2w, kf.K, 48, 36)
    I_ref, D_ref, A_ref = oracle.render(cfg, P, kf.c2w, kf.K, 48, 36, t_min=1e-2)
    _, _, A_full = oracle.render(cfg, P, kf.c2w, kf.K, 48, 36)
    assert np.mean(A_ref > 0.9) > 0.2 and np.abs(A_full - A_ref).max() > 1e-3   # termination matters
    assert np.allclose(rgb.reshape(-1, 3), I_ref, rtol=REL, atol=1e-6)
    assert np.allclose(D.ravel(), D_ref, rtol=REL, atol=1e-6)
    assert np.allclose(acc.ravel(), A_ref, rtol=REL, atol=1e-6)


def test_render_device_buffers_match_host():
    import torch
    cfg = synth.config_c1()
    P = synth.random_params(cfg, 1)
    m = _map(cfg, P, [synth.c1_keyframe(0)])
    kf = synth.c1_keyframe(2)
    rgb_h, d_h, a_h = m.render(kf.c2w, kf.K, 64, 48)
    out = torch.zeros((48, 64, 3), device="cuda")
    dep = torch.zeros((48, 64), device="cuda")
    m.render(kf.c2w, kf.K, 64, 48, out_rgb=out, out_depth=dep)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), rgb_h) and np.array_equal(dep.cpu().numpy(), d_h)


def test_occupancy_refresh_parity():
    cfg = synth.config_small(occ_res=16, occ_thresh=np.float32(1.5))
    P = synth.random_params(cfg, 12, table_scale=1.0, mlp_std=0.3)
    m = _map(cfg, P, [synth.c1_keyframe(0, W=8, H=8)])
    dens0 = np.random.default_rng(13).uniform(0, 0.03, 16 ** 3).astype(np.float32)
    m.set_occupancy_density(dens0)
    m.refresh_occupancy()
    m.refresh_occupancy()
    bits, dens = m.get_occupancy()
    d1, _, _ = oracle.occupancy_refresh(cfg, P, dens0.astype(np.float64), 0, cfg.seed)
    d2, bits_ref, _ = oracle.occupancy_refresh(cfg, P, d1, 1, cfg.seed)
    assert np.allclose(dens, d2, rtol=REL, atol=0)
    near = np.abs(d2 - float(cfg.occ_thresh)) < 1e-4 * float(cfg.occ_thresh)
    b_gpu = np.unpackbits(bits, bitorder="little").astype(bool)
    b_ref = np.unpackbits(bits_ref, bitorder="little").astype(bool)
    assert np.array_equal(b_gpu[~near], b_ref[~near])
    assert 0.05 < b_ref.mean() < 0.95


def test_edge_cases():
    from paper_2210_13641_gb300 import MapError, NerfMap
    cfg = synth.config_c1()
    P = synth.random_params(cfg, 2)
    m = NerfMap(cfg, occ_every=0)
    with pytest.raises(MapError) as e:
        m.step(16, seed=0)
    assert e.value.code == -3                  # no keyframes
    from paper_2210_13641_gb300 import pack_params
    m.set_params(pack_params(P))
    # camera outside the box looking away: no ray has a sample
    kf = synth.c1_keyframe(3)
    kf.c2w = synth.look_at_pose([3.0, 3.0, 3.0], [6.0, 6.0, 6.0])
    m.add_keyframe(kf)
    loss = m.step(100, seed=1, no_update=True)
    ref = oracle.forward_backward(cfg, P, [kf], 100, 1, 0)
    assert len(ref["t"]) == 0 and m.stats().n_samples == 0
    assert loss == pytest.approx(ref["loss"], rel=REL)
    assert not np.any(m.get_grads())
    with pytest.raises(MapError):
        m.step(0, seed=1)
    # replacing the keyframe by id changes what the next step sees
    kf2 = synth.c1_keyframe(4)
    kf2.kf_id = kf.kf_id
    m.add_keyframe(kf2)
    assert m.stats().n_keyframes == 1
    loss = m.step(1, seed=5, no_update=True)
    ref = oracle.forward_backward(cfg, P, [kf2], 1, 5, 0)
    assert loss == pytest.approx(ref["loss"], rel=REL)


@pytest.fixture(scope="module")
def room_workload():
    cfg = synth.config_c2(precision="fp32")
    room = synth.make_room(0)
    kfs = synth.room_keyframes(room, 20, seed=1)
    bits = synth.room_occupancy_bits(room, cfg.occ_res, cfg.grid_origin, cfg.grid_inv_size)
    P = synth.random_params(cfg, 0)
    return cfg, kfs, bits, P


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_full_size_room_step_sampled(room_workload, prec):
    """2^18 rays over 20 keyframes of 640x480 at L=16, T=2^19 with the 128^3
    bitfield (the benchmark's workload, in the benchmark's launch configuration):
    the sample lists of 512 sampled rays are bit-exact, their renders and loss terms
    match the oracle (FP32: 1e-5; FP16: 2e-3 against the oracle's FP16 rounding model), and the batch loss equals the mean of the per-ray terms."""
    cfg, kfs, bits, P = room_workload
    cfg = cfg.replace(precision=prec)
    tol = REL if prec == "fp32" else 2e-3
    n = 1 << 18
    m = _map(cfg, P, kfs, bits)
    loss = m.step(n, seed=21, no_update=True)
    rid, t = m.samples()
    rgb, D, acc = m.ray_outputs(n)
    kf, u, v = oracle.draw_rays(21, 0, n, [(k.W, k.H) for k in kfs])
    pick = np.sort(np.random.default_rng(22).choice(n, 512, replace=False))
    sub = (kf[pick], u[pick], v[pick])
    ref = oracle.forward_backward(cfg, P, kfs, 512, 0, 0, occ_bits=bits, rays=sub, want_grad=False,
                                  mlp_bits=prec)
    starts = np.searchsorted(rid, np.arange(n + 1))
    counts = np.diff(starts)
    assert np.array_equal(counts[pick], np.bincount(ref["ray_id"], minlength=512))
    t_gpu = np.concatenate([t[starts[r]:starts[r + 1]] for r in pick])
    assert np.array_equal(t_gpu, ref["t"])
    assert np.allclose(rgb[pick], ref["I_hat"], rtol=tol, atol=1e-6 if prec == "fp32" else tol)
    assert np.allclose(D[pick], ref["D_hat"], rtol=tol, atol=1e-6 if prec == "fp32" else tol)
    # whole-batch loss from the per-ray renders, targets taken by the oracle's draw
    I, Dt, V = oracle.ray_targets(kf, u, v, kfs)
    per_ray = ((I - rgb) ** 2).sum(1) + float(cfg.lambda_d) * (Dt - D) ** 2 / V
    assert loss == pytest.approx(per_ray.mean(), rel=REL)
    assert counts.mean() > 5


_ROOM_PLAIN = {}


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_full_size_room_backward(room_workload, prec):
    """The backward of the benchmark's workload (L=16, T=2^19, N up to 2048, the
    128^3 bitfield, 20 keyframes of 640x480) on 16384 rays, through the same
    launches as the benchmark's step: the field kernels' persistent grids are sized
    by the SM count, not by the batch, so the ~1M samples give every backward block
    about 26 tiles of 128 samples and every forward block about 13.  FP32: loss 1e-5,
    every gradient tensor 1e-5 relative and element-wise against grads_abs.  FP16 and
    BF16: loss and every gradient tensor 2e-3 against the oracle's rounding model of
    the format, and 2e-3 plus that model's distance from the plain oracle against the
    plain oracle."""
    cfg, kfs, bits, P = room_workload
    cfg = cfg.replace(precision=prec)
    n, seed = 16384, 23
    m = _map(cfg, P, kfs, bits)
    loss = m.step(n, seed=seed, no_update=True)
    if "plain" not in _ROOM_PLAIN:
        _ROOM_PLAIN["plain"] = oracle.forward_backward(cfg.replace(precision="fp32"), P, kfs, n, seed, 0,
                                                       occ_bits=bits, magnitudes=True)
    plain = _ROOM_PLAIN["plain"]
    rid, t = m.samples()
    assert np.array_equal(rid, plain["ray_id"].astype(np.uint32)) and np.array_equal(t, plain["t"])
    assert len(rid) > 40 * n
    G = m.unpack(m.get_grads())
    if prec == "fp32":
        _check_step(m, plain, n, loss)
        _check_grads(G, plain)
    else:
        ref = oracle.forward_backward(cfg, P, kfs, n, seed, 0, occ_bits=bits, mlp_bits=prec)
        assert loss == pytest.approx(ref["loss"], rel=2e-3) and loss == pytest.approx(plain["loss"], rel=2e-3)
        for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
            err = _rel(G[k], ref["grads"][k])
            floor = _rel(ref["grads"][k], plain["grads"][k])
            assert err <= 2e-3, (k, err)
            assert _rel(G[k], plain["grads"][k]) <= 2e-3 + floor, (k, err, floor)
    m.close()


def test_render_in_chunks_matches_oracle_on_sampled_pixels():
    """A 600x450 view (270k pixels, more than one 2^18-ray chunk): pixels on both
    sides of the chunk boundary equal the oracle's forward on the same rays."""
    cfg = synth.config_small(occ_res=0, render_t_min=np.float32(0.0))
    P = synth.random_params(cfg, 21, table_scale=0.5, mlp_std=0.3)
    m = _map(cfg, P, [synth.c1_keyframe(0, W=8, H=8)])
    W, H = 600, 450
    kf = synth.c1_keyframe(22, W=W, H=H)
    kf.K = np.array([400.0, 400.0, 300.0, 225.0], np.float32)
    rgb, D, acc = m.render(kf.c2w, kf.K, W, H)
    pix = np.concatenate([np.arange((1 << 18) - 300, (1 << 18) + 300),
                          np.random.default_rng(23).choice(W * H, 400, replace=False)])
    v, u = np.divmod(pix, W)
    ref = oracle.forward_backward(cfg, P, [kf], len(pix), 0, 0, rays=(np.zeros(len(pix), int), u, v),
                                  want_grad=False)
    assert np.allclose(rgb.reshape(-1, 3)[pix], ref["I_hat"], rtol=REL, atol=1e-6)
    assert np.allclose(D.ravel()[pix], ref["D_hat"], rtol=REL, atol=1e-6)
    assert np.allclose(acc.ravel()[pix], ref["acc"], rtol=REL, atol=1e-6)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_two_pass_render_with_early_termination(prec):
    """A dense field (most rays opaque within their first 32 samples) rendered with
    the termination threshold: the render evaluates the field for the first 32
    samples of each ray and then only for the rays still above the threshold
    (map_stats.render_evaluated well below render_samples), and the image matches the
    oracle's render with the same threshold (FP32 1e-5 plus the termination bound
    t_min x max(colour, far); FP16 2e-3 against the oracle's FP16 rounding model),
    the rays that stop after their first 32 samples included (the second pass
    evaluated more than the first pass's share)."""
    cfg = synth.config_small(precision=prec, occ_res=0, step=np.float32(0.01), n_steps=300, max_samples=256)
    P = synth.random_params(cfg, 31, table_scale=0.5, mlp_std=0.15)
    P["W2"][0] += 2.6     # denser: about 3/4 of the rays stop within 32 samples, the rest later
    m = _map(cfg, P, [synth.c1_keyframe(0, W=8, H=8)])
    kf = synth.c1_keyframe(33, W=40, H=30)
    rgb, D, acc = m.render(kf.c2w, kf.K, 40, 30)
    st = m.stats()
    o, d = oracle.render_rays_f32(np.asarray(kf.c2w, np.float32), np.asarray(kf.K, np.float32), 40, 30)
    n_r = np.bincount(oracle.march(cfg, o, d)[0], minlength=40 * 30)
    assert st.render_samples == n_r.sum() and n_r.mean() > 64
    first = np.minimum(n_r, 32).sum()
    assert first < st.render_evaluated < 0.7 * st.render_samples, (first, st.render_evaluated, st.render_samples)
    I_ref, D_ref, A_ref = oracle.render(cfg, P, kf.c2w, kf.K, 40, 30, t_min=float(cfg.render_t_min), mlp_bits=prec)
    # a ray whose transmittance passes the threshold within a rounding of it may stop
    # one sample earlier or later in FP32 than in FP64: that sample's weight is below
    # t_min, so the termination bound adds t_min x max(colour, far) to the tolerance
    t_min = float(cfg.render_t_min)
    far = float(cfg.near) + cfg.n_steps * float(cfg.step)
    tol = REL if prec == "fp32" else 2e-3
    a_c, a_d = (t_min, t_min * far) if prec == "fp32" else (2e-3, 2e-3)
    assert np.allclose(rgb.reshape(-1, 3), I_ref, rtol=tol, atol=a_c)
    assert np.allclose(D.ravel(), D_ref, rtol=tol, atol=a_d)
    assert np.allclose(acc.ravel(), A_ref, rtol=tol, atol=a_c)
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_maximum_samples_per_ray(prec):
    """The largest per-ray sample budget (max_samples = 1024): rays with hundreds of
    samples (many 32-sample chunks in the warp-per-ray march and compositing, many
    128-sample tiles per ray in the field kernels), some truncated at 1024, a ragged
    ray count; FP32 to the FP32 tolerance, FP16 to 2e-3 against the oracle's FP16
    rounding model."""
    cfg = synth.config_small(precision=prec, occ_res=0, step=np.float32(4e-4), n_steps=5000,
                             max_samples=1024)
    P = synth.random_params(cfg, 9, table_scale=0.05, mlp_std=0.1)
    kf = synth.c1_keyframe(70, W=20, H=15)
    m = _map(cfg, P, [kf])
    n = 301
    loss = m.step(n, seed=3, no_update=True)
    ref = oracle.forward_backward(cfg, P, [kf], n, 3, 0, mlp_bits=prec, magnitudes=prec == "fp32")
    counts = np.bincount(ref["ray_id"], minlength=n)
    assert counts.max() == 1024 and (counts == 1024).sum() > 10 and np.median(counts) > 300
    if prec == "fp32":
        _check_step(m, ref, n, loss)
        _check_grads(m.unpack(m.get_grads()), ref)
    else:
        rid, t = m.samples()
        assert np.array_equal(rid, ref["ray_id"].astype(np.uint32)) and np.array_equal(t, ref["t"])
        assert loss == pytest.approx(ref["loss"], rel=2e-3)
        rgb, D, acc = m.ray_outputs(n)
        assert np.allclose(rgb, ref["I_hat"], rtol=2e-3, atol=2e-3)
        assert np.allclose(D, ref["D_hat"], rtol=2e-3, atol=2e-3)
        G = m.unpack(m.get_grads())
        for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
            err = np.linalg.norm(G[k] - ref["grads"][k]) / np.linalg.norm(ref["grads"][k])
            assert err <= 2e-3, (k, err)
