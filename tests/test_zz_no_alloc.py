"""The allocation-free march entry point (map_march_noalloc).

map_march_noalloc serves callers that cannot allocate device memory (memory owned
by another allocator or a fixed budget, or a host loop that must not stall on a
cudaMalloc): its only scratch is a static device array, and every input and output
comes from the caller.  Its sample lists must equal, bit for bit, the ones
map_render produces for the same rays (the tolerance of all integer and index work
in these tests), on two calls in a row so that the second call runs over the first
call's leftovers in the shared scratch; at the room workload's march length they
must equal the oracle's march.  The calls must not change the device memory in use.
This file is collected last so that a failure here does not hide the other tests'
results.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2210_13641_gb300 import binding
    return binding.load()


def _view_rays(kf):
    """The pixel rays of a view, cast with the same FP32 operations as the GPU."""
    n = kf.W * kf.H
    v, u = np.divmod(np.arange(n), kf.W)
    o, d = oracle.cast_rays_f32(np.broadcast_to(kf.c2w, (n, 3, 4)), np.broadcast_to(kf.K, (n, 4)), u, v)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def _call(lib, ccfg, d_bits, d_o, d_d, n, offsets, rid, t, cap, stream):
    return lib.map_march_noalloc(ctypes.byref(ccfg), 0 if d_bits is None else d_bits, d_o.data_ptr(),
                                 d_d.data_ptr(), n, offsets.data_ptr(), rid.data_ptr(), t.data_ptr(), cap,
                                 stream.cuda_stream)


def test_march_noalloc_matches_map_march_twice(lib):
    import torch
    from paper_2210_13641_gb300 import NerfMap, binding, pack_params

    cfg = synth.config_small(occ_res=16, step=np.float32(0.02), n_steps=150)
    P = synth.random_params(cfg, 1)
    bits = np.packbits(np.random.default_rng(2).uniform(size=16 ** 3) < 0.5, bitorder="little")
    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    m.set_occupancy(bits)
    ccfg = binding.make_config(cfg, occ_every=0)
    d_bits = torch.from_numpy(bits).cuda()
    stream = torch.cuda.current_stream()

    for call, seed in enumerate((31, 32)):                 # two calls in a row
        kf = synth.c1_keyframe(seed, W=48 + 13 * call, H=37)
        m.render(kf.c2w, kf.K, kf.W, kf.H)
        ref_rid, ref_t = m.samples()
        n = kf.W * kf.H
        o, d = _view_rays(kf)
        cap = n * cfg.max_samples
        d_o, d_d = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
        offsets = torch.full((n + 1,), 0xFFFFFFFF, dtype=torch.int64).to(torch.int32).cuda()
        rid = torch.zeros(cap, dtype=torch.int32, device="cuda")
        t = torch.zeros(cap, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        used0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        rc = _call(lib, ccfg, d_bits.data_ptr(), d_o, d_d, n, offsets, rid, t, cap, stream)
        assert rc == 0, lib.map_last_error(None)
        torch.cuda.synchronize()
        if call == 1:
            # the second call (the library's kernels and the scratch address already
            # loaded) takes no device memory: neither from torch nor from the driver
            assert torch.cuda.memory_allocated() == used0
            assert torch.cuda.mem_get_info()[0] == free0
        off = offsets.cpu().numpy().view(np.uint32)
        total = int(off[n])
        assert total == len(ref_rid) and total > n
        assert np.array_equal(np.diff(off), np.bincount(ref_rid, minlength=n))
        assert np.array_equal(rid.cpu().numpy()[:total].view(np.uint32), ref_rid)
        assert np.array_equal(t.cpu().numpy()[:total], ref_t)

    # sizes beyond the static scratch are refused with a message
    rc = lib.map_march_noalloc(ctypes.byref(ccfg), d_bits.data_ptr(), d_o.data_ptr(), d_d.data_ptr(),
                               (1 << 20) + 1, offsets.data_ptr(), rid.data_ptr(), t.data_ptr(),
                               ((1 << 20) + 1) * cfg.max_samples, stream.cuda_stream)
    assert rc == binding.MAP_EINVAL and b"scratch" in lib.map_last_error(None)
    # a bitfield that is not 4-byte aligned (an offset into a byte tensor) is refused
    # on the host, before any launch
    rc = _call(lib, ccfg, d_bits.data_ptr() + 1, d_o, d_d, n, offsets, rid, t, cap, stream)
    assert rc == binding.MAP_EINVAL and b"aligned" in lib.map_last_error(None)
    # a later successful call clears the message
    rc = _call(lib, ccfg, d_bits.data_ptr(), d_o, d_d, n, offsets, rid, t, cap, stream)
    assert rc == 0 and lib.map_last_error(None) == b""
    torch.cuda.synchronize()
    m.close()


def test_march_noalloc_room_length_matches_oracle(lib):
    """The room workload's march (1024 steps per ray, at most 128 samples, the 128^3
    bitfield of the analytic surfaces) on 8192 rays of camera poses inside the room:
    offsets, ray ids and sample distances equal the oracle's march bit for bit."""
    import torch
    from paper_2210_13641_gb300 import binding

    cfg = synth.config_c2(precision="fp32")
    room = synth.make_room(0)
    bits = synth.room_occupancy_bits(room, cfg.occ_res, cfg.grid_origin, cfg.grid_inv_size)
    poses = synth.room_spline_poses(room, 4, seed=3)
    rng = np.random.default_rng(4)
    n = 8192
    K = np.array([525.0, 525.0, 320.0, 240.0], np.float32)
    pose_of = rng.integers(0, len(poses), n)
    u, v = rng.integers(0, 640, n), rng.integers(0, 480, n)
    c2w = np.stack([poses[j] for j in pose_of]).astype(np.float32)
    o, d = oracle.cast_rays_f32(c2w, np.broadcast_to(K, (n, 4)), u, v)
    o, d = np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)
    ref_rid, _, ref_t, _ = oracle.march(cfg, o, d, bits)

    ccfg = binding.make_config(cfg, occ_every=0)
    stream = torch.cuda.current_stream()
    d_bits = torch.from_numpy(bits).cuda()
    d_o, d_d = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    cap = n * cfg.max_samples
    offsets = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    rid = torch.zeros(cap, dtype=torch.int32, device="cuda")
    t = torch.zeros(cap, dtype=torch.float32, device="cuda")
    rc = _call(lib, ccfg, d_bits.data_ptr(), d_o, d_d, n, offsets, rid, t, cap, stream)
    assert rc == 0, lib.map_last_error(None)
    torch.cuda.synchronize()
    off = offsets.cpu().numpy().view(np.uint32)
    total = int(off[n])
    counts = np.bincount(ref_rid, minlength=n)
    assert total == len(ref_rid) and counts.mean() > 20 and counts.max() == cfg.max_samples
    assert np.array_equal(np.diff(off), counts)
    assert np.array_equal(rid.cpu().numpy()[:total].view(np.uint32), ref_rid.astype(np.uint32))
    assert np.array_equal(t.cpu().numpy()[:total].view(np.uint32), ref_t.astype(np.float32).view(np.uint32))
