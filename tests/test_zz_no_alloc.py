"""The allocation-free march entry point (map_march_noalloc) against the map's own
march.

map_march_noalloc serves callers that cannot allocate device memory: its only
scratch is a static device array, and every input and output comes from the
caller.  Its sample lists must equal, bit for bit, the ones map_render produces for
the same rays (the tolerance of all integer and index work in these tests), on two
calls in a row so that the second call runs over the first call's leftovers in the
shared scratch.  This file is collected last so that a failure here does not hide
the other tests' results.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _view_rays(kf):
    """The pixel rays of a view, cast with the same FP32 operations as the GPU."""
    n = kf.W * kf.H
    v, u = np.divmod(np.arange(n), kf.W)
    o, d = oracle.cast_rays_f32(np.broadcast_to(kf.c2w, (n, 3, 4)), np.broadcast_to(kf.K, (n, 4)), u, v)
    return np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32)


def test_march_noalloc_matches_map_march_twice():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2210_13641_gb300 import NerfMap, binding, pack_params
    lib = binding.load()

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
        rc = lib.map_march_noalloc(ctypes.byref(ccfg), d_bits.data_ptr(), d_o.data_ptr(), d_d.data_ptr(), n,
                                   offsets.data_ptr(), rid.data_ptr(), t.data_ptr(), cap, stream.cuda_stream)
        assert rc == 0, lib.map_last_error(None)
        torch.cuda.synchronize()
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
    m.close()
