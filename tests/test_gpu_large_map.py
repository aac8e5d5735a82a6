"""The large-map configuration (L=16, T=2^22 per level, N 16..8192, 256^3 occupancy,
a 20 x 20 x 3 m multi-room floor, 1200x680 keyframes) in all three MLP forms against
the FP64 oracle on a 4096-ray batch: bit-exact sample lists; loss, per-ray colour,
depth and opacity, and every gradient tensor within the forms' tolerances (FP32:
1e-5 relative, per-tensor relative L2 for gradients; FP16 and BF16: 2e-3 against
the oracle's rounding model of the MLP precision, and gradients within 2e-3 plus the
model's own distance from the plain FP64 oracle against that oracle, as in
test_gpu_tc.py); and a render of a 1200x680 view subsampled to 120x68 pixels against
the oracle's render of the same rays.

The keyframes are rendered on the GPU (synth.multiroom) and copied to the host, and
both sides consume those arrays.  When NERFMAP_PRECISION_REPORT names a file the
measured errors are appended to it."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth.multiroom import make_multiroom, multiroom_poses, occupancy_bits_torch, render_keyframes_torch

pytestmark = pytest.mark.gpu

W, H = 1200, 680
K = np.array([600.0, 600.0, 600.0, 340.0], np.float32)
TOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-3}
_PLAIN = {}


@pytest.fixture(scope="module")
def scene():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    room = make_multiroom(0)
    poses = multiroom_poses(room, 3, seed=1)
    kfs = []
    for kf, rgb, depth, var in render_keyframes_torch(room, poses, W, H, K, seed=2, device="cuda"):
        kf.rgb, kf.depth, kf.var = rgb.cpu().numpy(), depth.cpu().numpy(), var.cpu().numpy()
        kfs.append(kf)
    cfg = synth.config_c5("fp32")
    bits = occupancy_bits_torch(room, cfg.occ_res, cfg.grid_origin, cfg.grid_inv_size, device="cuda")
    P = synth.random_params(cfg, 4, table_scale=0.5, mlp_std=0.15)
    return room, kfs, bits, P


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _report(case, prec, errs):
    path = os.environ.get("NERFMAP_PRECISION_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": case, "precision": prec, **errs}) + "\n")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_large_map_step_matches_oracle(scene, prec):
    from paper_2210_13641_gb300 import NerfMap, pack_params
    room, kfs, bits, P = scene
    cfg = synth.config_c5(prec)
    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    m.set_occupancy(bits)
    for kf in kfs:
        m.add_keyframe(kf)
    n, seed = 4096, 11
    loss = m.step(n, seed=seed, no_update=True)
    ref = oracle.forward_backward(cfg, P, kfs, n, seed, 0, occ_bits=bits, mlp_bits=prec)
    if prec != "fp32" and "grads" not in _PLAIN:
        _PLAIN.update(oracle.forward_backward(cfg.replace(precision="fp32"), P, kfs, n, seed, 0, occ_bits=bits))
    rid, t = m.samples()
    assert len(rid) > 20 * n                      # the batch really marches the occupied shells
    assert np.array_equal(rid, ref["ray_id"].astype(np.uint32)) and np.array_equal(t, ref["t"])
    rgb, D, acc = m.ray_outputs(n)
    G = m.unpack(m.get_grads())
    errs = {"samples": int(len(rid)), "loss": abs(loss - ref["loss"]) / abs(ref["loss"]),
            "rgb_max_abs": float(np.abs(rgb - ref["I_hat"]).max()),
            "depth_rel": _rel(D, ref["D_hat"]), "acc_max_abs": float(np.abs(acc - ref["acc"]).max())}
    for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
        errs["grad_" + k] = _rel(G[k], ref["grads"][k])
        if prec != "fp32":
            errs["plain_grad_" + k] = _rel(G[k], _PLAIN["grads"][k])
            errs["floor_grad_" + k] = _rel(ref["grads"][k], _PLAIN["grads"][k])
    _report("c5_large_map", prec, errs)
    tol = TOL[prec]
    assert errs["loss"] <= tol, errs
    assert np.allclose(rgb, ref["I_hat"], rtol=tol, atol=tol)
    assert np.allclose(D, ref["D_hat"], rtol=tol, atol=tol)
    assert np.allclose(acc, ref["acc"], rtol=tol, atol=tol)
    for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
        assert errs["grad_" + k] <= tol, (k, errs)
        if prec != "fp32":
            assert errs["plain_grad_" + k] <= tol + errs["floor_grad_" + k], (k, errs)
    # render: a 120x68 view with the intrinsics of a 1200x680 camera scaled by 1/10
    pose = multiroom_poses(room, 1, seed=7)[0]
    Kr = K / 10.0
    out_rgb, out_D, out_acc = m.render(pose, Kr, 120, 68)
    I_ref, D_ref, A_ref = oracle.render(cfg, P, pose, Kr, 120, 68, occ_bits=bits,
                                        t_min=float(cfg.render_t_min),
                                        mlp_bits=prec)
    rerr = {"render_rgb_max_abs": float(np.abs(out_rgb.reshape(-1, 3) - I_ref).max()),
            "render_depth_rel": _rel(out_D.ravel(), D_ref)}
    _report("c5_large_map_render", prec, rerr)
    assert np.allclose(out_rgb.reshape(-1, 3), I_ref, rtol=tol, atol=tol), rerr
    assert np.allclose(out_D.ravel(), D_ref, rtol=tol, atol=tol), rerr
    assert np.allclose(out_acc.ravel(), A_ref, rtol=tol, atol=tol), rerr
    m.close()
