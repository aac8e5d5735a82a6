"""The fused backward behind torch.autograd, checked against central finite
differences of the GPU's own loss (plain FP32 form) and against the oracle.

FP32 loss evaluations carry ~1e-7 relative rounding, so with h = 1e-3 a central
difference has an absolute error of ~1e-7 * |L| / h; entries are compared within
2e-2 relative plus that noise floor, and kinks (one-sided differences that
disagree) are skipped."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_autograd_gradient_matches_finite_differences_and_oracle():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2210_13641_gb300 import NerfMap, pack_params
    from paper_2210_13641_gb300.autograd import mapping_loss

    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 11, table_scale=0.3, mlp_std=0.3)
    kf = synth.c1_keyframe(12, W=16, H=12)
    kf.K = np.array([12.0, 12.0, 8.0, 6.0], np.float32)
    m = NerfMap(cfg, occ_every=0)
    m.add_keyframe(kf)
    n_rays, seed = 48, 13
    p = torch.from_numpy(pack_params(P)).cuda().requires_grad_(True)
    loss = mapping_loss(p, m, n_rays, seed)
    (3.0 * loss).backward()
    g = p.grad.detach().cpu().numpy() / 3.0
    ref = oracle.forward_backward(cfg, P, [kf], n_rays, seed, 0)
    assert float(loss) == pytest.approx(ref["loss"], rel=1e-5)
    G = m.unpack(g.copy())
    for k in ("tables", "W1", "W4"):
        assert np.linalg.norm(G[k] - ref["grads"][k]) <= 1e-5 * np.linalg.norm(ref["grads"][k])

    base = pack_params(P).astype(np.float32)
    L0 = float(loss)
    rng = np.random.default_rng(14)
    nt = cfg.n_levels * cfg.table_size * 2
    used = np.nonzero(np.abs(g[:nt]) > 1e-3 * np.abs(g[:nt]).max())[0]
    picks = list(rng.choice(used, 12, replace=False)) + list(nt + rng.choice(9408, 12, replace=False))
    h = 1e-3

    def L(idx, dv):
        q = base.copy()
        q[idx] += dv
        with torch.no_grad():
            return float(mapping_loss(torch.from_numpy(q).cuda(), m, n_rays, seed))

    checked = 0
    for idx in picks:
        lp, lm = L(idx, h), L(idx, -h)
        fwd, bwd = (lp - L0) / h, (L0 - lm) / h
        if abs(fwd - bwd) > 5e-2 * max(abs(fwd), abs(bwd)) + 1e-3:
            continue
        fd = (lp - lm) / (2 * h)
        noise = 1e-6 * abs(L0) / h
        assert g[idx] == pytest.approx(fd, rel=2e-2, abs=noise + 1e-6), idx
        checked += 1
    assert checked >= 16
    m.close()
