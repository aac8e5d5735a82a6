"""Pins of the oracle's pose gradient (joint pose refinement: the mapping loss is
minimised over the keyframe poses too, Sec. 3.2): the SH Jacobian and the encoding's
position derivative against central differences of the functions themselves, and the
per-keyframe pose gradient against central differences of the batch loss with that
keyframe moved (sample list held fixed).  CPU only."""

import numpy as np
import pytest

import oracle
import synth


def test_sh_jacobian_matches_central_differences():
    rng = np.random.default_rng(0)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    J = oracle.sh_deg4_jacobian(d)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3); e[a] = h
        fd = (oracle.sh_deg4(d + e) - oracle.sh_deg4(d - e)) / (2 * h)
        assert np.abs(J[:, :, a] - fd).max() < 1e-8


def test_encoding_position_derivative_matches_central_differences():
    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 1, table_scale=0.5)
    lr = oracle.level_resolutions(cfg)
    rng = np.random.default_rng(2)
    x = rng.uniform(0.05, 0.95, size=(200, 3))
    # keep points away from every level's cell boundaries (the encoding is only C0 there)
    h = 1e-7
    ok = np.ones(len(x), bool)
    for N in lr:
        q = x * N
        ok &= np.all(np.abs(q - np.round(q)) > 1e-4, axis=1)
    x = x[ok]
    J = oracle.hash_encode_dx(cfg, lr, P["tables"], x.astype(np.float32).astype(np.float64))
    for a in range(3):
        e = np.zeros(3); e[a] = h
        xx = x.astype(np.float32).astype(np.float64)
        fd = (oracle.hash_encode_f64(cfg, lr, P["tables"], xx + e)
              - oracle.hash_encode_f64(cfg, lr, P["tables"], xx - e)) / (2 * h)
        scale = np.abs(J[:, :, a]).max()
        assert np.abs(J[:, :, a] - fd).max() < 1e-6 * scale


def _pose_case():
    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 5, table_scale=0.3, mlp_std=0.3)
    kfs = []
    for j in range(2):
        kf = synth.c1_keyframe(30 + j, W=12, H=10, kf_id=j)
        kf.K = np.array([9.0, 9.0, 6.0, 5.0], np.float32)
        kfs.append(kf)
    return cfg, P, kfs


def test_pose_gradient_matches_central_differences():
    cfg, P, kfs = _pose_case()
    pg = oracle.pose_gradients(cfg, P, kfs, 64, 3, 0)
    fb = pg["fb"]
    h = 1e-6
    checked = 0
    for k in range(2):
        for comp in range(6):
            e = np.zeros(6); e[comp] = h
            L = lambda s: oracle.loss_moved_samples(cfg, P, fb, s * e[:3], s * e[3:], k)
            lp, l0, lm = L(1.0), L(0.0), L(-1.0)
            fwd, bwd = (lp - l0) / h, (l0 - lm) / h
            if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd)) + 1e-6:
                continue                                   # a sample crossed a cell or ReLU kink
            fd = (lp - lm) / (2 * h)
            assert pg["pose_grads"][k, comp] == pytest.approx(fd, rel=1e-4, abs=1e-7), (k, comp)
            checked += 1
    assert checked >= 9
    # the rotation part is not a copy of the translation part, and both are non-trivial
    assert np.abs(pg["pose_grads"][:, :3]).max() > 1e-3 and np.abs(pg["pose_grads"][:, 3:]).max() > 1e-3


def test_pose_gradient_sign_convention():
    """A planted mistake (the rotation term's cross products flipped) fails the pin."""
    cfg, P, kfs = _pose_case()
    pg = oracle.pose_gradients(cfg, P, kfs, 64, 3, 0)
    fb = pg["fb"]
    o, d = fb["o"].astype(np.float64), fb["d"].astype(np.float64)
    sel = fb["kf"] == 0
    wrong = (np.cross(pg["g_o"][sel], o[sel]) + np.cross(pg["g_d"][sel], d[sel])).sum(0)
    h = 1e-6
    fds = []
    for comp in range(3):
        e = np.zeros(3); e[comp] = h
        fds.append((oracle.loss_moved_samples(cfg, P, fb, np.zeros(3), e, 0)
                    - oracle.loss_moved_samples(cfg, P, fb, np.zeros(3), -e, 0)) / (2 * h))
    fds = np.array(fds)
    assert np.linalg.norm(pg["pose_grads"][0, 3:] - fds) < 1e-3 * np.linalg.norm(fds)
    assert np.linalg.norm(wrong - fds) > 0.5 * np.linalg.norm(fds)
