"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test fixes one part of the oracle against a closed form, an invariant, a
published value, brute force or finite differences, chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one of them.
"""

import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
f32 = np.float32


# ------------------------------------------------------------------ RNG

def test_splitmix64_published_sequence():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    states = np.array([(k * oracle.SM_GAMMA) % 2 ** 64 for k in range(4)], dtype=np.uint64)
    got = [int(v) for v in oracle.splitmix64(states)]
    assert got == want


def test_ray_draw_uniform_and_in_range():
    sizes = [(64, 48), (10, 7), (33, 5)]
    kf, u, v = oracle.draw_rays(3, 7, 30000, sizes)
    assert kf.min() >= 0 and kf.max() == 2
    for j, (W, H) in enumerate(sizes):
        m = kf == j
        assert u[m].max() < W and v[m].max() < H and u[m].min() >= 0 and v[m].min() >= 0
        assert abs(m.mean() - 1 / 3) < 0.02          # uniform over keyframes
    # different steps draw different batches
    kf2, u2, _ = oracle.draw_rays(3, 8, 30000, sizes)
    assert np.mean((kf2 == kf) & (u2 == u)) < 0.1


# ------------------------------------------------------------------ ray casting

def test_cast_rays_reproject_to_pixel_centre():
    rng = np.random.default_rng(1)
    c2w = synth.random_pose(rng)
    K = np.array([50, 60, 31.0, 22.5], f32)
    u = rng.integers(0, 64, 500)
    v = rng.integers(0, 48, 500)
    o, d = oracle.cast_rays_f32(np.broadcast_to(c2w, (500, 3, 4)), np.broadcast_to(K, (500, 4)), u, v)
    assert np.allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1, atol=1e-6)
    R = c2w[:, :3].astype(np.float64)
    pc = (o + 2.0 * d - c2w[:, 3]) @ R               # world -> camera
    px = K[0] * pc[:, 0] / pc[:, 2] + K[2]
    py = K[1] * pc[:, 1] / pc[:, 2] + K[3]
    assert np.allclose(px, u + 0.5, atol=1e-4) and np.allclose(py, v + 0.5, atol=1e-4)
    assert np.all(pc[:, 2] > 0)                      # looking along +z (OpenCV)


def test_depth_targets_z_to_ray_distance():
    kf = synth.c1_keyframe(0)
    kf.depth_is_z = True
    u = np.array([0, 31, 63]); v = np.array([0, 23, 47]); j = np.zeros(3, int)
    I, D, V = oracle.ray_targets(j, u, v, [kf])
    fx, fy, cx, cy = kf.K
    for a in range(3):
        ray = np.array([(u[a] + .5 - cx) / fx, (v[a] + .5 - cy) / fy, 1.0])
        pt = ray * kf.depth[v[a], u[a]]              # camera-space point at z-depth
        assert D[a] == pytest.approx(np.linalg.norm(pt), rel=1e-12)
        assert V[a] == pytest.approx(kf.var[v[a], u[a]] * ray @ ray, rel=1e-12)
    assert np.array_equal(I, kf.rgb[v, u])


# ------------------------------------------------------------------ march

def test_march_counts_match_slab_intersection():
    cfg = synth.config_c1()
    rng = np.random.default_rng(2)
    n = 400
    kf = synth.c1_keyframe(5)
    u = rng.integers(0, 64, n); v = rng.integers(0, 48, n)
    o, d = oracle.cast_rays_f32(np.broadcast_to(kf.c2w, (n, 3, 4)), np.broadcast_to(kf.K, (n, 4)), u, v)
    ray_id, step, t, x = oracle.march(cfg, o, d)
    counts = np.bincount(ray_id, minlength=n)
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    with np.errstate(divide="ignore"):
        a = (0 - o64) / d64
        b = (1 - o64) / d64
    t_in = np.max(np.minimum(a, b), axis=1)
    t_out = np.min(np.maximum(a, b), axis=1)
    ti = float(cfg.near) + np.arange(cfg.n_steps) * float(cfg.step)
    checked = 0
    for r in range(n):
        gap = np.minimum(np.abs(ti - t_in[r]), np.abs(ti - t_out[r]))
        if gap.min() < 1e-5:
            continue                                  # a sample on the box face: skip
        want = int(np.sum((ti >= t_in[r]) & (ti < t_out[r])))
        assert counts[r] == want, r
        checked += 1
    assert checked > 300
    # samples are in ray-major order and positions lie inside the box
    assert np.all(np.diff(ray_id) >= 0)
    assert np.all((x >= 0) & (x < 1))


def test_march_single_occupied_cell_and_truncation():
    cfg = synth.config_small(occ_res=4, max_samples=3, step=f32(0.03), n_steps=96)
    bits = np.zeros(8, np.uint8)
    cell = (1, 2, 3)
    b = cell[0] + 4 * (cell[1] + 4 * cell[2])
    bits[b >> 3] |= 1 << (b & 7)
    rng = np.random.default_rng(3)
    o = rng.uniform(0.05, 0.95, (2000, 3)).astype(f32)
    d = rng.normal(size=(2000, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True); d = d.astype(f32)
    ray_id, step, t, x = oracle.march(cfg, o, d, bits)
    cells = np.floor(x.astype(np.float64) * 4).astype(int)
    assert len(ray_id) > 0
    assert np.all(cells == np.array(cell))
    assert np.bincount(ray_id).max() <= 3
    # without truncation some ray keeps more than 3 samples in that cell
    r2, _, _, _ = oracle.march(cfg.replace(max_samples=64), o, d, bits)
    assert np.bincount(r2).max() > 3


# ------------------------------------------------------------------ hash grid

def test_level_resolutions_golden():
    rows = {l.split()[0]: [int(a) for a in l.split()[1:]] for l in open(os.path.join(GOLDEN, "level_res.txt"))
            if l.strip() and not l.startswith("#")}
    assert oracle.level_resolutions(synth.config_c1()) == rows["c1"]
    c2 = oracle.level_resolutions(synth.config_c2())
    assert c2[0] == rows["c2_first"][0] and c2[-1] == rows["c2_last"][0]
    assert all(b > a for a, b in zip(c2, c2[1:]))


def test_dense_index_bijection():
    N, T = 8, 1024
    g = np.stack(np.meshgrid(*[np.arange(N + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    idx = oracle.vertex_index(g, N, T)
    assert sorted(idx.tolist()) == list(range((N + 1) ** 3))
    assert oracle.vertex_index(np.array([1, 0, 0]), N, T) == 1
    assert oracle.vertex_index(np.array([0, 1, 0]), N, T) == N + 1
    assert oracle.vertex_index(np.array([0, 0, 1]), N, T) == (N + 1) ** 2


def test_hash_structure():
    N, T = 100, 1 << 12                               # 101^3 > 4096: hashed
    vi = lambda *c: int(oracle.vertex_index(np.array(c), N, T))
    assert vi(0, 0, 0) == 0
    assert vi(37, 0, 0) == 37                          # first prime is 1
    assert vi(0, 1, 0) == 0x9E3779B1 % T               # 2654435761
    assert vi(0, 2, 0) == (2 * 0x9E3779B1 - 2 ** 32) % T  # uint32 wrap-around
    assert vi(0, 0, 1) == 805459861 % T
    for a, b, c in [(3, 5, 7), (99, 1, 64), (12, 77, 3)]:
        assert vi(a, b, c) == (a ^ ((b * 2654435761) & 0xFFFFFFFF) ^ ((c * 805459861) & 0xFFFFFFFF)) % T
    g = np.random.default_rng(0).integers(0, N + 1, (200000, 3))
    h = np.bincount(oracle.vertex_index(g, N, T), minlength=T)
    chi2 = np.sum((h - h.mean()) ** 2 / h.mean())
    assert chi2 < T + 6 * math.sqrt(2 * T)             # uniform bucket fill


def _affine_tables(cfg, level_res, A, B):
    """Tables whose vertex v at level l stores A[l,f] . v + B[l,f] (collision-free
    levels only)."""
    tab = np.zeros((cfg.n_levels, cfg.table_size, cfg.n_features))
    for l, N in enumerate(level_res):
        g = np.stack(np.meshgrid(*[np.arange(N + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
        idx = oracle.vertex_index(g, N, cfg.table_size)
        for f in range(cfg.n_features):
            tab[l, idx, f] = g @ A[l, f] + B[l, f]
    return tab


def test_trilinear_reproduces_affine_field():
    cfg = synth.config_small(log2_table=16)            # all four levels dense
    lr = oracle.level_resolutions(cfg)
    rng = np.random.default_rng(4)
    A = rng.normal(size=(4, 2, 3)); B = rng.normal(size=(4, 2))
    tab = _affine_tables(cfg, lr, A, B)
    x = rng.uniform(0, 1, (1000, 3)).astype(f32)
    feat, idx, w = oracle.hash_encode(cfg, lr, tab, x)
    assert np.allclose(w.sum(-1), 1, atol=1e-14) and np.all(w >= 0)
    for l, N in enumerate(lr):
        q = x.astype(f32) * f32(N)
        for f in range(2):
            want = q.astype(np.float64) @ A[l, f] + B[l, f]
            assert np.allclose(feat[:, l * 2 + f], want, atol=1e-10)
    assert np.all(feat[:, 8:] == 0)                    # zero padding to 32


def test_trilinear_on_hashed_level_brute_force():
    cfg = synth.config_small()                         # levels 2, 3 hashed (T = 1024)
    lr = oracle.level_resolutions(cfg)
    rng = np.random.default_rng(5)
    tab = rng.normal(size=(4, 1024, 2))
    x = rng.uniform(0, 1, (50, 3)).astype(f32)
    feat, _, _ = oracle.hash_encode(cfg, lr, tab, x)
    for s in range(50):                                # one corner at a time, by hand
        for l in (2, 3):
            N = lr[l]
            p = float(f32(x[s, 0]) * f32(N)), float(f32(x[s, 1]) * f32(N)), float(f32(x[s, 2]) * f32(N))
            c = [min(int(math.floor(a)), N - 1) for a in p]
            acc = np.zeros(2)
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        wgt = ((p[0] - c[0]) if dx else (1 - p[0] + c[0])) * \
                              ((p[1] - c[1]) if dy else (1 - p[1] + c[1])) * \
                              ((p[2] - c[2]) if dz else (1 - p[2] + c[2]))
                        v = (c[0] + dx, c[1] + dy, c[2] + dz)
                        h = (v[0] ^ ((v[1] * 2654435761) % 2 ** 32) ^ ((v[2] * 805459861) % 2 ** 32)) % 1024
                        acc += wgt * tab[l, h]
            assert np.allclose(feat[s, 2 * l:2 * l + 2], acc, atol=1e-12)


# ------------------------------------------------------------------ SH

def test_sh_orthonormal_by_quadrature():
    ct, wt = np.polynomial.legendre.leggauss(24)
    phi = np.arange(48) * 2 * np.pi / 48
    C, P = np.meshgrid(ct, phi, indexing="ij")
    W = np.meshgrid(wt, phi, indexing="ij")[0] * (2 * np.pi / 48)
    st = np.sqrt(1 - C ** 2)
    d = np.stack([st * np.cos(P), st * np.sin(P), C], -1).reshape(-1, 3)
    Y = oracle.sh_deg4(d)
    G = (Y * W.reshape(-1, 1)).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_addition_theorem_and_constant():
    d = np.random.default_rng(6).normal(size=(100, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_deg4(d)
    assert np.allclose(Y[:, 0], 1 / (2 * math.sqrt(math.pi)), atol=0)
    for l in range(4):
        band = Y[:, l * l:(l + 1) * (l + 1)]
        assert np.allclose((band ** 2).sum(1), (2 * l + 1) / (4 * math.pi), atol=1e-13)
    # band 1 is proportional to the direction itself
    assert np.allclose(Y[:, 2], math.sqrt(3 / (4 * math.pi)) * d[:, 2])


# ------------------------------------------------------------------ MLPs

def test_mlp_hand_built_weights():
    P = {"W1": np.zeros((64, 32)), "W2": np.zeros((16, 64)), "W3": np.zeros((64, 32)),
         "W4": np.zeros((64, 64)), "W5": np.zeros((3, 64))}
    P["W1"][:32, :] = np.eye(32)
    P["W1"][32:, :] = -np.eye(32)                       # h1 = [relu(f); relu(-f)]
    P["W2"][0, :] = 1.0                                 # h_0 = sum |f|
    P["W2"][1, :32] = 1.0                               # h_1 = sum relu(f)
    P["W3"][np.arange(32), np.arange(32)] = 1.0         # h3 = relu([h; sh]) (first 32)
    P["W4"][np.arange(64), (np.arange(64) + 1) % 64] = 1.0   # h4_i = relu(h3_{i+1})
    P["W5"][0, 16] = 1.0                                # z0 = h4_16 = relu(sh_1)
    P["W5"][1, 0] = 2.0                                 # z1 = 2 h4_0 = 2 relu(h_1)
    P["W5"][2, 63] = -1.0                               # z2 = -h4_63 = -relu(h3_0) = -relu(h_0)
    f = np.array([[0.3, -0.2] + [0.0] * 29 + [0.1]])
    dvec = np.array([[0.0, -0.6, 0.8]])
    sh = oracle.sh_deg4(dvec)
    fw = oracle.field_forward(P, f, sh)
    s_abs, s_pos = 0.6, 0.4
    assert fw["sigma"][0] == pytest.approx(math.exp(s_abs), rel=1e-14)
    sig = lambda z: 1 / (1 + math.exp(-z))
    sh1 = -math.sqrt(3 / (4 * math.pi)) * (-0.6)
    assert fw["rgb"][0, 0] == pytest.approx(sig(sh1), rel=1e-14)
    assert fw["rgb"][0, 1] == pytest.approx(sig(2 * s_pos), rel=1e-14)
    assert fw["rgb"][0, 2] == pytest.approx(sig(-s_abs), rel=1e-14)


# ------------------------------------------------------------------ compositing

def test_constant_density_transmittance_closed_form():
    sigma, delta, t0, N = 1.7, 0.09, 0.1, 32
    t = t0 + np.arange(N) * delta
    c = np.tile([[0.2, 0.5, 0.9]], (N, 1))
    I, D, acc, w, T = oracle.composite_ray(np.full(N, sigma), c, t, delta)
    assert np.allclose(T, np.exp(-sigma * (t - t0)), rtol=1e-14)
    assert acc == pytest.approx(1 - math.exp(-sigma * N * delta), rel=1e-13)
    q = math.exp(-sigma * delta)
    a = 1 - q
    s0 = (1 - q ** N) / (1 - q)
    s1 = q * (1 - N * q ** (N - 1) + (N - 1) * q ** N) / (1 - q) ** 2
    assert D == pytest.approx(a * (t0 * s0 + delta * s1), rel=1e-13)
    assert np.allclose(I, acc * np.array([0.2, 0.5, 0.9]), rtol=1e-13)


def test_opaque_slab_renders_its_depth():
    delta, t0, N = 0.01, 0.1, 300
    t = t0 + np.arange(N) * delta
    a, b = 1.2345, 1.6
    sigma = np.where((t >= a) & (t <= b), 1e4, 0.0)
    c = np.where(((t >= a) & (t <= b))[:, None], [0.3, 0.6, 0.1], [1.0, 1.0, 1.0])
    I, D, acc, w, T = oracle.composite_ray(sigma, c, t, delta)
    tk = t[np.argmax(t >= a)]
    assert D == pytest.approx(tk, abs=1e-6)
    assert acc == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(I, [0.3, 0.6, 0.1], atol=1e-12)


def test_weights_nonnegative_and_bounded():
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = rng.integers(1, 200)
        sig = rng.exponential(rng.uniform(0.1, 50), n)
        I, D, acc, w, T = oracle.composite_ray(sig, rng.uniform(0, 1, (n, 3)), np.arange(n) * 0.05, 0.05)
        assert np.all(w >= 0) and w.sum() <= 1 + 1e-15 and np.all(np.diff(T) <= 0)


def test_early_termination_error_bound():
    rng = np.random.default_rng(8)
    sig = rng.exponential(5.0, 120)
    c = rng.uniform(0, 1, (120, 3)); t = 0.1 + np.arange(120) * 0.05
    I0, D0, _, _, _ = oracle.composite_ray(sig, c, t, 0.05)
    I1, D1, _, _, _ = oracle.composite_ray(sig, c, t, 0.05, t_min=1e-4)
    assert np.all(np.abs(I1 - I0) <= 1e-4) and abs(D1 - D0) <= 1e-4 * t[-1]


# ------------------------------------------------------------------ loss

def test_loss_special_cases():
    I = np.array([[1.0, 0, 0]]); Ih = np.array([[0.5, 0, 0]])
    L, _ = oracle.mapping_loss(Ih, np.array([1.0]), I, np.array([2.0]), np.array([4.0]), 1.0)
    assert L == pytest.approx(0.25 + 1.0 / 4.0, rel=1e-15)
    rng = np.random.default_rng(9)
    I = rng.uniform(size=(10, 3)); Ih = rng.uniform(size=(10, 3))
    D = rng.uniform(1, 2, 10); Dh = rng.uniform(1, 2, 10)
    L_inf, _ = oracle.mapping_loss(Ih, Dh, I, D, np.full(10, 1e300), 1.0)
    assert L_inf == pytest.approx(((I - Ih) ** 2).sum(1).mean(), rel=1e-12)   # colour only
    L_raw, _ = oracle.mapping_loss(Ih, Dh, I, D, np.ones(10), 1.0)
    assert L_raw == pytest.approx(((I - Ih) ** 2).sum(1).mean() + ((D - Dh) ** 2).mean(), rel=1e-12)


# ------------------------------------------------------------------ gradients

def test_composite_backward_one_sample_closed_form():
    s, dl, tt = 0.7, 0.3, 1.1
    c = np.array([[0.2, 0.4, 0.6]])
    I, D, acc, w, T = oracle.composite_ray(np.array([s]), c, np.array([tt]), dl)
    gI, gD = np.array([1.0, -2.0, 0.5]), 0.3
    dsig, drgb = oracle.composite_backward_ray(np.array([s]), c, np.array([tt]), dl, w, T, gI, gD)
    e = math.exp(-s * dl)
    assert dsig[0] == pytest.approx(dl * e * (c[0] @ gI + gD * tt), rel=1e-14)
    assert np.allclose(drgb[0], (1 - e) * gI, rtol=1e-14)


def test_composite_backward_finite_differences():
    rng = np.random.default_rng(10)
    n, dl = 17, 0.07
    sig = rng.exponential(3.0, n); c = rng.uniform(0, 1, (n, 3)); t = 0.2 + dl * np.arange(n)
    gI, gD = rng.normal(size=3), rng.normal()
    f = lambda s, cc: (lambda r: r[0] @ gI + gD * r[1])(oracle.composite_ray(s, cc, t, dl))
    I, D, acc, w, T = oracle.composite_ray(sig, c, t, dl)
    dsig, drgb = oracle.composite_backward_ray(sig, c, t, dl, w, T, gI, gD)
    h = 1e-6
    for i in range(n):
        e = np.zeros(n); e[i] = h
        assert dsig[i] == pytest.approx((f(sig + e, c) - f(sig - e, c)) / (2 * h), rel=1e-6, abs=1e-10)
        for ch in range(3):
            E = np.zeros((n, 3)); E[i, ch] = h
            assert drgb[i, ch] == pytest.approx((f(sig, c + E) - f(sig, c - E)) / (2 * h), rel=1e-6, abs=1e-10)


def _tiny_problem():
    cfg = synth.config_small(occ_res=0)
    P = synth.random_params(cfg, 11, table_scale=0.3, mlp_std=0.3)
    P = {k: v.astype(np.float64) for k, v in P.items()}
    kf = synth.c1_keyframe(12, W=16, H=12)
    kf.K = np.array([12.0, 12.0, 8.0, 6.0], f32)
    return cfg, P, kf


def test_full_gradient_central_differences():
    """Analytic gradient of L_M vs central differences (h = 1e-4, FP64) on 64 random
    hash entries and MLP weights; kinks (one-sided differences that disagree) are
    skipped."""
    cfg, P, kf = _tiny_problem()
    n_rays = 48
    out = oracle.forward_backward(cfg, P, [kf], n_rays, 13, 0)
    assert len(out["t"]) > 100
    G = out["grads"]
    rng = np.random.default_rng(14)
    L0 = out["loss"]
    checked = 0
    used = set(np.unique(np.nonzero(np.abs(G["tables"]) > 0)[1]).tolist())
    picks = []
    for _ in range(40):
        l = rng.integers(0, 4)
        nz = np.nonzero(np.abs(G["tables"][l, :, 0]) > 0)[0]
        picks.append(("tables", (l, rng.choice(nz), rng.integers(0, 2))))
    for name in ("W1", "W2", "W3", "W4", "W5"):
        for _ in range(5 if name != "W5" else 4):
            picks.append((name, tuple(rng.integers(0, s) for s in P[name].shape)))
    assert len(picks) == 64 and used
    h = 1e-4
    for name, ix in picks:
        def L(dv):
            Q = {k: v.copy() for k, v in P.items()}
            Q[name][ix] += dv
            return oracle.loss_only(cfg, Q, [kf], n_rays, 13, 0)
        lp, lm = L(h), L(-h)
        fwd, bwd = (lp - L0) / h, (L0 - lm) / h
        if abs(fwd - bwd) > 1e-3 * max(abs(fwd), abs(bwd), 1e-8) + 1e-9:
            continue                                   # a ReLU kink inside [-h, h]
        fd = (lp - lm) / (2 * h)
        g = G[name][ix]
        assert g == pytest.approx(fd, rel=1e-4, abs=1e-7 * max(1.0, abs(L0))), (name, ix)
        checked += 1
    assert checked >= 56


# ------------------------------------------------------------------ Adam

def test_adam_first_step_is_sign_step_and_second_step_by_hand():
    cfg = synth.config_c1()
    g = np.array([1e-3, -2.0, 0.0, 5e-9])
    P = {"p": np.array([1.0, 1.0, 1.0, 1.0])}
    z = {"p": np.zeros(4)}
    P1, M1, V1 = oracle.adam_update(P, {"p": g}, z, z, 1, cfg)
    lr = float(cfg.lr); eps = float(cfg.eps)
    assert np.allclose(P1["p"], 1 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-16)
    assert P1["p"][2] == 1.0
    g2 = np.array([2e-3, 1.0, 0.0, 0.0])
    P2, _, _ = oracle.adam_update(P1, {"p": g2}, M1, V1, 2, cfg)
    b1, b2 = float(cfg.beta1), float(cfg.beta2)
    m = b1 * (1 - b1) * g + (1 - b1) * g2
    v = b2 * (1 - b2) * g * g + (1 - b2) * g2 * g2
    want = P1["p"] - lr * (m / (1 - b1 ** 2)) / (np.sqrt(v / (1 - b2 ** 2)) + eps)
    assert np.allclose(P2["p"], want, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ occupancy

def test_occupancy_refresh_positions_bits_and_decay():
    cfg = synth.config_small(occ_res=8)
    P = synth.random_params(cfg, 15)
    dens0 = np.random.default_rng(16).uniform(0, 0.02, 512)
    newd, bits, x = oracle.occupancy_refresh(cfg, P, dens0, 3, 99)
    cells = np.floor(x.astype(np.float64) * 8).astype(int)
    want_cells = np.stack([np.arange(512) % 8, (np.arange(512) // 8) % 8, np.arange(512) // 64], 1)
    assert np.array_equal(cells, want_cells)            # one point inside each cell
    assert np.all(newd >= float(cfg.occ_decay) * dens0)
    assert np.array_equal(np.unpackbits(bits, bitorder="little").astype(bool), newd > float(cfg.occ_thresh))
    # with the density MLP forced to sigma = exp(-50) the EMA only decays
    Q = dict(P); Q["W2"] = np.zeros_like(P["W2"]); Q["W2"][0, 0] = 0.0
    Q["W1"] = np.zeros_like(P["W1"])
    newd2, _, _ = oracle.occupancy_refresh(cfg, Q, dens0 + 2.0, 0, 1)
    assert np.allclose(newd2, float(cfg.occ_decay) * (dens0 + 2.0), rtol=1e-15)


def test_render_matches_training_forward_on_same_rays():
    cfg, P, kf = _tiny_problem()
    I, D, A = oracle.render(cfg, P, kf.c2w, kf.K, kf.W, kf.H)
    v, u = np.divmod(np.arange(kf.W * kf.H), kf.W)
    out = oracle.forward_backward(cfg, P, [kf], kf.W * kf.H, 0, 0,
                                  rays=(np.zeros(kf.W * kf.H, int), u, v), want_grad=False)
    assert np.allclose(I, out["I_hat"], rtol=1e-14) and np.allclose(D, out["D_hat"], rtol=1e-14)


def test_gradient_magnitudes_bound_the_gradients():
    """grads_abs (sum of |terms|) bounds |grad| entry by entry and equals it where
    no term changes sign (a single-sample, single-ray batch of the plain chain)."""
    cfg, P, kf = _tiny_problem()
    out = oracle.forward_backward(cfg, P, [kf], 64, 13, 0, magnitudes=True)
    for k, g in out["grads"].items():
        assert np.all(np.abs(g) <= out["grads_abs"][k] * (1 + 1e-12) + 1e-300), k
    assert all(np.any(out["grads_abs"][k] > np.abs(out["grads"][k]) * 1.01) for k in ("W1", "W4"))


def test_round_sig_matches_the_library_conversions():
    """round_sig(x, 11) is IEEE binary16's rounding and round_sig(x, 8) bfloat16's
    (round to nearest, ties to even) for values in those formats' normal ranges:
    checked against numpy's float16 conversion and torch's bfloat16 conversion of
    float32 inputs, with ties placed on purpose."""
    import torch
    rng = np.random.default_rng(31)
    x = (rng.uniform(-1, 1, 20000) * np.exp2(rng.integers(-13, 15, 20000))).astype(np.float32)
    ties = np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, -(2 + 2 ** -10), 1 + 2 ** -9, 1 + 3 * 2 ** -9], np.float32)
    x = np.concatenate([x, ties])
    normal16 = np.abs(x) >= 2.0 ** -14                    # binary16's normal range
    assert normal16.mean() > 0.9
    f16 = x[normal16].astype(np.float16).astype(np.float64)
    assert np.array_equal(oracle.round_sig(x[normal16], 11), f16)
    b16 = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_sig(x, 8), b16)
    assert oracle.round_sig(np.array([1 + 2 ** -9]), 8)[0] == 1.0          # tie to even
    assert oracle.round_sig(np.array([0.0]), 8)[0] == 0.0


def _c1_problem():
    cfg = synth.config_c1()
    return cfg, synth.random_params(cfg, 0), synth.c1_keyframe(0)


def test_rounding_model_is_the_plain_chain_at_full_precision():
    """With 53 significant bits the rounding is the identity, and the rounded-operand
    forward and backward equal the plain FP64 chain bit for bit (so everything but
    the rounding is the pinned plain chain); with fewer bits the error falls as the
    significand grows."""
    cfg, P, kf = _c1_problem()
    plain = oracle.forward_backward(cfg, P, [kf], 1024, 7, 0)
    full = oracle.forward_backward(cfg, P, [kf], 1024, 7, 0, mlp_bits=53)
    assert full["loss"] == plain["loss"]
    for k in plain["grads"]:
        assert np.array_equal(full["grads"][k], plain["grads"][k]), k
    errs = []
    for bits in (8, 11, 16, 21, 26):
        m = oracle.forward_backward(cfg, P, [kf], 1024, 7, 0, mlp_bits=bits)
        errs.append(max(np.linalg.norm(m["grads"][k] - plain["grads"][k]) / np.linalg.norm(plain["grads"][k])
                        for k in plain["grads"]))
        assert abs(m["loss"] - plain["loss"]) <= 2.0 ** -bits * abs(plain["loss"])
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert errs[3] < 1e-5 and errs[0] > 1e-3


def test_rounding_model_rounds_every_operand():
    """The forward's rounding sites: a layer whose operands are exactly representable
    in the operand type gives the plain result, and perturbing the weights or the
    features by less than half a unit of the type's last place (operands that are
    dyadic with few bits sit far from a rounding boundary) leaves the rounded
    forward unchanged while the plain forward moves."""
    rng = np.random.default_rng(32)
    shapes = {"W1": (64, 32), "W2": (16, 64), "W3": (64, 32), "W4": (64, 64), "W5": (3, 64)}
    P = {k: rng.integers(-4, 5, s) / 8.0 for k, s in shapes.items()}
    feat = rng.integers(-8, 9, (50, 32)) / 16.0
    sh = rng.integers(-8, 9, (50, 16)) / 16.0
    plain = oracle.field_forward(P, feat, sh)
    m = oracle.field_forward(P, feat, sh, bits=11)
    assert np.array_equal(m["a1"], plain["a1"])          # dyadic operands: exact in 11 bits
    Q = dict(P)
    Q["W1"] = P["W1"] * (1 + 2.0 ** -14)                  # below half an FP16 ulp
    assert np.array_equal(oracle.field_forward(Q, feat, sh, bits=11)["a1"], m["a1"])
    assert not np.array_equal(oracle.field_forward(Q, feat, sh)["a1"], plain["a1"])
    f2 = feat * (1 + 2.0 ** -14)
    assert np.array_equal(oracle.field_forward(P, f2, sh, bits=11)["a1"], m["a1"])


def test_mlp_precision_floor_on_the_c1_step():
    """The error floor of an MLP with FP16 / BF16 operands against the plain FP64
    oracle, from the oracle alone: on the C1 step (4096 rays) the rounding model
    moves the table gradient by more than 2e-3 relative in both formats (a
    pre-activation within a rounding of zero takes the other ReLU branch and changes
    its sample's whole contribution), so 2e-3 against the plain oracle is out of
    reach for any MLP that rounds its operands; the GPU tests hold the kernels to
    2e-3 against this model and to 2e-3 plus this floor against the plain oracle."""
    cfg, P, kf = _c1_problem()
    plain = oracle.forward_backward(cfg, P, [kf], 4096, 7, 0)
    floor = {}
    for prec in ("fp16", "bf16"):
        m = oracle.forward_backward(cfg, P, [kf], 4096, 7, 0, mlp_bits=prec)
        floor[prec] = {k: np.linalg.norm(m["grads"][k] - plain["grads"][k]) / np.linalg.norm(plain["grads"][k])
                       for k in plain["grads"]}
    assert floor["fp16"]["tables"] > 2e-3 and floor["bf16"]["tables"] > 2e-3
    assert max(floor["bf16"].values()) > 5 * 2e-3 / 2
    assert all(floor["bf16"][k] > floor["fp16"][k] for k in floor["fp16"])


def test_near_kink_samples_flag_pre_activations_at_zero():
    """near_kink_samples flags a sample exactly when one of its ReLU pre-activations
    (or h_0 against the density cap) is within the tolerance of zero relative to the
    sum of its terms' magnitudes: built here with one unit cancelling exactly, one
    just outside the tolerance and one sample far from every kink."""
    shapes = {"W1": (64, 32), "W2": (16, 64), "W3": (64, 32), "W4": (64, 64), "W5": (3, 64)}
    P = {k: np.zeros(s) for k, s in shapes.items()}
    P["W1"][:, 0] = 1.0                                   # every layer-1 unit = f0 + ...
    P["W1"][0, 1] = -1.0                                  # ... unit 0 = f0 - f1
    feat = np.zeros((3, 32))
    feat[:, 0] = 1.0
    feat[0, 1] = 1.0                                      # sample 0: unit 0 is exactly 0
    feat[1, 1] = 1.0 - 3e-5                               # sample 1: |a| = 3e-5, terms sum to ~2
    feat[2, 1] = -1.0                                     # sample 2: unit 0 = 2
    sh = np.zeros((3, 16))
    sh[:, 0] = 1.0
    P["W3"][:, 16] = 1.0                                  # layer-3 units = sh_0 = 1: no kink
    P["W4"][:, 0] = 1.0
    fw = oracle.field_forward(P, feat, sh)
    assert list(oracle.near_kink_samples(P, fw)) == [True, False, False]
    assert list(oracle.near_kink_samples(P, fw, tol=2e-5)) == [True, True, False]


def test_density_cap_is_opaque_and_flat():
    """sigma = exp(min(h_0, 15)): above the cap the value is exp(15) and the loss
    does not depend on h_0 (zero derivative, checked by central differences)."""
    P = {"W1": np.zeros((64, 32)), "W2": np.zeros((16, 64)), "W3": np.zeros((64, 32)),
         "W4": np.zeros((64, 64)), "W5": np.zeros((3, 64))}
    P["W1"][0, 0] = 1.0
    P["W2"][0, 0] = 20.0                                 # h_0 = 20 * relu(f_0)
    f = np.zeros((1, 32)); f[0, 0] = 1.0
    sh = np.zeros((1, 16))
    fw = oracle.field_forward(P, f, sh)
    assert fw["sigma"][0] == pytest.approx(math.exp(15.0), rel=1e-15)
    g, _ = oracle.field_backward(P, fw, np.array([1.0]), np.zeros((1, 3)))
    assert g["W2"][0, 0] == 0.0 and g["W1"][0, 0] == 0.0
    P["W2"][0, 0] = 10.0                                 # below the cap: d sigma / d h_0 = sigma
    fw = oracle.field_forward(P, f, sh)
    g, _ = oracle.field_backward(P, fw, np.array([1.0]), np.zeros((1, 3)))
    assert g["W2"][0, 0] == pytest.approx(math.exp(10.0), rel=1e-12)
