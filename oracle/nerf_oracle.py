"""FP64 oracle of one NeRF-SLAM mapping step (test infrastructure only).

What it computes, in the paper's order (arXiv 2210.13641, Sec. 3.2 "Mapping:
Probabilistic Volumetric NeRF", Sec. 3.3 "Architecture", Sec. 3.4 "Implementation
Details"):

  a1  draw rays uniformly over all keyframes received (Sec. 3.3: the mapping thread
      optimises all keyframes) and cast them through the pinhole camera;
  a2  sample 3D positions along each ray (Sec. 3.2, depth rendering) on a uniform
      grid t_i = t_0 + i*Delta, keep those inside the box and in occupied cells;
  a3  encode each position with the multiresolution hash grid of Instant-NGP
      (Sec. 3.4 names it as the map) - trilinear interpolation of per-level tables;
  a4  encode the view direction with real spherical harmonics, bands 0..3;
  a5  density MLP, sigma = exp(h_0);  a6  colour MLP with a sigmoid output;
  a7  alpha compositing of colour and expected depth with the transmittance of
      Eq. (transmittance) - Sec. 3.2 equations for d* and I*;
  a8  mapping loss L_M = L_rgb + lambda_D * L_D of Eq. (mapping_loss), colour L2 and
      the Sigma_D-weighted squared depth residual;
  a9-a11 the analytic gradient of L_M with respect to the map parameters Theta;
  a12 Adam on Theta;  a13 occupancy refresh;  a14 forward-only render.

Precision rule: the geometry that decides integers (ray casting, sample positions,
box and occupancy tests, grid cells) is evaluated in IEEE float32 with a fixed
operation order, the precision the GPU kernels use, so both sides take every
integer decision identically.  Everything after that is FP64.

Readings of the paper (where it is silent or defers to Instant-NGP) are listed in
the repository's design notes; the ones that fix arithmetic here are: Sigma_D is a
per-pixel variance and the depth residual is divided by it; the colour loss sums
the three channels; both losses are averaged over rays; delta_i = Delta for every
sample including the last; samples outside the box or in empty cells are dropped
(equivalently sigma = 0); background colour 0.

Parity status: every function below is pinned by the not-gpu tests (closed forms,
invariants, brute force, finite differences, the published SplitMix64 output
sequence).  One constant set is "parity unpinned": the three spatial-hash primes of
vertex_index are taken from the cited Instant-NGP paper (the NeRF-SLAM paper does
not restate them); the tests pin the hash's structure (first prime 1, uint32
wrap-around, xor of the axis terms, uniform bucket fill) but nothing outside this
file fixes the primes' digits.
"""

from __future__ import annotations

import math

import numpy as np

f32 = np.float32
U64 = np.uint64
MASK32 = 0xFFFFFFFF

# ------------------------------------------------------------------ a1: counter RNG

# SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; the output function as published in
# Vigna's splitmix64.c): state advances by the golden gamma, then two xor-shift /
# odd-multiply rounds.  Used as a counter-based generator: output = mix(seed ^ ctr).
SM_GAMMA = 0x9E3779B97F4A7C15
SM_M1 = 0xBF58476D1CE4E5B9
SM_M2 = 0x94D049BB133111EB
OCC_STREAM = 1 << 30


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state z (uint64 array), wrap-around arithmetic."""
    z = np.asarray(z, dtype=U64)
    with np.errstate(over="ignore"):
        z = z + U64(SM_GAMMA)
        z = (z ^ (z >> U64(30))) * U64(SM_M1)
        z = (z ^ (z >> U64(27))) * U64(SM_M2)
    return z ^ (z >> U64(31))


def counter_rand(seed: int, stream: int, index: np.ndarray, k: int) -> np.ndarray:
    """u64 random number for (seed, stream, index, k): counter = stream<<33 | index<<1 | k."""
    index = np.asarray(index, dtype=U64)
    ctr = (U64(stream) << U64(33)) | (index << U64(1)) | U64(k)
    return splitmix64(U64(seed) ^ ctr)


def draw_rays(seed: int, step: int, n_rays: int, kf_sizes):
    """Uniform draw with replacement over (keyframe, pixel), Sec. 3.3 (all keyframes
    are optimised).  kf_sizes = [(W, H), ...] in insertion order.  Returns keyframe
    index, u, v (int64 arrays)."""
    r = np.arange(n_rays, dtype=U64)
    n_kf = len(kf_sizes)
    r0 = counter_rand(seed, step, r, 0)
    r1 = counter_rand(seed, step, r, 1)
    kf = (r0 % U64(n_kf)).astype(np.int64)
    Ws = np.array([s[0] for s in kf_sizes], dtype=U64)
    Hs = np.array([s[1] for s in kf_sizes], dtype=U64)
    pix = r1 % (Ws[kf] * Hs[kf])
    u = (pix % Ws[kf]).astype(np.int64)
    v = (pix // Ws[kf]).astype(np.int64)
    return kf, u, v


def cast_rays_f32(c2w: np.ndarray, K: np.ndarray, u: np.ndarray, v: np.ndarray):
    """Pinhole back-projection Pi^-1 of the pixel centre (u+1/2, v+1/2) (Sec. 3.1
    projection model), rotated to world and normalised; float32, fixed op order.
    c2w [N,3,4], K [N,4] -> origin o [N,3], unit direction d [N,3] (float32)."""
    c2w = c2w.astype(f32)
    K = K.astype(f32)
    dx = ((u.astype(f32) + f32(0.5)) - K[:, 2]) / K[:, 0]
    dy = ((v.astype(f32) + f32(0.5)) - K[:, 3]) / K[:, 1]
    R = c2w[:, :, :3]
    w = [(R[:, a, 0] * dx + R[:, a, 1] * dy) + R[:, a, 2] for a in range(3)]
    n = np.sqrt((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2])
    d = np.stack([w[0] / n, w[1] / n, w[2] / n], axis=1)
    o = c2w[:, :, 3].copy()
    return o, d


def ray_targets(kf, u, v, keyframes):
    """Targets I (3), D, Sigma_D of each drawn ray in ray-distance units (FP64).

    A z-depth D_z of pixel (u,v) lies at distance D_z * ||K^-1 [u+1/2, v+1/2, 1]||
    along the unit ray, and its variance scales with the square of that factor."""
    n = len(kf)
    I = np.zeros((n, 3))
    D = np.zeros(n)
    V = np.zeros(n)
    for j, k in enumerate(keyframes):
        m = kf == j
        if not np.any(m):
            continue
        uu, vv = u[m], v[m]
        I[m] = k.rgb[vv, uu].astype(np.float64)
        z = k.depth[vv, uu].astype(np.float64)
        var = k.var[vv, uu].astype(np.float64)
        if k.depth_is_z:
            fx, fy, cx, cy = [float(a) for a in k.K]
            sx = (uu + 0.5 - cx) / fx
            sy = (vv + 0.5 - cy) / fy
            s = np.sqrt(sx * sx + sy * sy + 1.0)
            D[m] = z * s
            V[m] = var * s * s
        else:
            D[m] = z
            V[m] = var
    return I, D, V


# ------------------------------------------------------------------ a2: march

def occupancy_bit(bits: np.ndarray, res: int, x: np.ndarray) -> np.ndarray:
    """Bit of the occupancy cell holding grid position x [N,3] (float32).
    Cell c_a = min(floor(x_a * res), res-1); linear index cx + res*(cy + res*cz);
    bit (b & 7) of byte (b >> 3)."""
    q = x * f32(res)
    c = np.minimum(np.floor(q).astype(np.int64), res - 1)
    c = np.maximum(c, 0)
    b = c[:, 0] + res * (c[:, 1] + res * c[:, 2])
    return ((bits[b >> 3] >> (b & 7).astype(np.uint8)) & 1).astype(bool)


def sample_positions_f32(cfg, o, d, i):
    """t_i = t_0 + i*Delta and the grid position x = (o + t d - origin) * inv_size,
    float32 with this exact operation order.  i: int array broadcast against rays."""
    t = f32(cfg.near) + i.astype(f32) * f32(cfg.step)
    p = o[..., None, :] + t[..., None] * d[..., None, :]
    x = (p - cfg.grid_origin.astype(f32)) * f32(cfg.grid_inv_size)
    return t, x


def march(cfg, o, d, occ_bits=None):
    """Sec. 3.2: sample positions along each ray.  Steps i = 0..n_steps-1; a step is
    kept when 0 <= x_a < box_a on every axis and (with a bitfield) its cell is
    occupied; the first max_samples kept steps of each ray are its samples.
    Returns ray id [S], step index [S], t [S] (float32), x [S,3] (float32), all in
    ray-major order."""
    n = o.shape[0]
    i = np.arange(cfg.n_steps)
    t, x = sample_positions_f32(cfg, o, d, np.broadcast_to(i, (n, cfg.n_steps)))
    box = cfg.box_max.astype(f32)
    keep = np.all((x >= f32(0)) & (x < box), axis=-1)
    if occ_bits is not None and cfg.occ_res > 0:
        flat = x.reshape(-1, 3)
        occ = np.zeros(flat.shape[0], bool)
        kf = keep.reshape(-1)
        occ[kf] = occupancy_bit(occ_bits, cfg.occ_res, flat[kf])
        keep &= occ.reshape(keep.shape)
    rank = np.cumsum(keep, axis=1) - 1
    keep &= rank < cfg.max_samples
    ray_id, step_idx = np.nonzero(keep)
    return ray_id, step_idx, t[ray_id, step_idx], x[ray_id, step_idx]


# ------------------------------------------------------------------ a3: hash grid

PI1, PI2, PI3 = 1, 2654435761, 805459861   # spatial-hash primes of Instant-NGP


def level_resolutions(cfg) -> list:
    """N_l = floor(N_min * b^l), b = growth or exp(ln(N_max/N_min)/(L-1)).  A 1e-9
    relative nudge keeps exactly-integral products (16 * 2^(7*15/15) = 2048) from
    flooring one below through FP64 rounding."""
    L = cfg.n_levels
    if cfg.growth is not None:
        b = float(cfg.growth)
    else:
        b = math.exp(math.log(cfg.n_max / cfg.n_min) / (L - 1))
    return [int(math.floor(cfg.n_min * b ** l * (1 + 1e-9))) for l in range(L)]


def vertex_index(c: np.ndarray, N: int, T: int) -> np.ndarray:
    """Table slot of integer grid vertices c [...,3] at resolution N (coords 0..N).
    Dense when the (N+1)^3 vertices fit in T slots: cx + cy(N+1) + cz(N+1)^2;
    otherwise the spatial hash (cx*pi1 xor cy*pi2 xor cz*pi3) mod 2^32 mod T."""
    c = c.astype(np.int64)
    if (N + 1) ** 3 <= T:
        return c[..., 0] + (N + 1) * (c[..., 1] + (N + 1) * c[..., 2])
    h = ((c[..., 0] * PI1) & MASK32) ^ ((c[..., 1] * PI2) & MASK32) ^ ((c[..., 2] * PI3) & MASK32)
    return (h & MASK32) % T


CORNERS = np.array([[(k >> 0) & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)])


def grid_cell_f32(x: np.ndarray, N: int):
    """Cell and fractional offset of x [S,3] at resolution N: q = x*N (float32),
    c = min(floor(q), N-1), w = q - c (exact).  Returns c int64 [S,3], w FP64 [S,3]."""
    q = x.astype(f32) * f32(N)
    c = np.minimum(np.floor(q).astype(np.int64), N - 1)
    w = q.astype(np.float64) - c
    return c, w


def hash_encode(cfg, level_res, tables: np.ndarray, x: np.ndarray):
    """Multiresolution grid encoding (Instant-NGP, the map named in Sec. 3.4).
    x [S,3] float32 in [0,1).  Returns features [S, enc_width] (FP64, zero padded
    beyond L*F), slot indices [S, L, 8] and trilinear weights [S, L, 8]."""
    S = x.shape[0]
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    feat = np.zeros((S, cfg.enc_width))
    idx = np.zeros((S, L, 8), dtype=np.int64)
    wts = np.zeros((S, L, 8))
    tab = tables.astype(np.float64)
    for l in range(L):
        N = level_res[l]
        c, w = grid_cell_f32(x, N)
        for k in range(8):
            b = CORNERS[k]
            wk = np.prod(np.where(b[None, :] == 1, w, 1.0 - w), axis=1)
            ik = vertex_index(c + b[None, :], N, T)
            idx[:, l, k] = ik
            wts[:, l, k] = wk
            feat[:, l * F:(l + 1) * F] += wk[:, None] * tab[l, ik]
    return feat, idx, wts


# ------------------------------------------------------------------ a4: SH

def sh_deg4(d: np.ndarray) -> np.ndarray:
    """Real spherical harmonics Y_l^m, l = 0..3 (16 values), of unit directions d
    [S,3]; orthonormal on the sphere, Condon-Shortley phase.  Each constant is the
    normalisation sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0)
    of the associated Legendre closed form."""
    x, y, z = d[:, 0].astype(np.float64), d[:, 1].astype(np.float64), d[:, 2].astype(np.float64)
    pi = math.pi
    out = np.empty((d.shape[0], 16))
    out[:, 0] = 0.5 * math.sqrt(1 / pi)
    a1 = math.sqrt(3 / (4 * pi))
    out[:, 1] = -a1 * y
    out[:, 2] = a1 * z
    out[:, 3] = -a1 * x
    out[:, 4] = 0.5 * math.sqrt(15 / pi) * x * y
    out[:, 5] = -0.5 * math.sqrt(15 / pi) * y * z
    out[:, 6] = 0.25 * math.sqrt(5 / pi) * (3 * z * z - 1)
    out[:, 7] = -0.5 * math.sqrt(15 / pi) * x * z
    out[:, 8] = 0.25 * math.sqrt(15 / pi) * (x * x - y * y)
    out[:, 9] = -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y)
    out[:, 10] = 0.5 * math.sqrt(105 / pi) * x * y * z
    out[:, 11] = -0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1)
    out[:, 12] = 0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3)
    out[:, 13] = -0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1)
    out[:, 14] = 0.25 * math.sqrt(105 / pi) * z * (x * x - y * y)
    out[:, 15] = -0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y)
    return out


# ------------------------------------------------------------------ a5, a6: MLPs

# Density activation: sigma = exp(min(h_0, 15)), the exponential with its value
# capped (a reading: the paper defers the activation to its map).  Beyond h_0 = 15 a
# sample is opaque already (sigma * delta > 10^4 at any spacing used here); the cap
# keeps sigma finite in FP32 and its derivative there is zero.  (Instant-NGP's
# "truncated exponential" is a different rule: it clamps only the argument of the
# derivative.)
SIGMA_H_MAX = 15.0

def relu(a):
    return np.maximum(a, 0.0)


# MLP operand precision (the benchmark spec's precision pattern: the MLP multiplies
# FP16 or BF16 operands and accumulates in FP32; everything else stays FP32).  The
# oracle's model of such an MLP rounds every operand of every product - weights,
# layer inputs and, in the backward pass, the gradient operands - to the operand
# type's significand (11 bits for FP16, 8 for BF16, round to nearest even, exponent
# range unbounded) and sums the products exactly (FP64).  It is a model of the
# number format, not of any kernel: no scaling, no saturation, no accumulation
# order.  With the rounding an identity it is the plain FP64 chain.
MLP_BITS = {"fp16": 11, "bf16": 8}


def bits_of(precision):
    """Significand bits of an MLP precision name (None / "fp32": no rounding)."""
    if precision is None or precision == "fp32":
        return None
    if isinstance(precision, (int, np.integer)):
        return int(precision)
    return MLP_BITS[precision]


def round_sig(x, bits):
    """x rounded to `bits` significant bits (round to nearest, ties to even), with
    no exponent limit: x = m 2^e with 1/2 <= |m| < 1, m rounded to a multiple of
    2^-bits.  Exact in FP64 for bits <= 53 (the rescalings are powers of two)."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def field_forward(P: dict, feat: np.ndarray, sh: np.ndarray, bits=None) -> dict:
    """sigma_i and c_i from one evaluation of the MLPs at the sample (Sec. 3.2: both
    are estimated simultaneously).  Density MLP: h = W2 relu(W1 feat), sigma =
    exp(min(h_0, 15)).  Colour MLP on [h; SH]: c = sigmoid(W5 relu(W4 relu(W3 [h; SH]))).
    No biases.  With `bits` every MLP operand (weights and layer inputs) is rounded
    to that many significant bits before its products (round_sig); sigma and the
    colour come from the exactly summed products.  Returns every intermediate (the
    rounded operands where rounded) for the backward pass."""
    R = (lambda a: a) if bits is None else (lambda a: round_sig(a, bits))
    W = {k: R(P[k].astype(np.float64)) for k in ("W1", "W2", "W3", "W4", "W5")}
    f = R(np.asarray(feat, np.float64))
    a1 = f @ W["W1"].T
    m1 = a1 > 0
    h1 = R(np.where(m1, a1, 0.0))
    h = h1 @ W["W2"].T
    sigma = np.exp(np.minimum(h[:, 0], SIGMA_H_MAX))
    x3 = R(np.concatenate([h, sh], axis=1))
    a3 = x3 @ W["W3"].T
    m3 = a3 > 0
    h3 = R(np.where(m3, a3, 0.0))
    a4 = h3 @ W["W4"].T
    m4 = a4 > 0
    h4 = R(np.where(m4, a4, 0.0))
    z = h4 @ W["W5"].T
    rgb = 1.0 / (1.0 + np.exp(-z))
    return dict(feat=f, a1=a1, m1=m1, h1=h1, h=h, sigma=sigma, x3=x3, a3=a3, m3=m3, h3=h3,
                a4=a4, m4=m4, h4=h4, z=z, rgb=rgb, W=W, bits=bits)


# ------------------------------------------------------------------ a7: compositing

def composite_ray(sigma, rgb, t, delta, t_min=None):
    """Sec. 3.2 for one ray: alpha_i = 1 - exp(-sigma_i delta), transmittance
    T_i = exp(-sum_{j<i} sigma_j delta) (Eq. transmittance), weight w_i = T_i alpha_i,
    I* = sum w_i c_i, d* = sum w_i t_i, acc = sum w_i.  With t_min (render only) the
    sum stops at the first sample whose T_i < t_min."""
    tau = sigma * delta
    Tcum = np.exp(-np.concatenate([[0.0], np.cumsum(tau)[:-1]]))
    alpha = -np.expm1(-tau)
    w = Tcum * alpha
    if t_min is not None:
        w = np.where(Tcum < t_min, 0.0, w)
        # once below t_min the ray stays terminated (T is non-increasing)
    I = (w[:, None] * rgb).sum(0) if len(w) else np.zeros(3)
    D = float((w * t).sum())
    return I, D, float(w.sum()), w, Tcum


def composite(ray_id, sigma, rgb, t, delta, n_rays, t_min=None):
    """composite_ray over every ray (rays with no samples render 0)."""
    I = np.zeros((n_rays, 3))
    D = np.zeros(n_rays)
    A = np.zeros(n_rays)
    w_all = np.zeros(len(sigma))
    T_all = np.zeros(len(sigma))
    starts = np.searchsorted(ray_id, np.arange(n_rays + 1))
    for r in range(n_rays):
        a, b = starts[r], starts[r + 1]
        if a == b:
            continue
        I[r], D[r], A[r], w_all[a:b], T_all[a:b] = composite_ray(
            sigma[a:b], rgb[a:b], t[a:b], delta, t_min)
    return I, D, A, w_all, T_all


# ------------------------------------------------------------------ a8: loss

def mapping_loss(I_hat, D_hat, I, D, V, lambda_d):
    """Eq. (mapping_loss): L_M = L_rgb + lambda_D L_D with L_rgb = ||I - I*||^2
    (summed over channels) and L_D = ||D - D*||^2_{Sigma_D} = (D - D*)^2 / Sigma_D,
    both averaged over the rays of the batch.  Returns (L_M, per-ray terms)."""
    lrgb = ((I - I_hat) ** 2).sum(1)
    ld = (D - D_hat) ** 2 / V
    per_ray = lrgb + lambda_d * ld
    return float(per_ray.mean()), per_ray


# ------------------------------------------------------------------ a9: composite bwd

def composite_backward_ray(sigma, rgb, t, delta, w, Tcum, gI, gD):
    """Gradient of g_I . I* + g_D d* for one ray with respect to sigma_i and c_i.
    dI*/dc_i = w_i; dI*/dsigma_i = delta (T_{i+1} c_i - sum_{j>i} w_j c_j), and the
    same for d* with t_i in place of c_i (from the compositing of Sec. 3.2)."""
    T_next = Tcum * np.exp(-sigma * delta)
    wc = w[:, None] * rgb
    wt = w * t
    suf_c = np.cumsum(wc[::-1], axis=0)[::-1] - wc      # sum_{j>i}
    suf_t = np.cumsum(wt[::-1])[::-1] - wt
    dsig = delta * ((T_next[:, None] * rgb - suf_c) @ gI + gD * (T_next * t - suf_t))
    drgb = w[:, None] * gI[None, :]
    return dsig, drgb


def composite_backward_ray_abs(sigma, rgb, t, delta, w, Tcum, gI, gD):
    """Sum of the absolute values of the terms of composite_backward_ray (every
    term is w, T, c, t >= 0 times |g|): the scale of that sum's rounding error."""
    T_next = Tcum * np.exp(-sigma * delta)
    wc = w[:, None] * rgb
    wt = w * t
    suf_c = np.cumsum(wc[::-1], axis=0)[::-1] - wc
    suf_t = np.cumsum(wt[::-1])[::-1] - wt
    dsig = delta * ((T_next[:, None] * rgb + suf_c) @ np.abs(gI) + abs(gD) * (T_next * t + suf_t))
    drgb = w[:, None] * np.abs(gI)[None, :]
    return dsig, drgb


# ------------------------------------------------------------------ a10, a11: backward

def field_backward(P: dict, fw: dict, dsigma, drgb, magnitude: bool = False, with_dsh: bool = False):
    """Chain rule through the MLPs (a10).  Returns weight gradients and dL/dfeat.
    With a rounded forward (field_forward with bits) the gradient operands are
    rounded the same way before their products: dL/dz, the masked dL/da of each
    hidden layer and dL/dh (the density branch's input gradient, after the
    dL/dsigma term is added).
    magnitude=True (with the absolute-term inputs of composite_backward_ray_abs)
    runs the same chain on |W| and on activation magnitudes (each activation
    replaced by the sum of the absolute values of its own terms, same ReLU
    branches): every output is then the sum of the absolute values of the products
    that make up the matching gradient entry, expanded down to the inputs - the
    scale of its rounding error in any summation order."""
    bits = fw.get("bits")
    R = (lambda a: a) if bits is None else (lambda a: round_sig(a, bits))
    W = fw["W"]
    if magnitude:
        if bits is not None:
            raise ValueError("magnitudes are defined for the plain chain only")
        W = {k: np.abs(v) for k, v in W.items()}
        f = np.abs(fw["feat"])
        h1 = np.where(fw["m1"], f @ W["W1"].T, 0.0)
        x3 = np.concatenate([h1 @ W["W2"].T, np.abs(fw["x3"][:, P["W2"].shape[0]:])], axis=1)
        h3 = np.where(fw["m3"], x3 @ W["W3"].T, 0.0)
        h4 = np.where(fw["m4"], h3 @ W["W4"].T, 0.0)
        fw = dict(fw, feat=f, h1=h1, x3=x3, h3=h3, h4=h4)
    rgb = fw["rgb"]
    dz = R(drgb * rgb * (1.0 - rgb))
    g = {"W5": dz.T @ fw["h4"]}
    dh4 = dz @ W["W5"]
    da4 = R(dh4 * fw["m4"])
    g["W4"] = da4.T @ fw["h3"]
    dh3 = da4 @ W["W4"]
    da3 = R(dh3 * fw["m3"])
    g["W3"] = da3.T @ fw["x3"]
    dx3 = da3 @ W["W3"]
    dh = dx3[:, :P["W2"].shape[0]].copy()
    dh[:, 0] += dsigma * fw["sigma"] * (fw["h"][:, 0] < SIGMA_H_MAX)
    dh = R(dh)
    g["W2"] = dh.T @ fw["h1"]
    dh1 = dh @ W["W2"]
    da1 = R(dh1 * fw["m1"])
    g["W1"] = da1.T @ fw["feat"]
    dfeat = da1 @ W["W1"]
    if with_dsh:
        return g, dfeat, dx3[:, P["W2"].shape[0]:]      # dL/d(SH inputs of the colour MLP)
    return g, dfeat


def hash_backward(cfg, idx, wts, dfeat):
    """a11: dL/dtable[l, idx_k] += w_k * dL/dfeat_l for every corner and level."""
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    g = np.zeros((L, T, F))
    for l in range(L):
        for f in range(F):
            np.add.at(g[l, :, f], idx[:, l, :].ravel(),
                      (wts[:, l, :] * dfeat[:, l * F + f][:, None]).ravel())
    return g


# ------------------------------------------------------------------ the step

def forward_backward(cfg, P, keyframes, n_rays, seed, step, occ_bits=None,
                     level_res=None, rays=None, want_grad=True, magnitudes=False,
                     mlp_bits=None):
    """a1-a11: loss L_M and its gradient for one batch.  Returns a dict with the
    loss, per-ray renders, the sample list and the named gradients; with
    magnitudes=True also `grads_abs`, per entry the sum of the absolute values of
    the products that form it (see field_backward).  mlp_bits = "fp16" | "bf16" (or
    a bit count) evaluates the MLPs with operands rounded to that precision
    (field_forward / field_backward); None is the plain FP64 chain."""
    level_res = level_resolutions(cfg) if level_res is None else level_res
    if rays is None:
        kf, u, v = draw_rays(seed, step, n_rays, [(k.W, k.H) for k in keyframes])
    else:
        kf, u, v = rays
    c2w = np.stack([keyframes[j].c2w for j in kf]) if n_rays else np.zeros((0, 3, 4), f32)
    K = np.stack([keyframes[j].K for j in kf]) if n_rays else np.zeros((0, 4), f32)
    o, d = cast_rays_f32(c2w, K, u, v)
    I, D, V = ray_targets(kf, u, v, keyframes)
    ray_id, step_idx, t, x = march(cfg, o, d, occ_bits)
    feat, idx, wts = hash_encode(cfg, level_res, P["tables"], x)
    sh = sh_deg4(d[ray_id])
    fw = field_forward(P, feat, sh, bits_of(mlp_bits))
    delta = float(cfg.step)
    t64 = t.astype(np.float64)
    I_hat, D_hat, acc, w, Tcum = composite(ray_id, fw["sigma"], fw["rgb"], t64, delta, n_rays)
    lam = float(cfg.lambda_d)
    loss, per_ray = mapping_loss(I_hat, D_hat, I, D, V, lam)
    out = dict(loss=loss, per_ray=per_ray, I_hat=I_hat, D_hat=D_hat, acc=acc, kf=kf, u=u,
               v=v, o=o, d=d, I=I, D=D, V=V, ray_id=ray_id, step_idx=step_idx, t=t, x=x,
               sigma=fw["sigma"], rgb=fw["rgb"], w=w, level_res=level_res)
    if not want_grad:
        return out
    gI = -2.0 * (I - I_hat) / n_rays
    gD = -2.0 * lam * (D - D_hat) / (V * n_rays)
    dsig = np.zeros(len(t))
    drgb = np.zeros((len(t), 3))
    starts = np.searchsorted(ray_id, np.arange(n_rays + 1))
    for r in range(n_rays):
        a, b = starts[r], starts[r + 1]
        if a == b:
            continue
        dsig[a:b], drgb[a:b] = composite_backward_ray(
            fw["sigma"][a:b], fw["rgb"][a:b], t64[a:b], delta, w[a:b], Tcum[a:b], gI[r], gD[r])
    g, dfeat = field_backward(P, fw, dsig, drgb)
    g["tables"] = hash_backward(cfg, idx, wts, dfeat)
    out.update(grads=g, dsigma=dsig, drgb=drgb, dfeat=dfeat)
    if magnitudes:
        dsa = np.zeros(len(t))
        dra = np.zeros((len(t), 3))
        gIa = 2.0 * (np.abs(I) + np.abs(I_hat)) / n_rays          # residual I - I*: two terms
        gDa = 2.0 * lam * (np.abs(D) + np.abs(D_hat)) / (V * n_rays)
        for r in range(n_rays):
            a, b = starts[r], starts[r + 1]
            if a == b:
                continue
            dsa[a:b], dra[a:b] = composite_backward_ray_abs(
                fw["sigma"][a:b], fw["rgb"][a:b], t64[a:b], delta, w[a:b], Tcum[a:b], gIa[r], gDa[r])
        ga, dfa = field_backward(P, fw, dsa, dra, magnitude=True)
        ga["tables"] = hash_backward(cfg, idx, wts, dfa)
        out["grads_abs"] = ga
        near = near_kink_samples(P, fw)
        touched = np.zeros((cfg.n_levels, cfg.table_size), bool)
        for l in range(cfg.n_levels):
            touched[l, idx[near, l, :].ravel()] = True
        out["near_kink"] = near
        out["near_kink_entries"] = touched
    return out


# A ReLU branch (and the density cap) is an integer decided by floating point: where
# a pre-activation lies within a rounding of zero, an FP32 evaluation may take the
# other branch than FP64, and the sample's whole contribution to the gradient
# changes; both results are correct evaluations of the method.  These samples are
# found from the sum of the absolute values of each pre-activation's terms.
KINK_TOL = 1e-5


def near_kink_samples(P: dict, fw: dict, tol: float = KINK_TOL) -> np.ndarray:
    """Samples with some ReLU pre-activation a satisfying |a| <= tol * sum|terms of a|
    (or with h_0 within tol of the density cap): bool [S]."""
    A = {k: np.abs(P[k].astype(np.float64)) for k in ("W1", "W3", "W4")}
    near = np.any(np.abs(fw["a1"]) <= tol * (np.abs(fw["feat"]) @ A["W1"].T), axis=1)
    near |= np.any(np.abs(fw["a3"]) <= tol * (np.abs(fw["x3"]) @ A["W3"].T), axis=1)
    near |= np.any(np.abs(fw["a4"]) <= tol * (np.abs(fw["h3"]) @ A["W4"].T), axis=1)
    near |= np.abs(fw["h"][:, 0] - SIGMA_H_MAX) <= tol * SIGMA_H_MAX
    return near


def loss_only(cfg, P, keyframes, n_rays, seed, step, occ_bits=None, level_res=None, rays=None):
    return forward_backward(cfg, P, keyframes, n_rays, seed, step, occ_bits, level_res,
                            rays, want_grad=False)["loss"]


# ------------------------------------------------------------------ a12: Adam

def adam_update(P: dict, G: dict, M: dict, Vm: dict, t: int, cfg):
    """Adam (Kingma & Ba 2015) with bias correction, dense over all parameters:
    m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  p -= lr * m_hat / (sqrt(v_hat) + eps),
    m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t).  t counts from 1.  FP64."""
    lr, b1, b2, eps = (float(cfg.lr), float(cfg.beta1), float(cfg.beta2), float(cfg.eps))
    newP, newM, newV = {}, {}, {}
    for k in P:
        g = G[k].astype(np.float64)
        m = b1 * M[k] + (1 - b1) * g
        v = b2 * Vm[k] + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        newP[k] = P[k].astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)
        newM[k], newV[k] = m, v
    return newP, newM, newV


# ------------------------------------------------------------------ a13: occupancy

def occupancy_refresh(cfg, P, density, refresh_idx, seed, level_res=None):
    """Cell density EMA: d <- max(decay * d, sigma(x_cell)) at one seeded point per
    cell, then bit = d > threshold.  x_cell = (c + u) / res per axis, u from three
    21-bit fields of one counter draw (stream OCC_STREAM + refresh_idx, index = cell).
    Returns (new density FP64 [res^3], packed bits uint8, positions [res^3, 3])."""
    level_res = level_resolutions(cfg) if level_res is None else level_res
    res = cfg.occ_res
    n = res ** 3
    cell = np.arange(n, dtype=np.int64)
    r = counter_rand(seed, OCC_STREAM + refresh_idx, cell.astype(U64), 0)
    u = np.stack([((r >> U64(21 * a)) & U64(0x1FFFFF)).astype(np.float64) for a in range(3)], 1)
    u = (u * 2.0 ** -21).astype(f32)          # exact: 21-bit fractions
    c = np.stack([cell % res, (cell // res) % res, cell // (res * res)], 1).astype(f32)
    x = (c + u) / f32(res)
    feat, _, _ = hash_encode(cfg, level_res, P["tables"], x)
    W1 = P["W1"].astype(np.float64)
    W2 = P["W2"].astype(np.float64)
    sig = np.exp(np.minimum((relu(feat @ W1.T) @ W2.T)[:, 0], SIGMA_H_MAX))
    newd = np.maximum(float(cfg.occ_decay) * density, sig)
    bits = np.packbits(newd > float(cfg.occ_thresh), bitorder="little")
    return newd, bits, x


# ------------------------------------------------------------------ a14: render

def render_rays_f32(c2w, K, W, H):
    """All pixel rays of one view, row-major (v outer, u inner)."""
    v, u = np.divmod(np.arange(W * H, dtype=np.int64), W)
    n = W * H
    o, d = cast_rays_f32(np.broadcast_to(c2w, (n, 3, 4)), np.broadcast_to(K, (n, 4)), u, v)
    return o, d


def render(cfg, P, c2w, K, W, H, occ_bits=None, level_res=None, t_min=None, mlp_bits=None):
    """Forward-only render of a W x H view (Sec. 3.3, the mapping thread also
    renders): colour [H*W, 3] and expected depth [H*W]; with t_min, samples after
    the transmittance drops below t_min are skipped.  mlp_bits as in
    forward_backward."""
    level_res = level_resolutions(cfg) if level_res is None else level_res
    o, d = render_rays_f32(np.asarray(c2w, f32), np.asarray(K, f32), W, H)
    ray_id, _, t, x = march(cfg, o, d, occ_bits)
    feat, _, _ = hash_encode(cfg, level_res, P["tables"], x)
    sh = sh_deg4(d[ray_id])
    fw = field_forward(P, feat, sh, bits_of(mlp_bits))
    I_hat, D_hat, acc, _, _ = composite(ray_id, fw["sigma"], fw["rgb"], t.astype(np.float64),
                                        float(cfg.step), W * H, t_min)
    return I_hat, D_hat, acc


# ------------------------------------------------------------------ joint pose refinement
# The mapping loss is minimised over the keyframe poses T as well as the map (Sec. 3.2:
# L_M(T, Theta)).  Here the gradient with respect to each keyframe pose, for a batch
# whose sample list (ray id, t) is held fixed: a pose moves every sample of its rays
# (p = o + t d) and turns their view directions, while the march's keep/drop
# decisions are integers that do not move.  Pose perturbation: left, in the world
# frame, T <- exp(xi) T with xi = (rho, phi): p -> R(phi) p + rho, so o -> o + rho +
# phi x o and d -> d + phi x d to first order, and
#   dL/drho = sum_rays dL/do,   dL/dphi = sum_rays (o x dL/do + d x dL/dd).

def sh_deg4_jacobian(d: np.ndarray) -> np.ndarray:
    """d/dd of the 16 SH values of sh_deg4 (each a polynomial in x, y, z): [S, 16, 3]."""
    x, y, z = d[:, 0].astype(np.float64), d[:, 1].astype(np.float64), d[:, 2].astype(np.float64)
    pi = math.pi
    a1 = math.sqrt(3 / (4 * pi))
    b = 0.5 * math.sqrt(15 / pi)
    c = 0.25 * math.sqrt(5 / pi)
    e = 0.25 * math.sqrt(15 / pi)
    f = 0.25 * math.sqrt(35 / (2 * pi))
    g = 0.5 * math.sqrt(105 / pi)
    h = 0.25 * math.sqrt(21 / (2 * pi))
    i = 0.25 * math.sqrt(7 / pi)
    j = 0.25 * math.sqrt(105 / pi)
    zero = np.zeros_like(x)
    one = np.ones_like(x)
    J = np.stack([
        np.stack([zero, zero, zero], -1),
        np.stack([zero, -a1 * one, zero], -1),
        np.stack([zero, zero, a1 * one], -1),
        np.stack([-a1 * one, zero, zero], -1),
        np.stack([b * y, b * x, zero], -1),
        np.stack([zero, -b * z, -b * y], -1),
        np.stack([zero, zero, 6 * c * z], -1),
        np.stack([-b * z, zero, -b * x], -1),
        np.stack([2 * e * x, -2 * e * y, zero], -1),
        np.stack([-6 * f * x * y, -f * (3 * x * x - 3 * y * y), zero], -1),
        np.stack([g * y * z, g * x * z, g * x * y], -1),
        np.stack([zero, -h * (5 * z * z - 1), -10 * h * y * z], -1),
        np.stack([zero, zero, i * (15 * z * z - 3)], -1),
        np.stack([-h * (5 * z * z - 1), zero, -10 * h * x * z], -1),
        np.stack([2 * j * x * z, -2 * j * y * z, j * (x * x - y * y)], -1),
        np.stack([-f * (3 * x * x - 3 * y * y), 6 * f * x * y, zero], -1),
    ], axis=1)
    return J


def hash_encode_dx(cfg, level_res, tables: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d(features)/dx of the grid encoding at x [S,3] (the derivative of the
    trilinear interpolation inside each cell): [S, enc_width, 3].  With
    w_k = prod_a (b_a ? w_a : 1 - w_a) and w_a = x_a N - c_a,
    dw_k/dx_a = N (b_a ? 1 : -1) prod_{a' != a} (b_a' ? w_a' : 1 - w_a')."""
    S = x.shape[0]
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    out = np.zeros((S, cfg.enc_width, 3))
    tab = tables.astype(np.float64)
    for l in range(L):
        N = level_res[l]
        c, w = grid_cell_f32(x, N)
        for k in range(8):
            bk = CORNERS[k]
            fac = np.where(bk[None, :] == 1, w, 1.0 - w)          # [S, 3]
            ik = vertex_index(c + bk[None, :], N, T)
            vals = tab[l, ik]                                       # [S, F]
            for a in range(3):
                others = np.prod(np.delete(fac, a, axis=1), axis=1)
                dw = N * (1.0 if bk[a] == 1 else -1.0) * others
                out[:, l * F:(l + 1) * F, a] += dw[:, None] * vals
    return out


def pose_gradients(cfg, P, keyframes, n_rays, seed, step, occ_bits=None, level_res=None, mlp_bits=None):
    """Gradient of the batch loss with respect to each keyframe pose (left world-frame
    perturbation, see above) for the batch of forward_backward, its sample list held
    fixed.  Returns dict(loss, pose_grads [n_kf, 6] = (dL/drho, dL/dphi) per keyframe,
    g_o [R, 3], g_d [R, 3] per ray, kf [R])."""
    fb = forward_backward(cfg, P, keyframes, n_rays, seed, step, occ_bits=occ_bits, level_res=level_res,
                          mlp_bits=mlp_bits)
    lr = fb["level_res"]
    feat, _, _ = hash_encode(cfg, lr, P["tables"], fb["x"])
    sh = sh_deg4(fb["d"][fb["ray_id"]])
    fw = field_forward(P, feat, sh, bits_of(mlp_bits))
    _, dfeat, dsh = field_backward(P, fw, fb["dsigma"], fb["drgb"], with_dsh=True)
    dfdx = hash_encode_dx(cfg, lr, P["tables"], fb["x"])             # [S, E, 3]
    dLdx = np.einsum("se,sea->sa", dfeat, dfdx)                       # [S, 3]
    dLdp = dLdx * float(cfg.grid_inv_size)
    Jsh = sh_deg4_jacobian(fb["d"][fb["ray_id"]])                    # [S, 16, 3]
    dLdd_sh = np.einsum("sk,ska->sa", dsh, Jsh)
    rid = fb["ray_id"]
    t = fb["t"].astype(np.float64)
    g_o = np.zeros((n_rays, 3))
    g_d = np.zeros((n_rays, 3))
    np.add.at(g_o, rid, dLdp)
    np.add.at(g_d, rid, t[:, None] * dLdp + dLdd_sh)
    o = fb["o"].astype(np.float64)
    d = fb["d"].astype(np.float64)
    pg = np.zeros((len(keyframes), 6))
    np.add.at(pg, fb["kf"], np.concatenate([g_o, np.cross(o, g_o) + np.cross(d, g_d)], axis=1))
    return dict(loss=fb["loss"], pose_grads=pg, g_o=g_o, g_d=g_d, kf=fb["kf"], fb=fb)


def loss_moved_samples(cfg, P, fb, drho, dphi, kf_index, level_res=None):
    """The batch loss of forward_backward's result `fb` with keyframe `kf_index`
    moved by the left perturbation (drho, dphi) (rotation by the vector dphi,
    Rodrigues' formula) and every sample kept at its t: positions and directions of
    that keyframe's rays move, the sample list and the targets do not.  FP64
    throughout (for finite differences of pose_gradients)."""
    lr = fb["level_res"] if level_res is None else level_res
    o = fb["o"].astype(np.float64).copy()
    d = fb["d"].astype(np.float64).copy()
    th = float(np.linalg.norm(dphi))
    if th > 0:
        k = np.asarray(dphi, np.float64) / th
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
    else:
        R = np.eye(3)
    sel = fb["kf"] == kf_index
    o[sel] = o[sel] @ R.T + np.asarray(drho, np.float64)
    d[sel] = d[sel] @ R.T
    rid = fb["ray_id"]
    t = fb["t"].astype(np.float64)
    p = o[rid] + t[:, None] * d[rid]
    x = (p - cfg.grid_origin.astype(np.float64)) * float(cfg.grid_inv_size)
    feat = hash_encode_f64(cfg, lr, P["tables"], x)
    sh = sh_deg4(d[rid])
    fw = field_forward(P, feat, sh)
    n_rays = len(fb["kf"])
    I_hat, D_hat, _, _, _ = composite(rid, fw["sigma"], fw["rgb"], t, float(cfg.step), n_rays)
    loss, _ = mapping_loss(I_hat, D_hat, fb["I"], fb["D"], fb["V"], float(cfg.lambda_d))
    return loss


def hash_encode_f64(cfg, level_res, tables, x):
    """hash_encode with the cell and offset taken in FP64 (for finite differences:
    a float32 position would swallow the perturbation)."""
    S = x.shape[0]
    L, F, T = cfg.n_levels, cfg.n_features, cfg.table_size
    feat = np.zeros((S, cfg.enc_width))
    tab = tables.astype(np.float64)
    for l in range(L):
        N = level_res[l]
        q = x * N
        c = np.minimum(np.floor(q).astype(np.int64), N - 1)
        w = q - c
        for k in range(8):
            bk = CORNERS[k]
            wk = np.prod(np.where(bk[None, :] == 1, w, 1.0 - w), axis=1)
            feat[:, l * F:(l + 1) * F] += wk[:, None] * tab[l, vertex_index(c + bk[None, :], N, T)]
    return feat


# ------------------------------------------------------------------ depth covariances
# The per-pixel depth variances Sigma_D that weight the depth loss come from the
# tracking frontend's dense bundle adjustment: its Hessian has the cameras/depths
# arrow structure H = [[C, E], [E^T, P]] (Sec. 3.1, Eq. hessian: C the camera block,
# P diagonal with one entry per pixel inverse depth, E the coupling), and the
# marginal covariances follow from the Schur complement (Sec. 3.1, Eq. cov):
#   H_T = C - E P^-1 E^T = L L^T,  Sigma_T = (L L^T)^-1,
#   Sigma_d = P^-1 + P^-T E^T Sigma_T E P^-1   (its diagonal: one variance per pixel).

def arrow_dense_E(c: int, blk: np.ndarray, e: np.ndarray) -> np.ndarray:
    """E [c, p] from the block-sparse form: column q holds e[q, b] at rows
    6 blk[q, b] .. 6 blk[q, b] + 5 (blocks with blk < 0 are unused)."""
    p, B = blk.shape
    E = np.zeros((c, p))
    for q in range(p):
        for b in range(B):
            k = int(blk[q, b])
            if k >= 0:
                E[6 * k:6 * k + 6, q] += e[q, b]
    return E


def marginal_covariances(C: np.ndarray, P: np.ndarray, blk: np.ndarray, e: np.ndarray):
    """Eq. (cov) in FP64: returns Sigma_T [c, c] and the per-pixel marginal variances
    diag(Sigma_d) [p]."""
    c = C.shape[0]
    E = arrow_dense_E(c, blk, e)
    EP = E / P[None, :]                                   # E P^-1
    HT = C - EP @ E.T                                     # reduced camera matrix
    L = np.linalg.cholesky(HT)
    Linv = np.linalg.inv(L)
    ST = Linv.T @ Linv                                    # (L L^T)^-1
    Sd = 1.0 / P + np.einsum("ip,ij,jp->p", EP, ST, EP)
    return ST, Sd
