"""Procedural indoor scene rendered analytically (stand-in for the paper's indoor
datasets, which are not available here).

A room is an axis-aligned box [0, E] (E = 6x4x3 m by default) holding random
spheres and boxes.  Every surface carries a procedural colour texture (sinusoids of
the world position).  Keyframes are rendered by exact ray/primitive intersection;
depth gets Gaussian noise whose standard deviation grows with depth squared, and the
per-pixel variance Sigma_D = sigma_d^2 is returned with it.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .workloads import Keyframe, look_at_pose


@dataclasses.dataclass
class Room:
    extent: np.ndarray       # [3] room size in metres (walls at 0 and extent)
    sph_c: np.ndarray        # [ns, 3]
    sph_r: np.ndarray        # [ns]
    box_c: np.ndarray        # [nb, 3]
    box_h: np.ndarray        # [nb, 3] half sizes
    tex_dir: np.ndarray      # [n_obj, 3, 3] unit directions per colour channel
    tex_freq: np.ndarray     # [n_obj, 3]
    tex_phase: np.ndarray    # [n_obj, 3]

    @property
    def n_obj(self) -> int:
        return 6 + len(self.sph_r) + len(self.box_h)


def make_room(seed: int = 0, extent=(6.0, 4.0, 3.0), n_prims: int = 30) -> Room:
    """Room with `n_prims` primitives, half spheres (r ~ U[0.1, 0.5]) and half boxes
    (side ~ U[0.2, 1.0]), placed fully inside the room."""
    rng = np.random.default_rng(seed)
    E = np.asarray(extent, np.float64)
    ns = n_prims // 2
    nb = n_prims - ns
    sph_r = rng.uniform(0.1, 0.5, size=ns)
    sph_c = rng.uniform(0, 1, size=(ns, 3)) * (E - 2 * sph_r[:, None]) + sph_r[:, None]
    box_h = rng.uniform(0.2, 1.0, size=(nb, 3)) / 2
    box_c = rng.uniform(0, 1, size=(nb, 3)) * (E - 2 * box_h) + box_h
    n_obj = 6 + ns + nb
    d = rng.normal(size=(n_obj, 3, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return Room(E, sph_c, sph_r, box_c, box_h, d,
                rng.uniform(2.0, 12.0, size=(n_obj, 3)),
                rng.uniform(0, 2 * math.pi, size=(n_obj, 3)))


def _texture(room: Room, p: np.ndarray, obj: np.ndarray) -> np.ndarray:
    dirs = room.tex_dir[obj]                       # [N, 3, 3]
    arg = np.einsum("nca,na->nc", dirs, p) * room.tex_freq[obj] + room.tex_phase[obj]
    return 0.5 + 0.45 * np.sin(arg)


def _intersect(room: Room, o: np.ndarray, d: np.ndarray):
    """Nearest hit along o + t d (t > 0) for rays starting inside the room.
    Returns t [N] and object id [N] (0..5 walls, then spheres, then boxes)."""
    n = d.shape[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (0.0 - o) * inv
        t1 = (room.extent - o) * inv
    tw = np.maximum(t0, t1)                        # exit distance per axis
    axis = np.argmin(tw, axis=1)
    t_best = tw[np.arange(n), axis]
    side = (d[np.arange(n), axis] > 0).astype(np.int64)
    obj = axis * 2 + side
    a = np.sum(d * d, axis=1)
    CH = 65536
    ns = len(room.sph_r)
    for s0 in range(0, n, CH):                     # chunks keep the [chunk, prims, 3] arrays small
        sl = slice(s0, min(n, s0 + CH))
        oc = o[sl, None, :] - room.sph_c[None]     # [c, ns, 3]
        b = np.einsum("ca,cpa->cp", d[sl], oc)
        cc = np.sum(oc * oc, axis=2) - room.sph_r[None] ** 2
        disc = b * b - a[sl, None] * cc
        ok = disc >= 0
        t = np.where(ok, (-b - np.sqrt(np.where(ok, disc, 0))) / a[sl, None], np.inf)
        t = np.where(t > 1e-6, t, np.inf)
        if ns:
            i = np.argmin(t, axis=1)
            tm = t[np.arange(t.shape[0]), i]
            hit = tm < t_best[sl]
            t_best[sl] = np.where(hit, tm, t_best[sl])
            obj[sl] = np.where(hit, 6 + i, obj[sl])
        lo = room.box_c - room.box_h
        hi = room.box_c + room.box_h
        with np.errstate(divide="ignore", invalid="ignore"):
            a0 = (lo[None] - o[sl, None, :]) * inv[sl, None, :]
            a1 = (hi[None] - o[sl, None, :]) * inv[sl, None, :]
        tn = np.max(np.minimum(a0, a1), axis=2)
        tf = np.min(np.maximum(a0, a1), axis=2)
        tn = np.where((tn <= tf) & (tn > 1e-6), tn, np.inf)
        if len(room.box_h):
            i = np.argmin(tn, axis=1)
            tm = tn[np.arange(tn.shape[0]), i]
            hit = tm < t_best[sl]
            t_best[sl] = np.where(hit, tm, t_best[sl])
            obj[sl] = np.where(hit, 6 + ns + i, obj[sl])
    return t_best, obj


def render_room(room: Room, c2w: np.ndarray, K: np.ndarray, W: int, H: int):
    """Analytic render: returns z-depth [H, W] and colour [H, W, 3] (float64)."""
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dc = np.stack([(u - K[2]) / K[0], (v - K[3]) / K[1], np.ones_like(u)], -1).reshape(-1, 3)
    R = c2w[:, :3].astype(np.float64)
    o = np.broadcast_to(c2w[:, 3].astype(np.float64), dc.shape)
    d = dc @ R.T                                   # z component of dc is 1: t is z-depth
    t, obj = _intersect(room, o, d)
    p = o + t[:, None] * d
    rgb = _texture(room, p, obj)
    return t.reshape(H, W), rgb.reshape(H, W, 3)


def _sdf_abs(room: Room, p: np.ndarray) -> np.ndarray:
    """Unsigned distance to the nearest surface (walls and primitives)."""
    dist = np.min(np.minimum(p, room.extent - p), axis=1)
    dist = np.abs(dist)
    for i in range(len(room.sph_r)):
        dist = np.minimum(dist, np.abs(np.linalg.norm(p - room.sph_c[i], axis=1) - room.sph_r[i]))
    for i in range(len(room.box_h)):
        q = np.abs(p - room.box_c[i]) - room.box_h[i]
        out = np.linalg.norm(np.maximum(q, 0), axis=1)
        inside = np.minimum(np.max(q, axis=1), 0)
        dist = np.minimum(dist, np.abs(out + inside))
    return dist


def _inside_prims(room: Room, p: np.ndarray, margin: float) -> np.ndarray:
    ins = np.zeros(p.shape[0], bool)
    for i in range(len(room.sph_r)):
        ins |= np.linalg.norm(p - room.sph_c[i], axis=1) < room.sph_r[i] + margin
    for i in range(len(room.box_h)):
        ins |= np.all(np.abs(p - room.box_c[i]) < room.box_h[i] + margin, axis=1)
    return ins


def room_keyframes(room: Room, n: int, seed: int = 0, W: int = 640, H: int = 480,
                   K=(525.0, 525.0, 320.0, 240.0), noise_k: float = 0.01,
                   poses=None, first_id: int = 0, sigma_floor: float = 0.0,
                   outlier_frac: float = 0.0, outlier_range: float = 2.0, outlier_sigma: float = 1.0):
    """`n` keyframes at seeded poses inside the room looking at random interior
    points.  depth = z + N(0, sigma_d^2), sigma_d = max(noise_k * z^2 * U[0.5, 2],
    sigma_floor), var = sigma_d^2 (z-depth units).  With outlier_frac > 0 that
    fraction of the pixels (drawn independently) gets a gross depth error instead,
    depth = max(z + U[-outlier_range, outlier_range], 0.1), reported with
    sigma_d = outlier_sigma (a depth estimator that knows where it is unsure)."""
    rng = np.random.default_rng(seed)
    K = np.asarray(K, np.float32)
    E = room.extent
    out = []
    for k in range(n):
        if poses is not None:
            c2w = poses[k]
        else:
            while True:
                eye = rng.uniform(0.4, E - 0.4)
                if not _inside_prims(room, eye[None], 0.15)[0]:
                    break
            while True:
                tgt = rng.uniform(0.2, E - 0.2)
                if np.linalg.norm(tgt - eye) > 1.0:
                    break
            c2w = look_at_pose(eye, tgt)
        z, rgb = render_room(room, c2w, K, W, H)
        sigma = np.maximum(noise_k * z * z * rng.uniform(0.5, 2.0, size=z.shape), sigma_floor)
        depth = z + rng.normal(size=z.shape) * sigma
        if outlier_frac > 0.0:
            bad = rng.uniform(size=z.shape) < outlier_frac
            depth = np.where(bad, np.maximum(z + rng.uniform(-outlier_range, outlier_range, size=z.shape), 0.1),
                             depth)
            sigma = np.where(bad, outlier_sigma, sigma)
        out.append(Keyframe(first_id + k, c2w.astype(np.float32), K, W, H,
                            rgb.astype(np.float32), depth.astype(np.float32),
                            (sigma * sigma).astype(np.float32), depth_is_z=True))
    return out


def room_occupancy_bits(room: Room, res: int, grid_origin, grid_inv_size) -> np.ndarray:
    """Occupancy bitfield of the cells within about one cell of a surface.

    Cell (cx, cy, cz) has linear index b = cx + res*(cy + res*cz); its bit is bit
    (b & 7) of byte (b >> 3).  Cells outside the room are empty."""
    side = 1.0 / float(grid_inv_size)
    cell = side / res
    org = np.asarray(grid_origin, np.float64)
    bits = np.zeros(res ** 3, dtype=bool)
    g = (np.arange(res) + 0.5) * cell
    gx, gy = np.meshgrid(g, g, indexing="xy")      # gx varies along x (fastest)
    for cz in range(res):
        p = np.stack([gx.ravel() + org[0], gy.ravel() + org[1],
                      np.full(res * res, g[cz] + org[2])], axis=1)
        inside = np.all((p > 0) & (p < room.extent), axis=1)
        near = _sdf_abs(room, p) < 1.5 * cell
        bits[cz * res * res:(cz + 1) * res * res] = inside & near
    return np.packbits(bits, bitorder="little")


def room_spline_poses(room: Room, n: int, seed: int = 0, n_ctrl: int = 8, clearance: float = 0.3):
    """`n` poses along a Catmull-Rom spline through `n_ctrl` seeded control points,
    each looking at a point further along the path.  Control points are redrawn
    until every camera centre on the path keeps `clearance` from the walls and from
    every primitive."""
    rng = np.random.default_rng(seed)
    E = room.extent
    for _ in range(1000):
        ctrl = []
        while len(ctrl) < n_ctrl:
            p = rng.uniform(0.6, E - 0.6)
            if not _inside_prims(room, p[None], clearance)[0]:
                ctrl.append(p)
        ctrl = np.array(ctrl)
        P = np.concatenate([ctrl[:1], ctrl, ctrl[-1:]], 0)

        def cr(s):
            s = np.clip(s, 0, n_ctrl - 1 - 1e-9)
            i = int(s)
            u = s - i
            p0, p1, p2, p3 = P[i], P[i + 1], P[i + 2], P[i + 3]
            return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)

        eyes = np.array([cr(k * (n_ctrl - 1) / max(n - 1, 1)) for k in range(n)])
        clear = (np.all((eyes > clearance) & (eyes < E - clearance))
                 and not np.any(_inside_prims(room, eyes, clearance)))
        if clear:
            break
    poses = []
    for k in range(n):
        s = k * (n_ctrl - 1) / max(n - 1, 1)
        eye = eyes[k]
        tgt = cr(min(s + 0.5, n_ctrl - 1)) + np.array([0.0, 0.0, -0.1])
        if np.linalg.norm(tgt - eye) < 0.5:
            tgt = eye + np.array([1.0, 0.3, -0.1])
        poses.append(look_at_pose(eye, tgt))
    return poses
