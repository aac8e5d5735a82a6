"""Procedural multi-room floor (stand-in for a large indoor map): a 20 x 20 x 3 m
box divided by interior walls into a grid of rooms joined by doorways, each room
holding random spheres and boxes with procedural colour textures.

The scene is a `Room` (outer walls = the box, interior walls and furniture = axis-
aligned boxes, plus spheres), so the analytic renderer, occupancy and pose helpers
of `room.py` apply to it.  Thousands of megapixel keyframes are too many for the
host renderer, so this module also renders with PyTorch on any device: per keyframe
the ray/sphere test is one [rays x 3] x [3 x spheres] product (all rays of a camera
share its centre) and the ray/box slab test one broadcast over [rays, boxes].
Nothing here is part of the mapping method.
"""

from __future__ import annotations

import math

import numpy as np

from .room import Room, _inside_prims
from .workloads import Keyframe, look_at_pose


def make_multiroom(seed: int = 0, extent=(20.0, 20.0, 3.0), rooms=(4, 4), prims_per_room: int = 8,
                   wall: float = 0.1, door_w: float = 1.0, door_h: float = 2.2) -> Room:
    """Interior walls on the lines x = k E_x / rooms_x and y = k E_y / rooms_y; every
    wall segment between two crossings has one doorway (width door_w, height door_h,
    centred at a seeded position at least 1 m from the segment's ends) and a lintel
    above it.  Each room gets `prims_per_room` primitives (half spheres r ~ U[0.1,
    0.5], half boxes of side U[0.2, 1.0]) kept 0.2 m clear of its walls."""
    rng = np.random.default_rng(seed)
    E = np.asarray(extent, np.float64)
    nx, ny = rooms
    sx, sy = E[0] / nx, E[1] / ny
    box_c, box_h = [], []

    def add_box(lo, hi):
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        box_c.append((lo + hi) / 2)
        box_h.append((hi - lo) / 2)

    def wall_line(axis, pos, seg_len, n_seg):
        # a wall perpendicular to `axis` at coordinate `pos`, made of n_seg segments
        other = 1 - axis
        for s in range(n_seg):
            a0, a1 = s * seg_len, (s + 1) * seg_len
            dc = rng.uniform(a0 + 1.0, a1 - 1.0)
            pieces = [(a0, dc - door_w / 2, 0.0, E[2]), (dc + door_w / 2, a1, 0.0, E[2]),
                      (dc - door_w / 2, dc + door_w / 2, door_h, E[2])]
            for b0, b1, z0, z1 in pieces:
                lo, hi = np.zeros(3), np.zeros(3)
                lo[axis], hi[axis] = pos - wall / 2, pos + wall / 2
                lo[other], hi[other] = b0, b1
                lo[2], hi[2] = z0, z1
                add_box(lo, hi)

    for k in range(1, nx):
        wall_line(0, k * sx, sy, ny)
    for k in range(1, ny):
        wall_line(1, k * sy, sx, nx)
    n_walls = len(box_c)

    sph_c, sph_r = [], []
    for i in range(nx):
        for j in range(ny):
            lo = np.array([i * sx, j * sy, 0.0]) + np.array([wall / 2 + 0.2, wall / 2 + 0.2, 0.0])
            hi = np.array([(i + 1) * sx, (j + 1) * sy, E[2]]) - np.array([wall / 2 + 0.2, wall / 2 + 0.2, 0.0])
            for p in range(prims_per_room):
                if p % 2 == 0:
                    r = rng.uniform(0.1, 0.5)
                    sph_r.append(r)
                    sph_c.append(rng.uniform(lo + r, hi - r))
                else:
                    h = rng.uniform(0.2, 1.0, size=3) / 2
                    box_h.append(h)
                    box_c.append(rng.uniform(lo + h, hi - h))
    sph_c = np.array(sph_c).reshape(-1, 3)
    sph_r = np.array(sph_r)
    box_c = np.array(box_c).reshape(-1, 3)
    box_h = np.array(box_h).reshape(-1, 3)
    n_obj = 6 + len(sph_r) + len(box_h)
    d = rng.normal(size=(n_obj, 3, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    room = Room(E, sph_c, sph_r, box_c, box_h, d, rng.uniform(2.0, 12.0, size=(n_obj, 3)),
                rng.uniform(0, 2 * math.pi, size=(n_obj, 3)))
    room.n_walls = n_walls
    room.rooms = (nx, ny)
    return room


def multiroom_poses(room: Room, n: int, seed: int = 0, clearance: float = 0.15):
    """`n` seeded camera poses: the eye uniform over the floor plan at height
    U[0.4, 2.6] (redrawn while within `clearance` of a wall or primitive), looking at
    a point of the same room at least 1 m away."""
    rng = np.random.default_rng(seed)
    E = room.extent
    nx, ny = room.rooms
    sx, sy = E[0] / nx, E[1] / ny
    poses = []
    while len(poses) < n:
        eye = np.array([rng.uniform(0.3, E[0] - 0.3), rng.uniform(0.3, E[1] - 0.3), rng.uniform(0.4, 2.6)])
        if _inside_prims(room, eye[None], clearance)[0]:
            continue
        i, j = int(eye[0] // sx), int(eye[1] // sy)
        lo = np.array([i * sx + 0.3, j * sy + 0.3, 0.2])
        hi = np.array([(i + 1) * sx - 0.3, (j + 1) * sy - 0.3, E[2] - 0.2])
        for _ in range(100):
            tgt = rng.uniform(lo, hi)
            if np.linalg.norm(tgt - eye) > 1.0:
                break
        poses.append(look_at_pose(eye, tgt))
    return poses


class TorchScene:
    """The scene's geometry and textures as tensors on `device` (float32)."""

    def __init__(self, room: Room, device):
        import torch
        f = dict(dtype=torch.float32, device=device)
        self.torch = torch
        self.device = device
        self.E = torch.tensor(room.extent, **f)
        self.sph_c = torch.tensor(room.sph_c, **f).reshape(-1, 3)
        self.sph_r2 = torch.tensor(room.sph_r, **f) ** 2
        self.lo = torch.tensor(room.box_c - room.box_h, **f).reshape(-1, 3)
        self.hi = torch.tensor(room.box_c + room.box_h, **f).reshape(-1, 3)
        self.tex_dir = torch.tensor(room.tex_dir, **f)
        self.tex_freq = torch.tensor(room.tex_freq, **f)
        self.tex_phase = torch.tensor(room.tex_phase, **f)
        self.ns = self.sph_c.shape[0]

    def intersect(self, o, d):
        """Nearest hit of the rays o + t d (o: [3], d: [N, 3]); returns t [N] (in units
        of |d|) and the object id [N] (0..5 outer walls, then spheres, then boxes)."""
        torch = self.torch
        inv = 1.0 / d
        tw = torch.maximum((0.0 - o) * inv, (self.E - o) * inv)
        t, axis = tw.min(dim=1)
        side = (d.gather(1, axis[:, None])[:, 0] > 0).long()
        obj = axis * 2 + side
        if self.ns:
            oc = o[None] - self.sph_c                          # [ns, 3]
            b = d @ oc.T                                       # [N, ns]
            a = (d * d).sum(1, keepdim=True)
            cc = (oc * oc).sum(1) - self.sph_r2                # [ns]
            disc = b * b - a * cc
            ts = (-b - torch.sqrt(disc.clamp_min(0))) / a
            ts = torch.where((disc >= 0) & (ts > 1e-6), ts, torch.full_like(ts, float("inf")))
            tm, i = ts.min(dim=1)
            hit = tm < t
            t = torch.where(hit, tm, t)
            obj = torch.where(hit, 6 + i, obj)
        if self.lo.shape[0]:
            tn = torch.full((d.shape[0], self.lo.shape[0]), -float("inf"), device=d.device)
            tf = torch.full_like(tn, float("inf"))
            for ax in range(3):
                a0 = (self.lo[None, :, ax] - o[ax]) * inv[:, ax:ax + 1]
                a1 = (self.hi[None, :, ax] - o[ax]) * inv[:, ax:ax + 1]
                tn = torch.maximum(tn, torch.minimum(a0, a1))
                tf = torch.minimum(tf, torch.maximum(a0, a1))
            tn = torch.where((tn <= tf) & (tn > 1e-6), tn, torch.full_like(tn, float("inf")))
            tm, i = tn.min(dim=1)
            hit = tm < t
            t = torch.where(hit, tm, t)
            obj = torch.where(hit, 6 + self.ns + i, obj)
        return t, obj

    def texture(self, p, obj):
        arg = torch_einsum(self.torch, self.tex_dir[obj], p) * self.tex_freq[obj] + self.tex_phase[obj]
        return 0.5 + 0.45 * self.torch.sin(arg)


def torch_einsum(torch, dirs, p):
    return torch.einsum("nca,na->nc", dirs, p)


def render_keyframes_torch(room: Room, poses, W: int, H: int, K, seed: int = 0, noise_k: float = 0.01,
                           sigma_floor: float = 0.0, device="cuda", first_id: int = 0, chunk: int = 1 << 19):
    """Renders one keyframe per pose on `device`.  Yields (Keyframe with c2w/K/W/H
    and no host arrays, rgb [H, W, 3], z-depth [H, W], variance [H, W]) with the
    image tensors on `device`; depth = z + N(0, sigma_d^2), sigma_d =
    max(noise_k z^2 U[0.5, 2], sigma_floor) (torch generator seeded by `seed`)."""
    import torch
    sc = TorchScene(room, device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    K = np.asarray(K, np.float32)
    u = (torch.arange(W, device=device, dtype=torch.float32) + 0.5 - float(K[2])) / float(K[0])
    v = (torch.arange(H, device=device, dtype=torch.float32) + 0.5 - float(K[3])) / float(K[1])
    vv, uu = torch.meshgrid(v, u, indexing="ij")
    dc = torch.stack([uu, vv, torch.ones_like(uu)], -1).reshape(-1, 3)
    for k, c2w in enumerate(poses):
        R = torch.tensor(np.asarray(c2w)[:, :3], dtype=torch.float32, device=device)
        o = torch.tensor(np.asarray(c2w)[:, 3], dtype=torch.float32, device=device)
        d = dc @ R.T                                           # z component of dc is 1: t is z-depth
        zs, rgbs = [], []
        for s0 in range(0, d.shape[0], chunk):
            dd = d[s0:s0 + chunk]
            t, obj = sc.intersect(o, dd)
            zs.append(t)
            rgbs.append(sc.texture(o[None] + t[:, None] * dd, obj))
        z = torch.cat(zs).reshape(H, W)
        rgb = torch.cat(rgbs).reshape(H, W, 3).contiguous()
        sig = torch.clamp_min(noise_k * z * z * (0.5 + 1.5 * torch.rand((H, W), generator=g, device=device)),
                              sigma_floor)
        depth = (z + torch.randn((H, W), generator=g, device=device) * sig).contiguous()
        var = (sig * sig).contiguous()
        kf = Keyframe(first_id + k, np.asarray(c2w, np.float32), K, W, H, None, None, None, depth_is_z=True)
        yield kf, rgb, depth, var


def occupancy_bits_torch(room: Room, res: int, grid_origin, grid_inv_size, device="cuda",
                         band: float = 1.5) -> np.ndarray:
    """Occupancy bitfield (the layout of `room_occupancy_bits`) of the cells whose
    centre lies within `band` cells of a surface, computed with tensors on `device`."""
    import torch
    sc = TorchScene(room, device)
    side = 1.0 / float(grid_inv_size)
    cell = side / res
    org = torch.tensor(np.asarray(grid_origin, np.float64), dtype=torch.float32, device=device)
    g = (torch.arange(res, device=device, dtype=torch.float32) + 0.5) * cell
    gy, gx = torch.meshgrid(g, g, indexing="ij")               # x fastest within a z slice
    bits = torch.zeros(res ** 3, dtype=torch.bool, device=device)
    sph_r = torch.sqrt(sc.sph_r2)
    bc, bh = (sc.lo + sc.hi) / 2, (sc.hi - sc.lo) / 2
    for cz in range(res):
        p = torch.stack([gx.reshape(-1) + org[0], gy.reshape(-1) + org[1],
                         torch.full((res * res,), float(g[cz]), device=device) + org[2]], 1)
        dist = torch.minimum(p, sc.E - p).min(dim=1).values.abs()
        if sc.ns:
            ds = (torch.cdist(p, sc.sph_c) - sph_r).abs().min(dim=1).values
            dist = torch.minimum(dist, ds)
        if bc.shape[0]:
            q = (p[:, None, :] - bc[None]).abs() - bh[None]
            out = q.clamp_min(0).norm(dim=2)
            inside = q.max(dim=2).values.clamp_max(0)
            dist = torch.minimum(dist, (out + inside).abs().min(dim=1).values)
        inside_box = ((p > 0) & (p < sc.E)).all(dim=1)
        bits[cz * res * res:(cz + 1) * res * res] = inside_box & (dist < band * cell)
    return np.packbits(bits.cpu().numpy(), bitorder="little")
