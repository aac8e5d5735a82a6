"""Configurations, parameters and keyframes for the mapping workloads.

Every value the GPU path and the oracle must agree on bit for bit (sample spacing,
grid origin, box extents) is stored here as an IEEE float32 number, so both sides
read the same input instead of re-deriving it.  The level resolution table is NOT
stored here: it is part of the method (multiresolution grid, Instant-NGP as cited
in the paper's implementation details) and each side computes it on its own.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

F32 = np.float32


@dataclasses.dataclass
class FieldConfig:
    """Hyper-parameters of one radiance-field map and its mapping step."""

    name: str
    n_levels: int                 # L
    log2_table: int               # T = 2**log2_table entries per level
    n_min: int                    # coarsest grid resolution
    growth: Optional[float]       # per-level scale b (None: derived from n_max)
    n_max: Optional[int]          # finest resolution (used when growth is None)
    near: np.float32              # t of the first march step
    step: np.float32              # Delta, the march spacing (also delta_i of every sample)
    n_steps: int                  # march length (positions t_0 .. t_{n_steps-1})
    max_samples: int              # retained samples per ray (S_max)
    grid_origin: np.ndarray       # float32[3], world position of grid coordinate 0
    grid_inv_size: np.float32     # world -> grid scale (1 / cube side)
    box_max: np.ndarray           # float32[3], AABB upper corner in grid coordinates
    n_features: int = 2           # F
    enc_width: int = 32           # width of the density-MLP input (L*F zero padded)
    density_hidden: int = 64
    geo_width: int = 16
    color_hidden: int = 64
    occ_res: int = 0              # occupancy grid resolution (0: no bitfield)
    occ_every: int = 16
    occ_decay: np.float32 = F32(0.95)
    occ_thresh: np.float32 = F32(0.01)
    lambda_d: np.float32 = F32(1.0)
    lr: np.float32 = F32(1e-2)
    beta1: np.float32 = F32(0.9)
    beta2: np.float32 = F32(0.99)
    eps: np.float32 = F32(1e-15)
    render_t_min: np.float32 = F32(1e-4)
    precision: str = "fp32"       # "fp32" | "fp16" | "bf16" (MLP arithmetic)
    table_init: float = 1e-4      # hash tables ~ U(-table_init, table_init)
    mlp_init_std: float = 0.05    # MLP weights ~ N(0, mlp_init_std)
    seed: int = 0

    @property
    def table_size(self) -> int:
        return 1 << self.log2_table

    def replace(self, **kw) -> "FieldConfig":
        return dataclasses.replace(self, **kw)


def _cube(origin, side, extent):
    origin = np.asarray(origin, dtype=np.float64)
    extent = np.asarray(extent, dtype=np.float64)
    inv = F32(1.0 / side)
    box = (extent / side).astype(np.float32)
    return origin.astype(np.float32), inv, box


def config_small(precision: str = "fp32", occ_res: int = 16, **kw) -> FieldConfig:
    """A few-tile test field: L=4, T=2^10, N = 4..32 (two dense, two hashed levels),
    24 march steps on [0.1, 3], at most 16 retained samples (so truncation occurs)."""
    org, inv, box = _cube((0, 0, 0), 1.0, (1.0, 1.0, 1.0))
    cfg = FieldConfig(
        name="small", n_levels=4, log2_table=10, n_min=4, growth=2.0, n_max=None,
        near=F32(0.1), step=F32(2.9 / 24), n_steps=24, max_samples=16,
        grid_origin=org, grid_inv_size=inv, box_max=box, occ_res=occ_res,
        precision=precision)
    return cfg.replace(**kw)


def config_c1(precision: str = "fp32", **kw) -> FieldConfig:
    """Plain one-step workload: L=8, F=2, T=2^14, base 16, growth 1.5, 32 uniform
    samples over [0.1, 3] (Delta = 2.9/32), unit-cube AABB, no bitfield."""
    org, inv, box = _cube((0, 0, 0), 1.0, (1.0, 1.0, 1.0))
    cfg = FieldConfig(
        name="c1_L8_T2^14_4096rays", n_levels=8, log2_table=14, n_min=16, growth=1.5,
        n_max=None, near=F32(0.1), step=F32(2.9 / 32), n_steps=32, max_samples=32,
        grid_origin=org, grid_inv_size=inv, box_max=box, occ_res=0,
        precision=precision)
    return cfg.replace(**kw)


ROOM_EXTENT = (6.0, 4.0, 3.0)


def config_c2(precision: str = "fp16", **kw) -> FieldConfig:
    """Instant-NGP-scale step: L=16, F=2, T=2^19, N 16..2048, 128^3 bitfield, room
    6x4x3 m mapped into a 6 m cube, Delta = |diag|/1024, <=128 samples per ray."""
    org, inv, box = _cube((0, 0, 0), 6.0, ROOM_EXTENT)
    diag = math.sqrt(sum(e * e for e in ROOM_EXTENT))
    cfg = FieldConfig(
        name="c2_room_L16_T2^19_262144rays", n_levels=16, log2_table=19, n_min=16,
        growth=None, n_max=2048, near=F32(0.05), step=F32(diag / 1024), n_steps=1024,
        max_samples=128, grid_origin=org, grid_inv_size=inv, box_max=box, occ_res=128,
        precision=precision)
    return cfg.replace(**kw)


MULTIROOM_EXTENT = (20.0, 20.0, 3.0)


def config_c5(precision: str = "bf16", **kw) -> FieldConfig:
    """Large map: L=16, F=2, T=2^22, N 16..8192 over a 20x20x3 m multi-room scene."""
    org, inv, box = _cube((0, 0, 0), 20.0, MULTIROOM_EXTENT)
    diag = math.sqrt(sum(e * e for e in MULTIROOM_EXTENT))
    cfg = FieldConfig(
        name="c5_multiroom_L16_T2^22", n_levels=16, log2_table=22, n_min=16,
        growth=None, n_max=8192, near=F32(0.05), step=F32(diag / 4096), n_steps=4096,
        max_samples=128, grid_origin=org, grid_inv_size=inv, box_max=box, occ_res=256,
        precision=precision)
    return cfg.replace(**kw)


# --------------------------------------------------------------------------- params

def random_params(cfg: FieldConfig, seed: int = 0, table_scale: Optional[float] = None,
                  mlp_std: Optional[float] = None) -> dict:
    """Seeded initial parameters as named float32 arrays.

    tables [L, T, F] ~ U(-s, s); W1 [64, 32], W2 [16, 64], W3 [64, 32], W4 [64, 64],
    W5 [3, 64] ~ N(0, std).  Matrices are (out, in): layer output = W @ input.
    """
    rng = np.random.default_rng(seed)
    s = cfg.table_init if table_scale is None else table_scale
    std = cfg.mlp_init_std if mlp_std is None else mlp_std
    T = cfg.table_size
    p = {
        "tables": rng.uniform(-s, s, size=(cfg.n_levels, T, cfg.n_features)).astype(np.float32),
        "W1": rng.normal(0, std, size=(cfg.density_hidden, cfg.enc_width)).astype(np.float32),
        "W2": rng.normal(0, std, size=(cfg.geo_width, cfg.density_hidden)).astype(np.float32),
        "W3": rng.normal(0, std, size=(cfg.color_hidden, cfg.geo_width + 16)).astype(np.float32),
        "W4": rng.normal(0, std, size=(cfg.color_hidden, cfg.color_hidden)).astype(np.float32),
        "W5": rng.normal(0, std, size=(3, cfg.color_hidden)).astype(np.float32),
    }
    return p


# ------------------------------------------------------------------------- keyframes

@dataclasses.dataclass
class Keyframe:
    """One posed keyframe: colour, depth and per-pixel depth variance Sigma_D.

    c2w is the 3x4 camera-to-world matrix (OpenCV axes: x right, y down, z forward),
    K = (fx, fy, cx, cy).  depth_is_z says whether `depth`/`var` hold z-depth (as a
    depth sensor or a tracking frontend gives it) or distance along the unit ray.
    """

    kf_id: int
    c2w: np.ndarray        # float32 [3, 4]
    K: np.ndarray          # float32 [4]
    W: int
    H: int
    rgb: np.ndarray        # float32 [H, W, 3]
    depth: np.ndarray      # float32 [H, W]
    var: np.ndarray        # float32 [H, W]
    depth_is_z: bool = True


def quat_to_rot(q) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def random_pose(rng: np.random.Generator, lo=0.2, hi=0.8) -> np.ndarray:
    """Camera centre ~ U[lo, hi]^3, rotation from a normalised 4-Gaussian quaternion."""
    c = rng.uniform(lo, hi, size=3)
    R = quat_to_rot(rng.normal(size=4))
    return np.concatenate([R, c[:, None]], axis=1).astype(np.float32)


def look_at_pose(eye, target) -> np.ndarray:
    """OpenCV camera at `eye` looking at `target`, image y axis towards world -z."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    down = np.array([0.0, 0.0, -1.0])
    x = np.cross(down, f)
    if np.linalg.norm(x) < 1e-6:
        x = np.cross(np.array([0.0, 1.0, 0.0]), f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f], axis=1)
    return np.concatenate([R, eye[:, None]], axis=1).astype(np.float32)


def c1_keyframe(seed: int = 0, W: int = 64, H: int = 48, kf_id: int = 0) -> Keyframe:
    """The one-keyframe workload: 64x48 pinhole (fx=fy=50), seeded pose in the unit
    cube, targets RGB ~ U[0,1], ray depth ~ U[0.5, 2.5], sigma_d = 10^U[-2,0],
    Sigma_D = sigma_d^2."""
    rng = np.random.default_rng(seed)
    c2w = random_pose(rng)
    K = np.array([50.0, 50.0, W / 2.0, H / 2.0], dtype=np.float32)
    rgb = rng.uniform(0, 1, size=(H, W, 3)).astype(np.float32)
    depth = rng.uniform(0.5, 2.5, size=(H, W)).astype(np.float32)
    sigma_d = 10.0 ** rng.uniform(-2, 0, size=(H, W))
    var = (sigma_d ** 2).astype(np.float32)
    return Keyframe(kf_id, c2w, K, W, H, rgb, depth, var, depth_is_z=False)
