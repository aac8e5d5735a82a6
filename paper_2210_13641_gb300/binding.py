"""ctypes binding of libnerfmap.so (include/nerfmap.h), argument marshalling only.

Every computation of the mapping path runs in the library's CUDA kernels; this
module converts configurations, numpy arrays and torch tensors to the C ABI's plain
pointers and sizes.  It fails loudly when the library is missing: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnerfmap.so")

MAP_OK, MAP_EINVAL, MAP_ENOMEM, MAP_ENOKF, MAP_ETIMEOUT, MAP_ECUDA = 0, -1, -2, -3, -4, -5
MAP_MEM_HOST, MAP_MEM_DEVICE = 0, 1
MAP_STEP_NO_UPDATE = 1
MAP_STEP_POSE_GRAD = 2
MAP_SAVE_KEYFRAMES = 1
PRECISION = {"fp32": 0, "fp16": 1, "bf16": 2}
MLP_SHAPES = [("W1", (64, 32)), ("W2", (16, 64)), ("W3", (64, 32)), ("W4", (64, 64)), ("W5", (3, 64))]
MLP_PARAMS = sum(a * b for _, (a, b) in MLP_SHAPES)


class MapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"nerfmap error {code}: {msg}")
        self.code = code


class MapConfig(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_uint32), ("n_features", ctypes.c_uint32),
        ("log2_table", ctypes.c_uint32), ("level_res", ctypes.c_uint32 * 32),
        ("enc_width", ctypes.c_uint32), ("density_hidden", ctypes.c_uint32),
        ("geo_width", ctypes.c_uint32), ("color_hidden", ctypes.c_uint32),
        ("near_t", ctypes.c_float), ("step_t", ctypes.c_float),
        ("n_steps", ctypes.c_uint32), ("max_samples", ctypes.c_uint32),
        ("grid_origin", ctypes.c_float * 3), ("grid_inv_size", ctypes.c_float),
        ("box_max", ctypes.c_float * 3), ("occ_res", ctypes.c_uint32),
        ("occ_every", ctypes.c_uint32), ("occ_decay", ctypes.c_float),
        ("occ_thresh", ctypes.c_float), ("lambda_d", ctypes.c_float), ("lr", ctypes.c_float),
        ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
        ("render_t_min", ctypes.c_float), ("precision", ctypes.c_uint32),
        ("reserved0", ctypes.c_uint32), ("seed", ctypes.c_uint64),
    ]


class MapStats(ctypes.Structure):
    _fields_ = [("step", ctypes.c_uint64), ("n_samples", ctypes.c_uint64), ("n_rays", ctypes.c_uint32),
                ("n_keyframes", ctypes.c_uint32), ("param_count", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("render_samples", ctypes.c_uint64), ("render_evaluated", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_scenes", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("step_rays", ctypes.c_uint32), ("group_renders", ctypes.c_uint32),
                ("hbm_reserve_bytes", ctypes.c_size_t), ("kf_reserve_bytes", ctypes.c_size_t),
                ("seed", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("step_index", ctypes.c_uint64), ("scene", ctypes.c_uint32),
                ("kind", ctypes.c_uint32), ("status", ctypes.c_int32), ("loss", ctypes.c_float),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("t_now", ctypes.c_double), ("rays_done", ctypes.c_uint64), ("steps_done", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("n_scenes", ctypes.c_uint32), ("pending", ctypes.c_uint32),
                ("grouped_renders", ctypes.c_uint64), ("group_batches", ctypes.c_uint64)]


REQ_KEYFRAME, REQ_STEP, REQ_RENDER = 0, 1, 2

PHASES = ["ray_gen", "march", "field_fwd", "composite", "field_bwd", "adam", "occupancy", "output"]


_SIGS = {
    "map_config_init": (ctypes.c_int, [ctypes.POINTER(MapConfig), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_double]),
    "map_create": (ctypes.c_int, [ctypes.POINTER(MapConfig), ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "map_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "map_add_keyframe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "map_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                ctypes.c_void_p, ctypes.c_void_p]),
    "map_loss_device": (ctypes.c_void_p, [ctypes.c_void_p]),
    "map_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_void_p]),
    "map_render_group": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_void_p]),
    "map_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "map_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "map_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "map_get_pose_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int,
                                          ctypes.c_void_p]),
    "map_get_keyframe_ids": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32]),
    "map_evict_keyframe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "map_restore_keyframe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "map_keyframe_resident": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "map_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_uint32, ctypes.c_void_p]),
    "map_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "map_marginal_covariances": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "map_set_keyframe_pose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "map_get_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_int, ctypes.c_void_p]),
    "map_reset_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "map_set_occupancy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "map_get_occupancy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "map_set_occupancy_density": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                                 ctypes.c_void_p]),
    "map_refresh_occupancy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "map_get_samples": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "map_get_ray_outputs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "map_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(MapStats)]),
    "map_abi_config_size": (ctypes.c_size_t, []),
    "map_set_wait_polls": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "map_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "map_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "map_server_add_scene": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(MapConfig), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_uint32)]),
    "map_server_scene_handle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
    "map_server_submit_keyframe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_uint64)]),
    "map_server_submit_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_uint64)]),
    "map_server_submit_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.POINTER(ctypes.c_uint64)]),
    "map_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint32)]),
    "map_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "map_march_noalloc": (ctypes.c_int, [ctypes.POINTER(MapConfig), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "map_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "map_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "map_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}

_lib = None


def exported_symbols() -> list:
    return list(_SIGS)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnerfmap.so (built in-tree by build.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnerfmap.so not built at {path}: run paper_2210_13641_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.map_abi_config_size() != ctypes.sizeof(MapConfig):
        raise RuntimeError("map_config layout mismatch between the binding and libnerfmap.so")
    _lib = lib
    return lib


# ------------------------------------------------------------------ config helpers

def make_config(cfg, occ_every: Optional[int] = None) -> MapConfig:
    """C configuration from a field-config object (attributes as in the header);
    the level table comes from the library (map_config_init)."""
    lib = load()
    c = MapConfig()
    rc = lib.map_config_init(ctypes.byref(c), cfg.n_levels, cfg.log2_table, cfg.n_min, cfg.n_max or 0,
                             float(cfg.growth) if cfg.growth is not None else 0.0)
    if rc != MAP_OK:
        raise MapError(rc, lib.map_last_error(None).decode())
    if (cfg.n_features, cfg.enc_width, cfg.density_hidden, cfg.geo_width, cfg.color_hidden) != (2, 32, 64, 16, 64):
        raise ValueError("the library's field has F = 2 and MLP widths 32/64/16/64")
    c.near_t = float(cfg.near)
    c.step_t = float(cfg.step)
    c.n_steps = cfg.n_steps
    c.max_samples = cfg.max_samples
    for a in range(3):
        c.grid_origin[a] = float(cfg.grid_origin[a])
        c.box_max[a] = float(cfg.box_max[a])
    c.grid_inv_size = float(cfg.grid_inv_size)
    c.occ_res = cfg.occ_res
    c.occ_every = cfg.occ_every if occ_every is None else occ_every
    c.occ_decay = float(cfg.occ_decay)
    c.occ_thresh = float(cfg.occ_thresh)
    c.lambda_d = float(cfg.lambda_d)
    c.lr, c.beta1, c.beta2, c.eps = float(cfg.lr), float(cfg.beta1), float(cfg.beta2), float(cfg.eps)
    c.render_t_min = float(cfg.render_t_min)
    c.precision = PRECISION[cfg.precision]
    c.seed = cfg.seed
    return c


def level_resolutions(cfg) -> list:
    """The level table the library computes for a field config (map_config_init)."""
    c = make_config(cfg)
    return [int(c.level_res[l]) for l in range(cfg.n_levels)]


def pack_params(named: dict) -> np.ndarray:
    """Named parameters -> flat FP32 vector in the library layout."""
    parts = [np.ascontiguousarray(named["tables"], np.float32).ravel()]
    parts += [np.ascontiguousarray(named[k], np.float32).ravel() for k, _ in MLP_SHAPES]
    return np.concatenate(parts)


def unpack_params(flat: np.ndarray, n_levels: int, log2_table: int, n_features: int = 2) -> dict:
    T = 1 << log2_table
    nt = n_levels * T * n_features
    out = {"tables": flat[:nt].reshape(n_levels, T, n_features)}
    off = nt
    for k, (a, b) in MLP_SHAPES:
        out[k] = flat[off:off + a * b].reshape(a, b)
        off += a * b
    return out


# ------------------------------------------------------------------ pointers

def _ptr(x):
    """(address, mem_kind) of a numpy array or torch tensor (None -> (None, host))."""
    if x is None:
        return None, MAP_MEM_HOST
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data, MAP_MEM_HOST
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), (MAP_MEM_DEVICE if x.is_cuda else MAP_MEM_HOST)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class NerfMap:
    """One map (hash tables, MLP weights, Adam state, occupancy, keyframes) on the
    current GPU, driven through the C ABI."""

    def __init__(self, cfg, hbm_budget: int = 0, occ_every: Optional[int] = None):
        self.lib = load()
        self.cfg = cfg
        self.ccfg = make_config(cfg, occ_every)
        h = ctypes.c_void_p()
        rc = self.lib.map_create(ctypes.byref(self.ccfg), hbm_budget, ctypes.byref(h))
        if rc != MAP_OK:
            raise MapError(rc, self.lib.map_last_error(None).decode())
        self.h = h
        self.n_params = self.stats().param_count

    @classmethod
    def load(cls, path, cfg, hbm_budget: int = 0) -> "NerfMap":
        """The map saved in `path` by save() (map_load).  cfg: the field configuration it
        was created with (used by the Python-side helpers such as unpack)."""
        self = cls.__new__(cls)
        self.lib = load()
        self.cfg = cfg
        self.ccfg = None
        h = ctypes.c_void_p()
        rc = self.lib.map_load(os.fsencode(str(path)), hbm_budget, ctypes.byref(h))
        if rc != MAP_OK:
            raise MapError(rc, self.lib.map_last_error(None).decode())
        self.h = h
        self.n_params = self.stats().param_count
        return self

    def save(self, path, keyframes: bool = True, stream=None):
        """Checkpoint of the map's state into `path` (map_save); with keyframes=True the
        keyframe images too, so that a loaded map resumes bit for bit."""
        self._check(self.lib.map_save(self.h, os.fsencode(str(path)), MAP_SAVE_KEYFRAMES if keyframes else 0,
                                      _stream(stream)))

    def _check(self, rc):
        if rc != MAP_OK:
            raise MapError(rc, self.lib.map_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.map_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- keyframes
    def add_keyframe(self, kf, rgb=None, depth=None, var=None, stream=None):
        """kf: object with kf_id, c2w [3,4], K [4], W, H, rgb, depth, var, depth_is_z.
        rgb/depth/var override the arrays (e.g. torch tensors on the device)."""
        c2w = np.ascontiguousarray(kf.c2w, np.float32).reshape(12)
        K = np.ascontiguousarray(kf.K, np.float32).reshape(4)
        rgb = np.ascontiguousarray(kf.rgb, np.float32) if rgb is None else rgb
        depth = np.ascontiguousarray(kf.depth, np.float32) if depth is None else depth
        var = np.ascontiguousarray(kf.var, np.float32) if var is None else var
        (pr, kind), (pd, _), (pv, _) = _ptr(rgb), _ptr(depth), _ptr(var)
        self._check(self.lib.map_add_keyframe(self.h, kf.kf_id, c2w.ctypes.data, K.ctypes.data, kf.W, kf.H,
                                              pr, pd, pv, int(bool(kf.depth_is_z)), kind, _stream(stream)))

    # -------------------------------------------------------------- step / render
    def step(self, n_rays: int, seed: int, no_update: bool = False, want_loss: bool = True, stream=None,
             pose_grad: bool = False):
        loss = ctypes.c_float()
        flags = (MAP_STEP_NO_UPDATE if no_update else 0) | (MAP_STEP_POSE_GRAD if pose_grad else 0)
        self._check(self.lib.map_step(self.h, n_rays, seed, flags,
                                      ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def keyframe_ids(self) -> list:
        n = self.lib.map_get_keyframe_ids(self.h, None, 0)
        ids = (ctypes.c_uint32 * max(n, 1))()
        self.lib.map_get_keyframe_ids(self.h, ids, n)
        return list(ids[:n])

    def pose_grads(self, stream=None) -> np.ndarray:
        """[n_kf, 6] = (dL/drho, dL/dphi) per keyframe slot of the last POSE_GRAD step."""
        n = len(self.keyframe_ids())
        out = np.zeros((n, 6), np.float32)
        self._check(self.lib.map_get_pose_grads(self.h, out.ctypes.data, n, MAP_MEM_HOST, _stream(stream)))
        return out

    def evict_keyframe(self, kf_id: int, stream=None):
        self._check(self.lib.map_evict_keyframe(self.h, kf_id, _stream(stream)))

    def restore_keyframe(self, kf_id: int, stream=None):
        self._check(self.lib.map_restore_keyframe(self.h, kf_id, _stream(stream)))

    def keyframe_resident(self, kf_id: int) -> bool:
        rc = self.lib.map_keyframe_resident(self.h, kf_id)
        self._check(min(rc, 0))
        return rc == 1

    def set_pose(self, kf_id: int, c2w, stream=None):
        c2w = np.ascontiguousarray(c2w, np.float32).reshape(12)
        self._check(self.lib.map_set_keyframe_pose(self.h, kf_id, c2w.ctypes.data, _stream(stream)))

    def loss_device_ptr(self) -> int:
        return self.lib.map_loss_device(self.h)

    def render(self, c2w, K, W: int, H: int, out_rgb=None, out_depth=None, out_acc=None, stream=None):
        """Renders into the given buffers (torch CUDA tensors or numpy arrays); with no
        buffers, returns host numpy arrays (rgb [H,W,3], depth [H,W], acc [H,W])."""
        c2w = np.ascontiguousarray(c2w, np.float32).reshape(12)
        K = np.ascontiguousarray(K, np.float32).reshape(4)
        if out_rgb is None and out_depth is None and out_acc is None:
            out_rgb = np.zeros((H, W, 3), np.float32)
            out_depth = np.zeros((H, W), np.float32)
            out_acc = np.zeros((H, W), np.float32)
        (p1, kind), (p2, k2), (p3, k3) = _ptr(out_rgb), _ptr(out_depth), _ptr(out_acc)
        if out_rgb is None:
            kind = k2 if out_depth is not None else k3
        self._check(self.lib.map_render(self.h, c2w.ctypes.data, K.ctypes.data, W, H, p1, p2, p3, kind,
                                        _stream(stream)))
        return out_rgb, out_depth, out_acc

    # -------------------------------------------------------------- parameters
    def get_params(self, out=None, stream=None) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32) if out is None else out
        p, kind = _ptr(out)
        self._check(self.lib.map_get_params(self.h, p, self.n_params, kind, _stream(stream)))
        return out

    def set_params(self, flat, stream=None):
        if isinstance(flat, dict):
            flat = pack_params(flat)
        if isinstance(flat, np.ndarray):
            flat = np.ascontiguousarray(flat, np.float32)
        p, kind = _ptr(flat)
        self._check(self.lib.map_set_params(self.h, p, self.n_params, kind, _stream(stream)))

    def get_grads(self, out=None, stream=None) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32) if out is None else out
        p, kind = _ptr(out)
        self._check(self.lib.map_get_grads(self.h, p, self.n_params, kind, _stream(stream)))
        return out

    def get_adam(self, stream=None):
        m = np.zeros(self.n_params, np.float32)
        v = np.zeros(self.n_params, np.float32)
        self._check(self.lib.map_get_adam(self.h, m.ctypes.data, v.ctypes.data, self.n_params, MAP_MEM_HOST,
                                          _stream(stream)))
        return m, v

    def reset_adam(self, stream=None):
        self._check(self.lib.map_reset_adam(self.h, _stream(stream)))

    def unpack(self, flat) -> dict:
        return unpack_params(flat, self.cfg.n_levels, self.cfg.log2_table, self.cfg.n_features)

    # -------------------------------------------------------------- occupancy
    def set_occupancy(self, bits: np.ndarray, stream=None):
        bits = np.ascontiguousarray(bits, np.uint8)
        self._check(self.lib.map_set_occupancy(self.h, bits.ctypes.data, bits.size, MAP_MEM_HOST, _stream(stream)))

    def set_occupancy_density(self, dens: np.ndarray, stream=None):
        dens = np.ascontiguousarray(dens, np.float32)
        self._check(self.lib.map_set_occupancy_density(self.h, dens.ctypes.data, dens.size, MAP_MEM_HOST,
                                                       _stream(stream)))

    def get_occupancy(self, stream=None):
        n = self.cfg.occ_res ** 3
        bits = np.zeros(n // 8, np.uint8)
        dens = np.zeros(n, np.float32)
        self._check(self.lib.map_get_occupancy(self.h, bits.ctypes.data, dens.ctypes.data, MAP_MEM_HOST,
                                               _stream(stream)))
        return bits, dens

    def refresh_occupancy(self, stream=None):
        self._check(self.lib.map_refresh_occupancy(self.h, _stream(stream)))

    # -------------------------------------------------------------- inspection
    def stats(self) -> MapStats:
        s = MapStats()
        self._check(self.lib.map_get_stats(self.h, ctypes.byref(s)))
        return s

    def profile(self, enable: bool = True):
        self._check(self.lib.map_profile_enable(self.h, int(enable)))

    def set_wait_polls(self, polls: int):
        """Poll limit of the tensor-core kernels' MMA waits (0: expire at once)."""
        self._check(self.lib.map_set_wait_polls(self.h, polls))

    def profile_read(self) -> dict:
        ms = np.zeros(8, np.float64)
        cnt = np.zeros(8, np.uint64)
        lch = np.zeros(8, np.uint64)
        self._check(self.lib.map_profile_read(self.h, ms.ctypes.data, cnt.ctypes.data, lch.ctypes.data))
        return {name: dict(ms=float(ms[i]), count=int(cnt[i]), launches=int(lch[i]))
                for i, name in enumerate(PHASES)}

    def samples(self):
        n = self.stats().n_samples
        rid = np.zeros(n, np.uint32)
        t = np.zeros(n, np.float32)
        self._check(self.lib.map_get_samples(self.h, rid.ctypes.data, t.ctypes.data, n, None))
        return rid, t

    def ray_outputs(self, n_rays: int):
        rgb = np.zeros((n_rays, 3), np.float32)
        d = np.zeros(n_rays, np.float32)
        a = np.zeros(n_rays, np.float32)
        self._check(self.lib.map_get_ray_outputs(self.h, rgb.ctypes.data, d.ctypes.data, a.ctypes.data, n_rays,
                                                 None))
        return rgb, d, a


class MapServer:
    """Multi-scene serving loop (map_server_* of the C ABI).  One request per scene on
    the GPU at a time by default: with several scenes the device stays busy with the
    others' work, and a new keyframe or render waits behind one mapping step of its
    scene instead of two."""

    def __init__(self, max_scenes=4, max_inflight=1, step_rays=1 << 18, hbm_reserve=1 << 30,
                 kf_reserve=1 << 30, seed=0, group_renders=True):
        self.lib = load()
        c = ServerConfig(max_scenes, max_inflight, step_rays, int(group_renders), hbm_reserve, kf_reserve, seed)
        h = ctypes.c_void_p()
        rc = self.lib.map_server_create(ctypes.byref(c), ctypes.byref(h))
        if rc != MAP_OK:
            raise MapError(rc, "map_server_create failed")
        self.h = h
        self._keep = {}          # render output buffers, alive until polled
        self._done = {}          # polled completions not yet handed out by wait()

    def close(self):
        if getattr(self, "h", None):
            self.lib.map_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, cfg, continuous_mapping=True, occ_every=0):
        ccfg = make_config(cfg, occ_every)
        sid = ctypes.c_uint32()
        rc = self.lib.map_server_add_scene(self.h, ctypes.byref(ccfg), int(continuous_mapping), ctypes.byref(sid))
        if rc != MAP_OK:
            raise MapError(rc, "scene not admitted" if rc == MAP_ENOMEM else "add_scene failed")
        return sid.value

    def scene_map(self, scene, cfg):
        """A NerfMap view of the scene's map (for parameter / occupancy I/O while the
        scene has no pending request); it does not own the map."""
        h = ctypes.c_void_p()
        rc = self.lib.map_server_scene_handle(self.h, scene, ctypes.byref(h))
        if rc != MAP_OK:
            raise MapError(rc, "bad scene")
        m = NerfMap.__new__(NerfMap)
        m.lib, m.cfg, m.h = self.lib, cfg, h
        m.n_params = m.stats().param_count
        m.close = lambda: None
        return m

    def submit_keyframe(self, scene, kf):
        rid = ctypes.c_uint64()
        c2w = np.ascontiguousarray(kf.c2w, np.float32).reshape(12)
        K = np.ascontiguousarray(kf.K, np.float32).reshape(4)
        rgb = np.ascontiguousarray(kf.rgb, np.float32)
        dep = np.ascontiguousarray(kf.depth, np.float32)
        var = np.ascontiguousarray(kf.var, np.float32)
        rc = self.lib.map_server_submit_keyframe(self.h, scene, kf.kf_id, c2w.ctypes.data, K.ctypes.data, kf.W,
                                                 kf.H, rgb.ctypes.data, dep.ctypes.data, var.ctypes.data,
                                                 int(bool(kf.depth_is_z)), ctypes.byref(rid))
        if rc != MAP_OK:
            raise MapError(rc, "submit_keyframe failed")
        return rid.value

    def submit_step(self, scene, n_rays, want_loss=True):
        rid = ctypes.c_uint64()
        rc = self.lib.map_server_submit_step(self.h, scene, n_rays, int(want_loss), ctypes.byref(rid))
        if rc != MAP_OK:
            raise MapError(rc, "submit_step failed")
        return rid.value

    def submit_render(self, scene, c2w, K, W, H):
        """Returns (request id, rgb [H,W,3], depth [H,W]); the arrays are filled when
        the request's completion is polled."""
        rid = ctypes.c_uint64()
        c2w = np.ascontiguousarray(c2w, np.float32).reshape(12)
        K = np.ascontiguousarray(K, np.float32).reshape(4)
        rgb = np.zeros((H, W, 3), np.float32)
        dep = np.zeros((H, W), np.float32)
        rc = self.lib.map_server_submit_render(self.h, scene, c2w.ctypes.data, K.ctypes.data, W, H,
                                               rgb.ctypes.data, dep.ctypes.data, ctypes.byref(rid))
        if rc != MAP_OK:
            raise MapError(rc, "submit_render failed")
        self._keep[rid.value] = (rgb, dep)
        return rid.value, rgb, dep

    def poll(self, cap=256):
        buf = (Completion * cap)()
        n = ctypes.c_uint32()
        rc = self.lib.map_server_poll(self.h, buf, cap, ctypes.byref(n))
        if rc != MAP_OK:
            raise MapError(rc, "poll failed")
        out = []
        for i in range(n.value):
            c = buf[i]
            self._keep.pop(c.req_id, None)
            out.append({"id": c.req_id, "scene": c.scene, "kind": c.kind, "status": c.status,
                        "step_index": c.step_index, "loss": c.loss, "t_submit": c.t_submit,
                        "t_start": c.t_start, "t_done": c.t_done})
        return out

    def wait(self, ids, timeout=120.0):
        """Polls until every request in `ids` has completed; returns their records."""
        import time
        want = set(ids)
        t0 = time.time()
        while want - set(self._done):
            for c in self.poll():
                self._done[c["id"]] = c
            if time.time() - t0 > timeout:
                raise TimeoutError(f"requests not done: {sorted(want - set(self._done))[:5]}")
            time.sleep(0.0005)
        return {i: self._done.pop(i) for i in ids}

    def stats(self):
        st = ServerStats()
        self.lib.map_server_get_stats(self.h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}


def render_group(maps, views, outs, stream=None):
    """map_render_group: maps [n] NerfMap, views [n] of (c2w [3,4], K [4], W, H), outs
    [n] of (rgb, depth) CUDA tensors ([H,W,3] and [H,W], either may be None)."""
    n = len(maps)
    lib = load()
    hs = (ctypes.c_void_p * n)(*[m.h.value for m in maps])
    c2w = np.ascontiguousarray(np.stack([np.asarray(v[0], np.float32).reshape(12) for v in views]))
    K = np.ascontiguousarray(np.stack([np.asarray(v[1], np.float32).reshape(4) for v in views]))
    W = np.array([v[2] for v in views], np.uint32)
    H = np.array([v[3] for v in views], np.uint32)
    rgb = (ctypes.c_void_p * n)(*[o[0].data_ptr() if o[0] is not None else None for o in outs])
    dep = (ctypes.c_void_p * n)(*[o[1].data_ptr() if o[1] is not None else None for o in outs])
    rc = lib.map_render_group(hs, n, c2w.ctypes.data, K.ctypes.data, W.ctypes.data, H.ctypes.data, rgb, dep,
                              _stream(stream))
    if rc != MAP_OK:
        raise MapError(rc, lib.map_last_error(maps[0].h).decode())


def marginal_covariances(C, P, blk, e, stream=None):
    """Sigma_T [c, c] and the per-pixel depth variances Sigma_d [p] of a dense-BA arrow
    Hessian (map_marginal_covariances).  Host numpy inputs (FP64; blk int32)."""
    lib = load()
    C = np.ascontiguousarray(C, np.float64)
    P = np.ascontiguousarray(P, np.float64)
    blk = np.ascontiguousarray(blk, np.int32)
    e = np.ascontiguousarray(e, np.float64)
    c, p, B = C.shape[0], P.shape[0], blk.shape[1]
    ST = np.zeros((c, c))
    Sd = np.zeros(p)
    rc = lib.map_marginal_covariances(C.ctypes.data, c, P.ctypes.data, p, blk.ctypes.data, e.ctypes.data, B,
                                      ST.ctypes.data, Sd.ctypes.data, MAP_MEM_HOST, _stream(stream))
    if rc != 0:
        raise MapError(rc, lib.map_last_error(None).decode())
    return ST, Sd
