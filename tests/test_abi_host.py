"""Host-side checks (no GPU): the library builds, loads and exports every symbol the
header declares; configuration marshalling and parameter packing are consistent with
the oracle's own definitions."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "nerfmap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(map_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_13641_gb300 import binding
    return binding.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2210_13641_gb300 import binding
    names = _header_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert sorted(binding.exported_symbols()) == names


def test_config_struct_layout(lib):
    from paper_2210_13641_gb300 import binding
    assert lib.map_abi_config_size() == ctypes.sizeof(binding.MapConfig)


def test_create_without_gpu_fails_cleanly(lib):
    """Without a device map_create returns an error code with a message (no crash)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2210_13641_gb300 import MapError, NerfMap
    with pytest.raises(MapError):
        NerfMap(synth.config_small())


def test_invalid_configs_rejected_before_device_use(lib):
    from paper_2210_13641_gb300 import binding
    for bad in (dict(n_levels=0), dict(log2_table=30), dict(max_samples=0), dict(occ_res=12)):
        c = binding.make_config(synth.config_small())
        for k, v in bad.items():
            setattr(c, k, v)
        h = ctypes.c_void_p()
        rc = lib.map_create(ctypes.byref(c), 0, ctypes.byref(h))
        assert rc == binding.MAP_EINVAL, bad
        assert lib.map_last_error(None)


def test_checkpoint_refusals_before_device_use(lib, tmp_path):
    """map_load rejects a missing, foreign or truncated file (and map_save a null map)
    with MAP_EINVAL and a message, before it touches a device."""
    from paper_2210_13641_gb300 import binding
    h = ctypes.c_void_p()
    assert lib.map_load(str(tmp_path / "missing.ckpt").encode(), 0, ctypes.byref(h)) == binding.MAP_EINVAL
    assert b"cannot open" in lib.map_last_error(None) and not h.value
    foreign = tmp_path / "foreign.ckpt"
    foreign.write_bytes(b"not a map checkpoint at all" * 4)
    assert lib.map_load(str(foreign).encode(), 0, ctypes.byref(h)) == binding.MAP_EINVAL
    assert b"not a checkpoint" in lib.map_last_error(None)
    truncated = tmp_path / "truncated.ckpt"
    truncated.write_bytes(b"NMAPCKPT" + (1).to_bytes(4, "little"))
    assert lib.map_load(str(truncated).encode(), 0, ctypes.byref(h)) == binding.MAP_EINVAL
    assert lib.map_load(None, 0, ctypes.byref(h)) == binding.MAP_EINVAL
    assert lib.map_load(str(foreign).encode(), 0, None) == binding.MAP_EINVAL
    assert lib.map_save(None, str(tmp_path / "x.ckpt").encode(), 1, None) == binding.MAP_EINVAL


@pytest.mark.parametrize("mk", [synth.config_small, synth.config_c1, synth.config_c2, synth.config_c5])
def test_level_table_matches_oracle(lib, mk):
    """The library's level table (map_config_init, host only) equals the oracle's."""
    from paper_2210_13641_gb300 import binding
    cfg = mk()
    assert binding.level_resolutions(cfg) == oracle.level_resolutions(cfg)


def test_config_init_defaults_and_refusals(lib):
    from paper_2210_13641_gb300 import binding
    c = binding.MapConfig()
    assert lib.map_config_init(ctypes.byref(c), 16, 19, 16, 2048, 0.0) == 0
    assert lib.map_last_error(None) == b""
    assert (c.n_features, c.enc_width, c.density_hidden, c.geo_width, c.color_hidden) == (2, 32, 64, 16, 64)
    assert c.level_res[0] == 16 and c.level_res[15] == 2048 and c.level_res[16] == 0
    assert c.precision == binding.PRECISION["fp16"] and c.max_samples == 128 and c.step_t == 0.0
    for args in ((0, 19, 16, 2048, 0.0), (17, 19, 16, 2048, 0.0), (16, 9, 16, 2048, 0.0), (16, 19, 1, 2048, 0.0),
                 (16, 19, 16, 16, 0.0), (16, 19, 16, 0, -1.0), (16, 19, 2, 0, 4.0)):
        assert lib.map_config_init(ctypes.byref(c), *args) == binding.MAP_EINVAL, args
        assert lib.map_last_error(None).startswith(b"map_config_init"), args
    assert lib.map_config_init(None, 16, 19, 16, 2048, 0.0) == binding.MAP_EINVAL


def test_march_noalloc_allocates_nothing_in_source():
    """The allocation-free march's translation unit calls no allocating routine
    (comments aside): no cudaMalloc / cudaFree in any form, no cudaMallocHost."""
    src = open(os.path.join(ROOT, "paper_2210_13641_gb300", "csrc", "k_march_noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    assert "cudaGetSymbolAddress" in code
    for bad in ("cudaMalloc", "cudaFree", "cuMemAlloc", "cuMemFree", "malloc(", "new "):
        assert bad not in code, bad


def test_pack_unpack_roundtrip():
    from paper_2210_13641_gb300 import pack_params, unpack_params
    cfg = synth.config_small()
    P = synth.random_params(cfg, 1)
    flat = pack_params(P)
    assert flat.size == cfg.n_levels * cfg.table_size * 2 + 9408
    Q = unpack_params(flat, cfg.n_levels, cfg.log2_table)
    for k in P:
        assert np.array_equal(P[k], Q[k])


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2210_13641_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f


def _header_defines():
    src = open(os.path.join(ROOT, "include", "nerfmap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(MAP_\w+)\s+\(?(-?\d+)u?\)?", src)}


def test_binding_constants_match_the_header():
    """The binding's status codes, memory kinds, step flags, precisions, phases and
    serving request kinds are the header's values (a drifted constant would pass
    the wrong flag or misread a status without any other test noticing)."""
    from paper_2210_13641_gb300 import binding
    d = _header_defines()
    for name in ("MAP_OK", "MAP_EINVAL", "MAP_ENOMEM", "MAP_ENOKF", "MAP_ETIMEOUT", "MAP_ECUDA",
                 "MAP_MEM_HOST", "MAP_MEM_DEVICE", "MAP_STEP_NO_UPDATE", "MAP_STEP_POSE_GRAD", "MAP_SAVE_KEYFRAMES"):
        assert getattr(binding, name) == d[name], name
    assert binding.PRECISION == {"fp32": d["MAP_PREC_FP32"], "fp16": d["MAP_PREC_FP16"], "bf16": d["MAP_PREC_BF16"]}
    assert (binding.REQ_KEYFRAME, binding.REQ_STEP, binding.REQ_RENDER) == \
        (d["MAP_REQ_KEYFRAME"], d["MAP_REQ_STEP"], d["MAP_REQ_RENDER"])
    ph = {k: v for k, v in d.items() if k.startswith("MAP_PH_")}
    assert len(binding.PHASES) == d["MAP_PHASES"] == len(ph)
    order = ["MAP_PH_RAYGEN", "MAP_PH_MARCH", "MAP_PH_FIELD_FWD", "MAP_PH_COMPOSITE", "MAP_PH_FIELD_BWD",
             "MAP_PH_ADAM", "MAP_PH_OCC", "MAP_PH_OUTPUT"]
    assert [ph[k] for k in order] == list(range(len(order)))
    assert binding.PHASES[ph["MAP_PH_FIELD_BWD"]] == "field_bwd" and binding.PHASES[ph["MAP_PH_ADAM"]] == "adam"
    assert binding.MapConfig.level_res.size == 4 * d["MAP_MAX_LEVELS"]
