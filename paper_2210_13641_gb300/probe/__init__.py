"""Ceilings of the GPU for the hash-grid traffic (benchmark-side measurement tool;
not part of the mapping library or its ABI).

    python -m paper_2210_13641_gb300.probe

libnerfmap_probe.so (built by build.build_probe from probe/k_probe.cu) times:
  - uniformly random 8-byte reads and 8-byte FP32 vector reductions into tables of
    1 MB, 64 MB (the room workload's grid, L2-resident) and 1 GB (HBM-resident);
  - the streaming L2 bandwidth: coalesced 16-byte reads (L2 only) and 16-byte FP32
    vector reductions sweeping a buffer the size of the room workload's grid.
"""

from __future__ import annotations

import ctypes
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.path.dirname(HERE), "libnerfmap_probe.so")
_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnerfmap_probe.so not built at {LIB_PATH}: run paper_2210_13641_gb300.build.build_probe()")
    lib = ctypes.CDLL(LIB_PATH)
    lib.nmprobe_random_access.restype = ctypes.c_int
    lib.nmprobe_random_access.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    lib.nmprobe_l2_stream.restype = ctypes.c_int
    lib.nmprobe_l2_stream.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    _lib = lib
    return lib


def _best_ms(launch, reps: int) -> float:
    """Best CUDA-event time of `launch` over `reps` timed calls after one untimed."""
    import torch
    s = torch.cuda.current_stream()
    best = None
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        rc = launch(r, s.cuda_stream)
        e1.record(s)
        if rc != 0:
            raise RuntimeError(f"probe launch failed ({rc})")
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if r > 0 and (best is None or ms < best):
            best = ms
    return best


def random_access(table, per_thread: int, mode: int, n_threads: int = 152 * 2048, seed: int = 1,
                  reps: int = 5) -> dict:
    """Uniformly random 8-byte reads (mode 0) or FP32 vector reductions (mode 1) into
    a CUDA float32 tensor `table` ([n, 2], n a power of two): accesses/s and payload
    GB/s (best of `reps`)."""
    import torch
    lib = load()
    sink = torch.zeros(4, device=table.device)
    n = table.numel() // 2
    ms = _best_ms(lambda r, s: lib.nmprobe_random_access(table.data_ptr(), n, n_threads, per_thread, mode,
                                                         seed + r, sink.data_ptr(), s), reps)
    acc = n_threads * per_thread
    return {"accesses_per_s": acc / (ms / 1e3), "payload_gbs": acc * 8 / (ms / 1e3) / 1e9, "ms": ms}


def l2_stream(mbytes: float, mode: int, sweeps: int = 16, reps: int = 5, blocks_per_sm: int = 4) -> dict:
    """Streaming bandwidth over a buffer of `mbytes` MB: coalesced 16-byte L2 reads
    (mode 0) or 16-byte FP32 vector reductions (mode 1), `sweeps` sweeps per launch;
    payload GB/s (best of `reps`)."""
    import torch
    lib = load()
    n_vec = int(mbytes * (1 << 20)) // 16
    buf = torch.zeros(n_vec * 4, device="cuda")
    sink = torch.zeros(4, device="cuda")
    sms = torch.cuda.get_device_properties(buf.device).multi_processor_count
    ms = _best_ms(lambda r, s: lib.nmprobe_l2_stream(buf.data_ptr(), n_vec, sms * blocks_per_sm, sweeps, mode,
                                                     sink.data_ptr(), s), reps)
    del buf
    return {"buffer_mb": mbytes, "payload_gbs": n_vec * 16 * sweeps / (ms / 1e3) / 1e9, "ms": ms}


def main():
    import torch
    torch.cuda.set_device(0)
    out = []
    for mb in (1, 64, 1024):
        n = (mb << 20) // 8
        table = torch.zeros((n, 2), device="cuda")
        for mode, name in ((0, "gather"), (1, "atomic")):
            r = random_access(table, per_thread=64, mode=mode)
            out.append({"table_mb": mb, "op": name, **r})
            print(f"{mb:6d} MB  random {name:7s} {r['payload_gbs']:8.1f} GB/s", file=sys.stderr)
        del table
    for mb in (32, 64, 96):
        for mode, name in ((0, "read"), (1, "reduce")):
            r = l2_stream(mb, mode)
            out.append({"op": "stream_" + name, **r})
            print(f"{mb:6d} MB  stream {name:7s} {r['payload_gbs']:8.1f} GB/s", file=sys.stderr)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
