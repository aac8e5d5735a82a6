"""Random-access ceiling of the GPU for the hash-grid traffic (measurement tool).

    python -m paper_2210_13641_gb300.probe

Times uniformly random 8-byte reads and 8-byte FP32 vector reductions into tables
of 1 MB (the one-keyframe workload's grid), 64 MB (the room workload's grid,
L2-resident) and 1 GB (HBM-resident), through map_probe_random_access.
"""

import json
import sys


def main():
    import torch
    from paper_2210_13641_gb300 import binding
    torch.cuda.set_device(0)
    out = []
    for mb in (1, 64, 1024):
        n = (mb << 20) // 8
        table = torch.zeros((n, 2), device="cuda")
        for mode, name in ((0, "gather"), (1, "atomic")):
            r = binding.probe_random_access(table, per_thread=64, mode=mode)
            out.append({"table_mb": mb, "op": name, **r})
            print(f"{mb:6d} MB  {name:7s} {r['accesses_per_s'] / 1e9:8.1f} G/s  {r['payload_gbs']:8.1f} GB/s",
                  file=sys.stderr)
        del table
    print(json.dumps(out))


if __name__ == "__main__":
    main()
