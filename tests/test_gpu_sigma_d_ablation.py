"""The paper's depth-weighting claim on the synthetic room: with 20 % of the keyframe
pixels carrying a gross depth error (uniform within +-2 m) that the depth estimator
reports with sigma_d = 1 m, the Sigma_D-weighted depth loss fits better geometry than
the raw depth loss (every pixel at the median variance of the good pixels, so the
same overall depth weight without down-weighting the outliers) and than colour only
(lambda_D = 0), with colour quality far above the raw loss and near colour only.  Two
3000-step FP16 fits per variant (ray seeds 0 and 1, one workload; held-out views of
the camera path, as in bench.quality_run), compared on their means.

Bounds, from GB300 runs (single fits: weighted 18.6-20.6 dB / 0.314-0.327 m over
eleven fits, FP16 and FP32 alike, plus one FP16 fit whose colours stalled at 15.9 dB
with the same 0.321 m depth-L1; raw 15.3-15.8 dB / 0.339-0.351 m; colour only
20.0-20.7 dB / 0.463-0.488 m; the table gradients are summed by atomics in a varying
order, which a 3000-step fit amplifies into this spread): mean weighted depth-L1 at
most 0.97 x raw (a single-fit bound of 0.95 sat inside the spread: 0.3237 against
0.3388 m in one run) and 0.8 x colour only (the claim under test: the weighting buys
geometry); mean weighted PSNR not below raw and at least colour only - 5 dB."""

import json
import os

import pytest

pytestmark = pytest.mark.gpu


def test_sigma_d_weighting_beats_raw_and_colour_only():
    import torch
    import __graft_entry__
    import bench
    __graft_entry__.build()
    torch.cuda.set_device(0)
    wl = bench.quality_workload(n_poses=60, every=6, view_W=160, view_H=120, seed=0, sigma_floor=0.05,
                                outlier_frac=0.2)
    fits = {m: [bench.quality_fit(wl, "fp16", 3000, 1 << 16, ray_seed=rs, depth_weighting=m) for rs in (0, 1)]
            for m in ("sigma_d", "raw", "none")}
    path = os.environ.get("NERFMAP_QUALITY_REPORT")
    if path:
        with open(path, "a") as f:
            for m, xs in fits.items():
                for rs, x in enumerate(xs):
                    f.write(json.dumps({"run": "ablation_" + m, "ray_seed": rs, **x}) + "\n")
    mean = {m: {k: sum(x[k] for x in xs) / len(xs) for k in ("depth_l1_m", "psnr_db")} for m, xs in fits.items()}
    w, raw, none = mean["sigma_d"], mean["raw"], mean["none"]
    assert w["depth_l1_m"] <= 0.97 * raw["depth_l1_m"], mean
    assert w["depth_l1_m"] <= 0.8 * none["depth_l1_m"], mean
    assert w["psnr_db"] >= raw["psnr_db"], mean
    assert w["psnr_db"] >= none["psnr_db"] - 5.0, mean
