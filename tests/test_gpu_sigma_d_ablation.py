"""The paper's depth-weighting claim on the synthetic room: with 20 % of the keyframe
pixels carrying a gross depth error (uniform within +-2 m) that the depth estimator
reports with sigma_d = 1 m, the Sigma_D-weighted depth loss fits better geometry than
the raw depth loss (every pixel at the median variance of the good pixels, so the
same overall depth weight without down-weighting the outliers) and than colour only
(lambda_D = 0), with colour quality far above the raw loss and near colour only.  One 3000-step FP16 fit per variant
(ray seed 0; held-out views of the camera path, as in bench.quality_run).

Bounds, from GB300 runs (weighted 18.6-20.6 dB / 0.314-0.327 m over eleven fits,
FP16 and FP32 alike, plus one FP16 fit whose colours stalled at 15.9 dB with the
same 0.321 m depth-L1; raw 15.3-15.8 dB / 0.342-0.351 m; colour only 20.0-20.7 dB /
0.463-0.488 m): weighted depth-L1 at most 0.95 x raw and 0.8 x colour only (the
claim under test: the weighting buys geometry); weighted PSNR not below raw and at
least colour only - 5 dB."""

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
    r = {m: bench.quality_run("fp16", steps=3000, outlier_frac=0.2, depth_weighting=m, sigma_floor=0.05)
         for m in ("sigma_d", "raw", "none")}
    path = os.environ.get("NERFMAP_QUALITY_REPORT")
    if path:
        with open(path, "a") as f:
            for m, x in r.items():
                f.write(json.dumps({"run": "ablation_" + m, **x}) + "\n")
    w, raw, none = r["sigma_d"], r["raw"], r["none"]
    assert w["depth_l1_m"] <= 0.95 * raw["depth_l1_m"], r
    assert w["depth_l1_m"] <= 0.8 * none["depth_l1_m"], r
    assert w["psnr_db"] >= raw["psnr_db"], r
    assert w["psnr_db"] >= none["psnr_db"] - 5.0, r
