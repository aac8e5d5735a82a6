"""Parity of the tensor-core (FP16 / BF16 MLP) mapping path with the FP64 oracle.

Two oracles.  The rounding model (oracle mlp_bits: every MLP operand rounded to the
format's 11 or 8 significant bits, products summed exactly) is the FP64 oracle of
an MLP whose operands are FP16 / BF16, which the precision pattern prescribes; the
plain oracle is the unrounded FP64 chain.

Tolerances: against the rounding model, the benchmark spec's 2e-3 relative on the loss,
on per-ray colour, depth and opacity (plus 2e-3 absolute) and on every gradient
tensor (relative L2), in both formats.  Against the plain oracle, every gradient
tensor within 2e-3 plus the rounding model's own distance from the plain oracle on
the same inputs (the floor no FP16 / BF16 MLP can go below: a pre-activation within
a rounding of zero takes the other ReLU branch; test_oracle_pins pins that floor
above 2e-3 on the C1 step), and the loss within 2e-3.  Sample lists are bit-exact
(they do not depend on the MLP).  When NERFMAP_PRECISION_REPORT names a file, the
measured errors are appended to it as JSON lines.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 2e-3


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    torch.cuda.init()
    yield


def _map(cfg, P, kfs, occ_bits=None):
    from paper_2210_13641_gb300 import NerfMap, pack_params
    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    for kf in kfs:
        m.add_keyframe(kf)
    if occ_bits is not None:
        m.set_occupancy(occ_bits)
    return m


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _report(case, prec, errs):
    path = os.environ.get("NERFMAP_PRECISION_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": case, "precision": prec, **errs}) + "\n")


def _step_case(name, cfg, P, kfs, n, seed, bits=None):
    m = _map(cfg, P, kfs, bits)
    loss = m.step(n, seed=seed, no_update=True)
    ref = oracle.forward_backward(cfg, P, kfs, n, seed, 0, occ_bits=bits, mlp_bits=cfg.precision)
    plain = oracle.forward_backward(cfg, P, kfs, n, seed, 0, occ_bits=bits)
    rid, t = m.samples()
    assert np.array_equal(rid, ref["ray_id"].astype(np.uint32)) and np.array_equal(t, ref["t"])
    rgb, D, acc = m.ray_outputs(n)
    G = m.unpack(m.get_grads())
    errs = {"loss": abs(loss - ref["loss"]) / abs(ref["loss"]),
            "rgb_max_abs": float(np.abs(rgb - ref["I_hat"]).max()),
            "depth_rel": _rel(D, ref["D_hat"]), "acc_max_abs": float(np.abs(acc - ref["acc"]).max())}
    for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
        errs["grad_" + k] = _rel(G[k], ref["grads"][k])
        errs["plain_grad_" + k] = _rel(G[k], plain["grads"][k])
        errs["floor_grad_" + k] = _rel(ref["grads"][k], plain["grads"][k])
    errs["plain_loss"] = abs(loss - plain["loss"]) / abs(plain["loss"])
    _report(name, cfg.precision, errs)
    assert errs["loss"] <= TOL and errs["plain_loss"] <= TOL, errs
    assert np.allclose(rgb, ref["I_hat"], rtol=TOL, atol=TOL)
    assert np.allclose(D, ref["D_hat"], rtol=TOL, atol=TOL)
    assert np.allclose(acc, ref["acc"], rtol=TOL, atol=TOL)
    for k in ("tables", "W1", "W2", "W3", "W4", "W5"):
        assert errs["grad_" + k] <= TOL, (k, errs)
        assert errs["plain_grad_" + k] <= TOL + errs["floor_grad_" + k], (k, errs)
    return m


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_c1_step_tensor_cores(prec):
    cfg = synth.config_c1(precision=prec)
    _step_case("c1", cfg, synth.random_params(cfg, 0), [synth.c1_keyframe(0)], 4096, 7)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_trained_scale_field_tensor_cores(prec):
    """Table values of a fitted field (|f| ~ 0.1..1) and larger weights, several
    keyframes, occupancy and truncation, a ragged ray count."""
    cfg = synth.config_small(precision=prec, occ_res=16, step=np.float32(0.02), n_steps=150)
    P = synth.random_params(cfg, 3, table_scale=0.5, mlp_std=0.15)
    kfs = []
    for j, (W, H) in enumerate([(40, 30), (23, 17)]):
        kf = synth.c1_keyframe(20 + j, W=W, H=H, kf_id=j)
        kf.depth_is_z = True
        kfs.append(kf)
    bits = np.packbits(np.random.default_rng(5).uniform(size=16 ** 3) < 0.7, bitorder="little")
    _step_case("small_trained", cfg, P, kfs, 2999, 13, bits)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_render_tensor_cores(prec):
    cfg = synth.config_small(precision=prec, occ_res=0)
    P = synth.random_params(cfg, 8, table_scale=0.5, mlp_std=0.15)
    P["W2"][0] += 0.5
    m = _map(cfg, P, [synth.c1_keyframe(0, W=8, H=8)])
    kf = synth.c1_keyframe(9, W=40, H=30)
    rgb, D, acc = m.render(kf.c2w, kf.K, 40, 30)
    I_ref, D_ref, A_ref = oracle.render(cfg, P, kf.c2w, kf.K, 40, 30, t_min=float(cfg.render_t_min),
                                        mlp_bits=prec)
    errs = {"rgb_max_abs": float(np.abs(rgb.reshape(-1, 3) - I_ref).max()),
            "depth_rel": _rel(D.ravel(), D_ref), "acc_max_abs": float(np.abs(acc.ravel() - A_ref).max())}
    _report("render_small", prec, errs)
    assert np.allclose(rgb.reshape(-1, 3), I_ref, rtol=TOL, atol=TOL)
    assert np.allclose(D.ravel(), D_ref, rtol=TOL, atol=TOL)
    assert np.allclose(acc.ravel(), A_ref, rtol=TOL, atol=TOL)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_steps_with_adam_stay_finite_and_reduce_loss(prec):
    cfg = synth.config_c1(precision=prec)
    P = synth.random_params(cfg, 1)
    m = _map(cfg, P, [synth.c1_keyframe(3)])
    losses = [m.step(4096, seed=s) for s in range(30)]
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-5:]) < 0.9 * np.mean(losses[:5])
    assert np.all(np.isfinite(m.get_params()))
