"""The bounded-wait error path of the tensor-core kernels, made to run out on purpose.

With the poll limit of the MMA-completion waits set to zero (map_set_wait_polls),
every wait of the forward and backward field kernels expires at once: nothing waits
forever and nothing faults.  The kernels must then stop, wait for the MMAs they have
issued, free their tensor memory and raise the device flag, and the host must report
MAP_ETIMEOUT.  Afterwards the same map, with the default limit back, and a fresh map
must step and render exactly as the oracle says (the FP16 tolerance of
test_gpu_tc.py).
"""

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


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_expired_waits_report_timeout_and_the_map_recovers(prec):
    from paper_2210_13641_gb300 import MapError, NerfMap, pack_params
    from paper_2210_13641_gb300.binding import MAP_ETIMEOUT
    cfg = synth.config_c1(precision=prec)
    P = synth.random_params(cfg, 0)
    kf = synth.c1_keyframe(0)
    ref = oracle.forward_backward(cfg, P, [kf], 512, 3, 0, mlp_bits=prec)

    m = NerfMap(cfg, occ_every=0)
    m.set_params(pack_params(P))
    m.add_keyframe(kf)
    m.set_wait_polls(0)
    with pytest.raises(MapError) as e:
        m.step(512, seed=3, no_update=True)
    assert e.value.code == MAP_ETIMEOUT
    with pytest.raises(MapError) as e:
        m.render(kf.c2w, kf.K, 16, 12)
    assert e.value.code == MAP_ETIMEOUT

    # the same map with the default limit: correct again
    m.set_wait_polls(1 << 24)
    m.set_params(pack_params(P))
    loss = m.step(512, seed=3, no_update=True)
    assert abs(loss - ref["loss"]) <= TOL * abs(ref["loss"])
    G = m.unpack(m.get_grads())
    for k in ("tables", "W1", "W5"):
        err = np.linalg.norm(G[k] - ref["grads"][k]) / np.linalg.norm(ref["grads"][k])
        assert err <= TOL, (k, err)
    m.close()

    # and a fresh map
    m2 = NerfMap(cfg, occ_every=0)
    m2.set_params(pack_params(P))
    m2.add_keyframe(kf)
    loss2 = m2.step(512, seed=3, no_update=True)
    assert abs(loss2 - ref["loss"]) <= TOL * abs(ref["loss"])
    m2.close()
