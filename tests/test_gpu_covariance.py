"""The GPU marginal covariances of a dense-BA arrow Hessian (map_marginal_covariances,
Sec. 3.1 Eq. cov) against the FP64 oracle (pinned by the block-inverse identity in
test_oracle_covariance.py): Sigma_T and the per-pixel depth variances within 1e-9
relative (both sides FP64; the summation orders differ), invalid inputs refused."""

import numpy as np
import pytest

import oracle
from synth.arrow import arrow_hessian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    yield


@pytest.mark.parametrize("K,n,m", [(3, 50, 1), (10, 400, 3), (24, 200, 7)])
def test_marginal_covariances_match_oracle(K, n, m):
    from paper_2210_13641_gb300.binding import marginal_covariances
    h = arrow_hessian(K, n, m, seed=K)
    ST, Sd = marginal_covariances(h["C"], h["P"], h["blk"], h["e"])
    rST, rSd = oracle.marginal_covariances(h["C"], h["P"], h["blk"], h["e"])
    assert np.linalg.norm(ST - rST) <= 1e-9 * np.linalg.norm(rST)
    assert np.allclose(Sd, rSd, rtol=1e-9, atol=0)


def test_marginal_covariances_refuse_bad_input():
    from paper_2210_13641_gb300 import MapError
    from paper_2210_13641_gb300.binding import marginal_covariances
    h = arrow_hessian(3, 20, 1, seed=1)
    P = h["P"].copy()
    P[3] = -1.0
    with pytest.raises(MapError) as e:
        marginal_covariances(h["C"], P, h["blk"], h["e"])
    assert e.value.code == -1
    C = h["C"].copy()
    C[:6, :6] -= 1e7 * np.eye(6)                     # not positive definite
    with pytest.raises(MapError) as e:
        marginal_covariances(C, h["P"], h["blk"], h["e"])
    assert e.value.code == -1
