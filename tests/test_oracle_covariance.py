"""Pins of the oracle's marginal covariances (Sec. 3.1, Eq. cov): they are the blocks
of the inverse of the whole arrow Hessian (the block-inverse identity), computed
here by a dense inverse; the depth variances are at least the conditional ones
(1/P); a planted mistake (the Schur complement with a plus sign) fails.  CPU only."""

import numpy as np

import oracle
from synth.arrow import arrow_hessian, dense_hessian


def test_marginals_are_blocks_of_the_inverse_hessian():
    for seed, (K, n, m) in enumerate([(3, 8, 1), (5, 20, 2), (6, 30, 3)]):
        h = arrow_hessian(K, n, m, seed)
        ST, Sd = oracle.marginal_covariances(h["C"], h["P"], h["blk"], h["e"])
        Hinv = np.linalg.inv(dense_hessian(h))
        c = h["c"]
        assert np.allclose(ST, Hinv[:c, :c], rtol=1e-9, atol=1e-12)
        assert np.allclose(Sd, np.diag(Hinv)[c:], rtol=1e-9, atol=1e-12)
        assert np.all(Sd >= 1.0 / h["P"] * (1 - 1e-12))
        assert np.allclose(ST, ST.T) and np.linalg.eigvalsh(ST).min() > 0


def test_planted_schur_sign_mistake_fails():
    h = arrow_hessian(4, 12, 2, 7)
    c = h["c"]
    E = oracle.arrow_dense_E(c, h["blk"], h["e"])
    wrong = np.linalg.inv(h["C"] + (E / h["P"]) @ E.T)
    Hinv = np.linalg.inv(dense_hessian(h))
    assert not np.allclose(wrong, Hinv[:c, :c], rtol=1e-3)
