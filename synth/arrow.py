"""Seeded synthetic dense-BA Hessians with the cameras/depths arrow structure of the
tracking frontend's bundle adjustment (the producer of the mapping loss's per-pixel
depth variances): K keyframe poses (6 parameters each) and one inverse depth per
pixel of every keyframe.  Each keyframe is linked to `m` other keyframes; for every
link (i, j) and pixel u of keyframe i a 2-vector flow residual depends on pose i,
pose j and the pixel's inverse depth d_iu, with random Jacobians and a positive
diagonal weight.  Accumulating J^T W J gives the blocks of

    H = [[C, E], [E^T, P]],   C: 6K x 6K,  P: diagonal (one entry per pixel),

with E stored block-sparse: per pixel the 6-vectors of the poses it touches.  A
prior on pose 0 fixes the gauge, so H is positive definite.  Nothing here is part
of the covariance computation itself."""

from __future__ import annotations

import numpy as np


def arrow_hessian(n_kf: int = 6, px_per_kf: int = 48, links: int = 2, seed: int = 0, gauge_prior: float = 1e4):
    """Returns dict(C [c, c], P [p], blk [p, B] int32 (pose index per block, -1 =
    unused), e [p, B, 6], c = 6 n_kf, p = n_kf * px_per_kf, B = links + 1).  FP64."""
    rng = np.random.default_rng(seed)
    c = 6 * n_kf
    n = px_per_kf
    p = n_kf * n
    B = links + 1
    C = np.zeros((c, c))
    P = np.zeros(p)
    blk = -np.ones((p, B), np.int32)
    e = np.zeros((p, B, 6))
    for i in range(n_kf):
        others = rng.choice([k for k in range(n_kf) if k != i], size=min(links, n_kf - 1), replace=False)
        rows = slice(i * n, (i + 1) * n)
        blk[rows, 0] = i
        for jj, j in enumerate(others):
            blk[rows, jj + 1] = j
            Ji = rng.normal(size=(n, 2, 6))
            Jj = rng.normal(size=(n, 2, 6))
            Jd = rng.normal(size=(n, 2)) * 3.0
            w = rng.uniform(0.2, 2.0, size=(n, 2))             # diagonal flow weights
            for (a, Ja) in ((i, Ji), (j, Jj)):
                for (bb, Jb) in ((i, Ji), (j, Jj)):
                    C[6 * a:6 * a + 6, 6 * bb:6 * bb + 6] += np.einsum("nra,nr,nrb->ab", Ja, w, Jb)
            P[rows] += np.einsum("nr,nr,nr->n", Jd, w, Jd)
            e[rows, 0] += np.einsum("nra,nr,nr->na", Ji, w, Jd)
            e[rows, jj + 1] += np.einsum("nra,nr,nr->na", Jj, w, Jd)
    C[:6, :6] += gauge_prior * np.eye(6)
    return dict(C=C, P=P, blk=blk, e=e, c=c, p=p, B=B)


def dense_hessian(h: dict) -> np.ndarray:
    """The full (c + p) x (c + p) matrix H of an arrow_hessian result."""
    c, p = h["c"], h["p"]
    H = np.zeros((c + p, c + p))
    H[:c, :c] = h["C"]
    H[c:, c:] = np.diag(h["P"])
    for q in range(p):
        for b in range(h["B"]):
            k = h["blk"][q, b]
            if k < 0:
                continue
            H[6 * k:6 * k + 6, c + q] += h["e"][q, b]
            H[c + q, 6 * k:6 * k + 6] += h["e"][q, b]
    return H
