"""Random symmetric blocks with a prescribed spectrum (PSD-projection microbench).

Each block is Q diag(lam) Q^T with Q Haar-distributed (QR of a Gaussian with
the column-sign fix of Mezzadri 2007). The magnitudes are 10^(-4 t_i),
t_i ~ U(0,1) with one t pinned to 0 and one to 1 (condition number exactly
1e4), round(0.3 n) of the eigenvalues are negated (a seeded subset), and the
whole spectrum is multiplied by |g|, g ~ N(0,1).
"""
from __future__ import annotations

import numpy as np

MICROBENCH_SIZES = {8: 0.4, 36: 0.3, 78: 0.2, 136: 0.1}


def haar_orthogonal(rng, n):
    Z = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def sample_spectrum(rng, n):
    t = rng.uniform(0.0, 1.0, size=n)
    if n >= 2:
        t[0], t[1] = 0.0, 1.0
    lam = 10.0 ** (-4.0 * t)
    neg = rng.permutation(n)[: int(round(0.3 * n))]
    lam[neg] *= -1.0
    lam *= abs(rng.standard_normal())
    return lam


def known_spectrum_blocks(sizes, seed=1):
    """Blocks (list of n x n float64), their eigenvalues and eigenvectors."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    mats, lams, Qs = [], [], []
    for n in sizes:
        Q = haar_orthogonal(rng, n)
        lam = sample_spectrum(rng, n)
        A = (Q * lam) @ Q.T
        A = 0.5 * (A + A.T)
        mats.append(A)
        lams.append(lam)
        Qs.append(Q)
    return mats, lams, Qs


def microbench_sizes(nblocks=4096, seed=1, dist=None):
    dist = MICROBENCH_SIZES if dist is None else dist
    keys = sorted(dist)
    counts = [int(round(dist[k] * nblocks)) for k in keys]
    counts[-1] = nblocks - sum(counts[:-1])
    sizes = np.concatenate([np.full(c, k, dtype=np.int32) for k, c in zip(keys, counts)])
    rng = np.random.default_rng(np.random.PCG64(seed + 7919))
    return sizes[rng.permutation(len(sizes))]


def svec_pack(A):
    """Column-major upper triangle, off-diagonals times sqrt(2) (SDPT3 order)."""
    n = A.shape[0]
    iu = [(i, j) for j in range(n) for i in range(j + 1)]
    v = np.array([A[i, j] * (1.0 if i == j else np.sqrt(2.0)) for i, j in iu])
    return v


def psd_microbench(nblocks=4096, seed=1, dist=None):
    """(svec concatenation float64, block offsets int64, block sizes int32, mats)."""
    sizes = microbench_sizes(nblocks, seed, dist)
    mats, _, _ = known_spectrum_blocks(sizes, seed)
    parts = [svec_pack(A) for A in mats]
    off = np.zeros(len(parts) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    return np.concatenate(parts), off[:-1].copy(), sizes.astype(np.int32), mats
