"""Oracle: data-driven warm start from stored solutions (TEST INFRASTRUCTURE).

Sec. 5 (inverted pendulum) starts the solver from a convex combination of
the stored solutions of the three initial states nearest to the new one,
found through a Delaunay triangulation of the stored states. The paper does
not say how the combination is weighted; the reading used here:

  * neighbours: the min(d + 1, n) stored keys nearest to the query in
    Euclidean distance (d = key dimension), ties broken by lower index;
  * a query equal to a stored key takes that solution alone;
  * with d + 1 neighbours whose simplex is non-degenerate and contains the
    query (barycentric coordinates >= -1e-12), the weights are the query's
    barycentric coordinates in that simplex (clipped at 0, renormalised) --
    on a lattice whose Delaunay triangulation is unique this is the
    Delaunay triangle of the query (pinned against scipy's Delaunay);
  * otherwise weights proportional to 1 / distance;
  * X0 = sum_j w_j X_j, S0 = sum_j w_j S_j, y0 = 0 (Algorithm 1 takes X0, S0),
    sigma0 = prod_j sigma_j ** w_j.

Written from these definitions with NumPy; nothing here is shared with the
library.
"""
from __future__ import annotations

import numpy as np

BARY_SLACK = 1e-12      # barycentric coordinates down to -1e-12 count as inside
DEGENERATE = 1e-12      # simplex edge matrix with sigma_min <= 1e-12 * max|entry| is degenerate


def neighbours(keys: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Indices of the min(d + 1, n) stored keys nearest to key (ties: lower index first)."""
    keys = np.asarray(keys, dtype=np.float64).reshape(-1, np.size(key))
    key = np.asarray(key, dtype=np.float64).ravel()
    n, d = keys.shape
    dist2 = []
    for j in range(n):                       # squared distance, summed in coordinate order
        acc = 0.0
        for t in range(d):
            e = key[t] - keys[j, t]
            acc += e * e
        dist2.append(acc)
    order = sorted(range(n), key=lambda j: (dist2[j], j))
    return np.array(order[:min(d + 1, n)], dtype=np.int64), np.array(dist2)


def weights(keys: np.ndarray, key: np.ndarray):
    """(idx, w): neighbours of key and the convex weights of their solutions."""
    key = np.asarray(key, dtype=np.float64).ravel()
    keys = np.asarray(keys, dtype=np.float64).reshape(-1, key.size)
    d = key.size
    idx, dist2 = neighbours(keys, key)
    if idx.size == 0:
        return idx, np.zeros(0)
    if dist2[idx[0]] == 0.0:
        return idx[:1], np.ones(1)
    if idx.size == d + 1:
        E = (keys[idx[1:]] - keys[idx[0]]).T          # column c: k_{c+1} - k_0
        scale = np.max(np.abs(E))
        if scale > 0 and np.linalg.svd(E, compute_uv=False).min() > DEGENERATE * scale:
            lam = np.linalg.solve(E, key - keys[idx[0]])
            bary = np.concatenate([[1.0 - lam.sum()], lam])
            if np.all(bary >= -BARY_SLACK):
                bary = np.maximum(bary, 0.0)
                return idx, bary / bary.sum()
    inv = 1.0 / np.sqrt(dist2[idx])
    return idx, inv / inv.sum()


def combine(states, idx, w) -> np.ndarray:
    """sum_j w_j states[idx_j] (states: list or array of equal-length vectors)."""
    out = np.zeros_like(np.asarray(states[idx[0]], dtype=np.float64))
    for j, wj in zip(idx, w):
        out = out + wj * np.asarray(states[j], dtype=np.float64)
    return out


def sigma0(sigmas, idx, w) -> float:
    """Weighted geometric mean of the stored penalties."""
    return float(np.exp(sum(wj * np.log(sigmas[j]) for j, wj in zip(idx, w))))
