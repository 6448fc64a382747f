"""The seeded input recipes (CPU only): the 4096-block PSD microbench
(sizes {8: 40 %, 36: 30 %, 78: 20 %, 136: 10 %}; spectra with magnitudes
10^(-4 t), condition number exactly 1e4, round(0.3 n) negative eigenvalues,
Haar eigenvectors) and the pendulum batch (theta0 ~ U(-0.2, 0.2), request i
seeded with base + i)."""
import numpy as np

import workloads as wl
from workloads import psd_bench as PB
from workloads.problems import BASE_SEED


def test_microbench_size_mix_and_layout():
    x, off, n, mats = wl.psd_microbench()
    counts = {k: int(np.sum(n == k)) for k in (8, 36, 78, 136)}
    assert counts == {8: 1638, 36: 1229, 78: 819, 136: 410} and len(n) == 4096
    t = n.astype(np.int64) * (n + 1) // 2
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(t)[:-1]]))
    assert x.size == int(t.sum()) == 7_220_381
    assert np.array_equal(PB.microbench_sizes(), n)           # same seed, same order
    i = int(np.nonzero(n == 36)[0][0])
    A = mats[i]
    v = x[off[i]:off[i] + t[i]]
    # svec, column-major upper triangle: (0,0), sqrt(2) (0,1), (1,1), ...
    assert v[0] == A[0, 0] and abs(v[1] - np.sqrt(2) * A[0, 1]) <= 1e-15 * abs(A[0, 1]) and v[2] == A[1, 1]


def test_microbench_spectra():
    rng = np.random.default_rng(np.random.PCG64(3))
    for n in (8, 36, 78, 136):
        lam = PB.sample_spectrum(rng, n)
        mag = np.abs(lam)
        assert abs(mag.max() / mag.min() - 1e4) < 1e-6 * 1e4       # condition number exactly 1e4
        assert int(np.sum(lam < 0)) == int(round(0.3 * n))
    mats, lams, Qs = wl.known_spectrum_blocks([36, 78], seed=4)
    for A, lam, Q in zip(mats, lams, Qs):
        assert np.allclose(Q.T @ Q, np.eye(len(lam)), atol=1e-13)
        assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(lam), atol=1e-13)


def test_haar_sign_fix():
    """QR of a Gaussian with R's diagonal made positive (Mezzadri's fix): the
    returned Q times that R reproduces the Gaussian."""
    rng = np.random.default_rng(np.random.PCG64(9))
    Z = np.random.default_rng(np.random.PCG64(9)).standard_normal((6, 6))
    Q = PB.haar_orthogonal(rng, 6)
    Rm = Q.T @ Z
    assert np.allclose(np.tril(Rm, -1), 0, atol=1e-12) and np.all(np.diag(Rm) > 0)


def test_pendulum_batch_recipe():
    batch = wl.problem_batch("pendulum", 16, seed=BASE_SEED, N=4)
    th = np.array([p.meta["theta0"] for p in batch])
    assert np.all(np.abs(th) <= 0.2) and len(set(th.tolist())) == 16
    for i in (0, 5, 15):
        rng = np.random.default_rng(np.random.PCG64(BASE_SEED + i))
        assert th[i] == float(rng.uniform(-0.2, 0.2))
    assert all(p.N == 4 and p.nv == 7 for p in batch)


def test_serving_stream_recipe():
    """Config 5's stream: robots in the configured shares (50 / 30 / 20 %),
    horizons uniform over each robot's range, request j reproducible from
    its index alone; Poisson arrivals with the configured rate."""
    import numpy as np
    counts = {"pendulum": 0, "cartpole": 0, "rigid_body": 0}
    ranges = {k: rng for k, _, rng in wl.SERVING_MIX}
    seen = {k: set() for k in counts}
    n = 1500
    for j in range(n):
        kind, p = wl.mixed_request(j)
        counts[kind] += 1
        lo, hi = ranges[kind]
        assert lo <= p.N <= hi
        seen[kind].add(p.N)
    for kind, share, _ in wl.SERVING_MIX:
        assert abs(counts[kind] / n - share) < 0.04, (kind, counts)
    # every horizon of the pendulum's range appears (uniform over 51 values)
    assert seen["pendulum"] == set(range(10, 61))
    k0, p0 = wl.mixed_request(7)
    k1, p1 = wl.mixed_request(7)
    assert k0 == k1 and p0.N == p1.N and p0.meta == p1.meta
    t = wl.poisson_arrivals(40.0, 100.0)
    assert np.all(np.diff(t) > 0) and t[-1] < 100.0
    assert abs(len(t) - 4000) < 4 * np.sqrt(4000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 40.0) < 0.05 / 40.0
