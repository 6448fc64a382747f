"""Pins of the warm-start oracle (Sec. 5, nearest-neighbour warm start), and
parity of the library's host-side neighbour selection with it."""
import numpy as np
import pytest

from oracle import warm as W


def _tri_lattice(nx, ny, h=1.0):
    """Equilateral triangular lattice: no four points on a circle, so its Delaunay triangulation is unique."""
    pts = []
    for j in range(ny):
        for i in range(nx):
            pts.append((h * (i + 0.5 * (j % 2)), h * j * np.sqrt(3.0) / 2.0))
    return np.array(pts)


def test_affine_functions_are_reproduced_inside_the_hull():
    # barycentric weights interpolate affine data exactly: sum w_j f(k_j) = f(q)
    rng = np.random.default_rng(11)
    keys = _tri_lattice(8, 8)
    a, c = rng.normal(size=2), rng.normal()
    f = keys @ a + c
    for _ in range(200):
        q = rng.uniform([1.0, 1.0], [6.0, 5.0])
        idx, w = W.weights(keys, q)
        assert idx.size == 3 and np.all(w >= 0) and abs(w.sum() - 1) < 1e-15
        assert abs(w @ f[idx] - (q @ a + c)) < 1e-12
        assert np.allclose(w @ keys[idx], q, atol=1e-12)


def test_lattice_matches_scipy_delaunay():
    # the paper finds the neighbours through a Delaunay triangulation; on a
    # lattice with a unique triangulation the three nearest keys are the
    # vertices of the Delaunay triangle holding the query
    spatial = pytest.importorskip("scipy.spatial")
    keys = _tri_lattice(9, 9, h=0.37)
    tri = spatial.Delaunay(keys)
    rng = np.random.default_rng(12)
    for _ in range(300):
        q = rng.uniform([0.4, 0.4], [2.6, 2.4])
        s = int(tri.find_simplex(q))
        assert s >= 0
        T = tri.transform[s]
        b = T[:2] @ (q - T[2])
        bary = np.concatenate([b, [1.0 - b.sum()]])
        ref = dict(zip(tri.simplices[s].tolist(), bary))
        idx, w = W.weights(keys, q)
        assert sorted(idx.tolist()) == sorted(ref)
        for j, wj in zip(idx, w):
            assert abs(wj - ref[int(j)]) < 1e-12


def test_one_dimensional_keys_interpolate_linearly():
    keys = np.array([[0.0], [1.0], [3.0], [7.0]])
    idx, w = W.weights(keys, [2.5])
    assert sorted(idx.tolist()) == [1, 2]
    got = dict(zip(idx.tolist(), w))
    assert abs(got[1] - (3.0 - 2.5) / 2.0) < 1e-15 and abs(got[2] - (2.5 - 1.0) / 2.0) < 1e-15


def test_exact_key_takes_that_solution_alone():
    keys = _tri_lattice(4, 4)
    idx, w = W.weights(keys, keys[5])
    assert idx.tolist() == [5] and w.tolist() == [1.0]


def test_outside_the_hull_uses_inverse_distance():
    keys = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0]])
    q = np.array([0.0, -2.0])                     # distances sqrt5, sqrt5, 3: outside the triangle
    idx, w = W.weights(keys, q)
    assert idx.tolist() == [0, 1, 2]
    inv = np.array([1 / np.sqrt(5), 1 / np.sqrt(5), 1 / 3.0])
    assert np.allclose(w, inv / inv.sum(), rtol=0, atol=1e-15)


def test_degenerate_simplex_falls_back_to_inverse_distance():
    keys = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [5.0, 5.0]])
    q = np.array([0.9, 0.0])                      # the three nearest keys are collinear
    idx, w = W.weights(keys, q)
    assert idx.tolist() == [1, 0, 2]
    d = np.array([0.1, 0.9, 1.1])
    assert np.allclose(w, (1 / d) / (1 / d).sum(), rtol=0, atol=1e-15)


def test_neighbours_are_the_nearest():
    rng = np.random.default_rng(13)
    for d in (1, 2, 3, 4):
        keys = rng.normal(size=(40, d))
        for _ in range(20):
            q = rng.normal(size=d)
            idx, dist2 = W.neighbours(keys, q)
            far = np.setdiff1d(np.arange(40), idx)
            assert dist2[idx].max() <= dist2[far].min()


def test_combination_and_sigma():
    X = [np.full(5, 1.0), np.full(5, 3.0), np.arange(5.0)]
    out = W.combine(X, [2, 0], [0.25, 0.75])
    assert np.allclose(out, 0.25 * np.arange(5.0) + 0.75)
    assert abs(W.sigma0([2.0, 8.0], [0, 1], [0.5, 0.5]) - 4.0) < 1e-15


# ---- the library's host-side selection (strom_warm_select) against the oracle
def _lib():
    S = pytest.importorskip("paper_2406_05846_gb300")
    try:
        S.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    return S


@pytest.mark.parametrize("d", [1, 2, 3, 4, 8])
def test_library_selection_matches_oracle(d):
    S = _lib()
    rng = np.random.default_rng(100 + d)
    keys = rng.uniform(-1, 1, size=(60, d))
    qs = list(rng.uniform(-1.3, 1.3, size=(150, d))) + [keys[7], keys[59]]
    for q in qs:
        i_ref, w_ref = W.weights(keys, q)
        i_lib, w_lib = S.warm_select(keys, q)
        assert i_lib.tolist() == i_ref.tolist()
        assert np.allclose(w_lib, w_ref, rtol=0, atol=1e-12)


def test_library_selection_edge_cases():
    S = _lib()
    idx, w = S.warm_select(np.zeros((0, 2)), [0.3, 0.1])       # empty store: cold start
    assert idx.size == 0 and w.size == 0
    keys = np.array([[0.0, 0.0], [1.0, 0.0]])                   # fewer than d + 1 keys
    i_lib, w_lib = S.warm_select(keys, [0.25, 0.5])
    i_ref, w_ref = W.weights(keys, [0.25, 0.5])
    assert i_lib.tolist() == i_ref.tolist() and np.allclose(w_lib, w_ref, atol=1e-15)
    keys = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [5.0, 5.0]])   # collinear neighbours
    i_lib, w_lib = S.warm_select(keys, [0.9, 0.0])
    i_ref, w_ref = W.weights(keys, [0.9, 0.0])
    assert i_lib.tolist() == i_ref.tolist() and np.allclose(w_lib, w_ref, atol=1e-15)
    keys = _tri_lattice(5, 5)                                   # ties: lower index first
    q = keys[6] + (keys[7] - keys[6]) * 0.5
    assert S.warm_select(keys, q)[0].tolist() == W.weights(keys, q)[0].tolist()
    with pytest.raises(Exception):
        S.warm_select(keys, [np.nan, 0.0])
    with pytest.raises(Exception):
        S.warm_select(np.zeros((3, 9)), np.zeros(9))           # key dimension above the limit
