"""Flat-extension and partial rank-1 tests of a moment matrix (Sec. 2.2; the
car back-in experiment): oracle pins from moment matrices of atomic
measures, and parity of the library's host implementation with the oracle."""
import numpy as np
import pytest

from oracle import certify as OC
from oracle.relax import monomial_basis


def _vec(z):
    b = monomial_basis(len(z), 2)
    return np.array([np.prod([z[t] ** e[t] for t in range(len(z))]) for e in b])


def _moments(points, weights):
    """Moment matrix of order 2 of the measure sum_i w_i delta_{z_i}."""
    return sum(w * np.outer(_vec(z), _vec(z)) for z, w in zip(points, weights))


def test_rank_one_lifting():
    z = np.array([0.3, -0.5, 0.7, 0.1])
    r = OC.moment_rank_tests(_moments([z], [1.0]), 4)
    assert (r["rank"], r["rank_low"], r["flat"]) == (1, 1, True)
    assert abs(r["ratio_sub"]) < 1e-14
    assert np.allclose(r["zbar_sub"], z, atol=1e-12)


def test_two_atoms_are_flat_with_the_gram_spectrum():
    z1, z2, w = np.array([0.3, -0.5, 0.7]), np.array([-0.2, 0.4, 0.1]), 0.3
    r = OC.moment_rank_tests(_moments([z1, z2], [w, 1 - w]), 3)
    assert (r["rank"], r["rank_low"], r["flat"]) == (2, 2, True)
    # the nonzero eigenvalues of w v1 v1^T + (1-w) v2 v2^T are those of the
    # 2x2 Gram matrix of sqrt(w) v1 and sqrt(1-w) v2
    a, b = np.sqrt(w) * _vec(z1), np.sqrt(1 - w) * _vec(z2)
    G = np.array([[a @ a, a @ b], [a @ b, b @ b]])
    tr, det = np.trace(G), np.linalg.det(G)
    lo, hi = (tr - np.sqrt(tr * tr - 4 * det)) / 2, (tr + np.sqrt(tr * tr - 4 * det)) / 2
    assert abs(r["ratio_sub"] - lo / hi) < 1e-12
    assert abs(r["lambda_max"] - hi) < 1e-12 * hi


def test_three_atoms_on_a_line_are_not_flat():
    # one variable: [z]_2 = (1, x, x^2); three distinct atoms give a full-rank
    # 3x3 Hankel matrix while [z]_1 only spans rank 2
    r = OC.moment_rank_tests(_moments([[-0.5], [0.1], [0.8]], [0.2, 0.5, 0.3]), 1)
    assert (r["rank"], r["rank_low"], r["flat"]) == (3, 2, False)


def test_partial_rank_one_on_shared_variables():
    # two atoms that agree on the first two variables: M is rank 2, its
    # submatrix on those variables is rank 1 and yields them exactly
    z1, z2 = np.array([0.3, -0.5, 0.7, 0.2]), np.array([0.3, -0.5, -0.4, 0.9])
    M = _moments([z1, z2], [0.6, 0.4])
    full = OC.moment_rank_tests(M, 4)
    part = OC.moment_rank_tests(M, 4, vars_mask=[1, 1, 0, 0])
    assert full["rank"] == 2 and full["ratio_sub"] > 1e-3
    assert part["n_sub"] == 6 and abs(part["ratio_sub"]) < 1e-14
    assert np.allclose(part["zbar_sub"][:2], z1[:2], atol=1e-12) and np.all(np.isnan(part["zbar_sub"][2:]))


# ---- the library's host implementation against the oracle
@pytest.fixture(scope="module")
def S():
    pkg = pytest.importorskip("paper_2406_05846_gb300")
    try:
        pkg.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    return pkg


def _same(a, b):
    assert (a["n"], a["rank"], a["rank_low"], a["flat"], a["n_sub"]) == \
           (b["n"], b["rank"], b["rank_low"], b["flat"], b["n_sub"])
    assert abs(a["ratio_sub"] - b["ratio_sub"]) < 1e-10
    assert abs(a["lambda_max"] - b["lambda_max"]) <= 1e-12 * abs(b["lambda_max"])
    fa, fb = np.isfinite(a["zbar_sub"]), np.isfinite(b["zbar_sub"])
    assert np.array_equal(fa, fb)
    assert np.allclose(a["zbar_sub"][fa], b["zbar_sub"][fb], rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("nv", [1, 3, 7, 9])
def test_library_matches_oracle(S, nv):
    rng = np.random.default_rng(40 + nv)
    cases = []
    for atoms in (1, 2, 3):
        pts = rng.uniform(-1, 1, size=(atoms, nv))
        cases.append(_moments(pts, rng.dirichlet(np.ones(atoms))))
    n = (nv + 1) * (nv + 2) // 2
    B = rng.standard_normal((n, n))
    cases.append(B @ B.T / n)                                   # full rank
    for M in cases:
        masks = [None, rng.integers(0, 2, nv).astype(bool)]
        for vm in masks:
            _same(S.moment_rank_test(M, nv, vm), OC.moment_rank_tests(M, nv, vm))


def test_library_rejects_bad_input(S):
    M = _moments([np.array([0.1, 0.2])], [1.0])
    bad = M.copy()
    bad[0, 3] += 1.0
    with pytest.raises(RuntimeError, match="symmetric"):
        S.moment_rank_test(bad, 2)
    bad = M.copy()
    bad[1, 1] = np.nan
    with pytest.raises(RuntimeError, match="non-finite"):
        S.moment_rank_test(bad, 2)
    with pytest.raises(ValueError):
        S.moment_rank_test(M, 3)


def test_partial_rank_one_on_the_paper_car_backin_clique(S):
    """The car back-in's extraction: a clique of 18 variables (attitude and
    inputs of two steps, plus six separating-line variables) whose moments
    come from two trajectories that agree on the trajectory variables but use
    different separating lines. M_k (190 x 190) has rank 2; the submatrix on
    the trajectory variables has rank 1 and yields them; library == oracle."""
    rng = np.random.default_rng(9)
    nv = 18
    traj = np.ones(nv, bool)
    traj[8:14] = False                         # (x_{k-1} 4, v w f_c f_s, lines 6, x_k 4): the lines
    z1 = rng.uniform(-0.9, 0.9, nv)
    z2 = z1.copy()
    z2[~traj] = rng.uniform(-0.9, 0.9, (~traj).sum())
    M = _moments([z1, z2], [0.55, 0.45])
    want_full, want_part = OC.moment_rank_tests(M, nv), OC.moment_rank_tests(M, nv, traj)
    assert want_full["n"] == 190 and want_full["rank"] == 2 and want_full["ratio_sub"] > 1e-3
    assert abs(want_part["ratio_sub"]) < 1e-12
    assert np.allclose(want_part["zbar_sub"][traj], z1[traj], atol=1e-10)
    _same(S.moment_rank_test(M, nv), want_full)
    _same(S.moment_rank_test(M, nv, traj), want_part)
