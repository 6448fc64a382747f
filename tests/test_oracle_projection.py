"""Pins of the oracle's PSD projection Pi(X) = Q max(0, W) Q^T (Sec. 4) — CPU only."""
import numpy as np
import pytest

import workloads as wl
from oracle import relax as R
from oracle import sgs_admm as O


@pytest.mark.parametrize("n", [1, 2, 3, 8, 36, 78])
def test_known_spectrum(n):
    mats, lams, Qs = wl.known_spectrum_blocks([n, n], seed=11)
    for A, lam, Q in zip(mats, lams, Qs):
        want = (Q * np.maximum(lam, 0.0)) @ Q.T
        got = O.project_block(A)
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(lam)))


def test_closed_forms():
    for x in (-2.0, 0.0, 3.5):
        assert O.project_block(np.array([[x]]))[0, 0] == max(x, 0.0)
    # 2x2: [[a, b], [b, c]] with one negative eigenvalue, projection = lam+ v v^T
    a, b, c = 1.0, 2.0, -1.0
    lp = 0.5 * (a + c) + np.hypot(0.5 * (a - c), b)
    v = np.array([b, lp - a])
    v /= np.linalg.norm(v)
    assert np.allclose(O.project_block(np.array([[a, b], [b, c]])), lp * np.outer(v, v), atol=1e-14)


def test_moreau_idempotent_psd_identity():
    rng = np.random.default_rng(5)
    for n in (4, 10, 36):
        G = rng.standard_normal((n, n))
        X = 0.5 * (G + G.T)
        P, Pm = O.project_block(X), O.project_block(-X)
        assert np.allclose(P - Pm, X, atol=1e-12)                 # Moreau: Pi(X) - Pi(-X) = X
        assert abs(np.sum(P * (P - X))) < 1e-11                    # <Pi(X), Pi(X) - X> = 0
        assert np.allclose(O.project_block(P), P, atol=1e-12)      # idempotent
        assert np.min(np.linalg.eigvalsh(P)) > -1e-12
        Y = G @ G.T
        assert np.allclose(O.project_block(Y), Y, atol=1e-11)      # identity on PSD input


def test_svec_roundtrip_and_blocks():
    rng = np.random.default_rng(1)
    n = 7
    G = rng.standard_normal((n, n))
    M = 0.5 * (G + G.T)
    v = R.svec(M)
    assert np.allclose(R.smat(v, n), M)
    H = rng.standard_normal((n, n))
    H = H + H.T
    assert abs(R.svec(H) @ v - np.sum(H * M)) < 1e-12              # <A, B> = svec . svec
    x = np.concatenate([v, R.svec(-M)])
    out = O.project_psd(x, [(0, n), (len(v), n)])
    assert np.allclose(out[:len(v)] - out[len(v):], v, atol=1e-12)


# --------------------------------------------------------------------------
# the LAPACK-free cyclic Jacobi projection (Golub & Van Loan, Sec. 8.5)
# --------------------------------------------------------------------------
from oracle import jacobi as J  # noqa: E402


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 36])
def test_jacobi_known_spectrum(n):
    mats, lams, Qs = wl.known_spectrum_blocks([n, n], seed=12)
    for A, lam, Q in zip(mats, lams, Qs):
        w, V, sweeps = J.eig_jacobi(A)
        scale = max(1.0, np.max(np.abs(lam)))
        assert np.max(np.abs(np.sort(w) - np.sort(lam))) <= 1e-13 * scale
        assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13 * n
        assert np.max(np.abs((V * w) @ V.T - A)) <= 1e-13 * scale
        want = (Q * np.maximum(lam, 0.0)) @ Q.T
        assert np.max(np.abs(J.project_block(A) - want)) <= 1e-12 * scale
        assert sweeps <= 12


def test_jacobi_two_by_two_is_one_rotation():
    # a single Schur rotation diagonalises a 2 x 2 block exactly (closed form)
    a, b, c = 1.0, 2.0, -1.0
    A = np.array([[a, b], [b, c]])
    w, V, sweeps = J.eig_jacobi(A)
    lp, lm = 0.5 * (a + c) + np.hypot(0.5 * (a - c), b), 0.5 * (a + c) - np.hypot(0.5 * (a - c), b)
    assert sweeps <= 2                                                   # the second only sees rounding
    assert np.allclose(np.sort(w), [lm, lp], atol=1e-15, rtol=0)
    cs, sn = J.sym_schur2(A, 0, 1)
    assert abs(cs * cs + sn * sn - 1.0) <= 4e-16
    Jr = np.array([[cs, sn], [-sn, cs]])
    B = Jr.T @ A @ Jr
    assert abs(B[0, 1]) < 1e-15 and abs(B[1, 0]) < 1e-15
    assert J.eig_jacobi(np.diag([3.0, -1.0]))[2] == 0                  # already diagonal: no sweep


def test_jacobi_matches_the_eigh_projection_on_the_microbench_sizes():
    """Every block size of the 4096-block microbench, including the two large
    classes, projected by both oracle eigensolvers."""
    mats, _, _ = wl.known_spectrum_blocks([8, 36, 78, 136], seed=13)
    for A in mats:
        P1, P2 = J.project_block(A), O.project_block(A)
        assert np.max(np.abs(P1 - P2)) <= 1e-12 * np.max(np.abs(A))
