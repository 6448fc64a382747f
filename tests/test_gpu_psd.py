"""PSD projection kernels vs the oracle's Pi(X) = Q max(0, W) Q^T (Sec. 4)."""
import numpy as np
import pytest

import workloads as wl
from oracle import relax as OR
from oracle import sgs_admm as OA

from gpu_common import dev, host, lib, svec_blocks, torch

pytestmark = pytest.mark.gpu

RAGGED = [1, 2, 3, 5, 8, 12, 16, 17, 36, 40, 41, 78, 80, 81, 120, 136, 153, 160]


def _project(S, x, off, n, prec):
    xb = dev(x)
    out = torch.zeros_like(xb)
    S.kernel_psd_project(xb.data_ptr(), off, n, prec, out.data_ptr())
    return host(out)


def _rel_errors(x, off, n, got):
    """Per block, the larger of two relative errors of the projection: the
    Frobenius norm ||G - Pi||_F / ||X||_F and the element-wise
    max |G_ij - Pi_ij| / max |X_ij| (a wrong small entry of a large block
    shows in the second)."""
    errs = []
    for o, k in zip(off, n):
        t = k * (k + 1) // 2
        X = OR.smat(x[o:o + t], k)
        want = OA.project_block(X)
        G = OR.smat(got[o:o + t], k)
        fro = np.linalg.norm(G - want) / max(1e-300, np.linalg.norm(X))
        elem = np.max(np.abs(G - want)) / max(1e-300, np.max(np.abs(X)))
        errs.append(max(fro, elem))
    return np.array(errs)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_ragged_sizes(prec, tol):
    S = lib()
    mats, _, _ = wl.known_spectrum_blocks(RAGGED * 2, seed=5)
    x, off, n = svec_blocks(mats)
    got = _project(S, x, off, n, prec)
    e = _rel_errors(x, off, n, got)
    assert e.max() <= tol, dict(zip(n.tolist(), e.tolist()))


def test_degenerate_inputs():
    S = lib()
    mats = [np.zeros((7, 7)), np.eye(9), -np.eye(4), np.diag([3.0, -1.0, 0.0, 2.0]),
            np.ones((6, 6)), -np.ones((5, 5))]
    x, off, n = svec_blocks(mats)
    for prec, tol in ((0, 1e-13), (1, 1e-6)):
        e = _rel_errors(x, off, n, _project(S, x, off, n, prec))
        assert np.nan_to_num(e, nan=1.0).max() <= tol


def test_eigenvalues_output():
    S = lib()
    mats, lams, _ = wl.known_spectrum_blocks([3, 8, 36, 78, 136], seed=9)
    x, off, n = svec_blocks(mats)
    plan = S.PsdPlan(off, n, 0)
    xb = dev(x)
    lam = torch.zeros(int(n.sum()), dtype=torch.float64, device="cuda:0")
    plan.execute(xb.data_ptr(), 0, lam.data_ptr())
    got = host(lam)
    o = 0
    for k, l in zip(n, lams):
        assert np.allclose(got[o:o + k], np.sort(l), rtol=0, atol=1e-12 * np.abs(l).max())
        o += k


def test_microbench_full_size_sampled():
    """The 4096-block microbench in both precisions; 96 sampled blocks vs the oracle."""
    S = lib()
    x, off, n, _ = wl.psd_microbench()
    rng = np.random.default_rng(0)
    pick = np.concatenate([rng.choice(np.nonzero(n == k)[0], 24, replace=False) for k in (8, 36, 78, 136)])
    for prec, tol in ((0, 1e-10), (1, 1e-5)):
        got = _project(S, x, off, n, prec)
        e = _rel_errors(x, off[pick], n[pick], got)
        assert e.max() <= tol, (prec, e.max())
        assert np.all(np.isfinite(got))
