"""Shared helpers of the GPU parity tests (device memory through torch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def lib():
    from paper_2406_05846_gb300 import build
    build.build()
    import paper_2406_05846_gb300 as S
    S.lib()
    return S


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def svec_blocks(mats):
    from workloads.psd_bench import svec_pack
    parts = [svec_pack(A) for A in mats]
    off = np.zeros(len(parts), np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])[:-1]
    return np.concatenate(parts), off, np.array([A.shape[0] for A in mats], np.int32)


def assert_close(got, want, tol, floor=0.0, what=None):
    """got == want to relative tolerance tol, twice: in the 2-norm,
    ||got - want|| <= tol max(||want||, floor), and entry by entry,
    max |got - want| <= tol max(max |want|, floor), so that a wrong small
    entry of a large vector cannot hide inside the norm."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    d = got - want
    n = np.linalg.norm(d)
    assert n <= tol * max(np.linalg.norm(want), floor), (what, "norm", n / max(np.linalg.norm(want), floor, 1e-300))
    if d.size:
        e = np.max(np.abs(d))
        s = max(np.max(np.abs(want)), floor)
        assert e <= tol * s, (what, "max-abs", e / max(s, 1e-300))
