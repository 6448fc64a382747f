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
