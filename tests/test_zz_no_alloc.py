"""The allocation-free PSD projection matches the regular entry point.

strom_kernel_psd_project_noalloc serves callers that may not allocate device
memory themselves or through the library (a host framework that owns the
whole memory pool, a real-time loop that must not allocate after start-up).
It keeps its block table and FP64 scratch in a static device array instead.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

from gpu_common import dev, host, lib, svec_blocks, torch

pytestmark = pytest.mark.gpu


def _call(fn, x, off, n, prec):
    xb = dev(x)
    out = torch.zeros_like(xb)
    o = np.ascontiguousarray(off, np.int64)
    k = np.ascontiguousarray(n, np.int32)
    st = fn(C.c_void_p(xb.data_ptr()), o.ctypes.data_as(C.POINTER(C.c_int64)),
            k.ctypes.data_as(C.POINTER(C.c_int32)), len(k), prec, C.c_void_p(out.data_ptr()), None)
    assert st == 0, st
    return host(out)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_matches_regular_entry_point(prec, tol):
    S = lib()
    L = S.lib()
    # first call: every size class, and 40 FP64 blocks of size 136 (more than
    # the 16 the static scratch holds at once, so they run in chunks)
    sizes = [1, 3, 8, 12, 17, 36, 41, 78, 81, 120, 160] + [136] * 40
    mats, _, _ = wl.known_spectrum_blocks(sizes, seed=21)
    x, off, n = svec_blocks(mats)
    want = _call(L.strom_kernel_psd_project, x, off, n, prec)
    got = _call(L.strom_kernel_psd_project_noalloc, x, off, n, prec)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    # second call in a row, different and smaller input: the scratch keeps the
    # first call's contents and must not leak into this result
    mats2, _, _ = wl.known_spectrum_blocks([36, 8, 136, 2], seed=22)
    x2, off2, n2 = svec_blocks(mats2)
    want2 = _call(L.strom_kernel_psd_project, x2, off2, n2, prec)
    got2 = _call(L.strom_kernel_psd_project_noalloc, x2, off2, n2, prec)
    assert np.max(np.abs(got2 - want2)) <= tol * np.max(np.abs(want2))


def test_noalloc_rejects_too_many_blocks():
    S = lib()
    L = S.lib()
    n = np.full(65537, 2, np.int32)
    off = np.arange(65537, dtype=np.int64) * 3
    xb = torch.zeros(3 * 65537, dtype=torch.float64, device="cuda:0")
    out = torch.zeros_like(xb)
    st = L.strom_kernel_psd_project_noalloc(C.c_void_p(xb.data_ptr()), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                            n.ctypes.data_as(C.POINTER(C.c_int32)), len(n), 0,
                                            C.c_void_p(out.data_ptr()), None)
    assert st == -1
    assert b"65536" in L.strom_last_error()


_CHILD = r"""
import ctypes as C, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import torch
import workloads as wl
from gpu_common import lib, svec_blocks
torch.cuda.set_device(0)
S = lib()
L = S.lib()
calls = []
for seed, sizes in ((31, [8, 36, 78, 136, 136, 12]), (32, [160, 3, 41, 81])):
    mats, _, _ = wl.known_spectrum_blocks(sizes, seed=seed)
    x, off, n = svec_blocks(mats)
    xb = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    calls.append((xb, torch.zeros_like(xb), np.ascontiguousarray(off, np.int64), np.ascontiguousarray(n, np.int32)))
torch.cuda.synchronize()
def run(xb, out, off, n, prec):
    if xb is None:
        return L.strom_kernel_psd_project_noalloc(None, None, None, 0, prec, None, None)
    return L.strom_kernel_psd_project_noalloc(C.c_void_p(xb.data_ptr()), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                              n.ctypes.data_as(C.POINTER(C.c_int32)), len(n), prec,
                                              C.c_void_p(out.data_ptr()), None)
free = [torch.cuda.mem_get_info(0)[0]]
st = [run(None, None, None, None, 0)]
free.append(torch.cuda.mem_get_info(0)[0])
for prec in (0, 1):
    for c in calls:
        st.append(run(*c, prec))
        free.append(torch.cuda.mem_get_info(0)[0])
print(json.dumps({"status": st, "free": free}))
"""


def test_noalloc_allocates_nothing_after_setup():
    """In a fresh process where no library kernel has run yet: the set-up call
    (nblk = 0) may take device memory (module loading of the kernels and of
    the static array), every later call takes none."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CHILD, root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-4000:]
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    assert rec["status"] == [0] * 5, rec
    free = rec["free"]
    assert free[1] <= free[0]                          # set-up: module loading may take memory
    assert all(f == free[1] for f in free[2:]), free   # later calls: not one byte
