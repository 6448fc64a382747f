"""The C ABI library loads, exports every declared symbol, validates input,
and its host relaxation builder reproduces the oracle's SDP exactly (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as wl
from oracle import relax as OR

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_2406_05846_gb300 import build
    build.build()
    import paper_2406_05846_gb300 as pkg
    pkg.lib()
    return pkg


def test_exports_every_declared_symbol(S):
    hdr = open(os.path.join(ROOT, "include", "strom.h")).read()
    names = set(re.findall(r"^[a-z_0-9 \*]*?\b(strom_[A-Za-z_0-9]+)\s*\(", hdr, flags=re.M))
    assert len(names) > 25
    L = ctypes.CDLL(os.path.join(ROOT, "paper_2406_05846_gb300", "libstrom.so"))
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    from paper_2406_05846_gb300 import _native
    assert names == set(_native.SIGNATURES), names ^ set(_native.SIGNATURES)


@pytest.mark.parametrize("which", ["toy", "pendulum", "paper_pendulum", "cartpole", "rigid"])
def test_builder_matches_oracle(S, which):
    if which == "toy":
        p = wl.toy_problem(N=3)
    elif which == "paper_pendulum":
        p = wl.paper_pendulum_problem(N=3, theta0=0.4, thetadot0=-0.5)
    elif which == "pendulum":
        p = wl.pendulum_problem(N=5, theta0=0.13)
    elif which == "cartpole":
        p = wl.cartpole_problem(N=2, x0=0.2, theta0=0.1)
    else:
        p = wl.rigid_body_problem(N=2, disks=[(0.5, -0.3, 0.4), (-1.0, 1.0, 0.6)])
    a = S.Problem(p).relax().export()
    o = OR.relax(p)
    assert np.array_equal(a.block_n, [b.n for b in o.blocks])
    assert np.array_equal(a.block_off, [b.offset for b in o.blocks])
    assert np.array_equal(a.rowptr, o.A.indptr)
    assert np.array_equal(a.col, o.A.indices)
    assert np.max(np.abs(a.val - o.A.data)) <= 1e-15 * np.max(np.abs(o.A.data))
    assert np.max(np.abs(a.C - o.C)) <= 1e-15 * max(1.0, np.max(np.abs(o.C)))
    assert np.array_equal(a.b, o.b)
    assert np.array_equal(a.row_kind, o.row_kind)
    assert np.array_equal(a.row_clique, o.row_clique)


def _autonomous():
    """No control (du = 0): x_k = 0.9 x_{k-1}, one degree-1 inequality per clique."""
    from workloads.poly import Poly
    from workloads.problems import Clique, Problem
    X0, X1 = Poly.var(2, 0), Poly.var(2, 1)
    cl = [Clique(X0 * X0, [1.0 - X1], [X1 - 0.9 * X0] + ([X0 - 0.5] if k == 0 else [])) for k in range(3)]
    return Problem("autonomous", 3, 1, 0, cl, R=1.0)


def _no_inequalities():
    p = wl.toy_problem(N=3)
    for c in p.cliques:
        c.g = []
    return p


@pytest.mark.parametrize("make", [lambda: wl.toy_problem(N=1), lambda: wl.pendulum_problem(N=1),
                                  _no_inequalities, _autonomous],
                         ids=["toy-N1", "pendulum-N1", "no-inequalities", "no-control"])
def test_builder_matches_oracle_edge_cases(S, make):
    """Degenerate shapes: one clique (no consensus rows), no localizing blocks, du = 0."""
    p = make()
    a = S.Problem(p).relax().export()
    o = OR.relax(p)
    assert np.array_equal(a.block_n, [b.n for b in o.blocks])
    assert np.array_equal(a.rowptr, o.A.indptr) and np.array_equal(a.col, o.A.indices)
    assert np.max(np.abs(a.val - o.A.data)) <= 1e-15 * np.max(np.abs(o.A.data))
    assert np.max(np.abs(a.C - o.C)) <= 1e-15 * max(1.0, np.max(np.abs(o.C)))
    assert np.array_equal(a.b, o.b)
    assert np.array_equal(a.row_kind, o.row_kind) and np.array_equal(a.row_clique, o.row_clique)
    kinds = np.bincount(o.row_kind, minlength=5)
    if p.N == 1:
        assert kinds[OR.KIND_CONS] == 0
    if all(not c.g for c in p.cliques):
        assert kinds[OR.KIND_INEQ] == 0 and all(b.kind == "M" for b in o.blocks)


def test_tune_validates_arguments_without_a_gpu(S):
    """strom_solver_tune rejects a null solver, a null report and reps outside
    1..1000 before any CUDA call."""
    import ctypes as C
    from paper_2406_05846_gb300 import _native as N
    L = S.lib()
    rep = N.strom_tune_report()
    assert L.strom_solver_tune(None, 5, None, C.byref(rep)) == -1
    assert b"strom_solver_tune" in L.strom_last_error()
    assert L.strom_solver_tune(None, 5, None, None) == -1
    assert L.strom_solver_tune(None, 0, None, C.byref(rep)) == -1


def test_default_options_follow_the_same_readings_as_the_oracle(S):
    """Algorithm 1's inputs and the sigma rule are readings of the paper (it
    fixes only tau in (0, 2) and sigma > 0); the library's defaults and the
    oracle's must be the same readings, or whole-solve parity would compare
    two different methods."""
    from oracle import sgs_admm as OA
    o, ref = S.default_options(), OA.Options()
    for k in ("sigma0", "tau", "sigma_every", "sigma_ratio", "sigma_factor", "sigma_min", "sigma_max"):
        assert getattr(o, k) == getattr(ref, k), k
    assert o.rank_tol == OA.RANK_TOL
    assert 0 < o.tau < 2 and o.sigma0 > 0
    assert o.time_budget_s == 0.0 and S.default_options(time_budget_s=2.5).time_budget_s == 2.5
    with pytest.raises(KeyError):
        S.default_options(no_such_option=1)


@pytest.mark.parametrize("model", ["landing", "flying", "car"])
def test_builder_on_the_paper_robots(S, model):
    """18- and 20-variable cliques (monomial keys of 3 bits per variable):
    bit-exact parity with the oracle at N = 3, Table 1's sizes at the paper's
    horizon, and a solver that refuses their 190 / 231 blocks (the PSD
    kernels take up to 160) before touching the GPU."""
    import test_oracle_relax as T
    mk = getattr(wl, T.PAPER_ROBOTS[model])
    small = mk(N=3)
    a = S.Problem(small).relax().export()
    o = OR.relax(small)
    assert np.array_equal(a.block_n, [b.n for b in o.blocks])
    assert np.array_equal(a.rowptr, o.A.indptr) and np.array_equal(a.col, o.A.indices)
    assert np.max(np.abs(a.val - o.A.data)) <= 1e-15 * np.max(np.abs(o.A.data))
    assert np.max(np.abs(a.C - o.C)) <= 1e-15 * max(1.0, np.max(np.abs(o.C)))
    assert np.array_equal(a.b, o.b) and np.array_equal(a.row_kind, o.row_kind)
    want = T.paper_robot_sizes()[model]
    sd = S.Problem(mk()).relax()
    e = sd.export()
    assert sd.info.m == want["m"][0], want["m"][1]
    assert int(np.sum(e.block_kind == 0)) == want["nM"][0] and int(np.sum(e.block_kind == 1)) == want["nL"][0]
    assert set(e.block_n.tolist()) == {want["sizeM"][0], want["sizeL"][0]}
    from paper_2406_05846_gb300._native import StromError
    with pytest.raises(StromError, match="1..160"):
        S.Solver([S.Problem(small).relax()])


def test_binding_constants_match_the_header():
    """The Python constants are the values strom.h defines (status codes,
    precision modes, the warm-start key limit), and the oracle's row kinds
    are the header's STROM_ROW_* numbering."""
    import re
    from paper_2406_05846_gb300 import _native as N
    text = open(os.path.join(ROOT, "include", "strom.h")).read()
    vals = {k: int(v) for k, v in re.findall(r"\b(STROM_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    vals.update({k: int(v) for k, v in re.findall(r"#define\s+(STROM_[A-Z0-9_]+)\s+(\d+)", text)})
    for k in ("STROM_OK", "STROM_MAXITER", "STROM_PENDING", "STROM_PREC_FP64", "STROM_PREC_FP32",
              "STROM_PREC_MIXED", "STROM_WARM_MAX_KEY", "STROM_ERR_INVALID", "STROM_ERR_OOM", "STROM_ERR_NOT_PD",
              "STROM_ERR_NUMERICAL", "STROM_ERR_TIMEOUT", "STROM_ERR_CUDA"):
        assert getattr(N, k) == vals[k], k
    assert (OR.KIND_MOM, OR.KIND_INEQ, OR.KIND_EQ, OR.KIND_PHI0, OR.KIND_CONS) == \
        (vals["STROM_ROW_MOM"], vals["STROM_ROW_INEQ"], vals["STROM_ROW_EQ"], vals["STROM_ROW_PHI0"],
         vals["STROM_ROW_CONS"])


def test_problem_validation(S):
    p = wl.toy_problem(N=2)
    p.kappa = 3
    with pytest.raises(RuntimeError, match="kappa"):
        S.Problem(p)
    p = wl.toy_problem(N=2)
    p.cliques[0].g.append(wl.Poly.var(3, 0) ** 3)   # cubic inequality: degree too high
    with pytest.raises(RuntimeError, match="degree"):
        S.Problem(p)
    from workloads.problems import Clique, Problem   # 22 variables per clique: beyond the 64-bit monomial keys
    x = wl.Poly.var(22, 0)
    with pytest.raises(RuntimeError, match="21 variables"):
        S.Problem(Problem("wide", 1, 10, 2, [Clique(x * x, [], [])]))


def test_no_gpu_no_fallback(S):
    """Without a GPU the solver must fail loudly instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    sdp = S.Problem(wl.toy_problem(N=2)).relax()
    with pytest.raises(RuntimeError):
        S.Solver([sdp])


def test_binding_checks_array_lengths(S):
    """The binding rejects keys and warm states whose length does not match
    before the library would read past them."""
    from paper_2406_05846_gb300 import api
    api._key([0.1, 0.2], 2)
    with pytest.raises(ValueError, match="key"):
        api._key([0.1, 0.2, 0.3], 2)
    api._check_len(None, 5, "X0")
    api._check_len(np.zeros(5), 5, "X0")
    with pytest.raises(ValueError, match="X0"):
        api._check_len(np.zeros(4), 5, "X0")


def test_binding_checks_block_tables(S):
    """PSD plans and the one-shot projection refuse offset and size tables of
    different lengths before the library would read past the shorter one."""
    with pytest.raises(ValueError, match="blk_off"):
        S.PsdPlan([0, 3], [2], 0)
    with pytest.raises(ValueError, match="blk_off"):
        S.kernel_psd_project(0, [0], [2, 2], 0, 0)


def test_builder_reproduces_paper_pendulum_sizes(S):
    """Table 1's pendulum row and the sizes quoted in Sec. 1, from the C++ builder."""
    import test_oracle_relax as T
    want = T._paper_sizes()
    sd = S.Problem(wl.paper_pendulum_problem(N=30, theta0=0.4, thetadot0=-0.5)).relax()
    a = sd.export()
    assert int(np.sum(a.block_kind == 0)) == want["nM"][0]
    assert set(a.block_n[a.block_kind == 0].tolist()) == {want["sizeM"][0]}
    assert int(np.sum(a.block_kind == 1)) == want["nL"][0]
    assert set(a.block_n[a.block_kind == 1].tolist()) == {want["sizeL"][0]}
    assert sd.m == want["m"][0] and sd.nsvec == want["nvar"][0]


def test_plain_c_client(S, tmp_path):
    """A C program uses the library through include/strom.h alone (no Python):
    the toy problem built there relaxes to the same SDP as through the
    binding, and the host-only calls give the expected results."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_2406_05846_gb300")
    exe = str(tmp_path / "c_client")
    subprocess.run([cc, "-std=c99", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-lstrom", "-lm",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = dict(l.split(" ", 1) for l in out.stdout.strip().splitlines())
    info = S.Problem(wl.toy_problem(N=3)).relax().info
    assert lines["problem_create"] == "0" and lines["relax"] == "0"
    want = "nblocks %d nsvec %d m %d nnz %d kinds %s" % (info.nblocks, info.nsvec, info.m, info.nnz,
                                                         " ".join(str(x) for x in info.rows_by_kind))
    assert lines["info"] == want
    assert lines["export"] == "0 import 0 same 1"
    assert lines["bad_import"] == "-1"
    assert lines["warm_select"] == "0 k 3 idx 0 2 1 wt 0.500000 0.300000 0.200000"
    assert lines["rank_test"] == "0 rank 1 flat 1 zbar 0.500000 -0.250000 0.750000"
    assert lines["solver_create"] in ("ok", "cuda-unavailable")


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    that a C compiler gives the structures of strom.h."""
    import shutil
    import subprocess
    from paper_2406_05846_gb300 import _native as N
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"strom_options": N.strom_options, "strom_result": N.strom_result,
               "strom_certificate": N.strom_certificate, "strom_tune_report": N.strom_tune_report,
               "strom_server_class": N.strom_server_class, "strom_factor_info": N.strom_factor_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "strom.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append('  return 0;\n}')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe], check=True,
                   capture_output=True)
    got = dict(line.split() for line in subprocess.run([exe], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (name, fname)]) == getattr(cls, fname).offset, (name, fname)


def test_raw_csr_product_argument_checks(S):
    """strom_kernel_spmv_csr refuses a negative row count and missing
    pointers before touching the device, and does nothing for zero rows."""
    L = S.lib()
    assert L.strom_kernel_spmv_csr(None, None, None, -1, None, None, None) == -1
    assert b"bad arguments" in L.strom_last_error()
    assert L.strom_kernel_spmv_csr(None, None, None, 3, None, None, None) == -1
    assert L.strom_kernel_spmv_csr(None, None, None, 0, None, None, None) == 0
