"""Thin Python layer over the C ABI: marshalling of problems, SDPs, solvers and plans.

Every computation runs in libstrom (host C++ builder, CUDA kernels); this
module only converts arrays and keeps them alive across calls. Device
vectors are passed as raw pointers (e.g. torch tensors' data_ptr()).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _native as N
from ._native import check, lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Problem:
    """A polynomial trajectory problem handed to the library (strom_problem_create).

    `src` is any object with N, dx, du, kappa, R and cliques[k].f/.g/.h, where
    each polynomial exposes arrays() -> (coef float64[T], expo uint8[T, n_v]).
    """

    def __init__(self, src):
        self._keep = []
        nv = 2 * src.dx + src.du

        def poly(p):
            coef, expo = p.arrays() if hasattr(p, "arrays") else p
            coef = np.ascontiguousarray(coef, dtype=np.float64)
            expo = np.ascontiguousarray(expo, dtype=np.uint8).reshape(len(coef), nv)
            self._keep += [coef, expo]
            return N.strom_poly(len(coef), _ptr(coef, C.c_double), _ptr(expo, C.c_uint8))

        cl = (N.strom_clique * src.N)()
        for k, c in enumerate(src.cliques):
            g = (N.strom_poly * max(1, len(c.g)))(*[poly(x) for x in c.g])
            h = (N.strom_poly * max(1, len(c.h)))(*[poly(x) for x in c.h])
            self._keep += [g, h]
            cl[k] = N.strom_clique(poly(c.f), len(c.g), g, len(c.h), h)
        self._keep.append(cl)
        desc = N.strom_problem_desc(src.N, src.dx, src.du, getattr(src, "kappa", 2), float(src.R), cl)
        h = C.c_void_p()
        check(lib().strom_problem_create(C.byref(desc), C.byref(h)), "strom_problem_create")
        self.handle = h
        self.N, self.dx, self.du = src.N, src.dx, src.du
        self._keep = None  # the library copied the data

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_problem_destroy(self.handle)
            self.handle = None

    def relax(self) -> "Sdp":
        h = C.c_void_p()
        check(lib().strom_relax(self.handle, C.byref(h)), "strom_relax")
        return Sdp(h)


@dataclass
class SdpArrays:
    block_n: np.ndarray
    block_off: np.ndarray
    block_kind: np.ndarray
    block_clique: np.ndarray
    C: np.ndarray
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    b: np.ndarray
    row_kind: np.ndarray
    row_clique: np.ndarray


@dataclass
class StarData:
    rep: np.ndarray
    c: np.ndarray
    dsum: np.ndarray
    ptr: np.ndarray
    row: np.ndarray
    inv_s2: np.ndarray
    omega: np.ndarray
    inv_rep_s: np.ndarray


class Sdp:
    def __init__(self, handle):
        self.handle = handle
        self.info = N.strom_sdp_info()
        check(lib().strom_sdp_info_get(handle, C.byref(self.info)), "strom_sdp_info_get")

    @classmethod
    def from_arrays(cls, N_, dx, du, block_n, block_kind, block_clique, C_, rowptr, col, val, b, row_kind,
                    row_clique, block_index=None) -> "Sdp":
        """strom_sdp_import: an SDP given by arrays in the layout of export()."""
        keep = [np.ascontiguousarray(block_n, np.int32), np.ascontiguousarray(block_kind, np.int8),
                np.ascontiguousarray(block_clique, np.int32),
                None if block_index is None else np.ascontiguousarray(block_index, np.int32),
                np.ascontiguousarray(C_, np.float64), np.ascontiguousarray(rowptr, np.int64),
                np.ascontiguousarray(col, np.int32), np.ascontiguousarray(val, np.float64),
                np.ascontiguousarray(b, np.float64), np.ascontiguousarray(row_kind, np.int8),
                np.ascontiguousarray(row_clique, np.int32)]
        bn, bk, bc, bi, cc, rp, co, va, bb, rk, rc = keep
        d = N.strom_sdp_desc(int(N_), int(dx), int(du), bn.size, _ptr(bn, C.c_int32), _ptr(bk, C.c_int8),
                             _ptr(bc, C.c_int32), None if bi is None else _ptr(bi, C.c_int32),
                             _ptr(cc, C.c_double), bb.size, _ptr(rp, C.c_int64), _ptr(co, C.c_int32),
                             _ptr(va, C.c_double), _ptr(bb, C.c_double), _ptr(rk, C.c_int8), _ptr(rc, C.c_int32))
        h = C.c_void_p()
        check(lib().strom_sdp_import(C.byref(d), C.byref(h)), "strom_sdp_import")
        return cls(h)

    def star_data(self) -> StarData:
        """strom_sdp_star_export: the star elimination and Gram weights used by the y-solve."""
        nc, ns = C.c_int64(), C.c_int64()
        check(lib().strom_sdp_star_export(self.handle, C.byref(nc), C.byref(ns), *([None] * 8)),
              "strom_sdp_star_export")
        o = StarData(np.empty(nc.value, np.int64), np.empty(nc.value), np.empty(nc.value),
                     np.empty(nc.value + 1, np.int32), np.empty(ns.value, np.int64), np.empty(ns.value),
                     np.empty(self.nsvec), np.empty(self.nsvec))
        check(lib().strom_sdp_star_export(self.handle, None, None, _ptr(o.rep, C.c_int64), _ptr(o.c, C.c_double),
                                          _ptr(o.dsum, C.c_double), _ptr(o.ptr, C.c_int32),
                                          _ptr(o.row, C.c_int64), _ptr(o.inv_s2, C.c_double),
                                          _ptr(o.omega, C.c_double), _ptr(o.inv_rep_s, C.c_double)),
              "strom_sdp_star_export")
        return o

    def factor_info(self) -> dict:
        """strom_sdp_factor_info: size of the y-solve's sparse factor for this SDP."""
        fi = N.strom_factor_info()
        check(lib().strom_sdp_factor_info(self.handle, C.byref(fi)), "strom_sdp_factor_info")
        return {k: getattr(fi, k) for k, _ in fi._fields_}

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_sdp_destroy(self.handle)
            self.handle = None

    @property
    def m(self):
        return self.info.m

    @property
    def nsvec(self):
        return self.info.nsvec

    def export(self) -> SdpArrays:
        i = self.info
        a = SdpArrays(np.empty(i.nblocks, np.int32), np.empty(i.nblocks, np.int64), np.empty(i.nblocks, np.int8),
                      np.empty(i.nblocks, np.int32), np.empty(i.nsvec), np.empty(i.m + 1, np.int64),
                      np.empty(i.nnz, np.int32), np.empty(i.nnz), np.empty(i.m), np.empty(i.m, np.int8),
                      np.empty(i.m, np.int32))
        check(lib().strom_sdp_export(self.handle, _ptr(a.block_n, C.c_int32), _ptr(a.block_off, C.c_int64),
                                     _ptr(a.block_kind, C.c_int8), _ptr(a.block_clique, C.c_int32),
                                     _ptr(a.C, C.c_double), _ptr(a.rowptr, C.c_int64), _ptr(a.col, C.c_int32),
                                     _ptr(a.val, C.c_double), _ptr(a.b, C.c_double), _ptr(a.row_kind, C.c_int8),
                                     _ptr(a.row_clique, C.c_int32)), "strom_sdp_export")
        return a


def default_options(**kw) -> N.strom_options:
    o = N.strom_options()
    lib().strom_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclass
class Result:
    status: int
    iterations: int
    pobj: float
    dobj: float
    eta_p: float
    eta_d: float
    eta_g: float
    sigma: float
    m_kept: int


@dataclass
class Certificate:
    max_ratio: float
    lower_bound: float
    phat: float
    xi: float
    hmax: float
    gmin: float
    feasible: bool
    rank_one: bool
    certified: bool
    zbar: np.ndarray
    zhat: np.ndarray


def certify_host(problem: "Problem", block_n, block_kind, block_clique, lamX, topX, lamZ, by,
                 rank_tol=1e-4, xi_tol=1e-2) -> Certificate:
    """strom_certify_host: the host half of the certificate from eigen data
    computed elsewhere (eigenvalues of X's and Z's blocks, top eigenvectors of
    X's blocks, packed block after block; <b, y>)."""
    bn = np.ascontiguousarray(block_n, np.int32)
    bk = np.ascontiguousarray(block_kind, np.int8)
    bc = np.ascontiguousarray(block_clique, np.int32)
    tot = int(bn.sum())
    lx, tx, lz = (np.ascontiguousarray(v, np.float64).ravel() for v in (lamX, topX, lamZ))
    if not (len(bk) == len(bc) == len(bn)) or not (lx.size == tx.size == lz.size == tot):
        raise ValueError("block lists must have one length and eigen data sum(block_n) entries")
    nz = problem.N * (problem.dx + problem.du) + problem.dx
    zb, zh = np.empty(nz), np.empty(nz)
    c = N.strom_certificate()
    check(lib().strom_certify_host(problem.handle, len(bn), _ptr(bn, C.c_int32), _ptr(bk, C.c_int8),
                                   _ptr(bc, C.c_int32), _ptr(lx, C.c_double), _ptr(tx, C.c_double),
                                   _ptr(lz, C.c_double), float(by), rank_tol, xi_tol, C.byref(c),
                                   _ptr(zb, C.c_double), _ptr(zh, C.c_double)), "strom_certify_host")
    return Certificate(c.max_ratio, c.lower_bound, c.phat, c.xi, c.hmax, c.gmin, bool(c.feasible),
                       bool(c.rank_one), bool(c.certified), zb, zh)


class Solver:
    """strom_solver: sGS-ADMM (Algorithm 1) on a batch of SDPs on the current GPU."""

    def __init__(self, sdps, **opts):
        self.sdps = list(sdps)
        arr = (C.c_void_p * len(self.sdps))(*[s.handle.value for s in self.sdps])
        self.opt = default_options(**opts)
        h = C.c_void_p()
        check(lib().strom_solver_create(arr, len(self.sdps), C.byref(self.opt), C.byref(h)), "strom_solver_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_solver_destroy(self.handle)
            self.handle = None

    def __len__(self):
        return lib().strom_solver_count(self.handle)

    @property
    def factor_kind(self) -> int:
        """STROM_FACTOR_DENSE or STROM_FACTOR_SPARSE: the y-solve factor in use."""
        return lib().strom_solver_factor_kind(self.handle)

    def factor(self, stream=None):
        """Row reduction + factorisation from device-resident data, fresh state."""
        check(lib().strom_solver_factor(self.handle, stream), "strom_solver_factor")

    def certify_batch(self, problems, rank_tol=1e-4, xi_tol=1e-2):
        n = len(self)
        arr = (C.c_void_p * n)(*[pr.handle.value for pr in problems])
        out = (N.strom_certificate * n)()
        check(lib().strom_certify_batch(self.handle, arr, rank_tol, xi_tol, out), "strom_certify_batch")
        return [Certificate(c.max_ratio, c.lower_bound, c.phat, c.xi, c.hmax, c.gmin, bool(c.feasible),
                            bool(c.rank_one), bool(c.certified), None, None) for c in out]

    def solve(self, stream=None) -> int:
        return check(lib().strom_solve(self.handle, stream), "strom_solve")

    def step(self, iters, stream=None) -> int:
        n = C.c_int32()
        check(lib().strom_solver_step(self.handle, iters, stream, C.byref(n)), "strom_solver_step")
        return n.value

    def reset(self, i=-1, X0=None, S0=None, sigma=0.0):
        if i >= 0:
            _check_len(X0, self.sdps[i].nsvec, "X0")
            _check_len(S0, self.sdps[i].nsvec, "S0")
        elif X0 is not None or S0 is not None:
            raise ValueError("X0 / S0 need one instance (i >= 0)")
        px = None if X0 is None else _ptr(np.ascontiguousarray(X0, np.float64), C.c_double)
        ps = None if S0 is None else _ptr(np.ascontiguousarray(S0, np.float64), C.c_double)
        check(lib().strom_solver_reset(self.handle, i, px, ps, float(sigma)), "strom_solver_reset")

    def warm_start(self, i, store: WarmStore, key):
        """Reset instance i to the store's warm start for key (cold when the store is empty)."""
        _, pk = _key(key, store.key_dim)
        check(lib().strom_solver_warm_start(self.handle, i, store.handle, pk), "strom_solver_warm_start")

    def result(self, i=0) -> Result:
        r = N.strom_result()
        check(lib().strom_get_result(self.handle, i, C.byref(r)), "strom_get_result")
        return Result(r.status, r.iterations, r.pobj, r.dobj, r.eta_p, r.eta_d, r.eta_g, r.sigma, r.m_kept)

    def state(self, i=0):
        s = self.sdps[i]
        X, S, y = np.empty(s.nsvec), np.empty(s.nsvec), np.empty(s.m)
        check(lib().strom_get_state(self.handle, i, _ptr(X, C.c_double), _ptr(S, C.c_double), _ptr(y, C.c_double)),
              "strom_get_state")
        return X, S, y

    def kept_rows(self, i=0):
        k = np.empty(self.sdps[i].m, np.uint8)
        check(lib().strom_get_kept_rows(self.handle, i, _ptr(k, C.c_uint8)), "strom_get_kept_rows")
        return k.astype(bool)

    def moment(self, i, k):
        s = self.sdps[i]
        n = int(s.export().block_n[0])
        M = np.empty((n, n))
        check(lib().strom_get_moment(self.handle, i, k, _ptr(M, C.c_double)), "strom_get_moment")
        return M

    def certify(self, i, problem: Problem, rank_tol=1e-4, xi_tol=1e-2) -> Certificate:
        c = N.strom_certificate()
        nz = problem.N * (problem.dx + problem.du) + problem.dx
        zb, zh = np.empty(nz), np.empty(nz)
        check(lib().strom_certify(self.handle, i, problem.handle, rank_tol, xi_tol, C.byref(c),
                                  _ptr(zb, C.c_double), _ptr(zh, C.c_double)), "strom_certify")
        return Certificate(c.max_ratio, c.lower_bound, c.phat, c.xi, c.hmax, c.gmin, bool(c.feasible),
                           bool(c.rank_one), bool(c.certified), zb, zh)

    # kernel-level entry points (device pointers)
    @property
    def nsvec_total(self):
        return lib().strom_solver_nsvec_total(self.handle)

    @property
    def m_total(self):
        return lib().strom_solver_m_total(self.handle)

    def offsets(self, i):
        so, ro = C.c_int64(), C.c_int64()
        check(lib().strom_solver_offsets(self.handle, i, C.byref(so), C.byref(ro)), "strom_solver_offsets")
        return so.value, ro.value

    def kernel_A(self, x_ptr, out_ptr, stream=None):
        check(lib().strom_kernel_A(self.handle, x_ptr, out_ptr, stream), "strom_kernel_A")

    def kernel_At(self, y_ptr, out_ptr, stream=None):
        check(lib().strom_kernel_At(self.handle, y_ptr, out_ptr, stream), "strom_kernel_At")

    def kernel_solve(self, r_ptr, y_ptr, stream=None):
        check(lib().strom_kernel_solve(self.handle, r_ptr, y_ptr, stream), "strom_kernel_solve")

    def tune(self, reps=5, stream=None):
        """strom_solver_tune: time the y-solve launch shapes and the eigensolver's
        threads per CTA, keep the fastest. Returns ({tile: ms per y-solve},
        chosen tile); the eigensolver's choices are in self.eig_tuning
        ({precision: {size class: (threads, ms)}})."""
        rep = N.strom_tune_report()
        check(lib().strom_solver_tune(self.handle, int(reps), stream, C.byref(rep)), "strom_solver_tune")
        self.eig_tuning = {("fp64", "fp32")[p]: {k: (rep.eig_threads[p][k], rep.eig_ms[p][k])
                                                 for k in range(4) if rep.eig_threads[p][k] > 0}
                           for p in range(2)}
        return {rep.tile[i]: rep.ms[i] for i in range(rep.ncand)}, rep.chosen


def _check_len(a, n, name):
    if a is not None and np.asarray(a).size != n:
        raise ValueError("%s must have %d entries" % (name, n))


def _key(key, dim=None):
    """A key as a contiguous float64 array (checked against the store's key dimension)."""
    k = np.ascontiguousarray(np.atleast_1d(np.asarray(key, np.float64)).ravel())
    if dim is not None and k.size != dim:
        raise ValueError("warm-start key has %d entries, the store's keys have %d" % (k.size, dim))
    return k, _ptr(k, C.c_double)


def warm_select(keys, key):
    """Neighbour indices and convex weights of `key` among the rows of `keys` (host only)."""
    keys = np.ascontiguousarray(np.atleast_2d(np.asarray(keys, np.float64)))
    k, pk = _key(key)
    d = k.size
    if keys.size == 0:
        keys = np.zeros((0, d))
    if keys.shape[1] != d:
        raise ValueError("key dimension differs from the stored keys'")
    idx, wt, n = np.zeros(d + 1, np.int32), np.zeros(d + 1), C.c_int32()
    check(lib().strom_warm_select(_ptr(keys, C.c_double), keys.shape[0], d, pk, _ptr(idx, C.c_int32),
                                  _ptr(wt, C.c_double), C.byref(n)), "strom_warm_select")
    return idx[:n.value].copy(), wt[:n.value].copy()


class WarmStore:
    """strom_warm: solved states in device memory for data-driven warm starts."""

    def __init__(self, key_dim: int, nsvec: int, capacity: int):
        h = C.c_void_p()
        check(lib().strom_warm_create(key_dim, nsvec, capacity, C.byref(h)), "strom_warm_create")
        self.handle = h
        self.key_dim, self.nsvec, self.capacity = key_dim, nsvec, capacity

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_warm_destroy(self.handle)
            self.handle = None

    def __len__(self):
        return lib().strom_warm_count(self.handle)

    def add(self, key, X, S, sigma) -> int:
        _, pk = _key(key, self.key_dim)
        X = np.ascontiguousarray(X, np.float64).ravel()
        S = np.ascontiguousarray(S, np.float64).ravel()
        if X.size != self.nsvec or S.size != self.nsvec:
            raise ValueError("X and S must have nsvec = %d entries" % self.nsvec)
        j = C.c_int32()
        check(lib().strom_warm_add(self.handle, pk, _ptr(X, C.c_double), _ptr(S, C.c_double), float(sigma),
                                   C.byref(j)), "strom_warm_add")
        return j.value

    def add_from_solver(self, solver: "Solver", i: int, key) -> int:
        _, pk = _key(key, self.key_dim)
        j = C.c_int32()
        check(lib().strom_warm_add_from_solver(self.handle, solver.handle, i, pk, C.byref(j)),
              "strom_warm_add_from_solver")
        return j.value

    def query(self, key):
        _, pk = _key(key, self.key_dim)
        idx, wt, n = np.zeros(self.key_dim + 1, np.int32), np.zeros(self.key_dim + 1), C.c_int32()
        check(lib().strom_warm_query(self.handle, pk, _ptr(idx, C.c_int32), _ptr(wt, C.c_double), C.byref(n)),
              "strom_warm_query")
        return idx[:n.value].copy(), wt[:n.value].copy()

    def get(self, j):
        key, X, S, sg = np.empty(self.key_dim), np.empty(self.nsvec), np.empty(self.nsvec), C.c_double()
        check(lib().strom_warm_get(self.handle, j, _ptr(key, C.c_double), _ptr(X, C.c_double),
                                   _ptr(S, C.c_double), C.byref(sg)), "strom_warm_get")
        return key, X, S, sg.value


class Batch:
    """strom_batch: continuous batching of solve requests over `slots` solver slots."""

    def __init__(self, template: Sdp, slots: int, **opts):
        self.opt = default_options(**opts)
        h = C.c_void_p()
        check(lib().strom_batch_create(template.handle, slots, C.byref(self.opt), C.byref(h)), "strom_batch_create")
        self.handle = h
        self.slots = slots

    @staticmethod
    def slot_bytes(template: Sdp, **opts) -> int:
        """strom_batch_slot_bytes: device bytes per slot of a batch of this structure."""
        o = default_options(**opts)
        b, p, t = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().strom_batch_slot_bytes(template.handle, C.byref(o), C.byref(b), C.byref(p), C.byref(t)),
              "strom_batch_slot_bytes")
        return p.value

    @staticmethod
    def footprint(template: Sdp, **opts) -> dict:
        """strom_batch_slot_bytes: {'base', 'slot', 'transient'} device bytes."""
        o = default_options(**opts)
        b, p, t = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().strom_batch_slot_bytes(template.handle, C.byref(o), C.byref(b), C.byref(p), C.byref(t)),
              "strom_batch_slot_bytes")
        return {"base": b.value, "slot": p.value, "transient": t.value}

    @classmethod
    def with_budget(cls, template: Sdp, budget_bytes: int, **opts) -> "Batch":
        """strom_batch_create_budget: as many slots as budget_bytes of device memory hold."""
        self = cls.__new__(cls)
        self.opt = default_options(**opts)
        h, n = C.c_void_p(), C.c_int32()
        check(lib().strom_batch_create_budget(template.handle, int(budget_bytes), C.byref(self.opt), C.byref(h),
                                              C.byref(n)), "strom_batch_create_budget")
        self.handle = h
        self.slots = n.value
        return self

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_batch_destroy(self.handle)
            self.handle = None

    def submit(self, sdp: Sdp, problem: Problem | None = None, X0=None, S0=None) -> int:
        _check_len(X0, sdp.nsvec, "X0")
        _check_len(S0, sdp.nsvec, "S0")
        t = C.c_uint64()
        px = None if X0 is None else _ptr(np.ascontiguousarray(X0, np.float64), C.c_double)
        ps = None if S0 is None else _ptr(np.ascontiguousarray(S0, np.float64), C.c_double)
        check(lib().strom_batch_submit(self.handle, sdp.handle, problem.handle if problem else None, px, ps,
                                       C.byref(t)), "strom_batch_submit")
        return t.value

    def set_warm(self, store: "WarmStore | None", record=False):
        check(lib().strom_batch_set_warm(self.handle, store.handle if store is not None else None, int(bool(record))),
              "strom_batch_set_warm")
        self.warm = store     # keeps the store alive while attached

    def submit_keyed(self, sdp: Sdp, key, problem: Problem | None = None) -> int:
        t = C.c_uint64()
        store = getattr(self, "warm", None)
        _, pk = _key(key, store.key_dim if store is not None else None)
        check(lib().strom_batch_submit_keyed(self.handle, sdp.handle, problem.handle if problem else None, pk,
                                             C.byref(t)), "strom_batch_submit_keyed")
        return t.value

    def step(self, iters: int, stream=None):
        run, q = C.c_int32(), C.c_int32()
        check(lib().strom_batch_step(self.handle, iters, stream, C.byref(run), C.byref(q)), "strom_batch_step")
        return run.value, q.value

    def poll(self, ticket: int, with_service=False):
        """None while pending, else (Result, Certificate or None, latency_s[, service_s])."""
        r, c, lat, svc = N.strom_result(), N.strom_certificate(), C.c_double(), C.c_double()
        c.max_ratio = float("nan")
        st = check(lib().strom_batch_poll(self.handle, ticket, C.byref(r), C.byref(c), C.byref(lat),
                                          C.byref(svc)), "strom_batch_poll")
        if st == N.STROM_PENDING:
            return None
        res = Result(r.status, r.iterations, r.pobj, r.dobj, r.eta_p, r.eta_d, r.eta_g, r.sigma, r.m_kept)
        cert = None
        if c.max_ratio == c.max_ratio:
            cert = Certificate(c.max_ratio, c.lower_bound, c.phat, c.xi, c.hmax, c.gmin, bool(c.feasible),
                               bool(c.rank_one), bool(c.certified), None, None)
        if with_service:
            return res, cert, lat.value, svc.value
        return res, cert, lat.value


class Server:
    """strom_server: requests of several structures behind one front, one
    batch per structure class, sized from one device-memory budget."""

    def __init__(self, budget_bytes: int, max_slots: int, **opts):
        self.opt = default_options(**opts)
        h = C.c_void_p()
        check(lib().strom_server_create(int(budget_bytes), int(max_slots), C.byref(self.opt), C.byref(h)),
              "strom_server_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_server_destroy(self.handle)
            self.handle = None

    def submit(self, sdp: Sdp, problem: Problem | None = None) -> int:
        t = C.c_uint64()
        check(lib().strom_server_submit(self.handle, sdp.handle, problem.handle if problem else None, C.byref(t)),
              "strom_server_submit")
        return t.value

    def step(self, iters: int, stream=None):
        """Returns (requests in batches, requests waiting for a batch)."""
        run, w = C.c_int32(), C.c_int32()
        check(lib().strom_server_step(self.handle, iters, stream, C.byref(run), C.byref(w)), "strom_server_step")
        return run.value, w.value

    def poll(self, ticket: int, with_service=False):
        """None while pending, else (Result, Certificate or None, latency_s[, service_s])."""
        r, c, lat, svc = N.strom_result(), N.strom_certificate(), C.c_double(), C.c_double()
        c.max_ratio = float("nan")
        st = check(lib().strom_server_poll(self.handle, ticket, C.byref(r), C.byref(c), C.byref(lat), C.byref(svc)),
                   "strom_server_poll")
        if st == N.STROM_PENDING:
            return None
        res = Result(r.status, r.iterations, r.pobj, r.dobj, r.eta_p, r.eta_d, r.eta_g, r.sigma, r.m_kept)
        cert = None
        if c.max_ratio == c.max_ratio:
            cert = Certificate(c.max_ratio, c.lower_bound, c.phat, c.xi, c.hmax, c.gmin, bool(c.feasible),
                               bool(c.rank_one), bool(c.certified), None, None)
        if with_service:
            return res, cert, lat.value, svc.value
        return res, cert, lat.value

    def info(self):
        """([per-class dict], bytes of the budget reserved by current batches)."""
        n, used = C.c_int32(), C.c_int64()
        check(lib().strom_server_info(self.handle, 0, None, C.byref(n), C.byref(used)), "strom_server_info")
        arr = (N.strom_server_class * max(1, n.value))()
        check(lib().strom_server_info(self.handle, n.value, arr, C.byref(n), C.byref(used)), "strom_server_info")
        return [{k: getattr(arr[i], k) for k, _ in arr[i]._fields_ if k != "pad"} for i in range(n.value)], used.value


class PsdPlan:
    """strom_psd_plan: PSD projection of a fixed list of svec blocks."""

    def __init__(self, blk_off, blk_n, precision=N.STROM_PREC_FP64):
        self._off = np.ascontiguousarray(blk_off, np.int64).ravel()
        self._n = np.ascontiguousarray(blk_n, np.int32).ravel()
        _check_blocks(self._off, self._n)
        h = C.c_void_p()
        check(lib().strom_psd_plan_create(_ptr(self._off, C.c_int64), _ptr(self._n, C.c_int32), len(self._n),
                                          precision, C.byref(h)), "strom_psd_plan_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            lib().strom_psd_plan_destroy(self.handle)
            self.handle = None

    def execute(self, xb_ptr, out_ptr, lam_ptr=None, stream=None):
        check(lib().strom_psd_execute(self.handle, xb_ptr, out_ptr, lam_ptr, stream), "strom_psd_execute")


def moment_rank_test(M, nv: int, vars_mask=None, tol: float = 1e-8):
    """strom_moment_rank_test: flat-extension and partial rank-1 tests of one moment matrix."""
    M = np.asfortranarray(np.asarray(M, np.float64))
    n = (nv + 1) * (nv + 2) // 2
    if M.shape != (n, n):
        raise ValueError("M must be %d x %d for nv = %d" % (n, n, nv))
    vm = None if vars_mask is None else np.ascontiguousarray(np.asarray(vars_mask, bool).astype(np.uint8))
    if vm is not None and vm.size != nv:
        raise ValueError("vars_mask must have nv entries")
    out, z = N.strom_rank_test(), np.empty(nv)
    check(lib().strom_moment_rank_test(M.ctypes.data_as(C.POINTER(C.c_double)), nv,
                                       None if vm is None else _ptr(vm, C.c_uint8), float(tol), C.byref(out),
                                       _ptr(z, C.c_double)), "strom_moment_rank_test")
    return dict(n=out.n, rank=out.rank, rank_low=out.rank_low, flat=bool(out.flat), n_sub=out.n_sub,
                ratio_sub=out.ratio_sub, lambda_max=out.lambda_max, zbar_sub=z)


def launch_count() -> int:
    """Kernels launched by libstrom in this process (graph nodes counted per replay)."""
    return int(lib().strom_launch_count())


def transfer_bytes():
    """(host->device, device->host) bytes copied by libstrom in this process."""
    h, d = C.c_uint64(), C.c_uint64()
    lib().strom_transfer_bytes(C.byref(h), C.byref(d))
    return int(h.value), int(d.value)


def _check_blocks(off, n):
    """One offset per block size, so the library never reads past either array."""
    if off.size != n.size:
        raise ValueError("blk_off has %d entries but blk_n has %d" % (off.size, n.size))


def kernel_spmv_csr(rowptr_ptr, col_ptr, val_ptr, nrows, x_ptr, y_ptr, stream=None):
    """strom_kernel_spmv_csr: y = M x for a CSR matrix in device memory (int64
    row pointers, int32 columns, FP64 values): A(X) with A's rows, A^*(y)
    with A^T's."""
    check(lib().strom_kernel_spmv_csr(rowptr_ptr, col_ptr, val_ptr, int(nrows), x_ptr, y_ptr, stream),
          "strom_kernel_spmv_csr")


def kernel_psd_project(xb_ptr, blk_off, blk_n, precision, out_ptr, stream=None):
    off = np.ascontiguousarray(blk_off, np.int64).ravel()
    n = np.ascontiguousarray(blk_n, np.int32).ravel()
    _check_blocks(off, n)
    check(lib().strom_kernel_psd_project(xb_ptr, _ptr(off, C.c_int64), _ptr(n, C.c_int32), len(n), precision,
                                         out_ptr, stream), "strom_kernel_psd_project")
