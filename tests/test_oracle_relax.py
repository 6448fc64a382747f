"""Pins of the oracle's relaxation builder (Prop. 1, Sec. 2.3) — CPU only."""
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import relax as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toy_identities.txt")
DT = 0.1


def _golden():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, body, cite = [t.strip() for t in line.split("|")]
        out.append((kind, body.split(), cite))
    return out


@pytest.fixture(scope="module")
def toy():
    p = wl.toy_problem(N=3, dt=DT)
    return p, R.relax(p)


def _entry(sdp, name, i, j):
    """Global svec index and scale of 1-based entry (i, j) of block name (M2, M3, L21)."""
    if name[0] == "M":
        blk = [b for b in sdp.blocks if b.kind == "M"][int(name[1]) - 1]
    else:
        blk = [b for b in sdp.blocks if b.kind == "L" and b.clique == int(name[1]) - 1][int(name[2]) - 1]
    return blk.offset + R.svec_index(i - 1, j - 1), R.svec_scale(i - 1, j - 1)


def _row_as_entries(sdp, r):
    """Row r as {svec index: coefficient on the matrix ENTRY} (svec coef / entry scale)."""
    A = sdp.A
    cols = A.indices[A.indptr[r]:A.indptr[r + 1]]
    vals = A.data[A.indptr[r]:A.indptr[r + 1]]
    out = {}
    for c, v in zip(cols, vals):
        # find the entry scale of column c
        blk = max((b for b in sdp.blocks if b.offset <= c), key=lambda b: b.offset)
        p = c - blk.offset
        j = int((math.isqrt(8 * p + 1) - 1) // 2)
        i = p - j * (j + 1) // 2
        out[int(c)] = v / R.svec_scale(i, j)
    return out


def _find_row(sdp, target):
    """Index of a row proportional to target {svec index: entry coef}, else None."""
    keys = set(target)
    for r in range(sdp.m):
        e = _row_as_entries(sdp, r)
        if set(e) != keys:
            continue
        k0 = next(iter(keys))
        lam = e[k0] / target[k0]
        if all(abs(e[k] - lam * target[k]) <= 1e-14 * max(1.0, abs(lam * target[k])) for k in keys):
            return r
    return None


def _parse_coef(s):
    return eval(s, {"dt": DT})


def test_basis_matches_printed(toy):
    _, sdp = toy
    (kind, body, _), = [g for g in _golden() if g[0] == "basis"]
    names = ["x1", "u1", "x2"]
    got = []
    for e in R.monomial_basis(3, 2):
        s = "".join(n + ("^2" if k == 2 else "") for n, k in zip(names, e) if k)
        got.append(s or "1")
    assert got == body


def test_mom_identity(toy):
    _, sdp = toy
    for kind, body, cite in _golden():
        if kind != "mom":
            continue
        ents = [b.split(":") for b in body]
        ids = [_entry(sdp, n, *map(int, ij.split(","))) for n, ij in ents]
        # all of them hold the same monomial: each non-representative is tied to one representative
        mi = sdp.mindex
        monos = {tuple(a + b for a, b in zip(mi.basis[int(ij.split(',')[0]) - 1], mi.basis[int(ij.split(',')[1]) - 1]))
                 for _, ij in ents}
        assert len(monos) == 1, cite
        rep = mi.rep[monos.pop()]
        p_rep, _ = _entry(sdp, ents[0][0], rep[0] + 1, rep[1] + 1)
        for (p, s) in ids:
            if p == p_rep:
                continue
            assert _find_row(sdp, {p: 1.0, p_rep: -1.0}) is not None, cite


@pytest.mark.parametrize("kind", ["ineq", "eq"])
def test_linear_identities(toy, kind):
    _, sdp = toy
    for k, body, cite in _golden():
        if k != kind:
            continue
        tgt = {}
        for t in body:
            name, ij, c = t.split(":")
            p, _ = _entry(sdp, name, *map(int, ij.split(",")))
            tgt[p] = tgt.get(p, 0.0) + _parse_coef(c)
        assert _find_row(sdp, tgt) is not None, cite


def test_eq_count(toy):
    _, sdp = toy
    (_, body, cite), = [g for g in _golden() if g[0] == "eqcount"]
    # clique 2 has one equality h_{2,1} of degree 2 -> s(3, 2) rows
    n_eq = int(np.sum((sdp.row_kind == R.KIND_EQ) & (sdp.row_clique == 1)))
    assert n_eq == int(body[0]), cite


def test_consensus(toy):
    _, sdp = toy
    for kind, body, cite in _golden():
        if kind != "cons":
            continue
        (n1, ij1), (n2, ij2) = [b.split(":") for b in body]
        p1, _ = _entry(sdp, n1, *map(int, ij1.split(",")))
        p2, _ = _entry(sdp, n2, *map(int, ij2.split(",")))
        if ij1 == "1,1":
            # the constant monomial: both equal 1 through their phi_0 rows
            for p in (p1, p2):
                r = _find_row(sdp, {p: 1.0})
                assert r is not None and sdp.b[r] == 1.0, cite
        else:
            assert _find_row(sdp, {p1: 1.0, p2: -1.0}) is not None, cite


def test_table1_sizes():
    (_, body, cite), = [g for g in _golden() if g[0] == "sizes"]
    for t in body:
        nv, sM, sL = map(int, t.split(":"))
        assert len(R.monomial_basis(nv, 2)) == sM == R.s_count(nv, 2), cite
        assert len(R.monomial_basis(nv, 1)) == sL == R.s_count(nv, 1), cite


# --------------------------------------------------------------------------
# rank-1 lifting of a feasible point satisfies A(X(z)) = b and <C, X(z)> = sum f_k
# (eq. rank1-lifting and the identity chain of eq. inexact-lower-bound)
# --------------------------------------------------------------------------
def _toy_rollout(p, u):
    dt, x = p.meta["dt"], [p.meta["x_init"]]
    z = [x[0]]
    for uk in u:
        xn = z[-1] - dt * (1.0 + uk) * z[-1]
        z += [uk, xn]
    return np.array(z)


def _pend_rollout(p, U):
    """Explicit pendulum simulation in the rescaled variables (Cayley rotation, 2x2 solve)."""
    m = p.meta
    dt, wmax, umax, gl = m["dt"], m["w_max"], m["u_max"], m["g_l"]
    c, s, W = np.cos(m["theta0"]), np.sin(m["theta0"]), 0.0
    z = [c, s, W]
    h = 0.5 * dt * wmax
    for Uk in U:
        a = h * W
        # [1 a; -a 1] [c+; s+] = [c - a s; s + a c]
        rhs1, rhs2 = c - a * s, s + a * c
        det = 1.0 + a * a
        cn, sn = (rhs1 - a * rhs2) / det, (rhs2 + a * rhs1) / det
        Wn = W + dt / wmax * (umax * Uk - gl * s)
        z += [Uk, cn, sn, Wn]
        c, s, W = cn, sn, Wn
    return np.array(z)


@pytest.mark.parametrize("which", ["toy", "pendulum"])
def test_lifting_feasible(which):
    rng = np.random.default_rng(3)
    if which == "toy":
        p = wl.toy_problem(N=4, dt=DT)
        z = _toy_rollout(p, rng.uniform(-1, 1, 4))
    else:
        p = wl.pendulum_problem(N=4, theta0=0.15)
        z = _pend_rollout(p, rng.uniform(-1, 1, 4))
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    res = sdp.A @ X - sdp.b
    assert np.max(np.abs(res)) < 1e-12
    assert abs(sdp.C @ X - p.objective(z)) < 1e-12 * (1 + abs(p.objective(z)))


def test_lifting_detects_infeasible():
    p = wl.pendulum_problem(N=3, theta0=0.15)
    z = _pend_rollout(p, [0.3, -0.2, 0.5])
    z[5] += 1e-3               # break the dynamics of one state
    sdp = R.relax(p)
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-5


def test_pendulum_shapes():
    p = wl.pendulum_problem(N=10)
    sdp = R.relax(p)
    sizes = [b.n for b in sdp.blocks]
    assert sizes.count(36) == 10 and sizes.count(8) == 20
    assert sdp.nsvec == 10 * 666 + 20 * 36


# --------------------------------------------------------------------------
# the paper's own pendulum model reproduces the printed SDP sizes
# --------------------------------------------------------------------------
def _paper_sizes():
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_pendulum_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            k, v, cite = (x.strip() for x in line.split("|"))
            out[k] = (int(v), cite)
    return out


def test_paper_pendulum_sizes():
    sdp = R.relax(wl.paper_pendulum_problem(N=30, theta0=0.4, thetadot0=-0.5))
    want = _paper_sizes()
    M = [b for b in sdp.blocks if b.kind == "M"]
    L = [b for b in sdp.blocks if b.kind == "L"]
    assert len(M) == want["nM"][0], want["nM"][1]
    assert {b.n for b in M} == {want["sizeM"][0]}, want["sizeM"][1]
    assert len(L) == want["nL"][0], want["nL"][1]
    assert {b.n for b in L} == {want["sizeL"][0]}, want["sizeL"][1]
    assert sdp.m == want["m"][0], want["m"][1]
    assert sdp.nsvec == want["nvar"][0], want["nvar"][1]


def _paper_pend_rollout(p, U):
    """Explicit simulation of the paper's pendulum (rate update, then the
    rotation by the previous step's increment), rescaled control U = u / u_max."""
    m = p.meta
    dt, umax = m["dt"], m["u_max"]
    ml2, mgl, b = 1.0, 9.8, 0.1                     # m = l = 1, g = 9.8, b = 0.1 (the defaults)
    rc, rs = np.cos(m["theta0"]), np.sin(m["theta0"])
    fc, fs = np.cos(dt * m["thetadot0"]), np.sin(dt * m["thetadot0"])
    z = [rc, rs, fc, fs]
    for Uk in U:
        fs_n = fs + dt * dt / ml2 * (umax * Uk - mgl * rs - b * fs / dt)
        fc_n = np.sqrt(1.0 - fs_n * fs_n)
        rc_n, rs_n = rc * fc - rs * fs, rs * fc + rc * fs
        z += [Uk, rc_n, rs_n, fc_n, fs_n]
        rc, rs, fc, fs = rc_n, rs_n, fc_n, fs_n
    return np.array(z)


def test_paper_pendulum_lifting_feasible():
    # a rollout of the paper's dynamics satisfies every row exactly when
    # lifted to rank-1 moment matrices, and <C, X> is its cost
    rng = np.random.default_rng(4)
    p = wl.paper_pendulum_problem(N=5, theta0=0.3, thetadot0=0.7)
    z = _paper_pend_rollout(p, rng.uniform(-1, 1, 5))
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    assert np.max(np.abs(sdp.A @ X - sdp.b)) < 1e-12
    assert abs(sdp.C @ X - p.objective(z)) < 1e-12 * (1 + abs(p.objective(z)))
    for k, c in enumerate(p.cliques):                 # the bounds hold along the rollout
        zk = p.clique_vars(z, k)
        assert all(g.evaluate(zk) >= -1e-12 for g in c.g)
    z[5] += 1e-3                                      # break r_c of x_1
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-5


# --------------------------------------------------------------------------
# the paper's vehicle landing and flying robot reproduce the printed sizes
# --------------------------------------------------------------------------
def paper_robot_sizes():
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_robot_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            model, k, v, cite = (x.strip() for x in line.split("|"))
            out.setdefault(model, {})[k] = (int(v), cite)
    return out


PAPER_ROBOTS = {"landing": "paper_landing_problem", "flying": "paper_flying_robot_problem",
                "car": "paper_car_backin_problem"}


@pytest.mark.parametrize("model", ["landing", "flying", "car"])
def test_paper_robot_sizes(model):
    """Under the equality reading of the paper's pendulum (circles of x_{k-1}
    in cliques k >= 2, x_0 fixed by linear equalities) and with the printed
    number of localizing matrices, the oracle's SDP has every size of the
    model's Table 1 row, m included."""
    want = paper_robot_sizes()[model]
    p = getattr(wl, PAPER_ROBOTS[model])()
    if "dx" in want:
        assert (p.dx, p.du) == (want["dx"][0], want["du"][0])
    else:
        assert p.nv == want["nvars"][0], want["nvars"][1]
    sdp = R.relax(p)
    M = [b for b in sdp.blocks if b.kind == "M"]
    L = [b for b in sdp.blocks if b.kind == "L"]
    assert len(M) == want["nM"][0], want["nM"][1]
    assert {b.n for b in M} == {want["sizeM"][0]}, want["sizeM"][1]
    assert len(L) == want["nL"][0], want["nL"][1]
    assert {b.n for b in L} == {want["sizeL"][0]}, want["sizeL"][1]
    assert sdp.m == want["m"][0], want["m"][1]


def flying_robot_rollout(p, U, dt=0.2, alpha=0.2, beta=0.2, r_max=10.0, v_max=10.0, u_max=8.0,
                         x0=5.0, y0=-5.0, theta0=0.3):
    """Explicit simulation of the flying robot in physical units (controls U in
    [-1, 1]^4 map to u in [0, u_max]); returns the rescaled global vector."""
    rx, ry, vx, vy = x0, y0, 0.0, 0.0
    rc, rs, fc, fs = np.cos(theta0), np.sin(theta0), 1.0, 0.0
    scale = np.array([r_max, r_max, v_max, v_max, 1, 1, 1, 1])
    z = list(np.array([rx, ry, vx, vy, rc, rs, fc, fs]) / scale)
    for Uk in U:
        u = 0.5 * u_max * (np.asarray(Uk) + 1.0)
        T = u[0] - u[1] + u[2] - u[3]
        rx_n, ry_n = rx + dt * vx, ry + dt * vy
        vx_n, vy_n = vx + dt * T * rc, vy + dt * T * rs
        fs_n = fs + dt * dt * alpha * (u[1] - u[0]) + dt * dt * beta * (u[2] - u[3])
        fc_n = np.sqrt(1.0 - fs_n * fs_n)
        rc_n, rs_n = rc * fc - rs * fs, rs * fc + rc * fs
        rx, ry, vx, vy, rc, rs, fc, fs = rx_n, ry_n, vx_n, vy_n, rc_n, rs_n, fc_n, fs_n
        z += list(Uk) + list(np.array([rx, ry, vx, vy, rc, rs, fc, fs]) / scale)
    return np.array(z)


def test_paper_flying_robot_lifting_feasible():
    """A rollout of the flying robot's dynamics, lifted to rank-1 moment
    matrices, satisfies every row; its cost is <C, X>."""
    rng = np.random.default_rng(6)
    p = wl.paper_flying_robot_problem(N=4)
    U = rng.uniform(-0.3, 0.3, size=(4, 4))
    z = flying_robot_rollout(p, U)
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    assert np.max(np.abs(sdp.A @ X - sdp.b)) < 1e-12
    assert abs(sdp.C @ X - p.objective(z)) < 1e-12 * (1 + abs(p.objective(z)))
    for k, c in enumerate(p.cliques):
        assert all(g.evaluate(p.clique_vars(z, k)) >= -1e-12 for g in c.g)
    z[12 + 2] += 1e-4                  # v_x of x_1 (x_1 starts at z[12])
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-7


def landing_rollout(U, dt=0.2, m=1.0, inertia=50.0, lever=5.0, g=9.8, rx_max=100.0, ry_min=10.0, ry_max=120.0,
                    v_max=20.0, u_max=8.0, x0=20.0, y0=100.0, vx0=0.0, vy0=-5.0, theta0=0.1):
    """Explicit simulation of the vehicle landing in physical units (U in
    [-1, 1]^2 maps to u in [0, u_max]); returns the rescaled global vector."""
    rx, ry, vx, vy = x0, y0, vx0, vy0
    rc, rs, fc, fs = np.cos(theta0), np.sin(theta0), 1.0, 0.0

    def scaled(st):
        rx_, ry_, vx_, vy_ = st[:4]
        return [rx_ / rx_max, (ry_ - 0.5 * (ry_max + ry_min)) / (0.5 * (ry_max - ry_min)), vx_ / v_max,
                vy_ / v_max] + list(st[4:])
    z = scaled([rx, ry, vx, vy, rc, rs, fc, fs])
    for Uk in U:
        u = 0.5 * u_max * (np.asarray(Uk) + 1.0)
        T = u[0] + u[1]
        rx_n, ry_n = rx + dt * vx, ry + dt * vy
        vx_n = vx - dt * T * rs / m
        vy_n = vy + dt * (T * rc - m * g) / m
        fs_n = fs + lever * dt * dt * (u[1] - u[0]) / inertia
        fc_n = np.sqrt(1.0 - fs_n * fs_n)
        rc_n, rs_n = rc * fc - rs * fs, rs * fc + rc * fs
        rx, ry, vx, vy, rc, rs, fc, fs = rx_n, ry_n, vx_n, vy_n, rc_n, rs_n, fc_n, fs_n
        z += list(Uk) + scaled([rx, ry, vx, vy, rc, rs, fc, fs])
    return np.array(z)


def test_paper_landing_lifting_feasible():
    rng = np.random.default_rng(7)
    p = wl.paper_landing_problem(N=4)
    z = landing_rollout(rng.uniform(0.0, 0.6, size=(4, 2)))
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    assert np.max(np.abs(sdp.A @ X - sdp.b)) < 1e-12
    assert abs(sdp.C @ X - p.objective(z)) < 1e-12 * (1 + abs(p.objective(z)))
    for k, c in enumerate(p.cliques):
        assert all(g.evaluate(p.clique_vars(z, k)) >= -1e-12 for g in c.g)
    z[10 + 3] += 1e-4                  # v_y of x_1 (x_1 starts at z[10])
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-7


def car_rollout(V, Wr, dt=0.25, x0=2.0, y0=4.0, theta0=0.0, v_max=4.0, w_max=0.5, rx_max=4.0, ry_max=8.0):
    """Explicit simulation of the car (unicycle with the third-order rotation
    of the appendix), with the horizontal separating line y = 2 for both
    obstacles (positions divided by 8, (A, B, C) normalised)."""
    rx, ry, rc, rs = x0, y0, np.cos(theta0), np.sin(theta0)
    line = np.array([0.0, 1.0, -0.25]) / np.sqrt(1.0625)
    z = [rx / rx_max, ry / ry_max, rc, rs]
    for Vk, Wk in zip(V, Wr):
        v, w = v_max * Vk, w_max * Wk
        fs = dt * w - (dt * w) ** 3 / 6.0
        fc = np.sqrt(1.0 - fs * fs)
        rx, ry = rx + dt * v * rc, ry + dt * v * rs
        rc, rs = rc * fc - rs * fs, rs * fc + rc * fs
        z += [Vk, Wk, fc, fs] + list(line) + list(line) + [rx / rx_max, ry / ry_max, rc, rs]
    return np.array(z)


def test_paper_car_backin_lifting_feasible():
    """A rollout of the car with valid separating lines: every row of the SDP
    holds at its rank-1 lifting, every inequality (corners on either side of
    the lines, boxes) holds along it, and a perturbed position breaks it."""
    rng = np.random.default_rng(8)
    p = wl.paper_car_backin_problem(N=3)
    z = car_rollout(rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.5, 0.5, 3))
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    assert np.max(np.abs(sdp.A @ X - sdp.b)) < 1e-12
    assert abs(sdp.C @ X - p.objective(z)) < 1e-12 * (1 + abs(p.objective(z)))
    for k, c in enumerate(p.cliques):
        assert all(g.evaluate(p.clique_vars(z, k)) >= -1e-12 for g in c.g)
    z[14] += 1e-4                      # r_x of x_1 (x_1 starts at z[14])
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-7
