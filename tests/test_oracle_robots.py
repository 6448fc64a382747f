"""Pins of the cart-pole and planar rigid-body relaxations (CPU only).

The two robots are written in workloads/ as polynomial equalities after the
rescaling of every variable to [-1, 1] and, for the cart-pole, after clearing
the mass-matrix denominator. Here each robot is simulated from its physical
equations in divided form (no polynomial arithmetic, no rescaling inside the
step), and the rank-1 lifting of the rollout (eq. rank1-lifting) must satisfy
every row of the oracle's SDP, A(X(z)) = b, with <C, X(z)> equal to the
rollout's cost: a dropped term, a wrong sign or a wrong scale in either the
generator or the builder breaks one of these. The block sizes are those of
Prop. 1 for 11- and 16-variable cliques, and the seeded rigid-body batch
follows its stated recipe.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import relax as R

# cart-pole constants of the generator call below (m_c = 1, m_p = 0.1,
# l = 0.5, |f| <= 10, dt = 0.05; box limits on x, v, w)
CP = dict(dt=0.05, mc=1.0, mp=0.1, l=0.5, g=9.81, f_max=10.0, x_max=2.0, v_max=4.0, w_max=10.0)
# rigid-body constants of the generator call below
RB = dict(dt=0.1, p_max=2.5, v_max=2.0, w_max=2.0, a_max=1.0, lever=0.5)


def _cayley_step(c, s, a):
    """Implicit-midpoint rotation: [1 a; -a 1] [c+; s+] = [c - a s; s + a c]."""
    r1, r2 = c - a * s, s + a * c
    det = 1.0 + a * a
    return (r1 - a * r2) / det, (r2 + a * r1) / det


def cartpole_rollout(F, x0, theta0, dt, mc, mp, l, g, f_max, x_max, v_max, w_max):
    """Physical cart-pole (theta from hanging), explicit Euler on x, v, w and the
    Cayley rotation on (cos, sin) with the previous rate; returns the rescaled
    global vector z = (x_0, u_0, x_1, ..., x_N), x = (X, V, C, S, W), u = F."""
    x, v, c, s, w = x0, 0.0, math.cos(theta0), math.sin(theta0), 0.0
    z = [x / x_max, v / v_max, c, s, w / w_max]
    for Fk in F:
        f = f_max * Fk
        D = mc + mp * s * s
        xn = x + dt * v
        vn = v + dt * (f + mp * s * (g * c + l * w * w)) / D
        wn = w + dt * (-c * f - mp * l * c * s * w * w - (mc + mp) * g * s) / (l * D)
        cn, sn = _cayley_step(c, s, 0.5 * dt * w)
        z += [Fk, xn / x_max, vn / v_max, cn, sn, wn / w_max]
        x, v, c, s, w = xn, vn, cn, sn, wn
    return np.array(z)


def rigid_rollout(FC, FS, start, dt, p_max, v_max, w_max, a_max, lever):
    """Planar rigid body: body-frame force (fc, fs) rotated into the world frame,
    yaw torque lever * fs; x = (RX, RY, C, S, VX, VY, W), u = (FC, FS)."""
    rx, ry, th = start
    c, s, vx, vy, w = math.cos(th), math.sin(th), 0.0, 0.0, 0.0
    z = [rx / p_max, ry / p_max, c, s, 0.0, 0.0, 0.0]
    for fc, fs in zip(FC, FS):
        ax, ay = a_max * (c * fc - s * fs), a_max * (s * fc + c * fs)
        rxn, ryn = rx + dt * vx, ry + dt * vy
        vxn, vyn = vx + dt * ax, vy + dt * ay
        wn = w + dt * a_max * lever * fs
        cn, sn = _cayley_step(c, s, 0.5 * dt * w)
        z += [fc, fs, rxn / p_max, ryn / p_max, cn, sn, vxn / v_max, vyn / v_max, wn / w_max]
        rx, ry, c, s, vx, vy, w = rxn, ryn, cn, sn, vxn, vyn, wn
    return np.array(z)


def _cartpole(N, x0=0.3, theta0=0.25):
    return wl.cartpole_problem(N=N, x0=x0, theta0=theta0, **CP)


def _rigid(N, disks):
    return wl.rigid_body_problem(N=N, start=(-0.8, -0.6, 0.4), goal=(0.5, 0.5, 1.0), disks=disks, **RB)


def _check_lifting(p, z):
    sdp = R.relax(p)
    X = R.lift_rank1(p, sdp, z)
    res = sdp.A @ X - sdp.b
    assert np.max(np.abs(res)) < 1e-12
    cost = p.objective(z)
    assert abs(sdp.C @ X - cost) < 1e-12 * (1 + abs(cost))
    return sdp


def test_cartpole_lifting_feasible():
    rng = np.random.default_rng(11)
    F = rng.uniform(-1, 1, 4)
    p = _cartpole(4)
    z = cartpole_rollout(F, 0.3, 0.25, **CP)
    _check_lifting(p, z)
    # the rollout respects the boxes, so every localizing matrix is PSD at it
    for k, c in enumerate(p.cliques):
        assert all(g.evaluate(p.clique_vars(z, k)) >= 0 for g in c.g)


@pytest.mark.parametrize("where", ["v", "w", "c"])
def test_cartpole_lifting_detects_broken_dynamics(where):
    p = _cartpole(3)
    z = cartpole_rollout([0.4, -0.7, 0.2], 0.3, 0.25, **CP)
    # x_1 occupies z[6:11] = (X, V, C, S, W)
    z[{"v": 7, "w": 10, "c": 8}[where]] += 1e-4
    sdp = R.relax(p)
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-7


def test_cartpole_divided_form_is_not_the_undivided_one():
    """Dropping the denominator D = m_c + m_p s^2 from the rollout (a plausible
    slip) makes the lifting infeasible: the generator really multiplies it through."""
    cp = dict(CP)
    p = _cartpole(2, theta0=1.0)
    z = cartpole_rollout([0.5, -0.5], 0.3, 1.0, **cp)
    sdp = R.relax(p)
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) < 1e-12
    cp["mp"] = 0.0        # D -> m_c and the pole terms vanish: a different system
    z2 = cartpole_rollout([0.5, -0.5], 0.3, 1.0, **cp)
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z2) - sdp.b)) > 1e-6


def test_rigid_body_lifting_feasible():
    rng = np.random.default_rng(12)
    ang = rng.uniform(-np.pi, np.pi, 3)
    mag = rng.uniform(0, 1, 3)
    FC, FS = mag * np.cos(ang), mag * np.sin(ang)
    disks = [(1.5, -1.5, 0.4), (-1.8, 1.2, 0.6)]
    p = _rigid(3, disks)
    z = rigid_rollout(FC, FS, (-0.8, -0.6, 0.4), **RB)
    _check_lifting(p, z)
    for k, c in enumerate(p.cliques):
        assert all(g.evaluate(p.clique_vars(z, k)) >= 0 for g in c.g)
    z[9 + 4] += 1e-4         # VX of x_1 (x_1 starts at z[9])
    sdp = R.relax(p)
    assert np.max(np.abs(sdp.A @ R.lift_rank1(p, sdp, z) - sdp.b)) > 1e-7


def test_disk_constraint_sign():
    """A rollout that ends inside a disk violates that disk's polynomial: the
    obstacle inequality is ||r - o||^2 - rho^2 >= 0 in the rescaled frame."""
    z = rigid_rollout([0.0, 0.0], [0.0, 0.0], (0.2, 0.1, 0.0), **RB)   # stays at (0.2, 0.1)
    inside = _rigid(2, [(0.25, 0.1, 0.3)])
    outside = _rigid(2, [(1.5, 0.1, 0.3)])
    for p, sign in ((inside, -1), (outside, 1)):
        g_disk = p.cliques[0].g[4]
        assert sign * g_disk.evaluate(p.clique_vars(z, 0)) > 0


def test_block_sizes_of_the_robot_workloads():
    # cart-pole, N = 50: 11-variable cliques -> 50 moment blocks of s(11, 2) = 78
    # and 4 localizing blocks of s(11, 1) = 12 per clique
    sdp = R.relax(wl.cartpole_problem(N=50, x0=0.1, theta0=0.2))
    M = [b.n for b in sdp.blocks if b.kind == "M"]
    L = [b.n for b in sdp.blocks if b.kind == "L"]
    assert M == [R.s_count(11, 2)] * 50 == [78] * 50
    assert L == [R.s_count(11, 1)] * 200 == [12] * 200
    assert sdp.nsvec == 50 * 3081 + 200 * 78 == 169_650
    # rigid body: 16-variable cliques -> 153 and 17, 4 + (number of disks) localizing blocks
    sdp = R.relax(_rigid(3, [(1.5, -1.5, 0.4), (-1.8, 1.2, 0.6), (0.0, 1.9, 0.3)]))
    M = [b.n for b in sdp.blocks if b.kind == "M"]
    L = [b.n for b in sdp.blocks if b.kind == "L"]
    assert M == [R.s_count(16, 2)] * 3 == [153] * 3
    assert L == [R.s_count(16, 1)] * 21 == [17] * 21


def test_rigid_body_batch_recipe():
    """Seeded uneven batch: N ~ U{20..100}, 2-4 disks of radius U(0.3, 1.0) with
    centres in [-2, 2]^2 clear of start and goal, goal position in the unit box,
    heading in [-pi, pi]; a horizon given by the caller holds for every instance."""
    batch = wl.problem_batch("rigid_body", 12, seed=5)
    Ns = [p.N for p in batch]
    assert all(20 <= n <= 100 for n in Ns) and len(set(Ns)) > 1
    for p in batch:
        d = p.meta["disks"]
        assert 2 <= len(d) <= 4
        gx, gy, gth = p.meta["goal"]
        assert -1 <= gx <= 1 and -1 <= gy <= 1 and -np.pi <= gth <= np.pi
        for ox, oy, rho in d:
            assert 0.3 <= rho <= 1.0 and -2 <= ox <= 2 and -2 <= oy <= 2
            for px, py in (p.meta["start"][:2], (gx, gy)):
                assert math.hypot(ox - px, oy - py) > rho + 0.2
        assert len(p.cliques[0].g) == 4 + len(d)
    fixed = wl.problem_batch("rigid_body", 4, seed=5, N=7)
    assert [p.N for p in fixed] == [7] * 4
    # same seed, same instances
    again = wl.problem_batch("rigid_body", 12, seed=5)
    assert [p.meta["goal"] for p in again] == [p.meta["goal"] for p in batch]


def _cartpole_brute(p, x0, theta0):
    """min over (F_0, F_1) in [-1, 1]^2 of the rollout cost, boxes enforced:
    a 201 x 201 grid, then a bounded quasi-Newton refinement from its best point."""
    import scipy.optimize as so

    def cost(F):
        F = np.clip(F, -1, 1)
        z = cartpole_rollout(F, x0, theta0, **CP)
        for k in range(1, p.N + 1):
            xk = z[k * 6:k * 6 + 5]
            if max(abs(xk[0]), abs(xk[1]), abs(xk[4])) > 1.0:
                return np.inf
        return p.objective(z)
    g = np.linspace(-1, 1, 201)
    best, F0 = np.inf, None
    for a in g:
        for b in g:
            v = cost([a, b])
            if v < best:
                best, F0 = v, np.array([a, b])
    r = so.minimize(cost, F0, bounds=[(-1, 1)] * 2, method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
    return min(r.fun, best)


def test_cartpole_relaxation_matches_brute_force():
    """Theorem 1 on the cart-pole at N = 2: p*_kappa <= p* always, and with rank-1
    moment matrices the relaxation is tight, so the oracle's sGS-ADMM optimum
    equals a brute-force search of the nonconvex problem."""
    from oracle import certify as CE
    from oracle import sgs_admm as O
    x0, th0 = 0.2, 0.15
    p = _cartpole(2, x0=x0, theta0=th0)
    pbf = _cartpole_brute(p, x0, th0)
    red = O.reduce(R.relax(p))
    res = O.solve(red, O.Options(tol=1e-9, maxiter=40000))
    assert res.converged
    cert = CE.certify(p, red, res.X, res.y)
    assert res.pobj <= pbf + 1e-6 * (1 + abs(pbf))
    assert cert.lower_bound <= pbf + 1e-9
    assert cert.rank_one and cert.feasible
    assert abs(res.pobj - pbf) <= 1e-6 * (1 + abs(pbf))
    assert cert.phat >= pbf - 1e-9 * (1 + abs(pbf))
