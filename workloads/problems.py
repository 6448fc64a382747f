"""Polynomial trajectory problems with chain-like sparsity (Definition 1).

Every problem is a list of N cliques. Clique k (1-based, k = 1..N) holds the
variables z(I_k) = (x_{k-1}, u_{k-1}, x_k) in that order (Sec. 2.1), so the
overlap of cliques k and k+1 is x_k: the last dx variables of clique k and
the first dx variables of clique k+1. For each clique the data are the
objective term f_k, the inequality polynomials g_{k,i} >= 0 and the equality
polynomials h_{k,j} = 0, all in clique-local variables.

Variables are rescaled to [-1, 1] by their bounds and every constraint
polynomial is divided by its largest |coefficient| (Sec. 5, general setup);
the objective is divided by one global constant. The rotation (cos, sin)
pairs are propagated with the implicit-midpoint (Cayley) rotation
  c+ + h w s+ = c - h w s,   s+ - h w c+ = s + h w c,   h = dt/2,
which is polynomial of degree 2 and keeps c^2 + s^2 fixed exactly, so the
per-step circle equality c^2 + s^2 = 1 is consistent with the dynamics.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .poly import Poly


@dataclass
class Clique:
    f: Poly
    g: list
    h: list


@dataclass
class Problem:
    name: str
    N: int
    dx: int
    du: int
    cliques: list
    R: float = 1.0                 # bound on |z_i| after rescaling (Theorem 1)
    kappa: int = 2
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return 2 * self.dx + self.du

    def clique_arrays(self, k: int):
        """Clique k (0-based) as ((coef, expo) of f, [g...], [h...])."""
        c = self.cliques[k]
        return c.f.arrays(), [p.arrays() for p in c.g], [p.arrays() for p in c.h]

    def objective(self, z) -> float:
        """Sum_k f_k(z(I_k)) for a global vector z = (x0, u0, x1, u1, ..., xN)."""
        return sum(c.f.evaluate(self.clique_vars(z, k)) for k, c in enumerate(self.cliques))

    def clique_vars(self, z, k: int):
        s = k * (self.dx + self.du)
        return np.asarray(z, dtype=np.float64)[s:s + self.nv]

    @property
    def nz(self) -> int:
        return self.N * (self.dx + self.du) + self.dx


# --------------------------------------------------------------------------
# toy 1-D system of Example 1 (unscaled, exactly as printed)
# --------------------------------------------------------------------------
def toy_problem(N: int = 3, dt: float = 0.1, Pf: float = 1.0, x_init: float = 2.0) -> Problem:
    """Example 1: x_k = x_{k-1} - dt (1 + u_{k-1}) x_{k-1}, |u| <= 1, x_0 = x_init.

    Clique data follow eq. (toy-as-sparse-pop): f_k = u^2 + x_{k-1}^2 plus
    Pf x_N^2 in the last clique, g = 1 - u^2, h_1 = x_k + (dt-1) x_{k-1} +
    dt u x_{k-1}, and h_2 = x_0 - x_init in clique 1 only.
    """
    nv = 3
    X0, U, X1 = (Poly.var(nv, i) for i in range(3))
    cl = []
    for k in range(1, N + 1):
        f = U * U + X0 * X0
        if k == N:
            f = f + Pf * X1 * X1
        g = [1.0 - U * U]
        h = [X1 + (dt - 1.0) * X0 + dt * U * X0]
        if k == 1:
            h.append(X0 - x_init)
        cl.append(Clique(f, g, h))
    return Problem("toy", N, 1, 1, cl, R=max(1.0, abs(x_init)),
                   meta=dict(dt=dt, Pf=Pf, x_init=x_init))


def _cayley(c0, s0, w, c1, s1, hw):
    """Implicit-midpoint rotation by angle ~ 2*atan(hw*w), as two equalities."""
    e1 = c1 + hw * w * s1 - c0 + hw * w * s0
    e2 = s1 - hw * w * c1 - s0 - hw * w * c0
    return e1, e2


# --------------------------------------------------------------------------
# pendulum swing-up: state (c, s, w), control u
# --------------------------------------------------------------------------
def pendulum_problem(N: int = 10, dt: float = 0.1, theta0: float = 0.1, g_l: float = 9.81,
                     u_max: float = 2.0, w_max: float = 4.0, omega0: float = 0.0) -> Problem:
    """Pendulum: theta from hanging, c = cos(theta), s = sin(theta), w = theta-dot.

    Rescaled variables: w = w_max * W, u = u_max * U.
      rotation : Cayley step with w_{k-1}
      rate     : w_k = w_{k-1} + dt (u_{k-1} - g/l s_{k-1})
      circle   : c_k^2 + s_k^2 = 1
      bounds   : 1 - U^2 >= 0, 1 - W_k^2 >= 0
      cost     : sum_{k=0}^{N-1} 10 (1 + c_k)^2 + w_k^2 + 0.1 u_k^2
                 + 10 (1 + c_N)^2 + w_N^2     (terminal weight Pf = 1)
      initial  : c_0 = cos(theta0), s_0 = sin(theta0), w_0 = omega0 (clique 1)
    """
    nv = 7
    C0, S0, W0, U, C1, S1, W1 = (Poly.var(nv, i) for i in range(nv))
    hw = 0.5 * dt * w_max
    raw = []
    for k in range(1, N + 1):
        f = 10.0 * (1.0 + C0) ** 2 + (w_max ** 2) * W0 * W0 + 0.1 * (u_max ** 2) * U * U
        if k == N:
            f = f + 10.0 * (1.0 + C1) ** 2 + (w_max ** 2) * W1 * W1
        e1, e2 = _cayley(C0, S0, W0, C1, S1, hw)
        e3 = W1 - W0 - (dt / w_max) * (u_max * U - g_l * S0)
        e4 = C1 * C1 + S1 * S1 - 1.0
        h = [e1, e2, e3, e4]
        if k == 1:  # the initial state first: the same constraints, less fill in the y-solve's factor
            h = [C0 - np.cos(theta0), S0 - np.sin(theta0), W0 - omega0 / w_max] + h
        g = [1.0 - U * U, 1.0 - W1 * W1]
        raw.append((f, g, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in g], [p.normalized() for p in h])
          for f, g, h in raw]
    return Problem("pendulum", N, 3, 1, cl, R=1.0,
                   meta=dict(dt=dt, theta0=theta0, g_l=g_l, u_max=u_max, w_max=w_max,
                             fscale=fscale, x_init=[np.cos(theta0), np.sin(theta0), 0.0]))


# --------------------------------------------------------------------------
# the paper's pendulum (App. "Inverted Pendulum"): Lie-group variational
# integrator on SO(2), state x = (r_c, r_s, f_c, f_s), control u
# --------------------------------------------------------------------------
def paper_pendulum_problem(N: int = 30, dt: float = 0.1, theta0: float = 0.0, thetadot0: float = 0.0,
                           m: float = 1.0, l: float = 1.0, b: float = 0.1, g: float = 9.8,
                           fc_min: float = 0.5, u_max: float = 5.0, Pf: float = 1.0) -> Problem:
    """The inverted pendulum of the paper's experiments, 9-variable cliques.

    r = (r_c, r_s) is the attitude (cos, sin of theta) and f = (f_c, f_s) the
    rotation from one step to the next (f_s / dt ~ the angular rate). Per
    clique k, with u scaled to U = u / u_max:
      rate     : m l^2 (f_s,k - f_s,k-1) / dt^2 = u_{k-1} - m g l r_s,k-1 - b f_s,k-1 / dt
      rotation : r_c,k = r_c,k-1 f_c,k-1 - r_s,k-1 f_s,k-1,
                 r_s,k = r_s,k-1 f_c,k-1 + r_c,k-1 f_s,k-1
      SO(2)    : r_c^2 + r_s^2 = 1 and f_c^2 + f_s^2 = 1 for x_k, and for
                 x_{k-1} when k >= 2 (x_0 is fixed by the initial condition)
      bounds   : f_c,k - fc_min >= 0, 1 - U_{k-1}^2 >= 0 (two localizing blocks)
      initial  : x_0 = (cos theta0, sin theta0, cos(dt thetadot0), sin(dt thetadot0))
      cost     : the LQR-style loss to x_f = (-1, 0, 1, 0) (theta = pi, at rest)
                 with identity weights, Pf on x_N.
    With N = 30 this has the sizes of the paper's pendulum row of Table 1:
    30 moment blocks 55 x 55, 60 localizing blocks 10 x 10, 47,351 rows and
    49,500 svec entries.
    """
    nv = 9
    v = [Poly.var(nv, i) for i in range(nv)]
    rc0, rs0, fc0, fs0, U, rc1, rs1, fc1, fs1 = v
    xf = (-1.0, 0.0, 1.0, 0.0)
    x_prev, x_next = (rc0, rs0, fc0, fs0), (rc1, rs1, fc1, fs1)
    raw = []
    for k in range(1, N + 1):
        f = sum((xi - t) * (xi - t) for xi, t in zip(x_prev, xf)) + U * U
        if k == N:
            f = f + Pf * sum((xi - t) * (xi - t) for xi, t in zip(x_next, xf))
        h = [m * l * l / (dt * dt) * (fs1 - fs0) - u_max * U + m * g * l * rs0 + b / dt * fs0,
             rc1 - rc0 * fc0 + rs0 * fs0,
             rs1 - rs0 * fc0 - rc0 * fs0,
             rc1 * rc1 + rs1 * rs1 - 1.0,
             fc1 * fc1 + fs1 * fs1 - 1.0]
        if k >= 2:
            h += [rc0 * rc0 + rs0 * rs0 - 1.0, fc0 * fc0 + fs0 * fs0 - 1.0]
        else:
            h += [rc0 - np.cos(theta0), rs0 - np.sin(theta0), fc0 - np.cos(dt * thetadot0),
                  fs0 - np.sin(dt * thetadot0)]
        gg = [fc1 - fc_min, 1.0 - U * U]
        raw.append((f, gg, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in gg], [p.normalized() for p in h]) for f, gg, h in raw]
    return Problem("paper_pendulum", N, 4, 1, cl, R=1.0,
                   meta=dict(dt=dt, theta0=theta0, thetadot0=thetadot0, u_max=u_max, fc_min=fc_min,
                             fscale=fscale))


# --------------------------------------------------------------------------
# cart-pole swing-up: state (x, v, c, s, w), control force f
# --------------------------------------------------------------------------
def cartpole_problem(N: int = 50, dt: float = 0.05, x0: float = 0.0, theta0: float = 0.0,
                     mc: float = 1.0, mp: float = 0.1, l: float = 0.5, g: float = 9.81,
                     f_max: float = 10.0, x_max: float = 2.0, v_max: float = 4.0,
                     w_max: float = 10.0) -> Problem:
    """Cart-pole, theta from hanging, dynamics multiplied by D = mc + mp s^2.

      x_k = x_{k-1} + dt v_{k-1}
      D (v_k - v_{k-1}) = dt (f + mp s (g c + l w^2))
      l D (w_k - w_{k-1}) = dt (-c f - mp l c s w^2 - (mc + mp) g s)
      (c, s) Cayley step with w_{k-1};  c_k^2 + s_k^2 = 1
      boxes on f, x_k, v_k, w_k;  LQR-style cost towards (0, 0, -1, 0, 0).
    """
    nv = 11
    V = [Poly.var(nv, i) for i in range(nv)]
    X0, V0, C0, S0, W0, F, X1, V1, C1, S1, W1 = V
    hw = 0.5 * dt * w_max
    D = mc + mp * S0 * S0
    raw = []
    for k in range(1, N + 1):
        stage = (X0 * X0 + V0 * V0 + (C0 + 1.0) ** 2 + S0 * S0 + W0 * W0 + F * F)
        if k == N:
            stage = stage + X1 * X1 + V1 * V1 + (C1 + 1.0) ** 2 + S1 * S1 + W1 * W1
        e_x = x_max * X1 - x_max * X0 - dt * v_max * V0
        e_v = D * (v_max * V1 - v_max * V0) - dt * (f_max * F + mp * S0 * (g * C0 + l * w_max ** 2 * W0 * W0))
        e_w = l * D * (w_max * W1 - w_max * W0) - dt * (-f_max * C0 * F - mp * l * w_max ** 2 * C0 * S0 * W0 * W0
                                                       - (mc + mp) * g * S0)
        e1, e2 = _cayley(C0, S0, W0, C1, S1, hw)
        e_c = C1 * C1 + S1 * S1 - 1.0
        h = [e_x, e_v, e_w, e1, e2, e_c]
        if k == 1:  # the initial state first: the same constraints, less fill in the y-solve's factor
            h = [X0 - x0 / x_max, V0 - 0.0, C0 - np.cos(theta0), S0 - np.sin(theta0), W0 - 0.0] + h
        gg = [1.0 - F * F, 1.0 - X1 * X1, 1.0 - V1 * V1, 1.0 - W1 * W1]
        raw.append((stage, gg, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in gg], [p.normalized() for p in h])
          for f, gg, h in raw]
    return Problem("cartpole", N, 5, 1, cl, R=1.0,
                   meta=dict(dt=dt, x0=x0, theta0=theta0, fscale=fscale,
                             x_init=[x0 / x_max, 0.0, np.cos(theta0), np.sin(theta0), 0.0]))


# --------------------------------------------------------------------------
# planar rigid body among disk obstacles: state (rx, ry, c, s, vx, vy, w),
# control (fc, fs) with fc^2 + fs^2 <= 1 (body-frame force)
# --------------------------------------------------------------------------
def rigid_body_problem(N: int = 20, dt: float = 0.1, start=(-0.8, -0.8, 0.0), goal=(0.5, 0.5, 0.0),
                       disks=(), p_max: float = 2.5, v_max: float = 2.0, w_max: float = 2.0,
                       a_max: float = 1.0, lever: float = 0.5) -> Problem:
    nv = 16
    V = [Poly.var(nv, i) for i in range(nv)]
    RX0, RY0, C0, S0, VX0, VY0, W0, FC, FS, RX1, RY1, C1, S1, VX1, VY1, W1 = V
    hw = 0.5 * dt * w_max
    gx, gy, gth = goal
    gxs, gys = gx / p_max, gy / p_max
    raw = []
    for k in range(1, N + 1):
        stage = ((RX0 - gxs) ** 2 + (RY0 - gys) ** 2 + (C0 - np.cos(gth)) ** 2 + (S0 - np.sin(gth)) ** 2
                 + VX0 * VX0 + VY0 * VY0 + W0 * W0 + FC * FC + FS * FS)
        if k == N:
            stage = stage + ((RX1 - gxs) ** 2 + (RY1 - gys) ** 2 + (C1 - np.cos(gth)) ** 2
                             + (S1 - np.sin(gth)) ** 2 + VX1 * VX1 + VY1 * VY1 + W1 * W1)
        s = dt * v_max / p_max
        e_rx = RX1 - RX0 - s * VX0
        e_ry = RY1 - RY0 - s * VY0
        a = dt * a_max / v_max
        e_vx = VX1 - VX0 - a * (C0 * FC - S0 * FS)
        e_vy = VY1 - VY0 - a * (S0 * FC + C0 * FS)
        e_w = W1 - W0 - (dt * a_max * lever / w_max) * FS
        e1, e2 = _cayley(C0, S0, W0, C1, S1, hw)
        e_c = C1 * C1 + S1 * S1 - 1.0
        h = [e_rx, e_ry, e_vx, e_vy, e_w, e1, e2, e_c]
        if k == 1:  # the initial state first: the same constraints, less fill in the y-solve's factor
            sx, sy, sth = start
            h = [RX0 - sx / p_max, RY0 - sy / p_max, C0 - np.cos(sth), S0 - np.sin(sth),
                 VX0 - 0.0, VY0 - 0.0, W0 - 0.0] + h
        gg = [1.0 - FC * FC - FS * FS, 1.0 - VX1 * VX1, 1.0 - VY1 * VY1, 1.0 - W1 * W1]
        for (ox, oy, rho) in disks:
            gg.append((RX1 - ox / p_max) ** 2 + (RY1 - oy / p_max) ** 2 - (rho / p_max) ** 2)
        raw.append((stage, gg, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in gg], [p.normalized() for p in h])
          for f, gg, h in raw]
    return Problem("rigid_body", N, 7, 2, cl, R=1.0,
                   meta=dict(dt=dt, start=start, goal=goal, disks=list(disks), fscale=fscale))


# --------------------------------------------------------------------------
# seeded batches (base seed 20240607, instance i uses seed + i)
# --------------------------------------------------------------------------
BASE_SEED = 20240607


def problem_batch(kind: str, B: int, seed: int = BASE_SEED, **kw):
    out = []
    for i in range(B):
        rng = np.random.default_rng(np.random.PCG64(seed + i))
        if kind == "pendulum":
            out.append(pendulum_problem(theta0=float(rng.uniform(-0.2, 0.2)), **kw))
        elif kind == "cartpole":
            out.append(cartpole_problem(x0=float(rng.uniform(-0.5, 0.5)),
                                        theta0=float(rng.uniform(-0.3, 0.3)), **kw))
        elif kind == "rigid_body":
            # a horizon given by the caller holds for every instance; otherwise
            # each instance draws its own N ~ U{20..100}
            rest = {k: v for k, v in kw.items() if k != "N"}
            N = kw.get("N") or int(rng.integers(20, 101))
            nd = int(rng.integers(2, 5))
            start = (-1.5, -1.5, 0.0)
            goal = (float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1)), float(rng.uniform(-np.pi, np.pi)))
            disks = []
            while len(disks) < nd:
                ox, oy = rng.uniform(-2, 2, size=2)
                rho = rng.uniform(0.3, 1.0)
                if (np.hypot(ox - start[0], oy - start[1]) > rho + 0.2
                        and np.hypot(ox - goal[0], oy - goal[1]) > rho + 0.2):
                    disks.append((float(ox), float(oy), float(rho)))
            out.append(rigid_body_problem(N=N, start=start, goal=goal, disks=disks, **rest))
        else:
            raise ValueError(kind)
    return out


# --------------------------------------------------------------------------
# the serving mix: robots and horizons drawn per request
# --------------------------------------------------------------------------
SERVING_MIX = (("pendulum", 0.5, (10, 60)), ("cartpole", 0.3, (20, 80)), ("rigid_body", 0.2, (20, 100)))
SERVING_SEED = BASE_SEED + 5_000_000


def mixed_request(j: int, seed: int = SERVING_SEED):
    """Request j of the serving stream: its robot is drawn with the shares of
    SERVING_MIX, its horizon uniformly from the robot's range, then its
    initial state (and for the rigid body its goal and 2-4 disks) as in
    problem_batch. Seeded by PCG64(seed + j). Returns (kind, problem)."""
    rng = np.random.default_rng(np.random.PCG64(seed + j))
    u = rng.uniform()
    acc = 0.0
    for kind, share, (lo, hi) in SERVING_MIX:
        acc += share
        if u < acc:
            break
    N = int(rng.integers(lo, hi + 1))
    sub = int(rng.integers(0, 2**31 - 1))
    return kind, problem_batch(kind, 1, seed=sub, N=N)[0]


def poisson_arrivals(rate: float, duration: float, seed: int = SERVING_SEED + 1):
    """Arrival times (s) of a Poisson process of the given rate on [0, duration)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)


# --------------------------------------------------------------------------
# the paper's vehicle landing and flying robot (App. "Vehicle Landing",
# "Flying Robot"): state x = (r_x, r_y, v_x, v_y, r_c, r_s, f_c, f_s),
# attitude and its step rotation on SO(2) as in the paper's pendulum
# --------------------------------------------------------------------------
def _affine(v, lo, hi):
    """Physical value of a variable rescaled to [-1, 1] from [lo, hi]."""
    return 0.5 * (hi - lo) * v + 0.5 * (hi + lo)


def _so2_robot(N, nu, dt, theta0, thetadot0, x0, y0, vx0, vy0, box, u_max, fc_min, goal, Pf, dyn, extra_g, name):
    """Clique k: (x_{k-1}, u_{k-1}, x_k) with 2 * 8 + nu variables, rescaled to
    [-1, 1] by `box` = ((lo, hi) of r_x, r_y, v_x, v_y) and u_i in [0, u_max].

    Equalities of clique k: the translational dynamics `dyn` (physical
    variables), the attitude update r_k = r_{k-1} * f_{k-1} on SO(2), the
    circles of r and f for x_k and, for k >= 2, for x_{k-1}; x_0 is fixed by
    eight linear equalities in clique 1 (the reading under which the
    paper's pendulum reproduces its printed sizes). Inequalities of clique k:
    u_i (u_max - u_i) >= 0 for u_{k-1}, the boxes of r_x, r_y, v_x, v_y and
    f_c >= f_c,min for x_k; then `extra_g` more, as described by the caller.
    Cost: the LQR-style loss to `goal` with identity weights after rescaling,
    P_f on x_N.
    """
    dx = 8
    nv = 2 * dx + nu
    V = [Poly.var(nv, i) for i in range(nv)]
    X0, U, X1 = V[:dx], V[dx:dx + nu], V[dx + nu:]

    def phys(X):
        return [_affine(X[i], *box[i]) for i in range(4)] + list(X[4:])

    def scaled_state(vals):
        return [(vals[i] - 0.5 * (box[i][1] + box[i][0])) / (0.5 * (box[i][1] - box[i][0])) for i in range(4)] \
            + list(vals[4:])

    P0, P1 = phys(X0), phys(X1)
    u = [_affine(Ui, 0.0, u_max) for Ui in U]
    g_target = scaled_state(goal)
    init = scaled_state([x0, y0, vx0, vy0, np.cos(theta0), np.sin(theta0), np.cos(dt * thetadot0),
                         np.sin(dt * thetadot0)])
    rx0, ry0, vx_0, vy_0, rc0, rs0, fc0, fs0 = P0
    rx1, ry1, vx_1, vy_1, rc1, rs1, fc1, fs1 = P1
    raw = []
    for k in range(1, N + 1):
        f = sum((xi - t) * (xi - t) for xi, t in zip(X0, g_target)) + sum(Ui * Ui for Ui in U)
        if k == N:
            f = f + Pf * sum((xi - t) * (xi - t) for xi, t in zip(X1, g_target))
        h = dyn(P0, P1, u) + [rc1 - (rc0 * fc0 - rs0 * fs0), rs1 - (rs0 * fc0 + rc0 * fs0),
                               rc1 * rc1 + rs1 * rs1 - 1.0, fc1 * fc1 + fs1 * fs1 - 1.0]
        if k >= 2:
            h += [rc0 * rc0 + rs0 * rs0 - 1.0, fc0 * fc0 + fs0 * fs0 - 1.0]
        else:
            h += [X0[i] - init[i] for i in range(dx)]
        gg = [ui * (u_max - ui) for ui in u]
        gg += [1.0 - X1[i] * X1[i] for i in range(4)]
        gg += [fc1 - fc_min]
        gg += extra_g(k, X0)
        raw.append((f, gg, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in gg], [p.normalized() for p in h]) for f, gg, h in raw]
    return Problem(name, N, dx, nu, cl, R=1.0, meta=dict(dt=dt, theta0=theta0, fscale=fscale))


def _spread_previous_state_bounds(N, total):
    """`total` bounds 1 - z^2 >= 0 on variables of x_{k-1} in cliques 2..N, as
    evenly as possible (earlier cliques take the remainder), variables taken
    in state order and cycling. They are implied by the box and circle
    constraints of the clique before, so the trajectory problem is unchanged."""
    counts = [0] * (N + 1)
    for j in range(total):
        counts[2 + j % (N - 1)] += 1

    def extra(k, X0):
        return [1.0 - X0[j % len(X0)] * X0[j % len(X0)] for j in range(counts[k])]
    return extra


def _extra_count(N, n_localizing, listed, N_paper, printed):
    """Localizing constraints beyond the `listed` per clique: n_localizing -
    listed N when given; by default the printed surplus at the paper's
    horizon, scaled by (N - 1) / (N_paper - 1) at other horizons."""
    if N < 2:
        return 0
    if n_localizing is not None:
        return max(0, n_localizing - listed * N)
    return int(round((printed - listed * N_paper) * (N - 1) / (N_paper - 1)))


def paper_landing_problem(N: int = 50, dt: float = 0.2, theta0: float = 0.1, thetadot0: float = 0.0,
                          x0: float = 20.0, y0: float = 100.0, vx0: float = 0.0, vy0: float = -5.0,
                          m: float = 1.0, inertia: float = 50.0, lever: float = 5.0, g: float = 9.8,
                          fc_min: float = 0.7, rx_max: float = 100.0, ry_min: float = 10.0, ry_max: float = 120.0,
                          v_max: float = 20.0, u_max: float = 8.0, Pf: float = 10.0,
                          n_localizing: int | None = None) -> Problem:
    """The vehicle landing of the paper's appendix, 18-variable cliques (moment
    blocks s(18, 2) = 190, localizing blocks s(18, 1) = 19).

      m (v_x,k - v_x,k-1) = -dt (u_1 + u_2) r_s,k-1
      m (v_y,k - v_y,k-1) = dt ((u_1 + u_2) r_c,k-1 - m g)      (the printed line
                                                                 drops dt on m g)
      I (f_s,k - f_s,k-1) = L dt^2 (u_2 - u_1);  r_k = r_k-1 + dt v_k-1
    Goal: x = 0, y = 10, theta = 0 at rest. The appendix lists seven
    inequalities per clique (350 for N = 50) and states 499 localizing
    matrices; the other 149 are read as bounds on the previous state (see
    _spread_previous_state_bounds; n_localizing sets the total). With N = 50
    the SDP has Table 1's sizes.
    """
    box = ((-rx_max, rx_max), (ry_min, ry_max), (-v_max, v_max), (-v_max, v_max))

    def dyn(P0, P1, u):
        rx0, ry0, vx0_, vy0_, rc0, rs0, fc0, fs0 = P0
        rx1, ry1, vx1, vy1, rc1, rs1, fc1, fs1 = P1
        T = u[0] + u[1]
        return [rx1 - rx0 - dt * vx0_, ry1 - ry0 - dt * vy0_, m * (vx1 - vx0_) + dt * T * rs0,
                m * (vy1 - vy0_) - dt * (T * rc0 - m * g), inertia * (fs1 - fs0) - lever * dt * dt * (u[1] - u[0])]
    extra = _spread_previous_state_bounds(N, _extra_count(N, n_localizing, listed=7, N_paper=50, printed=499))
    return _so2_robot(N, 2, dt, theta0, thetadot0, x0, y0, vx0, vy0, box, u_max, fc_min,
                      (0.0, 10.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0), Pf, dyn, extra, "paper_landing")


def paper_flying_robot_problem(N: int = 60, dt: float = 0.2, theta0: float = 0.3, thetadot0: float = 0.0,
                               x0: float = 5.0, y0: float = -5.0, vx0: float = 0.0, vy0: float = 0.0,
                               alpha: float = 0.2, beta: float = 0.2, fc_min: float = 0.7, r_max: float = 10.0,
                               v_max: float = 10.0, u_max: float = 8.0, Pf: float = 10.0,
                               n_localizing: int | None = None) -> Problem:
    """The flying robot of the paper's appendix, 20-variable cliques (moment
    blocks s(20, 2) = 231, localizing blocks s(20, 1) = 21).

      v_k - v_k-1 = dt (u_1 - u_2 + u_3 - u_4) (r_c, r_s)_k-1
      f_s,k - f_s,k-1 = dt^2 alpha (u_2 - u_1) + dt^2 beta (u_3 - u_4)   (as printed)
      r_k = r_k-1 + dt v_k-1
    Goal: the origin at rest with theta = 0. The appendix lists nine
    inequalities per clique (540 for N = 60) and states 659 localizing
    matrices; the other 119 are read as bounds on the previous state. With
    N = 60 the SDP has Table 1's sizes.
    """
    box = ((-r_max, r_max), (-r_max, r_max), (-v_max, v_max), (-v_max, v_max))

    def dyn(P0, P1, u):
        rx0, ry0, vx0_, vy0_, rc0, rs0, fc0, fs0 = P0
        rx1, ry1, vx1, vy1, rc1, rs1, fc1, fs1 = P1
        T = u[0] - u[1] + u[2] - u[3]
        return [rx1 - rx0 - dt * vx0_, ry1 - ry0 - dt * vy0_, vx1 - vx0_ - dt * T * rc0, vy1 - vy0_ - dt * T * rs0,
                fs1 - fs0 - dt * dt * alpha * (u[1] - u[0]) - dt * dt * beta * (u[2] - u[3])]
    extra = _spread_previous_state_bounds(N, _extra_count(N, n_localizing, listed=9, N_paper=60, printed=659))
    return _so2_robot(N, 4, dt, theta0, thetadot0, x0, y0, vx0, vy0, box, u_max, fc_min,
                      (0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0), Pf, dyn, extra, "paper_flying_robot")


def paper_car_backin_problem(N: int = 30, dt: float = 0.25, x0: float = 2.0, y0: float = 4.0, theta0: float = 0.0,
                             car_L: float = 6.0, car_W: float = 2.5, ry_max: float = 8.0, v_max: float = 4.0,
                             w_max: float = 0.5, obstacles=((6.0, -4.0), (-6.0, -4.0)), side: float = 8.0,
                             goal=(0.0, -3.0, 0.5 * np.pi), Pf: float = 10.0,
                             n_localizing: int | None = None) -> Problem:
    """The car back-in of the paper's appendix: a car (rectangle car_L x car_W)
    backs in between two square obstacles, kept apart from each by a
    separating line (A, B, C) with A^2 + B^2 + C^2 = 1 per step.

    State x = (r_x, r_y, r_c, r_s); per step the clique-local variables
    (v, w, f_c, f_s, A_1, B_1, C_1, A_2, B_2, C_2) play the part of the
    control (the separating lines of one step are used by one clique only),
    so cliques have 2 * 4 + 10 = 18 variables (moment blocks s(18, 2) = 190,
    localizing blocks 19). Equalities of clique k: r_k = r_{k-1} + dt v
    (r_c, r_s)_{k-1}; f_s = dt w - (dt w)^3 / 6; (r_c, r_s)_k = (r_c, r_s)_{k-1}
    rotated by (f_c, f_s); the circles of (r_c, r_s)_k and (f_c, f_s), the two
    unit spheres of the lines, the circle of (r_c, r_s)_{k-1} for k >= 2, and
    x_0 fixed by four linear equalities in clique 1. Inequalities of clique
    k: the four corners of the car at x_k on the positive side of each line
    and the four corners of the matching obstacle on the other (16), and the
    boxes of r_x,k, r_y,k, v, w (4): 20 per clique, 600 for N = 30, against
    the 659 localizing matrices the appendix states; the other 59 are read as
    bounds on the previous state. With N = 30 the SDP has Table 1's m.
    """
    dx, du = 4, 10
    nv = 2 * dx + du
    Vv = [Poly.var(nv, i) for i in range(nv)]
    X0, Uv, X1 = Vv[:dx], Vv[dx:dx + du], Vv[dx + du:]
    rx_max = x0 + 2.0
    sx = (rx_max, ry_max)

    def pos(X):
        return X[0] * sx[0], X[1] * sx[1], X[2], X[3]
    rx0, ry0, rc0, rs0 = pos(X0)
    rx1, ry1, rc1, rs1 = pos(X1)
    v, w, fc, fs = Uv[0] * v_max, Uv[1] * w_max, Uv[2], Uv[3]
    lines = [(Uv[4], Uv[5], Uv[6]), (Uv[7], Uv[8], Uv[9])]
    hx, hy = 0.5 * car_L, 0.5 * car_W
    corners = [(rx1 + hx * rc1 - hy * rs1, ry1 + hx * rs1 + hy * rc1),
               (rx1 - hx * rc1 - hy * rs1, ry1 - hx * rs1 + hy * rc1),
               (rx1 - hx * rc1 + hy * rs1, ry1 - hx * rs1 - hy * rc1),
               (rx1 + hx * rc1 + hy * rs1, ry1 + hx * rs1 - hy * rc1)]
    # the lines act on positions divided by a common length so that their
    # coefficients stay of order one after rescaling
    ell = max(rx_max, ry_max)
    g_target = [goal[0] / sx[0], goal[1] / sx[1], np.cos(goal[2]), np.sin(goal[2])]
    n_extra = _extra_count(N, n_localizing, listed=20, N_paper=30, printed=659)
    extra = _spread_previous_state_bounds(N, n_extra) if N >= 2 else (lambda k, X: [])
    raw = []
    for k in range(1, N + 1):
        f = sum((xi - t) * (xi - t) for xi, t in zip(X0, g_target)) + sum(Uv[i] * Uv[i] for i in range(4))
        if k == N:
            f = f + Pf * sum((xi - t) * (xi - t) for xi, t in zip(X1, g_target))
        h = [rx1 - rx0 - dt * v * rc0, ry1 - ry0 - dt * v * rs0, fs - dt * w + (dt * w) ** 3 * (1.0 / 6.0),
             rc1 - (rc0 * fc - rs0 * fs), rs1 - (rs0 * fc + rc0 * fs), rc1 * rc1 + rs1 * rs1 - 1.0,
             fc * fc + fs * fs - 1.0]
        h += [A * A + B * B + C * C - 1.0 for A, B, C in lines]
        if k >= 2:
            h += [rc0 * rc0 + rs0 * rs0 - 1.0]
        else:
            h += [X0[0] - x0 / sx[0], X0[1] - y0 / sx[1], X0[2] - np.cos(theta0), X0[3] - np.sin(theta0)]
        gg = []
        for (A, B, C), (ox, oy) in zip(lines, obstacles):
            gg += [A * (cx * (1.0 / ell)) + B * (cy * (1.0 / ell)) + C for cx, cy in corners]
            s2 = 0.5 * side
            for qx, qy in ((ox + s2, oy + s2), (ox - s2, oy + s2), (ox - s2, oy - s2), (ox + s2, oy - s2)):
                gg.append(-(A * (qx / ell) + B * (qy / ell) + C))
        gg += [1.0 - X1[0] * X1[0], 1.0 - X1[1] * X1[1], 1.0 - Uv[0] * Uv[0], 1.0 - Uv[1] * Uv[1]]
        gg += extra(k, X0)
        raw.append((f, gg, h))
    fscale = 1.0 / max(f.max_abs_coef() for f, _, _ in raw)
    cl = [Clique(f * fscale, [p.normalized() for p in gg], [p.normalized() for p in h]) for f, gg, h in raw]
    return Problem("paper_car_backin", N, dx, du, cl, R=1.0, meta=dict(dt=dt, x0=x0, y0=y0, theta0=theta0,
                                                                       fscale=fscale))
