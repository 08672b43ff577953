"""Plain FP64 statement of Nievergelt's method as Barker describes it.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Slow on purpose:
numpy is used as a vector calculator over independent trajectories (samples or
basis columns), never to fuse or reorder the method's steps.

Array conventions (oracle side only):
  states          (d, K)     d state components, K independent trajectories
  PL table        (S, M)     final value of sample k on slice j
  bilinear table  (S, P, P, 2)  [j, p, q, :] = final state from (xi_p, eta_q)
  affine maps     A (S, n, n), b (S, n)
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Slice grid (Figure "pseudocode", Initialize step; Section 3, eq. localivp)
# ---------------------------------------------------------------------------


def slice_times(t0: float, T: float, S: int) -> np.ndarray:
    """T_j = t0 + j H with H = (T - t0)/S, j = 0..S, each computed directly."""
    H = (T - t0) / S
    return np.array([t0 + j * H for j in range(S + 1)], dtype=np.float64)


def steps_per_slice(t0: float, T: float, S: int, dt: float, fixed: int = 0) -> int:
    """Fine steps per slice.  The paper leaves a non-integer H/dt open; the
    reading that reproduces Table 1 is m = ceil(H/dt) (then h = H/m).  A guard
    of 1e-9 keeps ratios that are integers up to rounding at that integer."""
    if fixed > 0:
        return int(fixed)
    H = (T - t0) / S
    return max(1, int(math.ceil(H / dt - 1e-9)))


def step_size(t0: float, T: float, S: int, m: int) -> float:
    """h = H / m."""
    return ((T - t0) / S) / m


# ---------------------------------------------------------------------------
# Right-hand sides y' = f(t, y) (Figure "pseudocode", Given; eq. lineardiscrete)
# Each returns f(t, Y) for Y of shape (d, K).
# ---------------------------------------------------------------------------


def rhs_linear_scalar(lam: float):
    """y' = lambda y."""
    return lambda t, Y: lam * Y


def rhs_square():
    """y' = y^2, the model problem of Section 3 (eq. scalarmodel)."""
    return lambda t, Y: Y * Y


def rhs_cos_cubic():
    """y' = cos(t) y - y^3."""
    return lambda t, Y: math.cos(t) * Y - Y ** 3


def heat1d_grid(n: int) -> np.ndarray:
    """Interior points x_i = i/(n+1), i = 1..n."""
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def rhs_heat1d(n: int, kappa: float = 1.0, amp: float = 1.0, forcing: bool = True):
    """u_t = kappa u_xx + amp sin(pi x) cos(t), Dirichlet-0, second-order central
    differences on n interior points (eq. lineardiscrete with constant A and
    b(t) = amp sin(pi x) cos t).  With forcing=False this is the homogeneous
    system used for the basis solves (Section 4, before eq. linearreconstruct)."""
    dx = 1.0 / (n + 1)
    x = heat1d_grid(n)
    sx = np.sin(math.pi * x)[:, None]

    def f(t, U):
        P = np.zeros((n + 2, U.shape[1]))
        P[1:-1] = U
        lap = (P[:-2] - 2.0 * P[1:-1] + P[2:]) / (dx * dx)
        out = kappa * lap
        if forcing:
            out = out + amp * math.cos(t) * sx
        return out

    return f


def rhs_heat1d_varcoef(n: int):
    """Variable-coefficient heat equation of Section 5 (eq. heatequation):
    u_t = (1 + sin(t)/4) u_xx + b(t, x) with b chosen so that
    u = cos(t) sin(pi x) solves the continuous problem:
    b = -sin(t) sin(pi x) + (1 + sin(t)/4) pi^2 cos(t) sin(pi x).
    Returns (f_inhomogeneous, f_homogeneous)."""
    dx = 1.0 / (n + 1)
    x = heat1d_grid(n)
    sx = np.sin(math.pi * x)[:, None]

    def lap(U):
        P = np.zeros((n + 2, U.shape[1]))
        P[1:-1] = U
        return (P[:-2] - 2.0 * P[1:-1] + P[2:]) / (dx * dx)

    def f_hom(t, U):
        return (1.0 + 0.25 * math.sin(t)) * lap(U)

    def f_inh(t, U):
        a = 1.0 + 0.25 * math.sin(t)
        b = (-math.sin(t) + a * math.pi ** 2 * math.cos(t)) * sx
        return a * lap(U) + b

    return f_inh, f_hom


def rhs_vdp(mu: float):
    """Van der Pol: x' = y, y' = mu (1 - x^2) y - x."""
    def f(t, Y):
        x, y = Y[0], Y[1]
        return np.stack([y, mu * (1.0 - x * x) * y - x])
    return f


def rhs_chain3(k: float = 1.0, k3: float = 0.5, c: float = 0.05):
    """Three unit masses between two walls: wall-m1-m2-m3-wall.  A spring with
    extension d pulls with tension k d + k3 d^3; each mass has damping -c v.
    State (x1, x2, x3, v1, v2, v3)."""
    def tension(d):
        return k * d + k3 * d ** 3

    def f(t, Y):
        x1, x2, x3, v1, v2, v3 = Y
        t0_, t1_, t2_, t3_ = tension(x1), tension(x2 - x1), tension(x3 - x2), tension(-x3)
        a1 = -t0_ + t1_ - c * v1
        a2 = -t1_ + t2_ - c * v2
        a3 = -t2_ + t3_ - c * v3
        return np.stack([v1, v2, v3, a1, a2, a3])
    return f


def rhs_advdiff2d(nx: int, nu: float = 0.01, ax: float = 1.0, ay: float = 0.5):
    """u_t = nu (5-point Laplacian) - (ax D^-_x u + ay D^-_y u) on an nx x nx
    periodic grid with spacing 1/nx; first-order upwind (backward) differences
    for the positive velocity.  Flattened index iy * nx + ix."""
    dx = 1.0 / nx

    def f(t, U):
        K = U.shape[1]
        G = U.reshape(nx, nx, K)                  # [iy, ix, k]
        xm = np.roll(G, 1, axis=1)                # u[iy, ix-1]
        xp = np.roll(G, -1, axis=1)               # u[iy, ix+1]
        ym = np.roll(G, 1, axis=0)                # u[iy-1, ix]
        yp = np.roll(G, -1, axis=0)               # u[iy+1, ix]
        lap = (xm + xp + ym + yp - 4.0 * G) / (dx * dx)
        dxm = (G - xm) / dx
        dym = (G - ym) / dx
        return (nu * lap - (ax * dxm + ay * dym)).reshape(nx * nx, K)

    return f


# ---------------------------------------------------------------------------
# Fine schemes g_dt (Section 3; forward Euler as in Nievergelt's analysis,
# Section 4; classical RK4)
# ---------------------------------------------------------------------------


def euler_step(f, t, Y, h):
    """y_{i+1} = y_i + h f(t_i, y_i)."""
    return Y + h * f(t, Y)


def rk4_step(f, t, Y, h):
    """Classical fourth-order Runge-Kutta step."""
    k1 = f(t, Y)
    k2 = f(t + h / 2, Y + (h / 2) * k1)
    k3 = f(t + h / 2, Y + (h / 2) * k2)
    k4 = f(t + h, Y + h * k3)
    return Y + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)


STEPPERS = {"euler": euler_step, "rk4": rk4_step}


def integrate(f, scheme: str, t_start: float, Y0: np.ndarray, h: float, m: int) -> np.ndarray:
    """m fine steps from t_start with step times t_start + i h (Figure
    "pseudocode": solve y' = f on one slice from y(T_{j-1}) = xi)."""
    step = STEPPERS[scheme]
    Y = np.array(Y0, dtype=np.float64, copy=True)
    for i in range(m):
        Y = step(f, t_start + i * h, Y, h)
    return Y


def serial_fine(f, scheme: str, t0: float, T: float, S: int, m: int, y0) -> np.ndarray:
    """The serial fine solve over [t0, T] with the same step size and the same
    step times as the slices (slice j, step i at T_{j-1} + i h): the result the
    method approximates (Theorem of Section 4)."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    Y = np.array(y0, dtype=np.float64).reshape(-1, 1)
    for j in range(S):
        Y = integrate(f, scheme, Tj[j], Y, h, m)
    return Y[:, 0]


# ---------------------------------------------------------------------------
# Initial-value samples Xi_h (Section 3; Figure "pseudocode", Given)
# ---------------------------------------------------------------------------


def uniform_nodes(lo: float, hi: float, M: int) -> np.ndarray:
    """M equispaced nodes including both ends: xi_k = lo + k (hi - lo)/(M - 1)."""
    d = (hi - lo) / (M - 1)
    return np.array([lo + k * d for k in range(M)], dtype=np.float64)


# ---------------------------------------------------------------------------
# Computation phase: per-slice maps (Figure "pseudocode"; eqs. lineardiscrete,
# linearreconstruct)
# ---------------------------------------------------------------------------


def build_table_1d(f, scheme, t0, T, S, m, nodes) -> np.ndarray:
    """lambda_j^k = g_dt^j(xi_k) for every slice j and node k: the values of the
    piecewise-linear map phi^j at the nodes.  Returns (S, M)."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    out = np.empty((S, len(nodes)))
    for j in range(S):
        out[j] = integrate(f, scheme, Tj[j], nodes[None, :], h, m)[0]
    return out


def build_table_2d(f, scheme, t0, T, S, m, nodes_x, nodes_y) -> np.ndarray:
    """Final states from every grid point (xi_p, eta_q) on every slice.
    Returns (S, P, Q, 2) with [j, p, q] the state reached from (xi_p, eta_q)."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    P, Q = len(nodes_x), len(nodes_y)
    Xg, Yg = np.meshgrid(nodes_x, nodes_y, indexing="ij")      # [p, q]
    Y0 = np.stack([Xg.ravel(), Yg.ravel()])
    out = np.empty((S, P, Q, 2))
    for j in range(S):
        Yj = integrate(f, scheme, Tj[j], Y0, h, m)
        out[j] = Yj.T.reshape(P, Q, 2)
    return out


def build_affine(f_inh, f_hom, scheme, t0, T, S, m, n):
    """Exact affine slice maps for a linear system (eqs. lineardiscrete,
    linearreconstruct): b_j = g_dt^j(0) with the forcing on, column c of A_j =
    the homogeneous solve from e_c.  Returns A (S, n, n), b (S, n)."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    A = np.empty((S, n, n))
    b = np.empty((S, n))
    for j in range(S):
        b[j] = integrate(f_inh, scheme, Tj[j], np.zeros((n, 1)), h, m)[:, 0]
        A[j] = integrate(f_hom, scheme, Tj[j], np.eye(n), h, m)
    return A, b


def build_affine_slice(f_inh, f_hom, scheme, t0, T, S, m, n, j, columns=None):
    """One slice's map, optionally only some columns of A_j (for sampled checks
    at full size).  Returns (A_cols (n, len(columns)), b_j (n,))."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    cols = np.arange(n) if columns is None else np.asarray(columns)
    E = np.zeros((n, len(cols)))
    E[cols, np.arange(len(cols))] = 1.0
    b = integrate(f_inh, scheme, Tj[j], np.zeros((n, 1)), h, m)[:, 0]
    Ac = integrate(f_hom, scheme, Tj[j], E, h, m)
    return Ac, b


# ---------------------------------------------------------------------------
# Communication phase: phi^j evaluated at lambda_{j-1} (Figure "pseudocode")
# ---------------------------------------------------------------------------


def pl_eval(lo: float, hi: float, values: np.ndarray, lam: float):
    """Piecewise-linear interpolant through (xi_k, values[k]) on M equispaced
    nodes, evaluated at lam.  The segment is floor((lam - lo)/dxi) clamped to
    [0, M-2]; outside [lo, hi] the edge segment's line is extended.
    Returns (value, out_of_range)."""
    M = len(values)
    d = (hi - lo) / (M - 1)
    s = int(math.floor((lam - lo) / d))
    s = min(max(s, 0), M - 2)
    w = (lam - (lo + s * d)) / d
    return (1.0 - w) * values[s] + w * values[s + 1], bool(lam < lo or lam > hi)


def bilinear_eval(lo: float, hi: float, table: np.ndarray, lam):
    """Bilinear interpolant on the P x P grid over [lo, hi]^2 of a 2-D map
    (table[p, q] = state reached from (xi_p, eta_q)), evaluated at lam = (x, y).
    Cell indices clamp to [0, P-2]; outside the square the edge cell's bilinear
    formula is extended.  Returns (value (2,), out_of_range)."""
    P = table.shape[0]
    d = (hi - lo) / (P - 1)
    x, y = float(lam[0]), float(lam[1])
    p = min(max(int(math.floor((x - lo) / d)), 0), P - 2)
    q = min(max(int(math.floor((y - lo) / d)), 0), P - 2)
    wx = (x - (lo + p * d)) / d
    wy = (y - (lo + q * d)) / d
    v = ((1 - wx) * (1 - wy) * table[p, q] + wx * (1 - wy) * table[p + 1, q]
         + (1 - wx) * wy * table[p, q + 1] + wx * wy * table[p + 1, q + 1])
    oob = not (lo <= x <= hi and lo <= y <= hi)
    return v, oob


def compose_tables_1d(lo, hi, table, y0: float):
    """lambda_0 = y0, lambda_j = phi^j(lambda_{j-1}), j = 1..S.
    Returns (lambdas (S+1,), out_of_range count)."""
    lam = [float(y0)]
    oob = 0
    for j in range(table.shape[0]):
        v, o = pl_eval(lo, hi, table[j], lam[-1])
        lam.append(v)
        oob += o
    return np.array(lam), oob


def compose_tables_2d(lo, hi, table, y0):
    """Sequential bilinear composition; returns (lambdas (S+1, 2), oob count)."""
    lam = [np.array(y0, dtype=np.float64)]
    oob = 0
    for j in range(table.shape[0]):
        v, o = bilinear_eval(lo, hi, table[j], lam[-1])
        lam.append(v)
        oob += o
    return np.array(lam), oob


def compose_affine(A, b, y0):
    """lambda_j = A_j lambda_{j-1} + b_j (eq. linearreconstruct applied slice
    after slice).  Returns lambdas (S+1, n)."""
    lam = [np.array(y0, dtype=np.float64)]
    for j in range(A.shape[0]):
        lam.append(A[j] @ lam[-1] + b[j])
    return np.array(lam)


# ---------------------------------------------------------------------------
# Associative form of the composition.  Affine maps compose as
# (A2, b2) o (A1, b1) = (A2 A1, A2 b1 + b2); this is what lets the single
# final reduce of Figure "pseudocode" be evaluated as a scan.
# ---------------------------------------------------------------------------


def affine_combine(second, first):
    """(A2, b2) o (A1, b1): apply `first`, then `second`."""
    A2, b2 = second
    A1, b1 = first
    return A2 @ A1, A2 @ b1 + b2


def affine_prefix_sequential(A, b):
    """Prefix maps P_j = (A_j ... A_1, c_j) with lambda_j = P_j y0 + c_j."""
    n = A.shape[1]
    out = []
    cur = (np.eye(n), np.zeros(n))
    for j in range(A.shape[0]):
        cur = affine_combine((A[j], b[j]), cur)
        out.append(cur)
    return out


def affine_reduce_tree(A, b):
    """Total map of all slices by pairwise (tree) combination, in the order a
    log-depth reduce would use; equal to the sequential product up to rounding."""
    items = [(A[j], b[j]) for j in range(A.shape[0])]
    while len(items) > 1:
        nxt = []
        for i in range(0, len(items) - 1, 2):
            nxt.append(affine_combine(items[i + 1], items[i]))
        if len(items) % 2:
            nxt.append(items[-1])
        items = nxt
    return items[0]


# ---------------------------------------------------------------------------
# FP64 residual refinement of boundary states computed with reduced-precision
# maps: one parareal-style correction (the combination with parareal that the
# Conclusion proposes), the low-precision maps acting as the coarse propagator.
# ---------------------------------------------------------------------------


def refine_affine(f_inh, scheme, t0, T, S, m, lam_tilde, A_tilde):
    """Given approximate boundary states lam_tilde (S+1, n) with lam_tilde[0] =
    y0, and the reduced-precision maps A_tilde used to get them:
      d_j = g_dt^j(lam_tilde_{j-1}) - lam_tilde_j     (FP64 fine solve per slice)
      e_0 = 0, e_j = A_tilde_j e_{j-1} + d_j
      lambda_j = lam_tilde_j + e_j.
    For exact maps this returns the exact composition; the remaining error is
    (A_j - A_tilde_j) applied to the previous error.  Parity partly pinned: no
    paper value exists; the test checks the error contraction."""
    Tj = slice_times(t0, T, S)
    h = step_size(t0, T, S, m)
    lam_tilde = np.asarray(lam_tilde, dtype=np.float64)
    n = lam_tilde.shape[1]
    d = np.empty((S, n))
    for j in range(S):
        g = integrate(f_inh, scheme, Tj[j], lam_tilde[j][:, None], h, m)[:, 0]
        d[j] = g - lam_tilde[j + 1]
    e = np.zeros(n)
    out = [lam_tilde[0].copy()]
    for j in range(S):
        e = A_tilde[j] @ e + d[j]
        out.append(lam_tilde[j + 1] + e)
    return np.array(out)


# ---------------------------------------------------------------------------
# Workload helpers: the right-hand sides and maps for a workloads.Workload
# ---------------------------------------------------------------------------


def workload_rhs(w, forcing: bool = True):
    """f for a workloads.Workload (forcing=False gives the homogeneous part of a
    linear system)."""
    if w.rhs == "cos_cubic":
        return rhs_cos_cubic()
    if w.rhs == "square":
        return rhs_square()
    if w.rhs == "linear_scalar":
        return rhs_linear_scalar(w.params[0])
    if w.rhs == "heat1d":
        kappa, amp = w.params if w.params else (1.0, 1.0)
        return rhs_heat1d(w.dim, kappa, amp, forcing)
    if w.rhs == "heat1d_varcoef":
        fi, fh = rhs_heat1d_varcoef(w.dim)
        return fi if forcing else fh
    if w.rhs == "advdiff2d":
        nu, ax, ay, nx = w.params
        return rhs_advdiff2d(int(nx), nu, ax, ay)
    if w.rhs == "chain3":
        return rhs_chain3(*w.params)
    raise ValueError(w.rhs)


def workload_steps(w) -> int:
    return steps_per_slice(w.t0, w.T, w.S, w.dt, w.steps_per_slice)
