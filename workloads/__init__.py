"""Seeded synthetic inputs shared by the oracle, the GPU tests and the bench.

This module holds numbers only: random draws and the sizes/parameters of the
five workloads.  It contains none of the method's arithmetic (no stepping, no
interpolation, no composition), so the oracle and the CUDA path can both take
their inputs from here without sharing any of the computation they check.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out from its published
definition: the state advances by the golden-ratio increment 0x9E3779B97F4A7C15
and each output is the state passed through two xor-shift-multiply rounds and a
final xor-shift.  Uniform doubles take the top 53 bits; normals use the
Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream started at `seed`.

    Output i is mix(seed + (i + 1) * golden), so any slice of the stream can be
    produced independently (the generator is counter based).
    """
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential draws from one SplitMix64 stream (uniform, integer, normal)."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def _raw(self, count: int) -> np.ndarray:
        z = splitmix64(self.seed, count, self.pos)
        self.pos += count
        return z

    def uniform(self, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self._raw(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def integers(self, count: int, lo: int, hi_inclusive: int) -> np.ndarray:
        u = self.uniform(count)
        span = hi_inclusive - lo + 1
        return (lo + np.floor(u * span)).astype(np.int64)

    def normal(self, count: int) -> np.ndarray:
        u1 = self.uniform(count)
        u2 = self.uniform(count)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# Workload definitions.  Sizes follow the five benchmark configurations; the
# docstrings state the readings taken where a configuration leaves a point open.
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    rhs: str                 # rhs family name (see oracle / include/nvpit.h)
    dim: int
    t0: float
    T: float
    S: int
    scheme: str              # "euler" | "rk4"
    dt: float
    steps_per_slice: int     # 0 => ceil(H/dt)
    map_kind: str            # "pl1d" | "bilinear2d" | "affine" | "pairs"
    per_dim: int = 0
    lo: tuple = ()
    hi: tuple = ()
    params: tuple = ()
    y0: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def scalar_cos_cubic(S: int = 16, M: int = 64, steps: int = 10_000) -> Workload:
    """y' = cos(t) y - y^3 on [0,10], y(0)=0.5, forward Euler, PL tables on [-2,2]."""
    return Workload("scalar_cos_cubic_fe_pl", "cos_cubic", 1, 0.0, 10.0, S, "euler", 0.0, steps,
                    "pl1d", per_dim=M, lo=(-2.0,), hi=(2.0,), y0=np.array([0.5]))


def heat1d(n: int = 256, S: int = 1024, T: float = 0.1, dt: float = 1e-5, seed: int = 0) -> Workload:
    """u_t = u_xx + sin(pi x) cos t, Dirichlet-0, n interior points, RK4, affine maps.

    u0 = sin(pi x) + 0.1 N(0,1), x_i = i/(n+1).
    """
    x = np.arange(1, n + 1, dtype=np.float64) / (n + 1)
    u0 = np.sin(np.pi * x) + 0.1 * Stream(seed).normal(n)
    return Workload(f"heat1d_n{n}_S{S}_rk4_affine", "heat1d", n, 0.0, T, S, "rk4", dt, 0,
                    "affine", params=(1.0, 1.0), y0=u0)


def advdiff2d(nx: int = 64, S: int = 512, T: float = 1.0, dt: float = 2e-4, seed: int = 1) -> Workload:
    """u_t = 0.01 lap(u) - (1, 0.5).grad(u) on an nx x nx periodic grid, RK4, affine maps.

    u0 = exp(-r^2 / (2 * 0.1^2)) centred at (0.5, 0.5) plus N(0, 0.01^2) noise;
    grid points x_i = i/nx, flattened index iy * nx + ix.
    """
    g = np.arange(nx, dtype=np.float64) / nx
    X, Y = np.meshgrid(g, g, indexing="xy")           # Y[iy, ix], X[iy, ix]
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    u0 = (np.exp(-r2 / (2 * 0.1 ** 2)) + 0.01 * Stream(seed).normal(nx * nx).reshape(nx, nx)).ravel()
    return Workload(f"advdiff2d_{nx}x{nx}_S{S}_rk4_affine", "advdiff2d", nx * nx, 0.0, T, S, "rk4",
                    dt, 0, "affine", params=(0.01, 1.0, 0.5, float(nx)), y0=u0)


@dataclass
class VdpBatch:
    mu: np.ndarray       # (B,)
    T: np.ndarray        # (B,)
    S: np.ndarray        # (B,) int
    y0: np.ndarray       # (B, 2)
    dt: float = 1e-3
    per_dim: int = 32
    lo: float = -3.0
    hi: float = 3.0


def vdp_batch(B: int = 4096, seed: int = 2, s_lo: int = 8, s_hi: int = 256,
              t_lo: float = 5.0, t_hi: float = 20.0) -> VdpBatch:
    """Independent Van der Pol instances: mu ~ U[0.1,2], T ~ U[t_lo,t_hi], S ~ U{s_lo..s_hi},
    y0 ~ U[-2,2]^2, all drawn in that order from one stream."""
    st = Stream(seed)
    mu = st.uniform(B, 0.1, 2.0)
    T = st.uniform(B, t_lo, t_hi)
    S = st.integers(B, s_lo, s_hi)
    y0 = st.uniform(2 * B, -2.0, 2.0).reshape(B, 2)
    return VdpBatch(mu, T, S, y0)


def chain3(S: int = 128, M: int = 65536, T: float = 20.0, dt: float = 1e-3, seed: int = 3) -> Workload:
    """3 unit masses, wall-m1-m2-m3-wall, springs k=1 plus 0.5 d^3, damping 0.05."""
    return Workload(f"chain3_S{S}_M{M}_rk4", "chain3", 6, 0.0, T, S, "rk4", dt, 0, "pairs",
                    per_dim=M, lo=(-1.0,) * 6, hi=(1.0,) * 6, params=(1.0, 0.5, 0.05),
                    y0=np.array([0.3, -0.2, 0.1, 0.0, 0.0, 0.0]), extra={"seed": seed})


def chain3_samples(seed: int, S: int, M: int, slice_index: int) -> np.ndarray:
    """Sample points of one slice, U[-1,1]^6, shape (6, M).

    Point k of slice j, component c is output ((j*M + k)*6 + c) of the SplitMix64
    stream with this seed; a GPU kernel can regenerate any of them by index.
    """
    z = splitmix64(seed, M * 6, slice_index * M * 6)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (-1.0 + 2.0 * u).reshape(M, 6).T.copy()


def wave1d(M: int = 80, S: int = 512, T: float = 20.0) -> Workload:
    """u_tt = u_xx on [-1, 1], Dirichlet, Chebyshev points x_i = cos(i pi/M),
    leapfrog dt = 8/M^2 (Section 5, Table wave80 for M = 80, T = 20; Table
    wave40 for M = 40, T = 16).  State (u^n, u^{n-1}) of dimension 2(M-1); the
    initial state depends on the planned step h: see wave1d_initial."""
    return Workload(f"wave_cheb{M}_S{S}_leapfrog", "wave", 2 * (M - 1), 0.0, T, S, "leapfrog",
                    8.0 / (M * M), 0, "affine", params=(float(M),))


def wave1d_initial(M: int, h: float, width: float = 200.0) -> np.ndarray:
    """(u(x, 0), u(x, -h)) at the interior Chebyshev points for the single
    left-moving peak u(x, t) = exp(-width (x + t)^2)."""
    x = np.cos(np.pi * np.arange(1, M) / M)
    return np.concatenate([np.exp(-width * x ** 2), np.exp(-width * (x - h) ** 2)])


def square_paper(dt_exp: int = 14, S: int = 32, M: int = 4) -> Workload:
    """y' = y^2 on [0, 1/2], the scalar model problem of Section 3 (Table 3 sweep shape)."""
    return Workload(f"square_dt2^-{dt_exp}_N{S}_M{M}", "square", 1, 0.0, 0.5, S, "euler",
                    2.0 ** -dt_exp, 0, "pl1d", per_dim=M, lo=(0.0,), hi=(2.0,), y0=np.array([1.0]))
