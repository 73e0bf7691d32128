"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds particle lattices, wall layers, buffer boxes and
parameter sets.  It holds none of the method's arithmetic (no kernel, no
equation of state, no sweep), so both the CUDA path and the CPU oracle can
be fed from it.  Every random number is drawn here from numpy's PCG64 with an
explicit seed; random numbers the method itself draws during a step (inlet
fluctuation) come from Philox4x32-10 inside each implementation.

Shapes follow the paper's cases (Sec. 4): straight channel (4.1), U-shaped
channel (4.2), plane jet with bidirectional buffers on the open sides (4.3)
and a rotating-wall mixer (4.4).  The paper's own geometries exist only in
figures and its comparison data are not available, so these are stand-ins
with the same structure: lattice spacing dp, h = 1.3 dp (Sec. 2.2), four
wall-dummy layers, buffers of length 4 dp.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

H_FAC = 1.3  # h = 1.3 dp, Sec. 2.2
WALL_LAYERS = 4
C_MU = 0.09  # App. A; used only to size the inlet dissipation rate


@dataclass
class BufferSpec:
    """One bidirectional buffer (Sec. 2.4.1): an aligned box in its own frame.

    frame rows are (n_b, t1, t2): n_b points from the open face into the
    domain; the box is 0 <= x'_0 < length, |x'_1| <= half[0], |x'_2| <= half[1].
    """

    kind: str  # "velocity" | "pressure"
    origin: Sequence[float]
    frame: np.ndarray  # (3, 3) orthonormal rows
    length: float
    half: Sequence[float]
    p_ob: float = 0.0
    theta: Sequence[float] = (0.0,)
    noise: float = 0.0
    turb: str = "zero_gradient"  # | "freestream"
    k_in: float = 0.0
    eps_in: float = 0.0


@dataclass
class Case:
    name: str
    dim: int
    dp: float
    h: float
    rho0: float
    c0: float
    nu_l: float
    rans: bool
    U_ref: float
    lo: np.ndarray
    hi: np.ndarray
    periodic: Sequence[int]
    pos: np.ndarray  # (n, 3)
    vel: np.ndarray  # (n, 3)
    rho: np.ndarray
    mass: np.ndarray
    k: np.ndarray
    eps: np.ndarray
    wpos: np.ndarray  # (nw, 3)
    wvel: np.ndarray  # (nw, 3)
    buffers: List[BufferSpec] = field(default_factory=list)
    eta: float = 3.0
    g: Sequence[float] = (0.0, 0.0, 0.0)
    dt_mode: str = "dual"  # | "single" | "fixed"
    dt_ad_fixed: float = 0.0
    n_ac_fixed: int = 1
    seed: int = 0
    capacity: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nw(self) -> int:
        return int(self.wpos.shape[0])

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------
def frame_2d(normal) -> np.ndarray:
    n = np.asarray(normal, dtype=np.float64)[:2]
    n = n / np.linalg.norm(n)
    return np.array([[n[0], n[1], 0.0], [-n[1], n[0], 0.0], [0.0, 0.0, 1.0]])


def frame_3d(normal, t1) -> np.ndarray:
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    t = np.asarray(t1, dtype=np.float64)
    t = t - n * np.dot(n, t)
    t = t / np.linalg.norm(t)
    t2 = np.cross(n, t)
    return np.array([n, t, t2])


def lattice(counts, dp, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Cell-centred lattice: (i + 1/2) dp along each axis, z = 0 in 2D."""
    counts = list(counts)
    axes = [np.arange(c, dtype=np.float64) + 0.5 for c in counts]
    grids = np.meshgrid(*axes, indexing="ij")
    out = np.zeros((grids[0].size, 3))
    for a, gr in enumerate(grids):
        out[:, a] = origin[a] + gr.reshape(-1) * dp
    return out


def jitter(pos: np.ndarray, dim: int, amp: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = pos.copy()
    out[:, :dim] += rng.uniform(-amp, amp, size=(pos.shape[0], dim))
    return out


def _fluid_arrays(pos, dim, dp, rho0, vel=None, k=0.0, eps=0.0):
    n = pos.shape[0]
    v = np.zeros((n, 3)) if vel is None else np.asarray(vel, dtype=np.float64).copy()
    return dict(
        pos=np.ascontiguousarray(pos, dtype=np.float64),
        vel=v,
        rho=np.full(n, rho0),
        mass=np.full(n, rho0 * dp**dim),
        k=np.full(n, float(k)),
        eps=np.full(n, float(eps)),
    )


def _channel_walls(x0, x1, height, dp, layers=WALL_LAYERS):
    """Wall dummies below y = 0 and above y = height, columns spanning [x0, x1)."""
    nx = int(round((x1 - x0) / dp))
    xs = x0 + (np.arange(nx) + 0.5) * dp
    rows = []
    for l in range(layers):
        yb = -(l + 0.5) * dp
        yt = height + (l + 0.5) * dp
        rows.append(np.stack([xs, np.full(nx, yb), np.zeros(nx)], 1))
        rows.append(np.stack([xs, np.full(nx, yt), np.zeros(nx)], 1))
    return np.concatenate(rows, 0)


def inlet_turbulence(U: float, height: float, intensity: float = 0.05, mix_frac: float = 0.07):
    """Freestream k, eps for an inlet: k = 1.5 (I U)^2, eps = C_mu^(3/4) k^(3/2) / l,
    l = mix_frac * height (the usual inlet estimate; not given in the paper)."""
    k = 1.5 * (intensity * U) ** 2
    eps = C_MU**0.75 * k**1.5 / (mix_frac * height)
    return k, eps


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def poiseuille_channel(length=2.0, height=1.0, dp=0.05, p_in=0.2, p_out=0.1, nu=0.02,
                       rho0=1.0, jitter_frac=0.01, seed=1, buffer_cells=4,
                       capacity_factor=1.5) -> Case:
    """Laminar pressure-driven channel (Sec. 4.1 shape): pressure buffers at both
    ends, 4 wall layers top and bottom extending 4 dp beyond both open faces.

    U_max = G H^2 / (8 rho0 nu), G = (p_in - p_out) / length; c0 = 10 U_max.
    The pressure drop is 0.1 on a background of 0.1 (outlet 0.1, inlet 0.2,
    the pressures of the paper's laminar channel): without the transport-
    velocity correction a zero-pressure outlet is tensile-unstable.  The
    initial state is at rest with the density of the mean pressure.
    """
    nx, ny = int(round(length / dp)), int(round(height / dp))
    pos = jitter(lattice((nx, ny), dp), 2, jitter_frac * dp, seed)
    G = (p_in - p_out) / length
    umax = G * height**2 / (8.0 * rho0 * nu)
    c0 = 10.0 * umax
    h = H_FAC * dp
    wpos = _channel_walls(-WALL_LAYERS * dp, length + WALL_LAYERS * dp, height, dp)
    Lb = buffer_cells * dp
    bufs = [
        BufferSpec("pressure", (0.0, 0.5 * height, 0.0), frame_2d((1, 0)), Lb, (0.5 * height, 0.0),
                   p_ob=p_in),
        BufferSpec("pressure", (length, 0.5 * height, 0.0), frame_2d((-1, 0)), Lb,
                   (0.5 * height, 0.0), p_ob=p_out),
    ]
    margin = WALL_LAYERS * dp + 2 * h
    arr = _fluid_arrays(pos, 2, dp, rho0)
    arr["rho"][:] = rho0 * (1.0 + 0.5 * (p_in + p_out) / (rho0 * c0 * c0))
    return Case(name=f"poiseuille_2d_dp{dp:g}", dim=2, dp=dp, h=h, rho0=rho0, c0=c0, nu_l=nu,
                rans=False, U_ref=umax,
                lo=np.array([-margin, -margin, 0.0]), hi=np.array([length + margin, height + margin, 0.0]),
                periodic=(0, 0, 0), wpos=wpos, wvel=np.zeros_like(wpos), buffers=bufs,
                seed=seed, capacity=int(capacity_factor * pos.shape[0]) + 64, **arr)


def turbulent_channel(length=6.0, height=2.0, dp=0.005, U=1.0, Re=1.0e4, c0=10.0, rho0=1.0,
                      noise=0.05, seed=2, buffer_cells=4, jitter_frac=0.0,
                      capacity_factor=1.25) -> Case:
    """Turbulent straight channel with k-epsilon RANS (Sec. 4.1 turbulent shape):
    velocity inlet buffer (uniform U, seeded relative fluctuation `noise`,
    freestream k, eps) and a zero-pressure outlet buffer (zero-gradient k, eps).
    nu = U H / Re.  Initial state: uniform U, freestream k and eps.
    """
    nx, ny = int(round(length / dp)), int(round(height / dp))
    pos = lattice((nx, ny), dp)
    if jitter_frac:
        pos = jitter(pos, 2, jitter_frac * dp, seed)
    h = H_FAC * dp
    k_in, eps_in = inlet_turbulence(U, height)
    vel = np.zeros((pos.shape[0], 3))
    vel[:, 0] = U
    wpos = _channel_walls(-WALL_LAYERS * dp, length + WALL_LAYERS * dp, height, dp)
    Lb = buffer_cells * dp
    bufs = [
        BufferSpec("velocity", (0.0, 0.5 * height, 0.0), frame_2d((1, 0)), Lb, (0.5 * height, 0.0),
                   theta=(U,), noise=noise, turb="freestream", k_in=k_in, eps_in=eps_in),
        BufferSpec("pressure", (length, 0.5 * height, 0.0), frame_2d((-1, 0)), Lb,
                   (0.5 * height, 0.0), p_ob=0.0),
    ]
    margin = WALL_LAYERS * dp + 2 * h
    arr = _fluid_arrays(pos, 2, dp, rho0, vel=vel, k=k_in, eps=eps_in)
    return Case(name=f"turbulent_channel_2d_{length:g}x{height:g}_dp{dp:g}", dim=2, dp=dp, h=h,
                rho0=rho0, c0=c0, nu_l=U * height / Re, rans=True, U_ref=U,
                lo=np.array([-margin, -margin, 0.0]), hi=np.array([length + margin, height + margin, 0.0]),
                periodic=(0, 0, 0), wpos=wpos, wvel=np.zeros_like(wpos), buffers=bufs, seed=seed,
                capacity=int(capacity_factor * pos.shape[0]) + 1024, **arr)


def periodic_box(n_per_axis=16, dim=2, dp=0.1, jitter_frac=0.2, vel_amp=0.1, rho_amp=0.01,
                 rho0=1.0, c0=10.0, nu=0.01, rans=False, seed=5) -> Case:
    """Fully periodic box with a jittered lattice and random velocity/density
    (conservation pins; no walls, no buffers)."""
    counts = [n_per_axis] * dim
    pos = jitter(lattice(counts, dp), dim, jitter_frac * dp, seed)
    rng = np.random.default_rng(seed + 1)
    n = pos.shape[0]
    vel = np.zeros((n, 3))
    vel[:, :dim] = rng.uniform(-vel_amp, vel_amp, size=(n, dim))
    arr = _fluid_arrays(pos, dim, dp, rho0, vel=vel)
    arr["rho"] = rho0 * (1.0 + rng.uniform(-rho_amp, rho_amp, size=n))
    if rans:
        arr["k"] = rng.uniform(1e-3, 2e-3, size=n)
        arr["eps"] = rng.uniform(1e-3, 2e-3, size=n)
    L = n_per_axis * dp
    lo = np.zeros(3)
    hi = np.zeros(3)
    hi[:dim] = L
    per = tuple(1 if a < dim else 0 for a in range(3))
    return Case(name=f"periodic_box_{dim}d_{n_per_axis}", dim=dim, dp=dp, h=H_FAC * dp, rho0=rho0,
                c0=c0, nu_l=nu, rans=rans, U_ref=max(vel_amp, 1e-3), lo=lo, hi=hi, periodic=per,
                wpos=np.zeros((0, 3)), wvel=np.zeros((0, 3)), seed=seed, capacity=n + 16, **arr)


def lattice_block(n_per_axis=21, dim=2, dp=0.1, rho0=1.0, c0=10.0, nu=0.01, h_fac=H_FAC,
                  rans=False) -> Case:
    """An isolated perfect lattice (no walls, no periodicity): interior
    particles have full support, the outer rows are truncated."""
    pos = lattice([n_per_axis] * dim, dp)
    h = h_fac * dp
    L = n_per_axis * dp
    lo = np.zeros(3) - 4 * h
    hi = np.zeros(3)
    hi[:dim] = L + 4 * h
    arr = _fluid_arrays(pos, dim, dp, rho0)
    return Case(name=f"lattice_{dim}d_{n_per_axis}", dim=dim, dp=dp, h=h, rho0=rho0, c0=c0, nu_l=nu,
                rans=rans, U_ref=1.0, lo=lo, hi=hi, periodic=(0, 0, 0), wpos=np.zeros((0, 3)),
                wvel=np.zeros((0, 3)), capacity=pos.shape[0] + 16, **arr)
