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
    # open-boundary treatment (Sec. 4.1, Table of the four cases): "improved"
    # (case 4, the default), "vipo" (1), "vipo_rkgc" (2), "vipo_rkgc_mirror"
    # (3), or "minimal_mirror" (case 4 with B_i from the truncated support)
    obc: str = "improved"
    tvf: float = 0.0  # transport-velocity shift coefficient alpha (0 = off)
    tvf_pbuf: bool = False  # the shift also moves pressure-buffer particles (across the axis)
    density_sum: bool = False  # density reinitialised by summation every advection step
    wall_function: bool = False  # step-wise wall function at the walls (RANS)

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
                       capacity_factor=1.5, tvf=0.0, tvf_pbuf=False, density_sum=False) -> Case:
    """Laminar pressure-driven channel (Sec. 4.1 shape): pressure buffers at both
    ends, 4 wall layers top and bottom extending 4 dp beyond both open faces.

    U_max = G H^2 / (8 rho0 nu), G = (p_in - p_out) / length; c0 = 10 U_max.
    The pressure drop is 0.1 on a background of 0.1 (outlet 0.1, inlet 0.2,
    the pressures of the paper's laminar channel): without the transport-
    velocity correction a zero-pressure outlet is tensile-unstable.  The
    initial state is at rest with the density of the mean pressure.
    tvf, tvf_pbuf, density_sum: the transport-velocity shift (also of the
    pressure-buffer particles) and the density reinitialisation of Sec. 2.3,
    off by default (pressure_driven_channel turns them on).
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
                seed=seed, capacity=int(capacity_factor * pos.shape[0]) + 64, tvf=tvf, tvf_pbuf=tvf_pbuf,
                density_sum=density_sum, **arr)


def pressure_driven_channel(length=2.0, height=1.0, dp=0.05, p_in=0.1, p_out=0.0, nu=0.02, seed=1,
                            tvf=0.05, **kw) -> Case:
    """The laminar channel driven by pressure buffers at both ends with a
    zero-pressure outlet: 2.0 x 1.0, dp 0.05, inlet 0.1, outlet 0, nu 0.02,
    from rest (c0 = 10 U_max = 3.125).  With two pressure buffers nothing
    prescribes the motion of the buffer particles, so they crowd like fluid
    particles: the transport-velocity shift (alpha 0.05) acts on them too,
    across the buffer axis only, and the density is re-evaluated from the
    configuration every advection step (Sec. 2.3).  Without these the flow
    near the inlet runs away within a few hundred steps."""
    return poiseuille_channel(length=length, height=height, dp=dp, p_in=p_in, p_out=p_out, nu=nu, seed=seed,
                              tvf=tvf, tvf_pbuf=True, density_sum=True, **kw)


def laminar_channel(length=2.0, height=1.0, dp=0.05, U_max=0.3125, nu=0.02, p_out=0.1, rho0=1.0,
                    jitter_frac=0.01, seed=1, buffer_cells=4, n_theta=41, tvf=0.2, density_sum=True,
                    developed=True, capacity_factor=1.5) -> Case:
    """The laminar straight channel of Sec. 4.1 as the paper sets it up: a
    velocity inlet buffer with the parabolic profile U(y) = 4 U_max y (H - y)
    / H^2 (sampled at n_theta points across the width), a pressure outlet
    buffer at p_out (0.1 in the paper), 4 wall layers, 20 particles across.
    The plane Poiseuille flow of this inflow has the pressure gradient
    G = 8 rho0 nu U_max / H^2 (0.05 here, so the inlet pressure is
    p_out + G L = 0.2, the theoretical value the paper quotes).  developed:
    start from that flow (parabolic velocity, linear pressure) instead of
    rest.  The transport-velocity shift and the density reinitialisation
    (Sec. 2.3) are on."""
    nx, ny = int(round(length / dp)), int(round(height / dp))
    pos = jitter(lattice((nx, ny), dp), 2, jitter_frac * dp, seed)
    G = 8.0 * rho0 * nu * U_max / height**2
    c0 = 10.0 * U_max
    h = H_FAC * dp
    wpos = _channel_walls(-WALL_LAYERS * dp, length + WALL_LAYERS * dp, height, dp)
    Lb = buffer_cells * dp
    s = np.linspace(0.0, 1.0, n_theta)
    theta = tuple(U_max * 4.0 * s * (1.0 - s))
    bufs = [
        BufferSpec("velocity", (0.0, 0.5 * height, 0.0), frame_2d((1, 0)), Lb, (0.5 * height, 0.0),
                   theta=theta),
        BufferSpec("pressure", (length, 0.5 * height, 0.0), frame_2d((-1, 0)), Lb,
                   (0.5 * height, 0.0), p_ob=p_out),
    ]
    margin = WALL_LAYERS * dp + 2 * h
    arr = _fluid_arrays(pos, 2, dp, rho0)
    if developed:
        y, x = pos[:, 1], pos[:, 0]
        arr["vel"][:, 0] = U_max * 4.0 * (y / height) * (1.0 - y / height)
        p0 = p_out + G * (length - x)
    else:
        p0 = np.full(pos.shape[0], p_out)
    arr["rho"][:] = rho0 * (1.0 + p0 / (rho0 * c0 * c0))
    return Case(name=f"laminar_channel_2d_dp{dp:g}", dim=2, dp=dp, h=h, rho0=rho0, c0=c0, nu_l=nu,
                rans=False, U_ref=U_max,
                lo=np.array([-margin, -margin, 0.0]), hi=np.array([length + margin, height + margin, 0.0]),
                periodic=(0, 0, 0), wpos=wpos, wvel=np.zeros_like(wpos), buffers=bufs, seed=seed,
                capacity=int(capacity_factor * pos.shape[0]) + 64, tvf=tvf, density_sum=density_sum, **arr)


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


# --------------------------------------------------------------------------
# U-shaped channel and the batch of independent channels (Sec. 4.2 shape)
# --------------------------------------------------------------------------
def _arc_points(centre, radius, theta0, theta1, dp):
    """Points spaced ~dp along the arc of `radius` about `centre` from theta0 to theta1."""
    n = max(1, int(round(abs(theta1 - theta0) * radius / dp)))
    th = theta0 + (np.arange(n) + 0.5) * (theta1 - theta0) / n
    return np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th), np.zeros(n)], 1)


def u_channel(dp=0.05, width=1.0, r_inner=0.5, leg=1.5, nu=0.01, p_in=2.3, p_out=2.25, c0=15.0,
              rho0=1.0, jitter_frac=0.01, seed=7, buffer_cells=4, capacity_factor=1.5) -> Case:
    """Pressure-driven U-shaped channel: two straight legs of length `leg`
    joined by a half annulus (inner radius r_inner, outer r_inner + width).

    The lower leg occupies 0 <= y <= width, the upper leg
    width + 2 r_inner <= y <= 2 (width + r_inner), both for 0 <= x <= leg;
    the bend is centred at (leg, width + r_inner).  Inlet (lower leg) and
    outlet (upper leg) are pressure buffers at x = 0 with n_b = +x; four
    wall-dummy layers line every wall, straight walls extending 4 dp beyond
    the open faces.  The initial state is at rest with the density of the
    mean pressure.
    """
    Ro = r_inner + width
    cx, cy = leg, width + r_inner
    top = 2.0 * (width + r_inner)
    nx, ny = int(round((leg + Ro) / dp)), int(round(top / dp))
    pts = lattice((nx, ny), dp)
    x, y = pts[:, 0], pts[:, 1]
    rr = np.hypot(x - cx, y - cy)
    in_legs = (x < leg) & (((y > 0) & (y < width)) | ((y > width + 2 * r_inner) & (y < top)))
    in_bend = (x >= leg) & (rr > r_inner) & (rr < Ro)
    pos = jitter(pts[in_legs | in_bend], 2, jitter_frac * dp, seed)
    h = H_FAC * dp
    walls = []
    x0 = -WALL_LAYERS * dp
    ncol = int(round((leg - x0) / dp))
    xs = x0 + (np.arange(ncol) + 0.5) * dp
    for l in range(WALL_LAYERS):
        off = (l + 0.5) * dp
        for yy in (-off, width + off, width + 2 * r_inner - off, top + off):
            walls.append(np.stack([xs, np.full(ncol, yy), np.zeros(ncol)], 1))
        walls.append(_arc_points((cx, cy), Ro + off, -0.5 * np.pi, 0.5 * np.pi, dp))
        walls.append(_arc_points((cx, cy), r_inner - off, -0.5 * np.pi, 0.5 * np.pi, dp))
    wpos = np.concatenate(walls, 0)
    Lb = buffer_cells * dp
    bufs = [
        BufferSpec("pressure", (0.0, 0.5 * width, 0.0), frame_2d((1, 0)), Lb, (0.5 * width, 0.0), p_ob=p_in),
        BufferSpec("pressure", (0.0, top - 0.5 * width, 0.0), frame_2d((1, 0)), Lb, (0.5 * width, 0.0),
                   p_ob=p_out),
    ]
    margin = WALL_LAYERS * dp + 2 * h
    arr = _fluid_arrays(pos, 2, dp, rho0)
    arr["rho"][:] = rho0 * (1.0 + 0.5 * (p_in + p_out) / (rho0 * c0 * c0))
    return Case(name=f"u_channel_2d_dp{dp:g}", dim=2, dp=dp, h=h, rho0=rho0, c0=c0, nu_l=nu, rans=False,
                U_ref=c0 / 10.0, lo=np.array([-margin, -margin, 0.0]),
                hi=np.array([leg + Ro + margin, top + margin, 0.0]), periodic=(0, 0, 0), wpos=wpos,
                wvel=np.zeros_like(wpos), buffers=bufs, seed=seed,
                capacity=int(capacity_factor * pos.shape[0]) + 64, **arr)


def batched_channels(n_instances=64, seed=3, dps=(0.05, 0.025, 0.0125), re_range=(10.0, 200.0),
                     U=1.0, dt_mode="single", stable=False) -> List[Case]:
    """Independent laminar channels for one batched context: half straight
    2 x 1 channels, half U-channels (inner radius 0.5, width 1, legs 1.5),
    dp drawn from `dps` and Re uniform in `re_range`, nu = U W / Re.

    The pressure drop is the one of plane Poiseuille flow with mean velocity
    U over the centre-line length (dp/dx = 12 nu U / W^2); the outlet
    pressure is 0.01 rho0 c0^2 with c0 = 10 U_max = 15 U, the background that
    keeps the open boundaries free of tensile instability.

    stable: the form that holds long runs -- the transport-velocity shift
    (alpha 0.05, also on the buffer particles, across the buffer axis) and
    the density reinitialisation of Sec. 2.3 on every instance, with the
    outlet at zero pressure: the reinitialised density follows the particle
    spacing, which carries no background pressure, so a background at the
    buffers alone would start every instance out of balance.
    """
    rng = np.random.default_rng(seed)
    kinds = np.array([0, 1] * (n_instances // 2) + [0] * (n_instances % 2))
    rng.shuffle(kinds)
    out = []
    for q in range(n_instances):
        dp = float(rng.choice(np.asarray(dps)))
        Re = float(rng.uniform(*re_range))
        nu = U * 1.0 / Re
        c0 = 15.0 * U
        p_out = 0.0 if stable else 0.01 * c0 * c0
        if kinds[q] == 0:
            c = poiseuille_channel(length=2.0, height=1.0, dp=dp, p_in=p_out + 12 * nu * U * 2.0, p_out=p_out,
                                   nu=nu, seed=seed * 1000 + q)
        else:
            path = 2 * 1.5 + np.pi * 1.0
            c = u_channel(dp=dp, nu=nu, p_in=p_out + 12 * nu * U * path, p_out=p_out, c0=c0,
                          seed=seed * 1000 + q)
        c.name = f"batch{q:02d}_{c.name}_Re{Re:.0f}"
        c.dt_mode = dt_mode
        if stable:
            c.tvf, c.tvf_pbuf, c.density_sum = 0.05, True, True
        out.append(c)
    return out


# --------------------------------------------------------------------------
# plane jet with bidirectional buffers on the open sides (Sec. 4.3 shape)
# --------------------------------------------------------------------------
def plane_jet(dp=0.002, box=2.0, slot=0.1, U=1.0, Re=2.0e4, rho0=1.0, c0=10.0, n_theta=32,
              theta=None, rans=True, seed=4, buffer_cells=4, jitter_frac=0.0,
              capacity_factor=1.25) -> Case:
    """Turbulent plane jet entering a box x, y in [0, box] through a slot of
    width `slot` centred on the bottom side.

    Bottom side: a velocity buffer over the slot (profile theta, n_theta
    points across the slot, default uniform U; freestream k, eps) and
    zero-velocity inflow buffers over the rest.  Left, right and top sides:
    zero-pressure buffers (zero-gradient k, eps) that carry inflow and
    outflow.  No walls.  nu = U slot / Re.  Initial state at rest with the
    ambient k, eps.
    """
    n = int(round(box / dp))
    pos = lattice((n, n), dp)
    if jitter_frac:
        pos = jitter(pos, 2, jitter_frac * dp, seed)
    h = H_FAC * dp
    Lb = buffer_cells * dp
    k_in, eps_in = inlet_turbulence(U, slot)
    k_a, eps_a = inlet_turbulence(U, box, intensity=0.01)
    th = np.full(n_theta, U) if theta is None else np.asarray(theta, np.float64)
    s0, s1 = 0.5 * (box - slot), 0.5 * (box + slot)
    up = frame_2d((0, 1))
    bufs = [
        BufferSpec("velocity", (0.5 * box, 0.0, 0.0), up, Lb, (0.5 * slot, 0.0), theta=tuple(th),
                   turb="freestream", k_in=k_in, eps_in=eps_in),
        BufferSpec("velocity", (0.5 * s0, 0.0, 0.0), up, Lb, (0.5 * s0, 0.0), theta=(0.0,),
                   turb="freestream", k_in=k_a, eps_in=eps_a),
        BufferSpec("velocity", (0.5 * (s1 + box), 0.0, 0.0), up, Lb, (0.5 * (box - s1), 0.0), theta=(0.0,),
                   turb="freestream", k_in=k_a, eps_in=eps_a),
        BufferSpec("pressure", (0.0, 0.5 * box, 0.0), frame_2d((1, 0)), Lb, (0.5 * box - Lb, 0.0), p_ob=0.0),
        BufferSpec("pressure", (box, 0.5 * box, 0.0), frame_2d((-1, 0)), Lb, (0.5 * box - Lb, 0.0), p_ob=0.0),
        BufferSpec("pressure", (0.5 * box, box, 0.0), frame_2d((0, -1)), Lb, (0.5 * box, 0.0), p_ob=0.0),
    ]
    margin = 2 * h + Lb
    arr = _fluid_arrays(pos, 2, dp, rho0, k=k_a, eps=eps_a)
    return Case(name=f"plane_jet_2d_{box:g}_dp{dp:g}", dim=2, dp=dp, h=h, rho0=rho0, c0=c0,
                nu_l=U * slot / Re, rans=rans, U_ref=U, lo=np.array([-margin, -margin, 0.0]),
                hi=np.array([box + margin, box + margin, 0.0]), periodic=(0, 0, 0), wpos=np.zeros((0, 3)),
                wvel=np.zeros((0, 3)), buffers=bufs, seed=seed,
                capacity=int(capacity_factor * pos.shape[0]) + 1024, **arr)


# --------------------------------------------------------------------------
# 3D rotating-wall mixer (Sec. 4.4 shape)
# --------------------------------------------------------------------------
def _rings(R, z_levels, dp, centre=(0.0, 0.0)):
    """Wall points on the cylinder of radius R at the given heights, ~dp apart."""
    n = max(1, int(round(2 * np.pi * R / dp)))
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    xy = np.stack([centre[0] + R * np.cos(th), centre[1] + R * np.sin(th)], 1)
    z = np.asarray(z_levels, np.float64)
    out = np.zeros((n * z.size, 3))
    out[:, :2] = np.tile(xy, (z.size, 1))
    out[:, 2] = np.repeat(z, n)
    return out


def mixer_3d(dp=0.01, R=1.0, H=1.0, omega=2.0, r_in=0.15, x_in=0.5, U_in=0.5, r_out=0.3, stub_cells=8,
             Re=100.0, rho0=1.0, seed=6, buffer_cells=4, capacity_factor=1.25, tvf=0.0, tvf_pbuf=False,
             density_sum=False) -> Case:
    """Cylindrical chamber (radius R, height H) whose side wall rotates at
    omega about the axis, fed by two axial inlet stubs of radius r_in on the
    bottom at (+-x_in, 0) and drained by one outlet stub of radius r_out at
    the top centre; stubs are stub_cells * dp long.

    Inlets are velocity buffers (U_in along +z) whose boxes are the cuboids
    bounding the circular stubs, so region-constrained labelling sees
    corners outside the fluid; the outlet is a zero-pressure buffer.  Four
    wall layers line every wall.  nu = U_in (2 r_in) / Re; c0 = 10 max(U_in,
    omega R).  Initial state at rest.  tvf, tvf_pbuf, density_sum: the
    transport-velocity shift (also of the outlet's buffer particles) and the
    density reinitialisation of Sec. 2.3, off by default; mixer_3d_stable
    turns them on.
    """
    Ls = stub_cells * dp
    n_xy = int(round(2 * R / dp))
    nz = int(round(H / dp))
    pts = lattice((n_xy, n_xy, nz), dp, origin=(-R, -R, 0.0))
    keep = np.hypot(pts[:, 0], pts[:, 1]) < R
    fluid = [pts[keep]]
    n_st = int(round(Ls / dp))
    for (cx, rs, z0) in ((x_in, r_in, -Ls), (-x_in, r_in, -Ls), (0.0, r_out, H)):
        m = int(np.ceil(rs / dp)) + 1
        sp = lattice((2 * m, 2 * m, n_st), dp, origin=(cx - m * dp, -m * dp, z0))
        fluid.append(sp[np.hypot(sp[:, 0] - cx, sp[:, 1]) < rs])
    pos = np.concatenate(fluid, 0)
    walls, wv = [], []
    Lw = WALL_LAYERS * dp
    # rotating side wall
    zs = (np.arange(nz) + 0.5) * dp
    for l in range(WALL_LAYERS):
        ring = _rings(R + (l + 0.5) * dp, zs, dp)
        walls.append(ring)
        v = np.zeros_like(ring)
        v[:, 0] = -omega * ring[:, 1]
        v[:, 1] = omega * ring[:, 0]
        wv.append(v)
    # bottom and top plates with holes around the stubs, stub walls
    m = int(np.ceil((R + Lw) / dp))
    plate = lattice((2 * m, 2 * m), dp, origin=(-m * dp, -m * dp, 0.0))
    plate = plate[np.hypot(plate[:, 0], plate[:, 1]) < R + Lw]
    bot_ok = (np.hypot(plate[:, 0] - x_in, plate[:, 1]) >= r_in + Lw) & \
             (np.hypot(plate[:, 0] + x_in, plate[:, 1]) >= r_in + Lw)
    top_ok = np.hypot(plate[:, 0], plate[:, 1]) >= r_out + Lw
    for l in range(WALL_LAYERS):
        b = plate[bot_ok].copy()
        b[:, 2] = -(l + 0.5) * dp
        t = plate[top_ok].copy()
        t[:, 2] = H + (l + 0.5) * dp
        walls += [b, t]
        wv += [np.zeros_like(b), np.zeros_like(t)]
    n_sw = n_st + WALL_LAYERS
    for (cx, rs, zlev) in ((x_in, r_in, -(np.arange(n_sw) + 0.5) * dp),
                           (-x_in, r_in, -(np.arange(n_sw) + 0.5) * dp),
                           (0.0, r_out, H + (np.arange(n_sw) + 0.5) * dp)):
        for l in range(WALL_LAYERS):
            ring = _rings(rs + (l + 0.5) * dp, zlev, dp, centre=(cx, 0.0))
            walls.append(ring)
            wv.append(np.zeros_like(ring))
    wpos = np.concatenate(walls, 0)
    wvel = np.concatenate(wv, 0)
    h = H_FAC * dp
    Lb = buffer_cells * dp
    up = frame_3d((0, 0, 1), (1, 0, 0))
    down = frame_3d((0, 0, -1), (1, 0, 0))
    bufs = [
        BufferSpec("velocity", (x_in, 0.0, -Ls), up, Lb, (r_in, r_in), theta=(U_in,)),
        BufferSpec("velocity", (-x_in, 0.0, -Ls), up, Lb, (r_in, r_in), theta=(U_in,)),
        BufferSpec("pressure", (0.0, 0.0, H + Ls), down, Lb, (r_out, r_out), p_ob=0.0),
    ]
    c0 = 10.0 * max(U_in, omega * R)
    margin = Lw + 2 * h
    arr = _fluid_arrays(pos, 3, dp, rho0)
    lo = np.array([-R - margin, -R - margin, -Ls - margin])
    hi = np.array([R + margin, R + margin, H + Ls + margin])
    return Case(name=f"mixer_3d_R{R:g}_dp{dp:g}", dim=3, dp=dp, h=h, rho0=rho0, c0=c0,
                nu_l=U_in * 2 * r_in / Re, rans=False, U_ref=max(U_in, omega * R), lo=lo, hi=hi,
                periodic=(0, 0, 0), wpos=wpos, wvel=wvel, buffers=bufs, seed=seed,
                capacity=int(capacity_factor * pos.shape[0]) + 1024, tvf=tvf, tvf_pbuf=tvf_pbuf,
                density_sum=density_sum, **arr)


def mixer_3d_stable(dp=0.01, tvf=0.05, **kw) -> Case:
    """The 3D mixer with the transport-velocity shift (alpha 0.05, also on
    the particles of the outlet's pressure buffer, across its axis) and the
    density re-evaluated from the configuration every advection step
    (Sec. 2.3): the full-size mixer (dp 0.01, 3.18M particles) then runs its
    3000 steps (without them it runs away between steps 290 and 550)."""
    return mixer_3d(dp=dp, tvf=tvf, tvf_pbuf=True, density_sum=True, **kw)
