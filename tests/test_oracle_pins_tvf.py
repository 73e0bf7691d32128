"""Pins of two stages of the advection step that Sec. 2.3 names through the
schemes it cites, the transport-velocity correction and the density
re-evaluated from the configuration once per advection step:

* density reinitialisation rho_i = rho0 sigma_i / sigma_0 (sigma the kernel
  sum over the particle and its neighbours): a perfect lattice, continued
  by the wall dummies at a wall, has rho0 exactly; the reference sum
  equals the Wendland C2 lattice sum at h = 1.3 dp computed apart from the
  oracle (1.010473 in 2D, 1.009501 in 3D); a uniform compression
  raises the density by the inverse volume ratio;
* transport-velocity shift dr_i = -2 alpha h^2 sum_j V_j grad_i W_ij: zero
  on a perfect lattice, a displaced particle is moved back towards its
  site, the disorder of a jittered box decreases under repeated shifts, a
  particle close to a wall is pushed away from it, pressure-buffer particles
  (when the switch tvf_pbuf asks for it) are shifted only across their
  buffer's axis, and velocity-buffer particles and all velocities are left
  alone.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases


def _perfect_box(n, dim, **kw):
    return cases.periodic_box(n_per_axis=n, dim=dim, jitter_frac=0.0, vel_amp=0.0, rho_amp=0.0, **kw)


# --------------------------------------------------------------------------
# density reinitialisation
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,ref", [(2, 1.010473), (3, 1.009501)])
def test_density_sum_reference_and_perfect_lattice(orc, dim, ref):
    c = _perfect_box(12 if dim == 2 else 7, dim).replace(density_sum=True)
    o = orc.OracleSim(c)
    o.configure()
    # sigma_0 dp^d is the lattice kernel sum at h = 1.3 dp (values computed apart from the oracle)
    assert abs(o.lattice_kernel_sum() * c.dp ** dim - ref) < 1e-6
    o.a["rho"][: o.n] = 1.7  # a value the reinitialisation must replace
    o.density_sum()
    assert np.abs(o.a["rho"][: o.n] - c.rho0).max() < 1e-14


def test_density_sum_walls_continue_the_lattice(orc):
    """A channel lattice between four layers of wall dummies on the same
    lattice: fluid particles next to the walls see the lattice continued
    and get rho0 like the interior ones."""
    c = cases.poiseuille_channel(length=1.0, height=0.5, jitter_frac=0.0).replace(density_sum=True)
    c.buffers = []
    c.periodic = (1, 0, 0)
    c.lo = np.array([0.0, c.lo[1], 0.0])
    c.hi = np.array([1.0, c.hi[1], 0.0])
    c.wpos = c.wpos[(c.wpos[:, 0] > 0) & (c.wpos[:, 0] < 1.0)]
    c.wvel = np.zeros_like(c.wpos)
    o = orc.OracleSim(c)
    o.configure()
    o.density_sum()
    assert np.abs(o.a["rho"][: o.n] - c.rho0).max() < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_density_sum_uniform_compression(orc, dim):
    """Positions scaled by (1 - e) about the box centre (interior particles,
    full support): the density rises by the inverse volume ratio
    (1 - e)^-d to within the change of the lattice factor with h / dp
    (a small fraction of the rise)."""
    n = 21 if dim == 2 else 11
    c = cases.lattice_block(n, dim).replace(density_sum=True)
    o = orc.OracleSim(c)
    e = 2e-3
    ctr = 0.5 * n * c.dp
    o.a["pos"][: o.n, :dim] = ctr + (o.a["pos"][: o.n, :dim] - ctr) * (1 - e)
    o.configure()
    o.density_sum()
    pos = o.a["pos"][: o.n]
    inner = np.all((pos[:, :dim] > 2.5 * c.h) & (pos[:, :dim] < n * c.dp - 2.5 * c.h), axis=1)
    rise = (1 - e) ** (-dim) - 1
    got = o.a["rho"][: o.n][inner] / c.rho0 - 1
    assert inner.sum() > 0
    assert np.abs(got - rise).max() < 0.05 * rise


# --------------------------------------------------------------------------
# transport-velocity shift
# --------------------------------------------------------------------------
def _shift(orc, c):
    o = orc.OracleSim(c)
    o.configure()
    x0 = o.a["pos"][: o.n].copy()
    v0 = o.a["vel"][: o.n].copy()
    o.transport()
    assert np.array_equal(o.a["vel"][: o.n], v0)
    return o, o.a["pos"][: o.n] - x0


@pytest.mark.parametrize("dim", [2, 3])
def test_transport_shift_vanishes_on_perfect_lattice(orc, dim):
    _, s = _shift(orc, _perfect_box(12 if dim == 2 else 7, dim).replace(tvf=0.2))
    assert np.abs(s).max() < 1e-15


def test_transport_shift_restores_a_displaced_particle(orc):
    """One particle moved off its site in a perfect periodic lattice: the
    shift points back towards the site and shortens the displacement,
    by a fraction proportional to alpha."""
    c = _perfect_box(14, 2).replace(tvf=0.2)
    k = 14 * 7 + 7
    d = np.array([0.12, 0.05, 0.0]) * c.dp
    c.pos[k] += d
    o, s = _shift(orc, c)
    sk = s[k]
    assert np.dot(sk, d) < 0
    assert np.linalg.norm(d + sk) < np.linalg.norm(d)
    c2 = c.replace(tvf=0.1, pos=c.pos.copy())
    _, s2 = _shift(orc, c2)
    assert np.allclose(s2[k], 0.5 * sk, rtol=1e-12, atol=0)


def test_transport_shift_reduces_disorder(orc):
    """Repeated shifts of a jittered periodic box lower the RMS of
    sum_j V_j grad W_ij (zero on a regular arrangement) monotonically."""
    c = cases.periodic_box(n_per_axis=14, dim=2, jitter_frac=0.15, vel_amp=0.0).replace(tvf=0.2)
    o = orc.OracleSim(c)
    hist = []
    for _ in range(5):
        o.configure()
        hist.append(np.sqrt(np.mean(np.sum(o.kernel_gradient_sum() ** 2, axis=1))))
        o.transport()
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.5 * hist[0]


def test_transport_shift_pushes_from_walls_and_skips_buffers(orc):
    """The first row pressed towards the lower wall is pushed off it, in
    the fluid and, with tvf_pbuf, in the pressure buffers; a pressure-buffer
    particle takes only the part of the shift across its buffer's axis (its
    support is cut at the open face), so nothing moves it along the axis.
    Without tvf_pbuf the buffer particles stay where they are."""
    c = cases.poiseuille_channel(length=1.0, height=0.5, jitter_frac=0.0).replace(tvf=0.2)
    y = c.pos[:, 1]
    low = np.isclose(y, 0.5 * c.dp)
    c.pos[low, 1] = 0.3 * c.dp  # the first row pressed towards the lower wall

    def shift(case):
        o = orc.OracleSim(case)
        o.label()
        o.configure()
        x0 = o.a["pos"][: o.n].copy()
        o.transport()
        return x0, o.a["pos"][: o.n] - x0, o.a["label"][: o.n].copy(), o.n

    _, s_off, lab_off, _ = shift(c)
    assert lab_off.max() > 0 and np.all(s_off[lab_off > 0] == 0.0)
    x0, s, lab, n = shift(c.replace(tvf_pbuf=True))
    pushed = low[:n] & (lab == 0)
    assert pushed.sum() > 5 and np.all(s[pushed, 1] > 0)
    assert np.array_equal(s[lab == 0], s_off[lab_off == 0])
    inb = lab > 0
    assert inb.sum() > 0
    assert np.all(s[inb, 0] == 0.0)  # both buffer axes are +-x
    pushed_b = low[:n] & inb
    assert pushed_b.sum() >= 4 and np.all(s[pushed_b, 1] > 0)
    # untouched rows of a buffer: the transverse part vanishes by symmetry
    mid = inb & (np.abs(x0[:, 1] - 0.5 * c.pos[:, 1].max()) < 0.6 * c.dp)
    assert mid.sum() > 0 and np.abs(s[mid]).max() < 1e-12 * c.dp


def test_transport_shift_leaves_velocity_buffers(orc):
    """Velocity-buffer particles keep the motion their prescribed velocity
    gives them: the shift leaves them where they are."""
    c = cases.laminar_channel(jitter_frac=0.2).replace(tvf=0.2, tvf_pbuf=True)
    o = orc.OracleSim(c)
    o.label()
    o.configure()
    x0 = o.a["pos"][: o.n].copy()
    o.transport()
    s = o.a["pos"][: o.n] - x0
    lab = o.a["label"][: o.n]
    vel_ids = [q + 1 for q, b in enumerate(c.buffers) if b.kind == "velocity"]
    vb = np.isin(lab, vel_ids)
    assert vb.sum() > 0 and np.all(s[vb] == 0.0)
    assert np.abs(s[lab == 0]).max() > 0
