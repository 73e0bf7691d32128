"""Adjoint of differentiated windows against finite differences.

The gradient of the outlet mass flux J with respect to the inlet profile
theta, from the hand-written reverse kernels, must agree with central
finite differences of the same window (FP64, GPU forward) to a relative L2
of 1e-4, and with finite differences of the FP64 oracle along random
directions to the same bound.  Windows use a fixed time step and, for RANS
cases, frozen turbulence (k, eps, nu_t held), which both forwards apply.
"""
import math

import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def sph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_25702_gb300 import build
    from paper_2510_25702_gb300 import sph as S

    build.build()
    return S


def fixed_dt(case, n_ac=None):
    """Fixed advection step 0.25 h / U_ref split into the acoustic count of
    the dual criteria at rest (c0 + U_ref)."""
    dt_ad = 0.25 * case.h / case.U_ref
    dt_ac = 0.6 * case.h / (case.c0 + case.U_ref)
    n = n_ac or max(1, math.ceil(dt_ad / dt_ac))
    return case.replace(dt_mode="fixed", dt_ad_fixed=dt_ad, n_ac_fixed=n)


def small_jet(rans, box=0.4, dp=0.02, n_theta=8):
    th = 1.0 + 0.2 * np.sin(np.linspace(0, np.pi, n_theta))
    c = cases.plane_jet(dp=dp, box=box, slot=0.1, rans=rans, Re=100.0 if not rans else 2.0e4, theta=th,
                        jitter_frac=0.02)
    return fixed_dt(c), th


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def window_for(sph, case, theta, outlets, steps, K, warm=2):
    from paper_2510_25702_gb300.adjoint import Window

    sim = sph.Simulation(case, precision="fp64")
    sim.set_profile(0, 0, theta)
    sim.step(warm)
    start = sim.save_state()
    win = Window(sim, 0, 0, outlets, steps, K, 4 * case.dp)
    return sim, win, start


def adjoint_grad(win, theta, start):
    win.sim.restore_state(start)
    J = win.forward(theta)
    g = win.backward()
    return J, g


def test_laminar_jet_adjoint_matches_fd(sph):
    from paper_2510_25702_gb300.adjoint import fd_gradient

    case, th = small_jet(rans=False)
    sim, win, start = window_for(sph, case, th, [3, 4, 5], steps=12, K=5)
    J, g = adjoint_grad(win, th, start)
    assert J != 0.0 and np.any(g != 0.0)
    fd = fd_gradient(win, th, start)
    assert rel(g, fd) < TOL, (g, fd)


def test_checkpoint_interval_does_not_change_gradient(sph):
    case, th = small_jet(rans=False)
    sim, win, start = window_for(sph, case, th, [3, 4, 5], steps=9, K=1)
    _, g1 = adjoint_grad(win, th, start)
    win.checkpoint_every = 9
    _, g9 = adjoint_grad(win, th, start)
    win.checkpoint_every = 4
    _, g4 = adjoint_grad(win, th, start)
    assert rel(g9, g1) < 1e-12 and rel(g4, g1) < 1e-12


def test_backward_leaves_the_state_after_the_window(sph):
    case, th = small_jet(rans=False)
    sim, win, start = window_for(sph, case, th, [3, 4, 5], steps=6, K=2)
    sim.restore_state(start)
    win.forward(th)
    a = sim.read(["uid", "pos", "vel", "rho"])
    win.backward()
    b = sim.read(["uid", "pos", "vel", "rho"])
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_rans_jet_adjoint_matches_fd_and_oracle(sph, orc):
    """The 10k-particle version of the plane jet (dp 0.02, slot 5 particles,
    32-point profile), frozen turbulence."""
    from paper_2510_25702_gb300.adjoint import fd_gradient

    th = 1.0 + 0.1 * np.cos(np.linspace(0, 2 * np.pi, 32))
    case = fixed_dt(cases.plane_jet(dp=0.02, theta=th, jitter_frac=0.02))
    assert case.n == 10_000 and case.rans
    steps, K, warm = 16, 5, 2
    sim, win, start = window_for(sph, case, th, [3, 4, 5], steps=steps, K=K, warm=warm)
    J, g = adjoint_grad(win, th, start)
    fd = fd_gradient(win, th, start)
    assert rel(g, fd) < TOL, (g, fd)
    # the oracle's own finite differences along two random directions
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(2, th.size))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    h = 1e-6 * np.abs(th).max()
    for u in dirs:
        jj = []
        for sgn in (1, -1):
            o = orc.OracleSim(case, freeze_turb=0)
            o.set_profile(0, th)
            o.step(warm)
            o.cfg.freeze_turb = 1
            jj.append(oracle_window_J(o, case, th + sgn * h * u, [3, 4, 5], steps))
        d_or = (jj[0] - jj[1]) / (2 * h)
        assert abs(g @ u - d_or) <= TOL * max(abs(d_or), np.linalg.norm(g) * 1e-3), (g @ u, d_or)
    # the oracle and the GPU window give the same J
    o = orc.OracleSim(case)
    o.set_profile(0, th)
    o.step(warm)
    o.cfg.freeze_turb = 1
    assert abs(oracle_window_J(o, case, th, [3, 4, 5], steps) - J) <= 1e-9 * abs(J)


def oracle_window_J(o, case, theta, outlets, steps):
    """J of a window on the oracle: membership by label at the window start,
    flux after each step (live particles), n_out = -n_b."""
    o.set_profile(0, theta)
    f = o.fields()
    members = {}
    for u, lab in zip(f["uid"], f["label"]):
        if lab - 1 in outlets:
            members[int(u)] = lab - 1
    nout = {b: -np.asarray(case.buffers[b].frame)[0] for b in outlets}
    slab = 4 * case.dp
    J = 0.0
    for _ in range(steps):
        o.step(1)
        f = o.fields()
        for u, m, v in zip(f["uid"], f["mass"], f["vel"]):
            b = members.get(int(u))
            if b is not None:
                J += case.dt_ad_fixed * m * float(v @ nout[b]) / slab
    return J


def test_channel_with_walls_and_noise(sph):
    """Velocity inlet with seeded noise, walls, zero-pressure outlet
    (mirror B): gradient of the outlet flux w.r.t. a 4-point profile."""
    from paper_2510_25702_gb300.adjoint import fd_gradient

    # short channel: acoustic signals from the inlet reach the outlet
    # buffer within the window (c0 t > length)
    base = cases.turbulent_channel(length=0.1, height=0.1, dp=0.005, jitter_frac=0.05)
    th = np.array([0.9, 1.0, 1.1, 1.0])
    base.buffers[0].theta = tuple(th)
    case = fixed_dt(base)
    steps = 24
    assert case.c0 * steps * case.dt_ad_fixed > 2 * 0.1
    sim, win, start = window_for(sph, case, th, [1], steps=steps, K=7)
    J, g = adjoint_grad(win, th, start)
    fd = fd_gradient(win, th, start)
    assert np.linalg.norm(fd) > 1e-6 * abs(J)
    assert rel(g, fd) < TOL, (g, fd)


def test_mixer_3d_inlet_speed_gradient(sph):
    from paper_2510_25702_gb300.adjoint import fd_gradient

    case = fixed_dt(cases.mixer_3d(dp=0.05))
    th = np.array([0.5])
    steps = 10
    assert case.c0 * steps * case.dt_ad_fixed > 1.2  # inlet -> outlet stub, acoustically
    sim, win, start = window_for(sph, case, th, [2], steps=steps, K=4)
    J, g = adjoint_grad(win, th, start)
    fd = fd_gradient(win, th, start)
    assert np.linalg.norm(fd) > 1e-6 * abs(J)
    assert rel(g, fd) < TOL, (g, fd)


def test_autograd_function(sph):
    torch = pytest.importorskip("torch")
    from paper_2510_25702_gb300.adjoint import OutletFlux

    case, th = small_jet(rans=False)
    sim, win, start = window_for(sph, case, th, [3, 4, 5], steps=6, K=3)
    _, g = adjoint_grad(win, th, start)
    sim.restore_state(start)
    t = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    J = OutletFlux.apply(t, win)
    (2.0 * J).backward()
    assert rel(t.grad.numpy(), 2.0 * g) < 1e-12
