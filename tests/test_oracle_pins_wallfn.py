"""Pins of the oracle's step-wise wall function (Sec. 2.3 uses the one of
its reference at turbulent walls; the standard two-layer wall law):

* the friction velocity inverts the law it is defined by: the viscous
  sublayer u_t = u_tau^2 y / nu up to y+ = 11.225 and the log law
  u_t = (u_tau / kappa) ln(E y u_tau / nu) beyond, the two meeting there
  (u_tau continuous in u_t);
* log-layer equilibrium: with k = u_tau^2 / sqrt(C_mu) and eps at its wall
  value, a near-wall particle's production u_tau^3 / (kappa y) balances the
  dissipation, so k and eps stay where they are;
* the wall shear: the viscous force of the wall pairs goes as u_tau^2
  (not as u_t), the wall stress rho0 u_tau^2;
* particles off the wall and runs without the switch are untouched.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

KAPPA, E, YC, CMU = 0.4187, 9.793, 11.225, 0.09


@pytest.mark.parametrize("utau,y,nu", [(0.05, 0.01, 1e-5), (0.3, 0.002, 2e-5), (0.01, 0.5, 1e-4)])
def test_log_law_inverted(orc, utau, y, nu):
    yp = utau * y / nu
    assert yp > YC
    ut = utau / KAPPA * np.log(E * y * utau / nu)
    u, log_layer = orc.wall_utau(ut, y, nu)
    assert log_layer and abs(u / utau - 1) < 1e-13


@pytest.mark.parametrize("utau,y,nu", [(0.01, 0.01, 1e-4), (0.02, 0.001, 5e-5)])
def test_sublayer_inverted(orc, utau, y, nu):
    assert utau * y / nu < YC
    u, log_layer = orc.wall_utau(utau ** 2 * y / nu, y, nu)
    assert not log_layer and abs(u / utau - 1) < 1e-13


def test_laws_meet_at_crossover(orc):
    """kappa = 0.4187 and E = 9.793 make ln(E y+) / kappa = y+ at 11.225:
    u_tau is continuous across the switch from one law to the other."""
    assert abs(np.log(E * YC) / KAPPA - YC) < 5e-4
    y, nu = 0.01, 1e-4
    ut_c = (YC * nu / y) ** 2 * y / nu  # u_t at the crossover on the sublayer law
    lo, _ = orc.wall_utau(ut_c * (1 - 1e-9), y, nu)
    hi, lg = orc.wall_utau(ut_c * (1 + 1e-9), y, nu)
    assert lg and abs(hi / lo - 1) < 1e-4


def _wall_channel(u, k, eps, eta=3.0):
    """A turbulent channel lattice between flat static walls, uniform flow u
    along the walls, uniform k and eps; first fluid rows at dp/2 from the
    walls."""
    c = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.0).replace(
        wall_function=True, eta=eta)
    c.buffers = []
    c.periodic = (1, 0, 0)
    c.lo = np.array([0.0, c.lo[1], 0.0])
    c.hi = np.array([0.3, c.hi[1], 0.0])
    c.wpos = c.wpos[(c.wpos[:, 0] > 0) & (c.wpos[:, 0] < 0.3)]
    c.wvel = np.zeros_like(c.wpos)
    c.vel[:] = 0.0
    c.vel[:, 0] = u
    c.k[:] = k
    c.eps[:] = eps
    return c


def test_log_layer_equilibrium_keeps_k_and_eps(orc):
    dp, nu = 0.005, 5e-6
    y = 0.5 * dp
    u = 1.0
    utau, lg = orc.wall_utau(u, y, nu)
    assert lg
    k = utau ** 2 / np.sqrt(CMU)
    ew = CMU ** 0.75 * k ** 1.5 / (KAPPA * y)
    c = _wall_channel(u, k, ew).replace(nu_l=nu)
    o = orc.OracleSim(c)
    o.configure()
    first = np.isclose(o.a["pos"][: o.n, 1], y) | np.isclose(o.a["pos"][: o.n, 1], 0.1 - y)
    assert first.sum() == 2 * 60
    o.bmatrix()
    o.rans(1e-3)
    # uniform k: no diffusion; the wall particles' sources balance
    assert np.abs(o.a["k"][: o.n][first] / k - 1).max() < 1e-12
    assert np.abs(o.a["eps"][: o.n][first] / ew - 1).max() < 1e-12
    # interior particles follow the standard model (no production, uniform
    # flow): k decays by dt eps
    inner = np.abs(o.a["pos"][: o.n, 1] - 0.05) < 0.01
    assert np.allclose(o.a["k"][: o.n][inner], k - 1e-3 * ew, rtol=1e-12, atol=0)


def test_wall_shear_goes_as_utau_squared(orc):
    """The wall pairs carry nu_w = u_tau^2 y / u_t and the dummy velocity
    2 v_w - v_i, so their force is 2 u_tau^2 y sum_w (...): dividing the
    first-layer particles' viscous acceleration by u_tau^2 gives the same
    value for two flow speeds (limiter off, uniform flow: the fluid pairs
    add nothing)."""
    dp, nu = 0.005, 5e-6
    y = 0.5 * dp
    res = []
    for u in (0.5, 2.0):
        c = _wall_channel(u, 1e-3, 1e-3, eta=0.0).replace(nu_l=nu)
        o = orc.OracleSim(c)
        o.configure()
        o.viscous()
        first = np.isclose(o.a["pos"][: o.n, 1], y)
        utau, lg = orc.wall_utau(u, y, nu)
        assert lg
        res.append(o.a["acc_nu"][: o.n][first, 0] / utau ** 2)
        assert np.all(o.a["acc_nu"][: o.n][first, 0] < 0)  # the wall retards the flow
    assert np.allclose(res[0], res[1], rtol=1e-12, atol=0)


def test_switch_off_and_interior_untouched(orc):
    """The advection-step stages (B, viscous, k-eps) with and without the
    switch: particles farther than a support from every near-wall particle
    get the same viscous acceleration, k and eps; near-wall ones do not."""
    c_on = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05).replace(wall_function=True)
    out = []
    for c in (c_on, c_on.replace(wall_function=False)):
        o = orc.OracleSim(c)
        o.label()
        o.configure()
        o.bmatrix()
        o.viscous()
        o.rans(1e-4)
        out.append(o)
    a, b = out
    y = b.a["pos"][: b.n, 1]
    far = (y > c_on.dp + 2 * c_on.h + 0.1 * c_on.dp) & (y < 0.1 - c_on.dp - 2 * c_on.h - 0.1 * c_on.dp)
    assert far.sum() > 100
    for k in ("k", "eps", "acc_nu"):
        assert np.array_equal(a.a[k][: a.n][far], b.a[k][: b.n][far]), k
    near = (y < 0.8 * c_on.dp) & (b.a["label"][: b.n] == 0)
    assert near.sum() > 10
    assert not np.allclose(a.a["eps"][: a.n][near], b.a["eps"][: b.n][near])
