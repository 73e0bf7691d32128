"""The laminar straight channel of Sec. 4.1, run on the oracle to a steady
state: parabolic velocity inlet, pressure outlet 0.1, 20 particles across,
Re 10 (U_max 0.3125, nu 0.02), transport-velocity shift and density
reinitialisation on.  Plane Poiseuille flow fixes the answer: the profile
u(y) = 4 U_max y (H - y) / H^2 and the pressure gradient -G,
G = 8 rho0 nu U_max / H^2.

Measured on this oracle (time averages over steps 1000-2000, fluid
particles in 0.5 < x < 1.5): profile 5.7 % relative L2 below the parabola,
pressure gradient 0.95 G.  Of that, 2.7 % is the inflow itself: the inlet
buffer particles take the kick of the momentum sweep between two
imposures of the profile, and at the open face the pressure force of their
truncated support slows them, so they cross the generation line 3 % less
often than U / dp; the rest is the near-wall rows, slower than the parabola
(the discrete viscous term and the wall dummies).  The bounds below are
those measured values with a margin, not the 3 % of a converged method.

The open-boundary treatments of the Sec. 4.1 table on the same channel
reproduce the paper's findings: case 2 (correction applied directly) is
wrongly accelerated, case 3 (mirror support, uncorrected compensation)
under-predicts the pressure over the whole channel, cases 1 and 4 agree in
their pressure gradients.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.slow

H, L, NU, UMAX = 1.0, 2.0, 0.02, 0.3125
G = 8 * NU * UMAX / H ** 2


def _run(orc, obc):
    c = cases.laminar_channel().replace(obc=obc)
    o = orc.OracleSim(c)
    n0 = o.n
    o.step(1000)
    bins = np.linspace(0, H, 21)
    prof, grad, pcl, counts = [], [], [], []
    xb = np.linspace(0, L, 11)
    for _ in range(20):
        o.step(50)
        f = o.fields()
        x, y = f["pos"][:, 0], f["pos"][:, 1]
        sel = (f["label"] == 0) & (x > 0.5) & (x < 1.5)
        idx = np.clip(np.digitize(y[sel], bins) - 1, 0, 19)
        prof.append([f["vel"][sel, 0][idx == b].mean() for b in range(20)])
        A = np.stack([x[sel], np.ones(sel.sum())], 1)
        grad.append(-np.linalg.lstsq(A, f["p"][sel], rcond=None)[0][0])
        cl = (np.abs(y - 0.5 * H) < 0.15) & (f["label"] == 0)
        k = np.digitize(x, xb) - 1
        pcl.append([f["p"][cl & (k == b)].mean() for b in range(1, 9)])
        counts.append(o.stats["n"])
    yc = 0.5 * (bins[1:] + bins[:-1])
    ua = 4 * UMAX * yc * (H - yc) / H ** 2
    pm = np.mean(prof, 0)
    return dict(err=np.linalg.norm(pm - ua) / np.linalg.norm(ua), grad=np.mean(grad) / G,
                pcl=np.mean(pcl, 0), n0=n0, counts=np.array(counts))


@pytest.fixture(scope="module")
def runs(orc):
    return {obc: _run(orc, obc) for obc in ("improved", "vipo", "vipo_rkgc", "vipo_rkgc_mirror")}


def test_improved_scheme_holds_plane_poiseuille_flow(runs):
    r = runs["improved"]
    assert r["err"] < 0.07
    assert abs(r["grad"] - 1) < 0.08
    # no accumulation at the buffers: the particle count stays put
    assert np.abs(r["counts"] / r["n0"] - 1).max() < 0.02
    # the centre-line pressure falls monotonically from inlet to outlet
    assert np.all(np.diff(r["pcl"]) < 0)


def test_open_boundary_cases_of_the_ablation(runs):
    r4, r1, r2, r3 = runs["improved"], runs["vipo"], runs["vipo_rkgc"], runs["vipo_rkgc_mirror"]
    # case 2: flow wrongly accelerated (far off the parabola)
    assert r2["err"] > 0.5
    # case 3: the pressure is under-predicted over the whole channel
    assert np.all(r3["pcl"] < r4["pcl"])
    # cases 1 and 4: the same pressure gradient within a few per cent
    assert abs(r1["grad"] / r4["grad"] - 1) < 0.05
    assert r1["err"] < 0.07
