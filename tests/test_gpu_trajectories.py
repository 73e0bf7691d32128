"""Longer FP64 trajectories against the oracle (C1 as stated, C3 instances, a
section of C2, C5).

The plain-method channel at the pressures it is stated with: 2.0 x 1.0,
dp 0.05, pressure buffers at both ends with p_in 0.1 and p_out 0, nu 0.02,
FP64 (the laminar channel of Sec. 4.1 driven by two pressure buffers).

Over its first 200 steps -- inside the window before the flow near the
inlet runs away, which it does on the oracle and on the GPU alike between
steps 250 and 600 -- the GPU follows the oracle particle by particle:
the same particles (uid), labels and injected / deleted counts, and the
fields at 1e-9 relative L2.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def sph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_25702_gb300 import build
    from paper_2510_25702_gb300 import sph as S

    build.build()
    return S


def test_c1_as_stated_200_steps_fp64(sph, orc):
    case = cases.poiseuille_channel(length=2.0, height=1.0, dp=0.05, p_in=0.1, p_out=0.0, nu=0.02)
    sim = sph.Simulation(case, precision="fp64")
    o = orc.OracleSim(case)
    sim.step(200)
    o.step(200)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "p"])
    f = o.fields()
    st = sim.stats()
    assert o.stats["n_spawned"] > 0 and o.stats["n_deleted"] > 0
    assert st["spawned"] == o.stats["n_spawned"] and st["deleted"] == o.stats["n_deleted"]
    assert np.array_equal(g["uid"], f["uid"]) and np.array_equal(g["label"], f["label"])
    errs = {k: rel_l2(g[k], f[k]) for k in ("pos", "vel", "rho", "p")}
    print("C1 as stated, 200 steps", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(e < 1e-9 for e in errs.values()), errs


def test_batch_instances_follow_the_oracle_300_steps_fp64(sph, orc):
    """Three instances of the batched workload (a straight channel and
    U-channels, pressure buffers at every end, different viscosities) in
    one FP64 context replayed as CUDA graphs, 300 steps (injection and
    deletion at every instance): each instance, with its own time step and
    sub-step count, equals the oracle run on that instance alone (same
    particles and labels, fields at 1e-9)."""
    batch = cases.batched_channels(n_instances=3, dps=(0.05,), seed=11)
    sim = sph.Simulation(batch, precision="fp64")
    sim.set_graph(True)
    sim.step(300)
    g = sim.read(["inst", "uid", "label", "pos", "vel", "rho"])
    for q, c in enumerate(batch):
        o = orc.OracleSim(c)
        o.step(300)
        assert o.stats["n_spawned"] > 0 and o.stats["n_deleted"] > 0, q
        f = o.fields()
        gq = {k: v[g["inst"] == q] for k, v in g.items()}
        assert np.array_equal(gq["uid"], f["uid"]) and np.array_equal(gq["label"], f["label"]), q
        errs = {k: rel_l2(gq[k], f[k]) for k in ("pos", "vel", "rho")}
        print("instance", q, c.name, {k: f"{v:.2e}" for k, v in errs.items()})
        assert all(e < 1e-9 for e in errs.values()), (q, errs)


def test_mixer_3d_50_steps_fp64(sph, orc):
    """The 3D mixer (rotating wall, two velocity inlets, a pressure outlet;
    dp 0.05, 27k particles) in FP64 over 50 steps, with about 250 copies
    injected and 100 particles deleted: the same particles and labels as
    the oracle, fields at 1e-9."""
    case = cases.mixer_3d(dp=0.05)
    sim = sph.Simulation(case, precision="fp64")
    o = orc.OracleSim(case)
    sim.step(50)
    o.step(50)
    g = sim.read(["uid", "label", "pos", "vel", "rho"])
    f = o.fields()
    st = sim.stats()
    assert o.stats["n_spawned"] > 100 and o.stats["n_deleted"] > 50
    assert st["spawned"] == o.stats["n_spawned"] and st["deleted"] == o.stats["n_deleted"]
    assert np.array_equal(g["uid"], f["uid"]) and np.array_equal(g["label"], f["label"])
    errs = {k: rel_l2(g[k], f[k]) for k in ("pos", "vel", "rho")}
    print("mixer 3D, 50 steps", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(e < 1e-9 for e in errs.values()), errs


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-9)])
def test_turbulent_channel_100_steps(sph, orc, precision, bound):
    """A section of the turbulent channel (0.3 x 0.1, dp 0.005, k-epsilon,
    velocity inlet with its seeded fluctuation, pressure outlet) over 100
    steps with about 350 particles injected and as many deleted: the same
    particles and labels as the oracle; positions, velocities, density and
    k, epsilon, nu_t at 1e-9."""
    case = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    sim = sph.Simulation(case, precision=precision)
    o = orc.OracleSim(case)
    sim.step(100)
    o.step(100)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps", "nut"])
    f = o.fields()
    assert o.stats["n_spawned"] > 200 and o.stats["n_deleted"] > 200
    assert np.array_equal(g["uid"], f["uid"]) and np.array_equal(g["label"], f["label"])
    errs = {k: rel_l2(g[k], f[k]) for k in ("pos", "vel", "rho", "k", "eps", "nut")}
    print("turbulent channel, 100 steps", precision, {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(e < bound for e in errs.values()), errs
