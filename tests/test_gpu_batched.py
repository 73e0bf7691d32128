"""Batched instances, CUDA-graph stepping, snapshots and the autotuner.

Each instance of a batched context is an independent problem: its fields
must match the FP64 oracle run on that instance alone (same tolerance as the
single-instance parity tests).  Graph replay, block-size choice and
save/restore change no arithmetic, so their results must be bit-identical
to plain stepping.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
FIELDS = ("pos", "vel", "rho", "drho", "p")


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


def small_batch(n=6, seed=3):
    return cases.batched_channels(n_instances=n, seed=seed, dps=(0.05,))


def split(g, ninst):
    out = []
    for q in range(ninst):
        sel = g["inst"] == q
        out.append({k: v[sel] for k, v in g.items()})
    return out


def compare_instances(g, bat, orc, idx, nsteps, tol=TOL64):
    per = split(g, len(bat))
    for q in idx:
        o = orc.OracleSim(bat[q])
        o.step(nsteps)
        f = o.fields()
        gq = per[q]
        assert np.array_equal(gq["uid"], f["uid"]), f"instance {q}: uid sets differ"
        assert np.array_equal(gq["label"], f["label"]), f"instance {q}: labels differ"
        errs = {k: rel_l2(gq[k], f[k]) for k in FIELDS}
        bad = {k: e for k, e in errs.items() if not e < tol}
        assert not bad, f"instance {q} ({bat[q].name}): {bad}"


READ = ["inst", "uid", "label"] + list(FIELDS)


def test_batched_fp64_matches_oracle_per_instance(sph, orc):
    bat = small_batch()
    sim = sph.Simulation(bat, precision="fp64")
    sim.step(3)
    compare_instances(sim.read(READ), bat, orc, range(len(bat)), 3)


def test_graph_replay_is_bit_identical(sph):
    bat = small_batch(seed=11)
    a = sph.Simulation(bat, precision="fp32")
    a.step(7)
    b = sph.Simulation(bat, precision="fp32")
    b.set_graph(True)
    b.step(3)
    b.step(4)
    ga, gb = a.read(READ), b.read(READ)
    for k in READ:
        assert np.array_equal(ga[k], gb[k]), k
    assert a.stats()["step"] == b.stats()["step"] == 7


def test_graph_replay_with_buffer_traffic_fp64(sph, orc):
    # velocity-inlet channel with seeded noise: the Philox step counter is
    # read on the device, so replayed graphs draw the same numbers
    c = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    sim = sph.Simulation(c, precision="fp64")
    sim.set_graph(True)
    sim.step(5)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps"])
    o = orc.OracleSim(c)
    o.step(5)
    f = o.fields()
    assert np.array_equal(g["uid"], f["uid"])
    assert np.array_equal(g["label"], f["label"])
    for k in ("pos", "vel", "rho", "k", "eps"):
        assert rel_l2(g[k], f[k]) < TOL64, k


def test_save_restore_reproduces_steps(sph):
    c = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    sim = sph.Simulation(c, precision="fp32")
    sim.step(3)
    slot = sim.save_state()
    sim.step(4)
    a = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps", "nut", "p"])
    ta = sim.stats()
    sim.restore_state(slot)
    assert sim.stats()["step"] == 3
    sim.step(4)
    b = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps", "nut", "p"])
    tb = sim.stats()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert ta["t"] == tb["t"] and ta["spawned"] == tb["spawned"] and ta["deleted"] == tb["deleted"]
    sim.drop_state(slot)
    with pytest.raises(sph.SphError):
        sim.restore_state(slot)


def test_launch_config_does_not_change_results(sph):
    bat = small_batch(seed=5)
    a = sph.Simulation(bat, precision="fp32")
    a.step(3)
    b = sph.Simulation(bat, precision="fp32")
    b.set_launch([64, 256, 64, 256])
    assert b.get_launch() == [64, 256, 64, 256]
    b.step(3)
    ga, gb = a.read(READ), b.read(READ)
    for k in READ:
        assert np.array_equal(ga[k], gb[k]), k
    with pytest.raises(sph.SphError):
        b.set_launch([128, 128, 96, 128])


def test_autotune_keeps_state_and_caches(sph, tmp_path):
    bat = small_batch(seed=9)
    ref = sph.Simulation(bat, precision="fp32")
    ref.step(4)
    sim = sph.Simulation(bat, precision="fp32")
    sim.step(1)
    cache = str(tmp_path / "tune.txt")
    blocks, hit = sim.autotune(steps=2, cache_path=cache)
    assert not hit and all(b in (64, 128, 256) for b in blocks)
    assert sim.stats()["step"] == 1
    sim.step(3)
    g, r = sim.read(READ), ref.read(READ)
    for k in READ:
        assert np.array_equal(g[k], r[k]), k
    other = sph.Simulation(bat, precision="fp32")
    other.step(1)
    blocks2, hit2 = other.autotune(steps=2, cache_path=cache)
    assert hit2 and blocks2 == blocks


def test_full_batch_fp64_graph_sampled_instances(sph, orc):
    """All 64 channels (about 750k particles) in one context with graph
    stepping; sampled instances checked against the oracle."""
    bat = cases.batched_channels()
    sim = sph.Simulation(bat, precision="fp64")
    sim.set_graph(True)
    sim.step(2)
    g = sim.read(READ)
    n = np.array([c.n for c in bat])
    sample = sorted({int(np.argmin(n)), int(np.argmax(n)), int(np.argsort(n)[len(n) // 2]), 1})
    compare_instances(g, bat, orc, sample, 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multirate_batch_matches_single_instances(sph, precision):
    """Dual-criteria stepping with a different acoustic sub-step count per
    instance in one context (instances past their own count skip the
    surplus sub-steps inside the kernels, Sec. 2.3): every instance ends
    bit-identical to the same instance stepped alone."""
    a = cases.periodic_box(n_per_axis=12, dim=2, vel_amp=0.3).replace(dt_mode="dual", c0=3.0, nu_l=0.002)
    b = cases.periodic_box(n_per_axis=10, dim=2, vel_amp=0.2, seed=5).replace(dt_mode="dual", c0=3.0, nu_l=0.2)
    c = cases.poiseuille_channel(length=1.0, height=0.5).replace(dt_mode="dual")
    batch = [a, b, c]
    nac = []
    alone = []
    for q, case in enumerate(batch):
        s = sph.Simulation(case, precision=precision)
        s.set_graph(True)
        s.step(6)
        nac.append(s.stats()["n_ac"])
        alone.append(s.read(["uid", "pos", "vel", "rho"]))
        s.close()
    assert len(set(nac)) > 1, f"the instances should take different sub-step counts: {nac}"
    sim = sph.Simulation(batch, precision=precision)
    sim.set_graph(True)
    sim.step(6)
    per = split(sim.read(["inst", "uid", "pos", "vel", "rho"]), len(batch))
    for q in range(len(batch)):
        for k in ("uid", "pos", "vel", "rho"):
            assert np.array_equal(per[q][k], alone[q][k]), f"instance {q} ({batch[q].name}): {k} differs"
