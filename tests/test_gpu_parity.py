"""GPU path (C ABI) against the FP64 oracle, element by element by uid.

Integer stages (cell keys, neighbour sets, labels, injected / deleted sets,
uids) must be bit-exact given identical positions; FP64 float fields must
agree to a relative L2 of 1e-10; the FP32-sweep form is held to the error
bounds stated in each test.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


@pytest.fixture(scope="module")
def sph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_25702_gb300 import build
    from paper_2510_25702_gb300 import sph as S

    build.build()
    return S


def small_cases():
    c1 = cases.poiseuille_channel(length=1.0, height=0.5)
    c2 = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    box = cases.periodic_box(n_per_axis=14, dim=2, vel_amp=0.3)
    boxr = cases.periodic_box(n_per_axis=14, dim=2, vel_amp=0.3, rans=True)
    box3 = cases.periodic_box(n_per_axis=8, dim=3, vel_amp=0.3, jitter_frac=0.1)
    lat3 = cases.lattice_block(9, 3)
    lat3.buffers = [cases.BufferSpec("pressure", (0.0, 0.45, 0.45), cases.frame_3d((1, 0, 0), (0, 1, 0)),
                                     0.4, (0.5, 0.5), p_ob=0.05)]
    lat3.vel[:, 0] = 0.1
    uch = cases.u_channel(dp=0.05, nu=0.02)
    jet = cases.plane_jet(dp=0.02, jitter_frac=0.05)
    mix = cases.mixer_3d(dp=0.05)
    return {"channel": c1, "rans_channel": c2, "box2": box, "box2_rans": boxr, "box3": box3, "lattice3_buf": lat3,
            "u_channel": uch, "plane_jet": jet, "mixer3d": mix}


CASES = small_cases()


def compare_state(g, f, fields, tol=TOL64, skip_new=None):
    assert np.array_equal(g["uid"], f["uid"]), "uid sets differ"
    if "label" in g:
        assert np.array_equal(g["label"], f["label"]), "labels differ"
    errs = {}
    for k in fields:
        a, b = g[k], f[k]
        if skip_new is not None and k in ("B", "acc_nu"):
            keep = ~skip_new
            a, b = a[keep], b[keep]
        errs[k] = rel_l2(a, b)
    bad = {k: e for k, e in errs.items() if not e < tol}
    assert not bad, f"relative L2 above {tol}: {bad} (all: {errs})"
    return errs


# --------------------------------------------------------------------------
# integer stages
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(CASES))
def test_cell_keys_bit_exact(sph, orc, name):
    case = CASES[name]
    sim = sph.Simulation(case)
    g = sim.read(["key", "uid"])
    o = orc.OracleSim(case)
    keys = o.cell_keys()
    assert np.array_equal(g["key"], keys[g["uid"]])


@pytest.mark.parametrize("name", list(CASES))
def test_neighbour_pairs_bit_exact(sph, orc, name):
    case = CASES[name]
    sim = sph.Simulation(case)
    gp = sim.debug_pairs()
    o = orc.OracleSim(case, neighbor_mode=1)
    op = o.pairs()
    uid = o.a["uid"]
    oset = {(int(uid[i]), int(j if w else uid[j]), int(w)) for i, j, w in op}
    gset = {(int(a), int(b), int(w)) for a, b, w, _ in gp}
    assert len(gp) == len(op)
    assert gset == oset


# --------------------------------------------------------------------------
# one advection step, FP64
# --------------------------------------------------------------------------
FIELDS64 = ["pos", "vel", "rho", "drho", "p", "B", "acc_nu"]


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_fp64(sph, orc, name):
    case = CASES[name]
    sim = sph.Simulation(case, precision="fp64")
    sim.step(1)
    names = ["uid", "label", "pos", "vel", "rho", "drho", "p", "B", "acc_nu", "k", "eps", "nut"]
    g = sim.read(names)
    o = orc.OracleSim(case)
    o.step(1)
    f = o.fields()
    f["B"] = f["B"].reshape(-1, 9)
    new = g["uid"] >= case.n
    fields = FIELDS64 + (["k", "eps", "nut"] if case.rans else [])
    compare_state(g, f, fields, skip_new=new)
    st = sim.stats()
    assert st["n_ac"] == o.stats["n_ac"]
    assert st["dt_ad"] == o.stats["dt_ad"]  # identical state -> identical step


@pytest.mark.parametrize("obc", ["vipo", "vipo_rkgc", "vipo_rkgc_mirror", "minimal_mirror"])
def test_obc_ablation_cases_fp64(sph, orc, obc):
    """The open-boundary treatments of the Sec. 4.1 ablation (sph_config.obc)
    against the oracle with the same switches: three steps of the pressure
    buffer channel, every float field within the FP64 tolerance."""
    case = cases.poiseuille_channel(length=1.0, height=0.5).replace(obc=obc)
    case.vel[:, 0] = 0.2
    sim = sph.Simulation(case, precision="fp64")
    sim.step(3)
    o = orc.OracleSim(case)
    o.step(3)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "p", "B"])
    f = o.fields()
    f["B"] = f["B"].reshape(-1, 9)
    compare_state(g, f, ["pos", "vel", "rho", "p", "B"], skip_new=g["uid"] >= case.n)


def test_trajectory_fp64_channel(sph, orc):
    """Ten steps of the pressure-buffer channel: injection, recycling and
    deletion happen, uids of the copies agree, fields stay within 1e-9."""
    case = cases.poiseuille_channel(length=1.0, height=0.5)
    case.vel[:, 0] = 0.2  # start moving so the buffers work from step 1
    sim = sph.Simulation(case, precision="fp64")
    o = orc.OracleSim(case)
    for _ in range(10):
        sim.step(1)
        o.step(1)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "p"])
    f = o.fields()
    assert o.stats["n_spawned"] > 0 and o.stats["n_deleted"] > 0
    st = sim.stats()
    assert st["spawned"] == o.stats["n_spawned"] and st["deleted"] == o.stats["n_deleted"]
    compare_state(g, f, ["pos", "vel", "rho", "p"], tol=1e-9)


def test_trajectory_fp64_rans_channel(sph, orc):
    case = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005)
    sim = sph.Simulation(case, precision="fp64")
    o = orc.OracleSim(case)
    sim.step(8)
    o.step(8)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps", "nut"])
    f = o.fields()
    assert o.stats["n_spawned"] > 0
    compare_state(g, f, ["pos", "vel", "rho", "k", "eps", "nut"], tol=1e-9)


# --------------------------------------------------------------------------
# buffer stages with prescribed motion (kinematic mode): bit-exact
# --------------------------------------------------------------------------
def _kinematic_case(kind):
    dp = 0.05
    pos = cases.lattice((12, 20), dp)
    arr = cases._fluid_arrays(pos, 2, dp, 1.0)
    inlet = cases.BufferSpec("velocity", (0.0, 0.5, 0.0), cases.frame_2d((1, 0)), 4 * dp, (0.5, 0.0),
                             theta=(1.0,), noise=0.05)
    outlet = cases.BufferSpec("pressure", (0.6, 0.5, 0.0), cases.frame_2d((-1, 0)), 4 * dp, (0.5, 0.0),
                              p_ob=0.01)
    return cases.Case(name="kin", dim=2, dp=dp, h=1.3 * dp, rho0=1.0, c0=10.0, nu_l=0.01, rans=False,
                      U_ref=1.0, lo=np.array([-0.5, -0.5, 0]), hi=np.array([1.5, 1.5, 0]), periodic=(0, 0, 0),
                      wpos=np.zeros((0, 3)), wvel=np.zeros((0, 3)), buffers=[inlet, outlet],
                      capacity=2000, seed=11, **arr)


def _motion(pos, t):
    u = np.zeros_like(pos)
    u[:, 0] = 1.0 + 0.3 * np.sin(7.0 * pos[:, 1] + t)
    u[:, 1] = 0.05 * np.cos(5.0 * pos[:, 0])
    return u


def test_buffer_update_bit_exact(sph, orc):
    case = _kinematic_case("io")
    sim = sph.Simulation(case, kinematic=True)
    o = orc.OracleSim(case)
    dt = 0.2 * case.dp
    for s in range(40):
        g = sim.read(["pos", "uid"])
        g_new = g["pos"] + _motion(g["pos"], s * dt) * dt
        sim.write({"pos": g_new})
        sim.step(1)
        n = o.n
        live = o.a["dead"][:n] == 0
        p = o.a["pos"][:n]
        p[live] = p[live] + _motion(p[live], s * dt) * dt
        o.compact_sort()
        o.label()
        o.buffer_update(s)
        g = sim.read(["uid", "label", "pos", "vel"])
        f = o.fields()
        assert np.array_equal(g["uid"], f["uid"]), f"step {s}: particle sets differ"
        assert np.array_equal(g["label"], f["label"]), f"step {s}: labels differ"
        assert np.array_equal(g["pos"], f["pos"]), f"step {s}: positions differ"
        assert np.array_equal(g["vel"], f["vel"]), f"step {s}: boundary velocities differ"
    st = sim.stats()
    assert st["spawned"] == o.stats["n_spawned"] > 0
    assert st["deleted"] == o.stats["n_deleted"] > 0


def test_capacity_overflow_is_reported_and_not_committed(sph, orc):
    case = _kinematic_case("io")
    case.capacity = case.n
    sim = sph.Simulation(case, kinematic=True)
    g = sim.read(["pos"])
    sim.write({"pos": g["pos"] + np.array([1.1 * case.dp, 0.0, 0.0])})
    sim.step(1)  # labels the shifted particles
    before = sim.read(["pos", "uid"])
    sim.write({"pos": before["pos"] + np.array([1.1 * case.dp, 0.0, 0.0])})
    mid = sim.read(["pos", "uid"])
    rc = sim.step_rc(1)
    assert rc == -3
    after = sim.read(["pos", "uid"])
    assert np.array_equal(after["uid"], mid["uid"])


def test_nonfinite_state_is_reported(sph):
    case = cases.periodic_box(n_per_axis=10, dim=2)
    sim = sph.Simulation(case)
    v = sim.read(["vel"])["vel"]
    v[3, 0] = np.nan
    sim.write({"vel": v})
    assert sim.step_rc(1) == -4


def test_fp64_mass_momentum_reduction(sph, orc):
    """sph_reduce_mass_momentum (FP64, fixed summation order): equal to the
    oracle's totals after a step within the field tolerance, the same bits on
    a repeated call, and a mass budget that closes exactly over steps with
    injection and deletion (Sec. 2.4.2, 2.4.3: copies carry their parent's
    mass, deleted particles take theirs away; all masses are equal here)."""
    case = cases.poiseuille_channel(length=1.0, height=0.5)
    case.vel[:, 0] = 0.2
    sim = sph.Simulation(case, precision="fp64")
    m0, p0 = sim.mass_momentum()
    assert m0[0] == pytest.approx(case.mass.sum(), rel=1e-13)
    sim.step(1)
    o = orc.OracleSim(case)
    o.step(1)
    f = o.fields()
    m1, p1 = sim.mass_momentum()
    m1b, p1b = sim.mass_momentum()
    assert np.array_equal(m1, m1b) and np.array_equal(p1, p1b)
    assert rel_l2(m1, [f["mass"].sum()]) < 1e-13
    mom = (f["mass"][:, None] * f["vel"]).sum(0)
    assert rel_l2(p1[0], mom) < TOL64
    st0 = sim.stats()
    sim.step(12)
    st1 = sim.stats()
    m2, _ = sim.mass_momentum()
    net = (st1["spawned"] - st0["spawned"]) - (st1["deleted"] - st0["deleted"])
    assert st1["spawned"] > st0["spawned"] and st1["deleted"] > st0["deleted"]
    mp = float(case.mass[0])
    assert np.all(case.mass == mp)
    assert m2[0] - m1[0] == pytest.approx(net * mp, abs=1e-12 * m1[0])
    assert m2[0] == pytest.approx(sim.count() * mp, rel=1e-13)


def test_mass_momentum_async_equals_the_waiting_call(sph):
    """sph_reduce_mass_momentum_async into page-locked memory: after the
    stream has passed it, the same bits as sph_reduce_mass_momentum, for
    every instance of a batch; enqueued behind steps without a wait."""
    import torch

    batch = cases.batched_channels(n_instances=3, dps=(0.05,), seed=7)
    sim = sph.Simulation(batch, precision="fp32")
    sim.step(2)
    out = torch.full((4 * len(batch),), float("nan"), dtype=torch.float64, pin_memory=True)
    sim.step_async(2)
    sim.mass_momentum_async(out)
    ev = torch.cuda.Event()
    ev.record(torch.cuda.current_stream())
    ev.synchronize()
    m, p = sim.mass_momentum()
    tot = out.numpy().reshape(len(batch), 4)
    assert np.array_equal(tot[:, 0], m) and np.array_equal(tot[:, 1:], p)
    # pageable memory: the copy path; device memory: written directly; the same bits
    out2 = torch.full((4 * len(batch),), float("nan"), dtype=torch.float64)
    sim.mass_momentum_async(out2)
    out3 = torch.full((4 * len(batch),), float("nan"), dtype=torch.float64, device="cuda")
    sim.mass_momentum_async(out3)
    torch.cuda.synchronize()
    assert np.array_equal(out2.numpy(), out.numpy())
    assert np.array_equal(out3.cpu().numpy(), out.numpy())
    with pytest.raises(ValueError):
        sim.mass_momentum_async(torch.empty(3, dtype=torch.float64))


def test_async_stepping_matches_and_reports_status(sph):
    """sph_step_async + sph_get_stats (one wait per step, profiles staged
    in pinned memory) give the same state as sph_step, bit for bit, and the
    stats carry the device status word."""
    case = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    a = sph.Simulation(case, precision="fp32")
    b = sph.Simulation(case, precision="fp32")
    for s in range(6):
        theta = np.array([1.0 + 0.05 * s])
        a.set_profile(0, 0, theta)
        a.step(1)
        b.set_profile(0, 0, theta)
        theta[0] = -7.0  # the staged copy is independent of the caller's array
        b.step_async(1)
        assert b.stats()["status"] == 0
    fa, fb = a.read(["pos", "vel", "rho", "uid"]), b.read(["pos", "vel", "rho", "uid"])
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    box = cases.periodic_box(n_per_axis=10, dim=2)
    sim = sph.Simulation(box)
    v = sim.read(["vel"])["vel"]
    v[3, 0] = np.nan
    sim.write({"vel": v})
    sim.step_async(1)
    assert sim.stats()["status"] == -4


# --------------------------------------------------------------------------
# FP32 sweeps (precision pattern): error against the FP64 oracle
# --------------------------------------------------------------------------
def test_fp32_sweeps_error_bounds(sph, orc):
    """FP32 pair sweeps, FP64 integration.  Sweep results carry the FP32
    unit roundoff (6e-8) amplified by the cancellation in the pair sums
    (|sum of |terms|| / |sum| ~ 1e2 for the pressure force), so velocity,
    k and eps increments are good to ~1e-5 relative; FP64 state plus those
    increments gives a velocity error ~1e-6 of |v|; positions move by
    dt |v| ~ 1e-2 of their magnitude per step, so their error is ~1e-8."""
    case = cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05)
    sim = sph.Simulation(case, precision="fp32")
    sim.step(1)
    g = sim.read(["uid", "label", "pos", "vel", "rho", "k", "eps", "B"])
    o = orc.OracleSim(case)
    o.step(1)
    f = o.fields()
    f["B"] = f["B"].reshape(-1, 9)
    assert np.array_equal(g["uid"], f["uid"])
    errs = {k: rel_l2(g[k], f[k]) for k in ("pos", "vel", "rho", "k", "eps")}
    new = g["uid"] >= case.n
    errs["B"] = rel_l2(g["B"][~new], f["B"][~new])
    bounds = {"pos": 1e-8, "vel": 1e-5, "rho": 1e-7, "k": 1e-5, "eps": 1e-5, "B": 1e-5}
    assert all(errs[k] < bounds[k] for k in bounds), errs
