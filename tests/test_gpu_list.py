"""The neighbour list that the pair sweeps walk (the frozen configuration of
an advection step, Sec. 2.3; cell-linked-list search, Sec. 2.4.1), read back
through sph_debug_list, against the oracle's pairs 0 < |r_ij|^2 < (2h)^2 at
the same FP64 positions: bit-exact sets in the FP64 and in the FP32 form
(whose list builder decides candidates near the cut-off by the FP64 test),
after a few steps so that positions, injected copies and deletions are
those of a running case.  The FP64 test-aid pair search (sph_debug_pairs)
must give the same set.
"""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2510_25702_gb300 import build
    from paper_2510_25702_gb300 import sph as S

    build.build()
    return S


def row_keys(rows):
    """One int64 per (uid_i, uid_j | wall index, is_wall) row, sorted."""
    r = np.asarray(rows, np.int64)
    return np.sort(r[:, 0] * (1 << 32) + r[:, 2] * (1 << 31) + r[:, 1])


def oracle_keys(orc, case, g, neighbor_mode):
    """Oracle pairs at the GPU's FP64 positions (rows g sorted by uid)."""
    n = len(g["uid"])
    z = np.zeros(n)
    c = case.replace(pos=g["pos"].copy(), vel=np.zeros((n, 3)), rho=np.full(n, case.rho0),
                     mass=np.full(n, case.rho0 * case.dp ** case.dim), k=z + 1e-3, eps=z + 1e-3,
                     capacity=n + 16)
    o = orc.OracleSim(c, neighbor_mode=neighbor_mode)
    op = o.pairs()
    uid = g["uid"].astype(np.int64)
    j = op[:, 1].copy()
    real = op[:, 2] == 0
    j[real] = uid[j[real]]
    return np.sort(uid[op[:, 0]] * (1 << 32) + op[:, 2] * (1 << 31) + j)


def small_cases():
    lat3 = cases.lattice_block(9, 3)
    lat3.buffers = [cases.BufferSpec("pressure", (0.0, 0.45, 0.45), cases.frame_3d((1, 0, 0), (0, 1, 0)),
                                     0.4, (0.5, 0.5), p_ob=0.05)]
    lat3.vel[:, 0] = 0.1
    return {
        "channel": cases.poiseuille_channel(length=1.0, height=0.5),
        "rans_channel": cases.turbulent_channel(length=0.3, height=0.1, dp=0.005, jitter_frac=0.05),
        "box2": cases.periodic_box(n_per_axis=14, dim=2, vel_amp=0.3),
        "box2_rans": cases.periodic_box(n_per_axis=14, dim=2, vel_amp=0.3, rans=True),
        "box3": cases.periodic_box(n_per_axis=8, dim=3, vel_amp=0.3, jitter_frac=0.1),
        "lattice3_buf": lat3,
        "u_channel": cases.u_channel(dp=0.05, nu=0.02),
        "plane_jet": cases.plane_jet(dp=0.02, jitter_frac=0.05),
        "mixer3d": cases.mixer_3d(dp=0.05),
    }


CASES = small_cases()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_sweep_list_equals_oracle_pairs(sph, orc, name, precision):
    case = CASES[name]
    sim = sph.Simulation(case, precision=precision)
    sim.step(3)
    rows = sim.debug_list()
    g = sim.read(["uid", "pos"])
    got = row_keys(rows)
    assert len(np.unique(got)) == len(got), "an entry appears twice in a list"
    want = oracle_keys(orc, case, g, neighbor_mode=0)
    assert len(got) == len(want)
    assert np.array_equal(got, want)
    assert np.array_equal(row_keys(sim.debug_pairs()), want)
    # reading the list changes nothing that stepping sees
    sim.step(1)
    sim.close()


def test_fp32_list_band_decides_near_cutoff(sph, orc):
    """Pairs placed within FP32 rounding of the cut-off, far from the
    origin (where the FP32 coordinates are coarsest): for each offset the
    FP32 form's list holds exactly the pairs of the FP64 test."""
    dp = 0.005
    h = 1.3 * dp
    cut = 2 * h
    rng = np.random.default_rng(7)
    # lone pairs at x ~ 6 along random directions, separations cut * (1 + e)
    # with e within a few FP32 ulps of zero on both sides
    base = np.array([6.0, 1.0, 0.0])
    pos = []
    for q, e in enumerate(np.concatenate([np.linspace(-4e-7, 4e-7, 33), [0.0]])):
        th = rng.uniform(0, 2 * np.pi)
        p0 = base + np.array([0.0, 8 * cut * q, 0.0])
        d = (1 + e) * cut * np.array([np.cos(th), np.sin(th), 0.0])
        pos += [p0, p0 + d]
    pos = np.array(pos)
    n = len(pos)
    z = np.zeros(n)
    c = cases.Case(name="cutoff_pairs", dim=2, dp=dp, h=h, rho0=1.0, c0=10.0, nu_l=1e-3, rans=False,
                   U_ref=1.0, lo=np.array([5.9, 0.9, 0.0]), hi=np.array([6.1, 1.0 + 8 * cut * 35, 0.0]),
                   periodic=(0, 0, 0), pos=pos, vel=np.zeros((n, 3)), rho=z + 1.0, mass=z + dp * dp, k=z,
                   eps=z, wpos=np.zeros((0, 3)), wvel=np.zeros((0, 3)), capacity=n + 16)
    want = oracle_keys(orc, c, {"uid": np.arange(n), "pos": pos}, neighbor_mode=0)
    assert 5 < len(want) // 2 < 33  # some separations fall on each side of the cut-off
    for precision in ("fp64", "fp32"):
        sim = sph.Simulation(c, precision=precision)
        assert np.array_equal(row_keys(sim.debug_list()), want), precision
        sim.close()
