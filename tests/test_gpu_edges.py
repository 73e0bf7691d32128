"""Degenerate inputs of the GPU step, through the C ABI: a lone particle (no
neighbours: B falls back to I, nothing acts on it), an empty instance in a
batch (zero keys to sort, no cells occupied), and a context whose particles
are all deleted by an outlet (the live count drops to zero and stepping
goes on with nothing to do)."""
import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


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


def test_lone_particle_matches_oracle(sph, orc):
    case = cases.lattice_block(1, 2)
    case.vel[0, :2] = (0.3, -0.2)
    sim = sph.Simulation(case, precision="fp64")
    sim.step(2)
    g = sim.read(["uid", "pos", "vel", "rho", "B"])
    o = orc.OracleSim(case)
    o.step(2)
    f = o.fields()
    assert g["uid"].tolist() == [0]
    for k in ("pos", "vel", "rho"):
        assert rel_l2(g[k], f[k]) < TOL64, k
    assert np.array_equal(g["B"].reshape(-1, 9)[0], np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 0]))
    assert np.allclose(g["vel"][0, :2], (0.3, -0.2), rtol=0, atol=1e-14)


def test_empty_instance_in_a_batch(sph):
    box = cases.periodic_box(n_per_axis=10, dim=2, vel_amp=0.3)
    empty = cases.lattice_block(0, 2)
    assert empty.n == 0
    alone = sph.Simulation(box, precision="fp64")
    alone.step(3)
    ref = alone.read(["uid", "pos", "vel", "rho"])
    for order in ([box, empty], [empty, box]):
        sim = sph.Simulation(order, precision="fp64")
        sim.set_graph(True)
        assert sim.step_rc(3) == 0
        g = sim.read(["inst", "uid", "pos", "vel", "rho"])
        q = 0 if order[0] is box else 1
        assert np.all(g["inst"] == q)
        for k in ("uid", "pos", "vel", "rho"):
            assert np.array_equal(g[k], ref[k]), k


def test_every_particle_deleted(sph):
    """Kinematic stepping: the particles are put in the outlet buffer (they
    take its label), then behind its open face (x'_0 < 0: deleted), after
    which further steps run on an empty context."""
    dp = 0.05
    pos = cases.lattice((12, 20), dp)
    arr = cases._fluid_arrays(pos, 2, dp, 1.0)
    outlet = cases.BufferSpec("pressure", (0.6, 0.5, 0.0), cases.frame_2d((-1, 0)), 4 * dp, (0.5, 0.0),
                              p_ob=0.01)
    case = cases.Case(name="drain", dim=2, dp=dp, h=1.3 * dp, rho0=1.0, c0=10.0, nu_l=0.01, rans=False,
                      U_ref=1.0, lo=np.array([-0.5, -0.5, 0]), hi=np.array([1.5, 1.5, 0]), periodic=(0, 0, 0),
                      wpos=np.zeros((0, 3)), wvel=np.zeros((0, 3)), buffers=[outlet], capacity=400, seed=3,
                      **arr)
    sim = sph.Simulation(case, kinematic=True)
    n = case.n
    p = sim.read(["pos"])["pos"]
    p[:, 0] = 0.5 + 0.0005 * (np.arange(n) % 10)  # inside the box: 0.4 < x <= 0.6
    p[:, 1] = 0.02 + 0.96 * np.arange(n) / n
    sim.write({"pos": p})
    assert sim.step_rc(1) == 0
    assert (sim.read(["label"])["label"] == 1).all()
    p = sim.read(["pos"])["pos"]
    p[:, 0] = 0.7  # behind the open face
    sim.write({"pos": p})
    assert sim.step_rc(1) == 0
    assert sim.count() == 0
    assert sim.stats()["deleted"] == n
    assert sim.step_rc(3) == 0
    assert sim.count() == 0
    assert sim.read(["pos"])["pos"].shape == (0, 3)
    m, _ = sim.mass_momentum()
    assert m[0] == 0.0


def test_misaligned_allocator_is_refused(sph, monkeypatch):
    """The sweeps gather 32-byte records with 256-bit loads, so the ABI asks
    a caller's allocator for 256-byte aligned blocks: a context given blocks
    16 bytes off fails with SPH_ERR_ALLOC, runs nothing, and hands every
    block back."""
    made = []

    class Shifted(sph._TorchAlloc):
        def __init__(self):
            self.live = {}
            self.calls = 0
            super().__init__()
            made.append(self)

        def _do_alloc(self, user, nbytes, stream):
            base = int(self.torch.cuda.caching_allocator_alloc(int(nbytes) + 256, self.device, self.stream))
            self.calls += 1
            self.live[base + 16] = base
            return base + 16

        def _do_free(self, user, ptr, stream):
            self.torch.cuda.caching_allocator_delete(self.live.pop(int(ptr)))

    monkeypatch.setattr(sph, "_TorchAlloc", Shifted)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(cases.periodic_box(n_per_axis=10, dim=2), precision="fp32")
    assert e.value.code == -8
    assert made and made[0].calls > 0 and made[0].live == {}
    monkeypatch.undo()
    sim = sph.Simulation(cases.periodic_box(n_per_axis=10, dim=2), precision="fp32")
    assert sim.step_rc(2) == 0


def test_grid_barrier_wait_runs_out_and_recovers(sph):
    """The bounded wait of the grid barrier: a cooperative launch whose
    barrier can never complete ends with SPH_ERR_TIMEOUT in its status word
    (every block leaves at its poll limit or at the abort flag), resets the
    barrier words, and the context's following steps -- whose later
    sub-steps wait on the same words -- are bit-identical to a context that
    never saw it."""
    case = cases.poiseuille_channel(length=1.0, height=0.5)
    a = sph.Simulation(case, precision="fp64")
    for _ in range(2):
        st, words = a.debug_barrier_timeout()
        assert st == -5
        assert words == [0, 0, 0, 0]
    a.step(3)
    assert a.stats()["n_ac"] > 1  # the cooperative later-sub-steps launch ran
    b = sph.Simulation(case, precision="fp64")
    b.step(3)
    ga, gb = a.read(["uid", "pos", "vel", "rho"]), b.read(["uid", "pos", "vel", "rho"])
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    assert a.stats()["status"] == 0
