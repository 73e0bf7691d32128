"""Workload generators: sizes and structure of the synthetic inputs (CPU)."""
import numpy as np

from paper_2510_25702_gb300 import cases


def test_batched_channels_shape():
    bat = cases.batched_channels()
    assert len(bat) == 64
    kinds = [c.name.split("_")[1] for c in bat]
    assert kinds.count("u") == 32
    n = np.array([c.n for c in bat])
    assert 700_000 < n.sum() < 800_000 and n.min() >= 800 and n.max() < 40_000
    assert all(c.dt_mode == "single" for c in bat)
    assert all(len(c.buffers) == 2 and all(b.kind == "pressure" for b in c.buffers) for c in bat)
    # same seed, same batch
    again = cases.batched_channels()
    assert all(np.array_equal(a.pos, b.pos) and a.nu_l == b.nu_l for a, b in zip(bat, again))


def test_u_channel_fluid_inside_walls():
    c = cases.u_channel(dp=0.025)
    x, y = c.pos[:, 0], c.pos[:, 1]
    r = np.hypot(x - 1.5, y - 1.5)
    bend = x >= 1.5
    assert np.all((r[bend] > 0.5) & (r[bend] < 1.5))
    legs = ~bend
    assert np.all(((y[legs] > 0) & (y[legs] < 1)) | ((y[legs] > 2) & (y[legs] < 3)))
    # no wall dummy closer than dp / 2 to a fluid particle
    from scipy.spatial import cKDTree

    d, _ = cKDTree(c.wpos[:, :2]).query(c.pos[:, :2])
    assert d.min() > 0.4 * c.dp


def test_plane_jet_layout():
    c = cases.plane_jet(dp=0.02)
    assert c.n == 100 * 100 and c.nw == 0 and c.rans
    kinds = [b.kind for b in c.buffers]
    assert kinds.count("velocity") == 3 and kinds.count("pressure") == 3
    slot = c.buffers[0]
    assert len(slot.theta) == 32 and np.isclose(2 * slot.half[0], 0.1)
    assert np.isclose(c.nu_l, 0.1 / 2.0e4)


def test_mixer_layout():
    c = cases.mixer_3d(dp=0.05)
    r = np.hypot(c.pos[:, 0], c.pos[:, 1])
    body = (c.pos[:, 2] >= 0) & (c.pos[:, 2] <= 1)
    assert np.all(r[body] < 1.0)
    side = np.isclose(np.hypot(c.wpos[:, 0], c.wpos[:, 1]), 1.0 + 0.5 * c.dp) & \
        (c.wpos[:, 2] > 0) & (c.wpos[:, 2] < 1)
    # rotating side wall: v = omega x r with omega = 2
    assert np.allclose(c.wvel[side, 0], -2.0 * c.wpos[side, 1])
    assert np.allclose(c.wvel[side, 1], 2.0 * c.wpos[side, 0])
    full = cases.mixer_3d.__defaults__[0]
    assert full == 0.01
    from scipy.spatial import cKDTree

    d, _ = cKDTree(c.wpos).query(c.pos)
    assert d.min() > 0.4 * c.dp


def test_long_run_forms():
    """The forms that hold their stated lengths: the stated pressures of the
    pressure-driven channel, the switches of each, and the same geometry as
    the plain generators."""
    c1 = cases.pressure_driven_channel()
    plain = cases.poiseuille_channel(p_in=0.1, p_out=0.0)
    assert [b.kind for b in c1.buffers] == ["pressure", "pressure"]
    assert (c1.buffers[0].p_ob, c1.buffers[1].p_ob) == (0.1, 0.0)
    assert c1.n == 800 and np.isclose(c1.nu_l, 0.02) and np.isclose(c1.c0, 3.125)
    assert c1.tvf == 0.05 and c1.tvf_pbuf and c1.density_sum
    assert not plain.tvf and not plain.tvf_pbuf and not plain.density_sum
    assert np.array_equal(c1.pos, plain.pos) and np.array_equal(c1.wpos, plain.wpos)
    m = cases.mixer_3d_stable(dp=0.05)
    m0 = cases.mixer_3d(dp=0.05)
    assert m.tvf == 0.05 and m.tvf_pbuf and m.density_sum and not m0.tvf_pbuf
    assert np.array_equal(m.pos, m0.pos)
    st = cases.batched_channels(stable=True)
    pl = cases.batched_channels()
    for a, b in zip(st, pl):
        assert np.array_equal(a.pos, b.pos) and a.nu_l == b.nu_l
        assert a.tvf == 0.05 and a.tvf_pbuf and a.density_sum
        assert a.buffers[1].p_ob == 0.0
        # the same pressure drop on a zero background
        assert np.isclose(a.buffers[0].p_ob, b.buffers[0].p_ob - b.buffers[1].p_ob)
