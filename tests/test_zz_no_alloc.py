"""sph_cell_sort_noalloc: the cell sort for callers that cannot allocate
device memory (code inside a CUDA stream capture, applications with a fixed
device-memory budget).  Called through the C ABI and checked against the
cell keys that the stepping path reports (sph_read_fields), on two calls in
a row with different positions, so state left in the shared scratch array
by the first call cannot leak into the second.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2510_25702_gb300 import cases

pytestmark = pytest.mark.gpu


def test_noalloc_cell_sort_matches_the_stepping_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    from paper_2510_25702_gb300 import build, sph

    build.build()
    L = sph.lib()
    case = cases.turbulent_channel(length=0.6, height=0.2, dp=0.005)
    sim = sph.Simulation(case, precision="fp32")
    cfg = sph.make_config(case)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")

    # sizes beyond the stated maximum are rejected before any device work
    ncell = C.c_int64()
    rc = L.sph_cell_sort_noalloc(C.byref(cfg), dummy.data_ptr(), sph.NOALLOC_MAX_POINTS + 1,
                                 dummy.data_ptr(), dummy.data_ptr(), 4, C.byref(ncell), stream)
    assert rc == -1

    for call in range(2):
        if call == 1:
            sim.step(3)  # the particles move: a different input for the second call
        f = sim.read(["pos", "key"])
        keys = f["key"]
        n = keys.shape[0]
        pos = torch.from_numpy(np.ascontiguousarray(f["pos"])).cuda()
        # ncell query: a too-short cell_start is rejected after ncell is reported
        rc = L.sph_cell_sort_noalloc(C.byref(cfg), pos.data_ptr(), n, dummy.data_ptr(), dummy.data_ptr(), 0,
                                     C.byref(ncell), stream)
        assert rc == -1 and ncell.value > 0
        m = ncell.value
        order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        start = torch.full((m + 1,), -1, dtype=torch.int32, device="cuda")
        rc = L.sph_cell_sort_noalloc(C.byref(cfg), pos.data_ptr(), n, order.data_ptr(), start.data_ptr(), m + 1,
                                     C.byref(ncell), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = order.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, np.argsort(keys, kind="stable")), f"call {call}: order differs"
        expect_start = np.searchsorted(np.sort(keys), np.arange(m + 1), side="left")
        assert np.array_equal(start.cpu().numpy().view(np.uint32), expect_start), f"call {call}: cell starts differ"
    sim.close()


def test_noalloc_cell_sort_edges_empty_and_maximum():
    """The edges of the size range: no points (every cell start is 0) and
    exactly SPH_NOALLOC_MAX_POINTS points placed inside known cells (well
    away from cell faces), whose stable cell order is known here; the empty
    call leaves the order buffer untouched, the maximal one fills it."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    from paper_2510_25702_gb300 import build, sph

    build.build()
    L = sph.lib()
    case = cases.turbulent_channel(length=0.6, height=0.2, dp=0.005)
    cfg = sph.make_config(case)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cs = 2.0 * case.h
    nc = np.maximum(np.floor((case.hi - case.lo) / cs).astype(np.int64), 1)[:2]
    m = int(nc[0] * nc[1])
    ncell = C.c_int64()

    order = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    start = torch.full((m + 1,), -1, dtype=torch.int32, device="cuda")
    rc = L.sph_cell_sort_noalloc(C.byref(cfg), None, 0, order.data_ptr(), start.data_ptr(), m + 1,
                                 C.byref(ncell), stream)
    assert rc == 0 and ncell.value == m
    torch.cuda.synchronize()
    assert np.all(start.cpu().numpy() == 0)
    assert np.all(order.cpu().numpy() == -1)

    n = sph.NOALLOC_MAX_POINTS
    rng = np.random.default_rng(17)
    cells = rng.integers(0, nc, size=(n, 2))
    frac = rng.uniform(0.05, 0.95, size=(n, 2))
    pos = np.zeros((n, 3))
    pos[:, :2] = case.lo[:2] + (cells + frac) * cs
    keys = cells[:, 1] * nc[0] + cells[:, 0]
    d_pos = torch.from_numpy(pos).cuda()
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):  # twice: the second call starts from the first one's scratch
        rc = L.sph_cell_sort_noalloc(C.byref(cfg), d_pos.data_ptr(), n, order.data_ptr(), start.data_ptr(), m + 1,
                                     C.byref(ncell), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert np.array_equal(order.cpu().numpy().view(np.uint32), np.argsort(keys, kind="stable")), call
        expect_start = np.searchsorted(np.sort(keys), np.arange(m + 1), side="left")
        assert np.array_equal(start.cpu().numpy().view(np.uint32), expect_start), call
