"""The event voxel grid on the GPU against the oracle, bit for bit (needs a B300): random
records with skips and colour polarities, the device-side count, bin counts whose planes fill
one, two and eight groups of 256 planes (events whose two bins straddle a group boundary), a
1280-pixel-wide sensor next to small ones, and the grid of a synthesis step read in place
from the library's event buffer."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_08098_b300 import build
    build.build()
    import paper_2607_08098_b300 as m
    return m


def _records(rng, n, segs, junk_env=True):
    e = np.zeros(n, dtype=[("t", "<i8"), ("x", "<u2"), ("y", "<u2"), ("env", "<u2"), ("p", "<i2")])
    env = rng.integers(0, len(segs) + (1 if junk_env else 0), n)
    e["env"] = env
    for i, (W, H, t0, t1) in enumerate(segs + [(8, 8, 0, 1)]):
        m = env == i
        k = int(m.sum())
        e["t"][m] = rng.integers(t0 - (t1 - t0) // 20, t1 + (t1 - t0) // 20 + 1, k)
        e["x"][m] = rng.integers(0, W + 2, k)        # a few outside the sensor
        e["y"][m] = rng.integers(0, H, k)
    e["p"] = rng.choice([-3, -2, -1, 1, 2, 3], n)
    return e


@pytest.mark.parametrize("bins", [1, 7, 128, 129, 1024])
def test_voxel_grid_random_records(ev, oracle_mod, bins):
    rng = np.random.default_rng(bins)
    segs = [(64, 48, 1_000, 500_001_000), (37, 23, 0, 123_456_789), (1, 1, 5, 9), (346, 260, 0, 16_666_667)]
    rec = _records(rng, 400_000, segs)
    _, want = oracle_mod.voxel_grid(rec, segs, bins=bins)
    d = torch.from_numpy(rec.view(np.int64).reshape(-1)).cuda()
    got = ev.voxel_grid(d.data_ptr(), None, rec.size, segs, bins).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    # count on the device: only the first 250 000 records
    cnt = torch.tensor([250_000], dtype=torch.int64, device="cuda")
    _, want2 = oracle_mod.voxel_grid(rec[:250_000], segs, bins=bins)
    got2 = ev.voxel_grid(d.data_ptr(), cnt.data_ptr(), rec.size, segs, bins).cpu().numpy()
    np.testing.assert_array_equal(got2, want2)


def test_voxel_grid_large_planes(ev, oracle_mod):
    """A 1280 x 720 sensor (40 row segments per row) beside a small and a VGA one, in one
    call."""
    rng = np.random.default_rng(5)
    segs = [(1280, 720, 0, 50_000_000), (64, 48, 1_000, 2_001_000), (640, 480, 7, 99_999)]
    rec = _records(rng, 300_000, segs)
    _, want = oracle_mod.voxel_grid(rec, segs, bins=3)
    d = torch.from_numpy(rec.view(np.int64).reshape(-1)).cuda()
    got = ev.voxel_grid(d.data_ptr(), None, rec.size, segs, 3).cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_voxel_grid_of_a_synthesis_step(ev, oracle_mod, scenes_mod):
    """Events of two keyframe gaps of the 64 x 346x260 workload, gridded in place from the
    event buffer (device count) over each environment's 2-gap segment."""
    w = scenes_mod.config2(n_envs=16)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 26)
    for kf in kfs:
        ctx.step(torch.from_numpy(kf.L).cuda(), torch.from_numpy(kf.mv.reshape(-1)).cuda(),
                 torch.from_numpy(kf.Z).cuda(), w.dt_ns)
    segs = [(e.W, e.H, e.t0_ns, e.t0_ns + 2 * w.dt_ns) for e in w.envs]
    g1 = ctx.voxel_grid(segs, bins=128)
    g2 = ctx.voxel_grid(segs, bins=128)
    assert torch.equal(g1, g2)
    recs = ctx.read_events()
    assert len(recs) > 100_000
    _, want = oracle_mod.voxel_grid(recs, segs, bins=128)
    np.testing.assert_array_equal(g1.cpu().numpy(), want)
    ctx.close()


def test_voxel_grid_many_environments(ev, oracle_mod):
    """100 environments (more than the record passes stage in shared memory, so their
    descriptors are read from global memory), sizes from 1x1 to 40x33, ragged row segments."""
    rng = np.random.default_rng(11)
    segs = [(int(rng.integers(1, 41)), int(rng.integers(1, 34)), int(t0), int(t0) + int(rng.integers(1000, 10**8)))
            for t0 in rng.integers(0, 10**9, 100)]
    rec = _records(rng, 300_000, segs)
    _, want = oracle_mod.voxel_grid(rec, segs, bins=16)
    d = torch.from_numpy(rec.view(np.int64).reshape(-1)).cuda()
    got = ev.voxel_grid(d.data_ptr(), None, rec.size, segs, 16).cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_voxel_grid_without_records(ev, oracle_mod):
    """No records (max_events = 0, or a device count of 0): every plane is empty, so the
    grid is all zeros."""
    segs = [(64, 48, 0, 1_000_000), (37, 23, 5, 99)]
    d = torch.zeros(2 * 16, dtype=torch.int64, device="cuda")
    g0 = ev.voxel_grid(d.data_ptr(), None, 0, segs, 7)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    g1 = ev.voxel_grid(d.data_ptr(), cnt.data_ptr(), 16, segs, 7)
    assert g0.numel() == 2 * 7 * (64 * 48 + 37 * 23)
    assert not torch.any(g0) and not torch.any(g1)


def test_voxel_grid_into_a_grid_not_on_a_16_byte_boundary(ev, oracle_mod):
    """A grid pointer that is 4-byte but not 16-byte aligned (allowed by the header) takes the
    one-pixel-per-lane stores and gives the same grid."""
    import ctypes
    rng = np.random.default_rng(21)
    segs = [(64, 48, 1_000, 500_001_000), (640, 2, 0, 123_456_789)]
    bins = 8
    rec = _records(rng, 100_000, segs)
    _, want = oracle_mod.voxel_grid(rec, segs, bins=bins)
    d = torch.from_numpy(rec.view(np.int64).reshape(-1)).cuda()
    n_vox = sum(2 * bins * W * H for W, H, _, _ in segs)
    out = torch.zeros(n_vox + 4, dtype=torch.float32, device="cuda")
    wsb = ev.voxel_workspace_size(segs, bins, rec.size)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    arr = ev._voxel_envs(segs)
    st = ev.lib().evis_voxel_grid(d.data_ptr(), None, rec.size, ctypes.addressof(arr), len(segs), bins,
                                  ws.data_ptr(), wsb, out.data_ptr() + 4, None)
    assert st == ev.OK
    got = out[1:1 + n_vox].cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert out[0].item() == 0.0 and not torch.any(out[1 + n_vox:])
