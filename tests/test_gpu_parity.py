"""Parity of the CUDA path with the oracle, through the C ABI (needs a B300).

Bar (bit-exact unless stated): splat winners (z-buffer keys), interpolated log-intensity,
event streams in canonical order (env, t, y, x, p), reference levels, refractory times and
keyframe clocks.  The log conversion of linear inputs is the one step outside the exact
contract (CUDA logf vs the host log): it is checked within 2 ulp on its own.
"""
import numpy as np
import pytest

from evis_testutil import TinyEnv, packed_total

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).cuda()


def _frames(kf, mode, nc=1):
    if nc == 3:   # colour: three log-intensity planes, or linear RGB triples
        rgb = kf.rgb.reshape(-1, 3)
        if mode == 0:
            return np.concatenate([np.log(np.maximum(rgb[:, c] + 1e-4, 1e-30)).astype(np.float32)
                                   for c in range(3)])
        return kf.rgb.reshape(-1)
    if mode == 0:
        return kf.L
    if mode == 1:
        return kf.I
    return kf.rgb.reshape(-1)


def _trace_masks(envs, nc=1):
    """Sensor pixels (inside each environment's margin) of the trace layouts: keys
    [K][2][H*W] and interpolated L [K][nc][H*W] per environment, in order."""
    mk, ml = [], []
    for e in envs:
        m = int(getattr(e, "margin", 0))
        g = np.zeros((e.H, e.W), bool)
        g[m:e.H - m, m:e.W - m] = True
        g = g.ravel()
        mk.append(np.tile(g, 2 * e.K))
        ml.append(np.tile(g, e.K * nc))
    return np.concatenate(mk), np.concatenate(ml)


def run_both(ev, oracle_mod, envs, kfs, dt, flags=0, eps=1e-4, trace_steps=(), capacity=1 << 22,
             check_state=True, tile=None, noise=None):
    """Feed the same keyframes to the oracle and the library; compare everything."""
    mode = flags & 0x3
    nc = 3 if flags & 0x200 else 1
    o = oracle_mod.Oracle(envs, eps=eps, flags=flags & 0x2FF)
    ctx = ev.Context(envs, eps=eps, flags=flags, capacity=capacity)
    if tile is not None:
        ctx.set_tile_shape(*tile)
    if noise is not None:
        o.set_noise(noise)
        ctx.set_noise(noise)
    alive = []  # keeps inputs alive for EVIS_KEEP_INPUTS
    for s, kf in enumerate(kfs):
        fr = _frames(kf, mode, nc)
        g_in = (_dev(fr), _dev(kf.mv), _dev(kf.Z))
        alive.append(g_in)
        if s in trace_steps and s > 0:
            ok, ol = o.step(fr, kf.mv, kf.Z, dt, trace=True)
            gk, gl = ctx.step_trace(*g_in, dt)
            torch.cuda.synchronize()
            mk, ml = _trace_masks(envs, nc)   # with a margin only sensor pixels are traced
            gk = gk.cpu().numpy().view(np.uint64)[mk]
            gl = gl.cpu().numpy()[ml]
            ok, ol = ok[mk], ol[ml]
            bad = np.nonzero(gk != ok)[0]
            assert bad.size == 0, f"step {s}: {bad.size} splat keys differ, first at {bad[:5]}"
            np.testing.assert_array_equal(gl, ol, err_msg=f"step {s}: interpolated L")
        else:
            o.step(fr, kf.mv, kf.Z, dt)
            ctx.step(*g_in, dt)
        alive = alive[-2:]
    eo = oracle_mod.sort_events(o.events())
    eg = ev.sort_events(ctx.read_events())
    assert len(eg) == len(eo), (len(eg), len(eo))
    np.testing.assert_array_equal(eg.view(np.uint8), eo.view(np.uint8))
    if check_state:
        so, sg = o.state(), ctx.state()
        valid = np.zeros(o.total, dtype=bool)
        for e, off in zip(envs, o.offsets):
            m = int(getattr(e, "margin", 0))
            g = np.zeros((e.H, e.W), bool)
            g[m:e.H - m, m:e.W - m] = True
            valid[off:off + e.H * e.W] = g.ravel()
        valid = np.tile(valid, nc)   # state arrays hold nc planes
        np.testing.assert_array_equal(sg[0][valid], so[0][valid])
        if any(e.refractory_ns > 0 for e in envs):   # t_last is tracked only then
            np.testing.assert_array_equal(sg[1][valid], so[1][valid])
        else:
            assert np.all(sg[1] == np.iinfo(np.int64).min)
        np.testing.assert_array_equal(sg[2], so[2])
    ctx.close()
    return eo


def test_config1_plain_single_env(ev, oracle_mod, scenes_mod):
    """Plain single env 128x128, 10 frame pairs, K=8, C=0.2 -- the whole workload."""
    w = scenes_mod.config1()
    kfs = [scenes_mod.render(w.envs, k) for k in range(w.n_pairs + 1)]
    evs = run_both(ev, oracle_mod, w.envs, kfs, w.dt_ns, trace_steps=(1, 5, 10))
    assert len(evs) > 100_000


def _ragged_envs(scenes_mod):
    rng = np.random.default_rng(99)
    sizes = [(37, 23, 3, 0), (70, 41, 5, 300_000), (1, 1, 2, 0), (33, 1, 4, 0), (5, 40, 1, 0),
             (96, 64, 7, 50_000)]
    envs = []
    for i, (W, H, K, r) in enumerate(sizes):
        lay = scenes_mod._random_layers(rng, W, H, 3, vmax=6.0, wmax=0.1)
        e = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.15 + 0.01 * i, c_off=0.2, refractory_ns=r,
                                t0_ns=1000 * i, layers=lay)
        if i == 5:
            e.c_on_map = np.maximum(rng.normal(0.2, 0.03, W * H), 0.01).astype(np.float32)
            e.c_off_map = np.maximum(rng.normal(0.2, 0.03, W * H), 0.01).astype(np.float32)
        envs.append(e)
    return envs


@pytest.mark.parametrize("tile", [(32, 8), (32, 16), (32, 32), (64, 16), (64, 32), (128, 16)])
def test_ragged_multi_env(ev, oracle_mod, scenes_mod, tile):
    """Uneven sizes (1x1, single rows/columns, ragged tiles), per-env K, refractory, maps,
    for every tile shape of the synthesis kernel."""
    envs = _ragged_envs(scenes_mod)
    kfs = [scenes_mod.render(envs, k) for k in range(4)]
    run_both(ev, oracle_mod, envs, kfs, 16_666_667, trace_steps=(1, 2, 3), tile=tile)


def test_long_keyframe_gap_timestamps(ev, oracle_mod, scenes_mod):
    """Sub-frame intervals of 2^29 ns and more take the binary64 timestamp route, shorter ones
    the exact integer route; both must match the oracle's binary64 llrint."""
    w = scenes_mod.config1()
    envs = [scenes_mod.EnvScene(W=64, H=48, K=2, c_on=0.2, c_off=0.2, layers=w.envs[0].layers),
            scenes_mod.EnvScene(W=64, H=48, K=7, c_on=0.2, c_off=0.2, layers=w.envs[0].layers)]
    kfs = [scenes_mod.render(envs, k) for k in range(3)]
    run_both(ev, oracle_mod, envs, kfs, 3_000_000_001, trace_steps=(1,))


@pytest.mark.parametrize("flags", [0x10, 0x20, 0x30, 0x40, 0x60, 0x100, 0x110])
def test_modes(ev, oracle_mod, scenes_mod, flags):
    """B-primary blend, joint argmin, index-only tie-break and in-place (kept) inputs."""
    envs = _ragged_envs(scenes_mod)[:2] + _ragged_envs(scenes_mod)[5:]
    kfs = [scenes_mod.render(envs, k) for k in range(3)]
    run_both(ev, oracle_mod, envs, kfs, 16_666_667, flags=flags, trace_steps=(1, 2))


def test_adversarial_motion_and_depth(ev, oracle_mod):
    """NaN / inf / non-positive depths, NaN and huge motion vectors, exact half-pixel
    offsets and depth ties: winners, values and events still agree bit for bit."""
    rng = np.random.default_rng(5)
    envs = [TinyEnv(W=45, H=37, K=4, c_on=0.1, c_off=0.12, refractory_ns=10_000),
            TinyEnv(W=64, H=16, K=3, c_on=0.2, c_off=0.2)]
    n = packed_total(envs)

    class KF:
        pass

    kfs = []
    for _ in range(3):
        k = KF()
        mvc = np.array([0, 0.5, -0.5, 1, -1, 1.5, 2, -2.25, 0.25, 3, -7, 40, np.nan, 1e9],
                       dtype=np.float32)
        mv = rng.choice(mvc, size=(n, 2)).astype(np.float32)
        m = rng.random((n, 2)) < 0.5
        mv[m] = rng.uniform(-9, 9, size=m.sum()).astype(np.float32)
        zc = np.array([1, 2, 2, 3, 3, 3, 2.5, np.inf, np.nan, -1, 0], dtype=np.float32)
        z = rng.choice(zc, size=n).astype(np.float32)
        mz = rng.random(n) < 0.4
        z[mz] = rng.uniform(0.5, 4, size=mz.sum()).astype(np.float32)
        k.L = rng.normal(0, 1.5, size=n).astype(np.float32)
        k.mv, k.Z, k.I, k.rgb = mv, z, None, None
        kfs.append(k)
    run_both(ev, oracle_mod, envs, kfs, 5_000_000, trace_steps=(1, 2))


def test_statistics_count_sources_that_cannot_splat(ev, scenes_mod):
    """evis_get_stats: keyframes, gaps, and per environment the sources with depth not finite
    and > 0 or a non-finite motion vector, summed over the keyframes fed."""
    rng = np.random.default_rng(5)
    envs = [TinyEnv(W=40, H=30, K=2), TinyEnv(W=17, H=9, K=3)]
    n = packed_total(envs)
    ctx = ev.Context(envs, flags=ev.IN_LOG, capacity=1 << 16)
    assert ctx.stats()["keyframes"] == 0
    want = np.zeros(2, np.uint64)
    offs = [0, (40 * 30 + 3) // 4 * 4]
    for k in range(3):
        L = rng.normal(0, 1, n).astype(np.float32)
        mv = rng.normal(0, 2, (n, 2)).astype(np.float32)
        Z = rng.uniform(1, 5, n).astype(np.float32)
        bad = rng.random(n) < 0.1
        Z[bad] = rng.choice([0.0, -1.0, np.nan, np.inf], bad.sum())
        mvbad = rng.random(n) < 0.05
        mv[mvbad, 0] = np.nan
        for e, o in zip(envs, offs):
            m = slice(o, o + e.W * e.H)
            want[envs.index(e)] += np.sum(bad[m] | mvbad[m])
        ctx.step(_dev(L), _dev(mv), _dev(Z), 1_000_000)
    st = ctx.stats()
    assert st["keyframes"] == 3 and st["gaps"] == 2
    np.testing.assert_array_equal(st["invalid_sources"], want)
    ctx.close()


def test_misaligned_motion_vectors_are_rejected(ev, scenes_mod):
    """mv is read as float pairs: a pointer 4 bytes off an 8-byte boundary returns
    ERR_INVALID_ARG before any work, and the context steps on with aligned inputs."""
    rng = np.random.default_rng(6)
    envs = [TinyEnv(W=40, H=30, K=2)]
    n = packed_total(envs)
    L = _dev(rng.normal(0, 1, n).astype(np.float32))
    mv = torch.zeros(2 * n + 1, dtype=torch.float32, device="cuda")
    Z = _dev(rng.uniform(1, 5, n).astype(np.float32))
    ctx = ev.Context(envs, flags=ev.IN_LOG, capacity=1 << 16)
    ctx.step(L, mv[:2 * n], Z, 1_000_000)
    st = ev.lib().evis_step(ctx.handle, L.data_ptr(), mv.data_ptr() + 4, Z.data_ptr(), 1_000_000)
    assert st == ev.ERR_INVALID_ARG
    ctx.step(L, mv[:2 * n], Z, 1_000_000)
    assert ctx.stats()["gaps"] == 1
    ctx.close()


def test_wild_motion_overflows_candidate_lists(ev, oracle_mod):
    """Motion of up to +-300 px in every row segment: each tile's list of candidate source
    segments overflows and the kernel scans its whole source region instead."""
    rng = np.random.default_rng(11)
    envs = [TinyEnv(W=256, H=200, K=2, c_on=0.2, c_off=0.2)]
    n = packed_total(envs)

    class KF:
        pass

    kfs = []
    for _ in range(2):
        k = KF()
        k.mv = rng.uniform(-300, 300, size=(n, 2)).astype(np.float32)
        k.Z = rng.uniform(1, 5, size=n).astype(np.float32)
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        kfs.append(k)
    for tile in ((32, 16), (128, 16)):
        run_both(ev, oracle_mod, envs, kfs, 1_000_000, trace_steps=(1,), tile=tile)


@pytest.mark.parametrize("amp,tile", [(3.0, (64, 16)), (3.0, (64, 32)), (14.0, (128, 16)),
                                      (14.0, (32, 16))])
def test_splat_work_list_overflow(ev, oracle_mod, amp, tile):
    """Random per-pixel motion of +-amp px widens every segment's lane interval: at +-3 px on
    64-wide tiles the sources overflow the per-sub-frame item list into the per-segment
    overflow list; at +-14 px that list fills too and the kernel scans the region."""
    rng = np.random.default_rng(int(amp * 10) + tile[0])
    envs = [TinyEnv(W=200, H=120, K=3, c_on=0.2, c_off=0.2, refractory_ns=20_000)]
    n = packed_total(envs)

    class KF:
        pass

    kfs = []
    for _ in range(3):
        k = KF()
        k.mv = rng.uniform(-amp, amp, size=(n, 2)).astype(np.float32)
        k.Z = rng.uniform(1, 5, size=n).astype(np.float32)
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        kfs.append(k)
    run_both(ev, oracle_mod, envs, kfs, 1_000_000, trace_steps=(1, 2), tile=tile)


def test_static_scene_is_per_pixel_linear_esim(ev, oracle_mod):
    envs = [TinyEnv(W=50, H=30, K=8, c_on=0.2, c_off=0.2)]
    n = packed_total(envs)
    rng = np.random.default_rng(3)

    class KF:
        pass

    kfs = []
    for _ in range(4):
        k = KF()
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        k.mv = np.zeros((n, 2), dtype=np.float32)
        k.Z = np.ones(n, dtype=np.float32)
        kfs.append(k)
    run_both(ev, oracle_mod, envs, kfs, 10_000_000, trace_steps=(1, 3))


@pytest.mark.parametrize("tile", [(32, 16), (64, 16), (64, 32)])
def test_dense_crossings_overflow_the_event_stage(ev, oracle_mod, tile):
    """About 35 crossings per pixel and sub-frame (threshold 0.01 against unit-variance jumps):
    every tile-sub-frame stages far more events than the CTA's shared buffer holds, so most
    chunks go to global memory one warp reservation at a time, each warp's row needs many
    chunks, and the refractory period (100 us against crossings about 70 us apart) sends
    chunks to the per-pixel walk."""
    envs = [TinyEnv(W=70, H=35, K=4, c_on=0.01, c_off=0.012, refractory_ns=100_000)]
    n = packed_total(envs)
    rng = np.random.default_rng(11)

    class KF:
        pass

    kfs = []
    for _ in range(4):
        k = KF()
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        k.mv = np.zeros((n, 2), dtype=np.float32)
        k.Z = np.ones(n, dtype=np.float32)
        kfs.append(k)
    evs = run_both(ev, oracle_mod, envs, kfs, 10_000_000, trace_steps=(2,), tile=tile)
    assert len(evs) > 200_000


def test_constant_image_emits_nothing(ev, scenes_mod):
    w = scenes_mod.config2(n_envs=4)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG)
    for kf in kfs:
        ctx.step(_dev(np.full_like(kf.L, 0.3)), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    assert ctx.event_count() == 0


@pytest.mark.parametrize("mode", [1, 2])
def test_log_intensity_within_two_ulp(ev, oracle_mod, mode):
    rng = np.random.default_rng(8)
    n = 200_000
    x = (10.0 ** rng.uniform(-6, 6, size=n * (3 if mode == 2 else 1))).astype(np.float32)
    x[:8] = [0, -1, np.nan, np.inf, 1e-30, 1, 1e-4, 3.4e38]
    got = ev.log_intensity(_dev(x), mode=mode, eps=1e-4).cpu().numpy()
    want = oracle_mod.log_intensity(x, mode=mode, eps=1e-4)
    fin = np.isfinite(want)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ulp = np.spacing(np.abs(want[fin]).astype(np.float32))
    assert np.all(np.abs(got[fin] - want[fin]) <= 2 * ulp)


@pytest.mark.parametrize("mode", [1, 2])
def test_linear_inputs_end_to_end(ev, oracle_mod, scenes_mod, mode):
    """Linear / RGB radiance inputs.  The GPU log may differ from the host one by an ulp, which
    can move an interpolated timestamp by a few ns or, rarely, a crossing across a sub-frame
    boundary, so the streams are compared per pixel: >= 99.5 % of pixels with the same event
    count and polarities, and their timestamps within 1 ns at the median and 100 ns at the
    99th percentile."""
    w = scenes_mod.config1()
    for lay in w.envs[0].layers:
        lay.tint_r, lay.tint_g, lay.tint_b = 0.9, 1.1, 0.7
    kfs = [scenes_mod.render(w.envs, k, want=("L", "I", "rgb", "mv", "Z")) for k in range(4)]
    o = oracle_mod.Oracle(w.envs, eps=1e-4, flags=mode)
    ctx = ev.Context(w.envs, eps=1e-4, flags=mode)
    for kf in kfs:
        fr = _frames(kf, mode)
        o.step(fr, kf.mv, kf.Z, w.dt_ns)
        ctx.step(_dev(fr), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    _per_pixel_close(o.events(), ctx.read_events())


def _per_pixel_close(eo, eg):
    """Event streams that may differ where the log of linear input differs by an ulp: event
    totals within 0.2 %, >= 99.5 % of pixels with the same count and polarities, and their
    timestamps within 1 ns at the median and 100 ns at the 99th percentile."""
    assert len(eo) > 0 and abs(len(eg) - len(eo)) <= 0.002 * len(eo)

    def key(e):
        return (e["env"].astype(np.int64) << 32) | (e["y"].astype(np.int64) << 16) | e["x"]

    keys = np.union1d(key(eo), key(eg))

    def by_pixel(e):
        pix = np.searchsorted(keys, key(e))
        order = np.lexsort((e["t"], pix))
        return pix[order], e[order], np.bincount(pix, minlength=keys.size)

    po, so, co = by_pixel(eo)
    pg, sg, cg = by_pixel(eg)
    same = co == cg
    assert same.mean() >= 0.995
    ko, kg = same[po], same[pg]
    assert np.array_equal(so["p"][ko], sg["p"][kg])
    dt = np.abs(so["t"][ko] - sg["t"][kg])
    assert np.median(dt) <= 1 and np.percentile(dt, 99) <= 100


def test_step_host_matches_device_step(ev, scenes_mod):
    w = scenes_mod.config2(n_envs=3)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    a = ev.Context(w.envs, flags=ev.IN_LUM, capacity=1 << 24)
    b = ev.Context(w.envs, flags=ev.IN_LUM | ev.KEEP_INPUTS, capacity=1 << 24)
    alive = []
    for kf in kfs:
        g = (_dev(kf.I), _dev(kf.mv), _dev(kf.Z))
        alive = (alive + [g])[-2:]
        a.step(*g, w.dt_ns)
        b.step_host(kf.I, kf.mv, kf.Z, w.dt_ns)
    ea, eb = ev.sort_events(a.read_events()), ev.sort_events(b.read_events())
    assert len(ea) > 0
    np.testing.assert_array_equal(ea.view(np.uint8), eb.view(np.uint8))


def test_overflow_reports_total_and_keeps_state(ev, oracle_mod, scenes_mod):
    w = scenes_mod.config1()
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    o = oracle_mod.Oracle(w.envs)
    ctx = ev.Context(w.envs, capacity=5000)
    for kf in kfs:
        o.step(kf.L, kf.mv, kf.Z, w.dt_ns)
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    eo = o.events()
    got, produced = ctx.read_events(allow_overflow=True)
    assert produced == len(eo) > 5000 and len(got) == 5000
    so = set(map(bytes, eo.view(np.dtype((np.void, 16)))))
    assert all(bytes(r) in so for r in got.view(np.dtype((np.void, 16))))
    np.testing.assert_array_equal(ctx.state()[0], o.state()[0])
    assert ctx.event_count() == 0        # the read emptied the buffer
    kf = scenes_mod.render(w.envs, 3)
    ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    o.step(kf.L, kf.mv, kf.Z, w.dt_ns)
    assert ctx.event_count() == len(o.events())


def _subset(ev, oracle_mod, envs, kfs, dt, sample, flags=0, noise=None):
    """Oracle on a sample of environments (re-packed), for comparison with a full-size run.
    Noise seeds are remapped so that sampled environment j draws environment i's stream
    (the generator's key mixes the environment index into the seed's high word)."""
    import scenes
    sub = [envs[i] for i in sample]
    off, _ = scenes.pixel_offsets(envs)
    soff, stotal = scenes.pixel_offsets(sub)
    o = oracle_mod.Oracle(sub, flags=flags)
    if noise is not None:
        o.set_noise([dict(noise[i], seed=int(noise[i].get("seed", 0)) ^ ((i ^ j) << 32))
                     for j, i in enumerate(sample)])
    for kf in kfs:
        L = np.zeros(stotal, np.float32)
        mv = np.zeros((stotal, 2), np.float32)
        Z = np.ones(stotal, np.float32)
        for j, i in enumerate(sample):
            n = envs[i].H * envs[i].W
            L[soff[j]:soff[j] + n] = kf.L[off[i]:off[i] + n]
            mv[soff[j]:soff[j] + n] = kf.mv[off[i]:off[i] + n]
            Z[soff[j]:soff[j] + n] = kf.Z[off[i]:off[i] + n]
        o.step(L, mv, Z, dt)
    return o, off, soff


def test_config2_full_size_sampled(ev, oracle_mod, scenes_mod):
    """64 envs at 346x260, K=16, C=0.25, refractory 100 us -- the benchmarked launch -- with
    the oracle on three sampled environments."""
    w = scenes_mod.config2()
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 27)
    for kf in kfs:
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    eg = ctx.read_events()
    Lref, tl, clk = ctx.state()
    sample = [0, 31, 63]
    o, off, soff = _subset(ev, oracle_mod, w.envs, kfs, w.dt_ns, sample)
    eo = oracle_mod.sort_events(o.events())
    so = o.state()
    for j, i in enumerate(sample):
        mine = eg[eg["env"] == i].copy()
        mine["env"] = j
        theirs = eo[eo["env"] == j]
        mine = ev.sort_events(mine)
        assert len(mine) == len(theirs) > 1000
        np.testing.assert_array_equal(mine.view(np.uint8), theirs.view(np.uint8))
        n = w.envs[i].H * w.envs[i].W
        np.testing.assert_array_equal(Lref[off[i]:off[i] + n], so[0][soff[j]:soff[j] + n])
        np.testing.assert_array_equal(tl[off[i]:off[i] + n], so[1][soff[j]:soff[j] + n])
        assert clk[i] == so[2][j]


def test_determinism(ev, scenes_mod):
    w = scenes_mod.config2(n_envs=8)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    outs = []
    for _ in range(2):
        ctx = ev.Context(w.envs, capacity=1 << 24)
        for kf in kfs:
            ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
        outs.append(ev.sort_events(ctx.read_events()))
    np.testing.assert_array_equal(outs[0].view(np.uint8), outs[1].view(np.uint8))


def test_high_speed_full_size_sampled(ev, oracle_mod, scenes_mod):
    """High-speed workload at full per-environment size (640x480, K=32, C=0.15, flows up to
    40 px/frame, ~10 % holes), 8 environments on the GPU, two of them against the oracle."""
    w = scenes_mod.config4(n_envs=8)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 26)
    for kf in kfs:
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    eg = ctx.read_events()
    Lref, _, clk = ctx.state()
    sample = [0, 5]
    o, off, soff = _subset(ev, oracle_mod, w.envs, kfs, w.dt_ns, sample)
    eo = oracle_mod.sort_events(o.events())
    so = o.state()
    for j, i in enumerate(sample):
        mine = eg[eg["env"] == i].copy()
        mine["env"] = j
        mine = ev.sort_events(mine)
        theirs = eo[eo["env"] == j]
        assert len(mine) == len(theirs) > 10000
        np.testing.assert_array_equal(mine.view(np.uint8), theirs.view(np.uint8))
        n = w.envs[i].H * w.envs[i].W
        np.testing.assert_array_equal(Lref[off[i]:off[i] + n], so[0][soff[j]:soff[j] + n])
        assert clk[i] == so[2][j]


def _noise_specs(n):
    """All three noise sources at rates that fire often, one environment without noise, and
    environments sharing a seed (their streams still differ by the environment index)."""
    out = []
    for i in range(n):
        if i == 1:
            out.append({})
        else:
            out.append(dict(leak_hz=40.0 + 10.0 * i, shot_hz=80.0, hot_hz=300.0, hot_fraction=0.03,
                            lo=-3.0, hi=3.0, seed=0x1234_5678_9ABC + (i % 3)))
    return out


@pytest.mark.parametrize("tile", [(32, 8), (32, 16), (32, 32), (64, 16), (64, 32), (128, 16)])
def test_noise_ragged_multi_env(ev, oracle_mod, scenes_mod, tile):
    """Leak, shot and hot-pixel events (Sec. 3.4) with the signal events, refractory periods
    and threshold maps of the ragged set, through the production and the trace kernels."""
    envs = _ragged_envs(scenes_mod)
    kfs = [scenes_mod.render(envs, k) for k in range(4)]
    evs = run_both(ev, oracle_mod, envs, kfs, 16_666_667, trace_steps=(1, 3), tile=tile,
                   noise=_noise_specs(len(envs)))
    assert len(evs) > 1000


@pytest.mark.parametrize("flags", [0x10, 0x40])
def test_noise_modes(ev, oracle_mod, scenes_mod, flags):
    """Shot noise reads the blended sample, so the blend modes change it."""
    envs = _ragged_envs(scenes_mod)[:2] + _ragged_envs(scenes_mod)[5:]
    kfs = [scenes_mod.render(envs, k) for k in range(3)]
    run_both(ev, oracle_mod, envs, kfs, 16_666_667, flags=flags, noise=_noise_specs(len(envs)))


def test_noise_sub_frames_longer_than_2_32_ns(ev, oracle_mod, scenes_mod):
    """Noise times t_{i-1} + floor(u d / 2^32) with d above 2^32 (the high word of d)."""
    w = scenes_mod.config1()
    envs = [scenes_mod.EnvScene(W=40, H=24, K=1, c_on=0.2, c_off=0.2, layers=w.envs[0].layers),
            scenes_mod.EnvScene(W=40, H=24, K=3, c_on=0.2, c_off=0.2, layers=w.envs[0].layers)]
    kfs = [scenes_mod.render(envs, k) for k in range(3)]
    noise = [dict(leak_hz=0.05, shot_hz=0.1, hot_hz=0.2, hot_fraction=0.1, seed=3)] * 2
    evs = run_both(ev, oracle_mod, envs, kfs, (1 << 33) + 12345, noise=noise)
    assert np.sum(evs["t"] > (1 << 32)) > 100


def test_noise_graph_replay_and_switching(ev, oracle_mod, scenes_mod):
    """The gap counter lives on the device, so replayed gaps draw fresh noise like stepped
    ones; set_noise drops the captured graph; None turns noise off."""
    envs = _ragged_envs(scenes_mod)
    kfs = [scenes_mod.render(envs, k) for k in range(5)]
    noise = _noise_specs(len(envs))
    o = oracle_mod.Oracle(envs)
    o.set_noise(noise)
    for kf in kfs:
        o.step(kf.L, kf.mv, kf.Z, 16_666_667)
    want = oracle_mod.sort_events(o.events())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = ev.Context(envs, capacity=1 << 22, stream=stream)
        ctx.set_noise(noise)
        ctx.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), 16_666_667)
        ctx.step(_dev(kfs[1].L), _dev(kfs[1].mv), _dev(kfs[1].Z), 16_666_667)
        ctx.capture(16_666_667)
        for kf in kfs[2:]:
            ctx.write_inputs(_dev(kf.L), _dev(kf.mv), _dev(kf.Z))
            ctx.replay()
        got = ev.sort_events(ctx.read_events())
        np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
        ctx.set_noise(None)
        with pytest.raises(ev.EvisError):
            ctx.replay()
        with pytest.raises(ev.EvisError):
            ctx.set_noise([dict(hot_fraction=1.5)] * len(envs))
        with pytest.raises(ev.EvisError):
            ctx.set_noise([dict(leak_hz=float("inf"))] * len(envs))
        with pytest.raises(ev.EvisError):
            ctx.set_noise([dict(lo=1.0, hi=1.0)] * len(envs))
        ctx.close()
    # off again: the plain event stream
    run_both(ev, oracle_mod, envs, kfs[:3], 16_666_667, noise=[{}] * len(envs))


def test_noise_high_speed_full_size_sampled(ev, oracle_mod, scenes_mod):
    """All noise sources on the 8-env high-speed workload at full size, in the persistent
    autotuned launch with caller-kept inputs; two environments against the oracle."""
    w = scenes_mod.config4(n_envs=8)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    noise = [dict(leak_hz=2.0, shot_hz=5.0, hot_hz=50.0, hot_fraction=0.01, lo=-1.0, hi=5.0,
                  seed=77)] * len(w.envs)
    ctx = ev.Context(w.envs, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=1 << 26)
    ctx.set_noise(noise)
    g = [(_dev(kf.L), _dev(kf.mv), _dev(kf.Z)) for kf in kfs]
    ctx.step(*g[0], w.dt_ns)
    ctx.autotune(*g[1], w.dt_ns, reps=1)
    for t in g[1:]:
        ctx.step(*t, w.dt_ns)
    eg = ctx.read_events()
    ctx.close()
    sample = [0, 5]
    o, _, _ = _subset(ev, oracle_mod, w.envs, kfs, w.dt_ns, sample, noise=noise)
    eo = oracle_mod.sort_events(o.events())
    for j, i in enumerate(sample):
        mine = eg[eg["env"] == i].copy()
        mine["env"] = j
        mine = ev.sort_events(mine)
        theirs = eo[eo["env"] == j]
        assert len(mine) == len(theirs) > 10000
        np.testing.assert_array_equal(mine.view(np.uint8), theirs.view(np.uint8))


@pytest.mark.parametrize("tile", [(32, 16), (64, 32), (128, 16)])
def test_margin_crop(ev, oracle_mod, scenes_mod, tile):
    """Over-render margins (Appendix B) of 0..9 pixels, including a sensor one pixel wide and
    tails of every tile, with refractory periods, maps and noise drawn per sensor pixel."""
    envs = _ragged_envs(scenes_mod)
    margins = [3, 0, 0, 0, 2, 9]         # (37x23, 70x41, 1x1, 33x1, 5x40, 96x64)
    for e, m in zip(envs, margins):
        e.margin = m
    envs[0].margin = 11                  # 37x23 -> a 15x1 sensor
    kfs = [scenes_mod.render(envs, k) for k in range(4)]
    noise = [dict(leak_hz=30.0, hot_hz=200.0, hot_fraction=0.05, shot_hz=50.0, seed=9)] * len(envs)
    evs = run_both(ev, oracle_mod, envs, kfs, 16_666_667, trace_steps=(1, 3), tile=tile, noise=noise)
    for e in envs:
        m = e.margin
        sel = evs[evs["env"] == envs.index(e)]
        assert np.all(sel["x"] < e.W - 2 * m) and np.all(sel["y"] < e.H - 2 * m)


@pytest.mark.parametrize("mode", [1, 2])
def test_defocus_plane_bit_exact(ev, oracle_mod, mode):
    """The defocus kernel (Sec. 3.4) against the oracle's blur, bit for bit: single pixels,
    single rows and columns, tile tails, a radius (sigma 8: 24 px) wider than the image."""
    rng = np.random.default_rng(21)
    for H, W in [(1, 1), (1, 37), (29, 1), (8, 32), (37, 53), (260, 346)]:
        for sigma in (0.0, 0.3, 0.5, 1.3, 8.0):
            shape = (H, W, 3) if mode == 2 else (H, W)
            img = rng.uniform(0.0, 5.0, shape).astype(np.float32)
            got = ev.defocus(torch.from_numpy(img).cuda(), sigma).cpu().numpy()
            lum = img if mode == 1 else oracle_mod.rec709(img.reshape(-1, 3)).reshape(H, W)
            np.testing.assert_array_equal(got, oracle_mod.defocus(lum, sigma),
                                          err_msg=f"{H}x{W} sigma {sigma}")


@pytest.mark.parametrize("mode", [1, 2])
def test_defocus_in_the_pipeline(ev, oracle_mod, scenes_mod, mode):
    """Per-environment defocus before the log: (a) exactly the events of a plain luminance
    context fed the GPU-blurred keyframes; (b) the oracle's defocused events per pixel, up
    to the log's ulp."""
    envs = _ragged_envs(scenes_mod)
    sig = [0.5, 0.0, 1.5, 0.3, 8.0, 0.8]
    kfs = [scenes_mod.render(envs, k, want=("I", "rgb", "mv", "Z")) for k in range(4)]
    dt = 16_666_667
    a = ev.Context(envs, flags=mode, capacity=1 << 22)
    a.set_defocus(sig)
    b = ev.Context(envs, flags=ev.IN_LUM, capacity=1 << 22)
    o = oracle_mod.Oracle(envs, flags=mode)
    o.set_defocus(sig)
    off = o.offsets
    for kf in kfs:
        fr = _frames(kf, mode)
        a.step(_dev(fr), _dev(kf.mv), _dev(kf.Z), dt)
        o.step(fr, kf.mv, kf.Z, dt)
        pre = torch.zeros(kf.I.size, dtype=torch.float32, device="cuda")
        for e, s_, ofs in zip(envs, sig, off):
            n = e.W * e.H
            plane = (fr[ofs:ofs + n].reshape(e.H, e.W) if mode == 1
                     else fr.reshape(-1, 3)[ofs:ofs + n].reshape(e.H, e.W, 3))
            pre[ofs:ofs + n] = ev.defocus(torch.from_numpy(np.ascontiguousarray(plane)).cuda(), s_).reshape(-1)
        b.step(pre, _dev(kf.mv), _dev(kf.Z), dt)
    ga, gb = ev.sort_events(a.read_events()), ev.sort_events(b.read_events())
    assert len(ga) > 1000
    np.testing.assert_array_equal(ga.view(np.uint8), gb.view(np.uint8))
    _per_pixel_close(o.events(), ga)
    with pytest.raises(ev.EvisError):
        a.set_defocus([9.0] * len(envs))
    with pytest.raises(ev.EvisError):
        ev.Context(envs, flags=ev.IN_LOG).set_defocus(sig)


def _tint(envs, seed=31):
    rng = np.random.default_rng(seed)
    for e in envs:
        for lay in e.layers:
            lay.tint_r, lay.tint_g, lay.tint_b = rng.uniform(0.3, 1.6, 3)
    return envs


@pytest.mark.parametrize("tile", [(32, 8), (32, 16), (32, 32), (64, 16), (64, 32), (128, 16)])
def test_colour_planes_exact(ev, oracle_mod, scenes_mod, tile):
    """Colour events (Sec. 3.2) from three log-intensity planes: bit-exact events, traced
    winners and per-channel log-intensity, per-channel reference levels and refractory
    times, with noise, refractory periods, maps and margins, on every tile shape."""
    envs = _tint(_ragged_envs(scenes_mod))
    envs[5].margin = 3
    kfs = [scenes_mod.render(envs, k, want=("rgb", "mv", "Z")) for k in range(4)]
    noise = [dict(leak_hz=30.0, hot_hz=200.0, hot_fraction=0.05, shot_hz=50.0, lo=-3.0, hi=3.0,
                  seed=17)] * len(envs)
    evs = run_both(ev, oracle_mod, envs, kfs, 16_666_667, flags=ev.IN_LOG | ev.COLOR,
                   trace_steps=(1, 3), tile=tile, noise=noise)
    ch = np.abs(evs["p"])
    assert set(np.unique(ch)) == {1, 2, 3} and len(evs) > 3000


@pytest.mark.parametrize("flags", [0x10, 0x40, 0x100])
def test_colour_modes(ev, oracle_mod, scenes_mod, flags):
    envs = _tint(_ragged_envs(scenes_mod)[4:])
    kfs = [scenes_mod.render(envs, k, want=("rgb", "mv", "Z")) for k in range(3)]
    run_both(ev, oracle_mod, envs, kfs, 16_666_667, flags=ev.IN_LOG | ev.COLOR | flags,
             trace_steps=(2,))


def test_colour_linear_rgb_and_defocus(ev, oracle_mod, scenes_mod):
    """Linear RGB in colour mode: (a) exactly the events of a planar-log colour context fed
    the GPU's per-channel logs, with and without per-channel defocus; (b) the oracle's events
    per pixel, up to the log's ulp."""
    envs = _tint(_ragged_envs(scenes_mod))
    kfs = [scenes_mod.render(envs, k, want=("rgb", "mv", "Z")) for k in range(3)]
    dt = 16_666_667
    for sig in (None, [0.6, 0.0, 1.2, 0.4, 2.0, 0.8]):
        a = ev.Context(envs, flags=ev.IN_RGB | ev.COLOR, capacity=1 << 22)
        b = ev.Context(envs, flags=ev.IN_LOG | ev.COLOR, capacity=1 << 22)
        o = oracle_mod.Oracle(envs, flags=oracle_mod.IN_RGB | oracle_mod.COLOR)
        if sig is not None:
            a.set_defocus(sig)
            o.set_defocus(sig)
        keep = []
        for kf in kfs:
            rgb = kf.rgb.reshape(-1, 3)
            a.step(_dev(rgb), _dev(kf.mv), _dev(kf.Z), dt)
            o.step(rgb.reshape(-1), kf.mv, kf.Z, dt)
            planes = torch.zeros(3 * rgb.shape[0], dtype=torch.float32, device="cuda")
            n_tot = rgb.shape[0]
            for c in range(3):
                lin = torch.from_numpy(np.ascontiguousarray(rgb[:, c])).cuda()
                if sig is not None:
                    for e, s_, ofs in zip(envs, sig, o.offsets):
                        n = e.W * e.H
                        lin[ofs:ofs + n] = ev.defocus(lin[ofs:ofs + n].reshape(e.H, e.W).contiguous(),
                                                      s_).reshape(-1)
                planes[c * n_tot:(c + 1) * n_tot] = ev.log_intensity(lin, mode=ev.IN_LUM, eps=1e-4)
            keep.append(planes)
            b.step(planes, _dev(kf.mv), _dev(kf.Z), dt)
        ga, gb = ev.sort_events(a.read_events()), ev.sort_events(b.read_events())
        assert len(ga) > 1000
        np.testing.assert_array_equal(ga.view(np.uint8), gb.view(np.uint8))
        real = np.zeros(o.total, dtype=bool)   # packing pads hold no pixel
        for e, ofs in zip(envs, o.offsets):
            real[ofs:ofs + e.W * e.H] = True
        np.testing.assert_array_equal(a.state()[0][np.tile(real, 3)], b.state()[0][np.tile(real, 3)])
        eo = o.events()
        for c in range(3):
            _per_pixel_close(eo[np.abs(eo["p"]) == c + 1], ga[np.abs(ga["p"]) == c + 1])
    with pytest.raises(ev.EvisError):
        ev.Context(envs, flags=ev.IN_LUM | ev.COLOR)


@pytest.mark.parametrize("flags", [0x0, 0x200])
def test_checkpoint_resume(ev, oracle_mod, scenes_mod, flags):
    """State get/set: a context resumed from a checkpoint (state, clocks and noise gap
    counters, after re-feeding the retained keyframe) continues exactly like the
    uninterrupted one, in mono and colour mode, with noise and refractory periods."""
    envs = _tint(_ragged_envs(scenes_mod))
    kfs = [scenes_mod.render(envs, k, want=("L", "rgb", "mv", "Z")) for k in range(6)]
    noise = [dict(leak_hz=30.0, hot_hz=200.0, hot_fraction=0.05, shot_hz=50.0, seed=4)] * len(envs)
    dt = 16_666_667

    def fr(kf):   # log-intensity input: one plane, or three in colour mode
        return _dev(_frames(kf, 0, 3 if flags & 0x200 else 1))

    full = ev.Context(envs, flags=flags, capacity=1 << 22)
    full.set_noise(noise)
    for kf in kfs[:3]:
        full.step(fr(kf), _dev(kf.mv), _dev(kf.Z), dt)
    full.read_events()
    Lref, tl, clk = full.state()
    gaps = full.gaps()
    assert np.all(gaps == 2)
    for kf in kfs[3:]:
        full.step(fr(kf), _dev(kf.mv), _dev(kf.Z), dt)
    want = ev.sort_events(full.read_events())
    want_state = full.state()
    res = ev.Context(envs, flags=flags, capacity=1 << 22)
    res.set_noise(noise)
    with pytest.raises(ev.EvisError):
        res.set_state(Lref=Lref)            # no retained keyframe yet
    res.step(fr(kfs[2]), _dev(kfs[2].mv), _dev(kfs[2].Z), dt)
    res.read_events()
    res.set_state(Lref=Lref, t_last=tl, clocks=clk, gaps=gaps)
    for kf in kfs[3:]:
        res.step(fr(kf), _dev(kf.mv), _dev(kf.Z), dt)
    got = ev.sort_events(res.read_events())
    assert len(want) > 1000
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    for a, b in zip(res.state(), want_state):
        np.testing.assert_array_equal(a, b)
    full.close()
    res.close()


@pytest.mark.parametrize("tile", [(32, 16), (128, 16)])
def test_extreme_shapes_and_long_k(ev, oracle_mod, tile):
    """The size limits: a 65535-pixel-wide strip, a 65535-pixel-tall column (16-bit event
    coordinates, 2048 row segments per row, a tile column at x0 = 65504), one pixel with
    K = 700 sub-frames and a 4x3 image with K = 257, with motion, holes and refractory."""
    rng = np.random.default_rng(42)
    envs = [TinyEnv(W=65535, H=2, K=2, c_on=0.15, c_off=0.15, refractory_ns=1000),
            TinyEnv(W=3, H=65535, K=3, c_on=0.15, c_off=0.15),
            TinyEnv(W=1, H=1, K=700, c_on=0.01, c_off=0.01),
            TinyEnv(W=4, H=3, K=257, c_on=0.05, c_off=0.05, refractory_ns=30_000)]
    n = packed_total(envs)

    class KF:
        pass

    kfs = []
    for _ in range(3):
        k = KF()
        k.mv = rng.uniform(-2.5, 2.5, size=(n, 2)).astype(np.float32)
        k.Z = rng.uniform(1, 5, size=n).astype(np.float32)
        k.Z[rng.random(n) < 0.02] = 0.0
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        kfs.append(k)
    evs = run_both(ev, oracle_mod, envs, kfs, 16_666_667, trace_steps=(2,), tile=tile,
                   capacity=1 << 23)
    assert evs["x"].max() >= 65000 and evs["y"].max() >= 65000


def test_noise_with_long_k(ev, oracle_mod):
    """Sensor noise over K = 700, 257 and 300 sub-frames: the noise kernel's per-sub-frame
    constants come in chunks of 256, and the last block of four sub-frames is partial."""
    rng = np.random.default_rng(43)
    envs = [TinyEnv(W=1, H=1, K=700, c_on=0.05, c_off=0.05),
            TinyEnv(W=4, H=3, K=257, c_on=0.05, c_off=0.05, refractory_ns=30_000),
            TinyEnv(W=300, H=5, K=300, c_on=0.2, c_off=0.2)]
    n = packed_total(envs)

    class KF:
        pass

    kfs = []
    for _ in range(3):
        k = KF()
        k.mv = rng.uniform(-2.5, 2.5, size=(n, 2)).astype(np.float32)
        k.Z = rng.uniform(1, 5, size=n).astype(np.float32)
        k.L = rng.normal(0, 1, size=n).astype(np.float32)
        kfs.append(k)
    noise = [dict(leak_hz=200.0, shot_hz=400.0, hot_hz=900.0, hot_fraction=0.2, lo=-2.0, hi=2.0,
                  seed=77 + i) for i in range(3)]
    evs = run_both(ev, oracle_mod, envs, kfs, 16_666_667, noise=noise, capacity=1 << 22)
    assert len(evs) > 1000


@pytest.mark.parametrize("tile", [(32, 16), (64, 16), (32, 8)])
def test_crossing_limit_is_reported(ev, oracle_mod, tile):
    """Pixel-sub-frames whose Eq. 4 count n exceeds the per-pixel emission limit (4096):
    none of their crossings is emitted, the reference still moves by the whole p n C, the
    read reports ERR_RANGE (with every other event delivered), env_stats counts them per
    environment, and all of it equals the oracle bit for bit (refractory period on, an
    infinite and a NaN outcome included)."""
    C = 0.25
    envs = [TinyEnv(W=70, H=37, K=3, c_on=C, c_off=0.3, refractory_ns=30_000),
            TinyEnv(W=33, H=20, K=2, c_on=C, c_off=C)]
    n = packed_total(envs)
    rng = np.random.default_rng(21)
    lim = ev.MAX_CROSSINGS

    class KF:
        pass

    kfs = []
    for s in range(3):
        k = KF()
        k.L = rng.normal(0, 1, n).astype(np.float32)
        big = rng.random(n) < 0.04
        k.L[big] = np.float32((3 * (lim + 1) + 1.5) * C) * rng.choice([-1, 1], big.sum())
        k.L[rng.random(n) < 0.002] = np.float32(3e38)
        k.mv = np.zeros((n, 2), np.float32)
        k.Z = np.ones(n, np.float32)
        kfs.append(k)
    o = oracle_mod.Oracle(envs, flags=oracle_mod.IN_LOG)
    ctx = ev.Context(envs, flags=ev.IN_LOG | (ev.STATS if tile == (32, 16) else 0),
                     capacity=1 << 22)
    ctx.set_tile_shape(*tile)
    for s, k in enumerate(kfs):
        o.step(k.L, k.mv, k.Z, 1_000_000)
        ctx.step(_dev(k.L), _dev(k.mv), _dev(k.Z), 1_000_000)
        if s == 0:
            continue
        assert o.last_over_limit
        with pytest.raises(ev.EvisError) as ei:
            ctx.read_events()
        assert ei.value.status == ev.ERR_RANGE
        got = ev.sort_events(ei.value.events)
        want = oracle_mod.sort_events(o.events())
        assert len(got) == len(want) > 1000
        np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
        np.testing.assert_array_equal(ctx.env_stats()["over_limit"], o.over_limit())
    so, sg = o.state(), ctx.state()
    np.testing.assert_array_equal(sg[0], so[0])      # NaN where Eq. 4 met inf - inf
    np.testing.assert_array_equal(sg[1], so[1])
    # a gap without such pixels reads OK again
    k = kfs[-1]
    o.step(k.L, k.mv, k.Z, 1_000_000)
    ctx.step(_dev(k.L), _dev(k.mv), _dev(k.Z), 1_000_000)
    if not o.last_over_limit:
        assert len(ctx.read_events()) == len(o.events())
    ctx.close()


def test_env_stats_holes_polarity_and_noise(ev, oracle_mod, scenes_mod):
    """evis_get_env_stats against counts taken from the oracle: holes per warp direction and
    of both from its traced z-buffers (sensor pixels inside a margin), ON / OFF events from
    its stream, noise events as the difference to a noise-free oracle run."""
    w = scenes_mod.config4(n_envs=3, W=200, H=150)
    for e in w.envs:
        e.K, e.margin = 8, 5
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    noise = [dict(leak_hz=60.0, shot_hz=90.0, hot_hz=200.0, hot_fraction=0.02, lo=-3.0, hi=3.0,
                  seed=77 + i) for i in range(len(w.envs))]
    o = oracle_mod.Oracle(w.envs, flags=oracle_mod.IN_LOG)
    o.set_noise(noise)
    quiet = oracle_mod.Oracle(w.envs, flags=oracle_mod.IN_LOG)
    ctx = ev.Context(w.envs, flags=ev.IN_LOG | ev.STATS, capacity=1 << 23)
    ctx.set_noise(noise)
    plain = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 23)   # statistics off
    plain.set_noise(noise)
    holes = np.zeros((len(w.envs), 3), np.uint64)
    for s, kf in enumerate(kfs):
        tr = o.step(kf.L, kf.mv, kf.Z, w.dt_ns, trace=s > 0)
        quiet.step(kf.L, kf.mv, kf.Z, w.dt_ns)
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
        plain.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
        if s == 0:
            continue
        keys = tr[0]
        ko = 0
        for i, e in enumerate(w.envs):
            k = keys[ko:ko + e.K * 2 * e.H * e.W].reshape(e.K, 2, e.H, e.W)
            ko += e.K * 2 * e.H * e.W
            m = e.margin
            emp = k[:, :, m:e.H - m, m:e.W - m] == np.uint64(0xFFFFFFFFFFFFFFFF)
            holes[i] += np.array([emp[:, 0].sum(), emp[:, 1].sum(), (emp[:, 0] & emp[:, 1]).sum()],
                                 dtype=np.uint64)
    evs = o.events()
    n_quiet = np.bincount(quiet.events()["env"], minlength=len(w.envs))
    st = ctx.env_stats()
    got = ev.sort_events(ctx.read_events())
    np.testing.assert_array_equal(got.view(np.uint8), oracle_mod.sort_events(evs).view(np.uint8))
    for i, e in enumerate(w.envs):
        mine = evs[evs["env"] == i]
        assert st["target_subframes"][i] == (e.W - 2 * e.margin) * (e.H - 2 * e.margin) * e.K * 2
        assert [st["holes_a"][i], st["holes_b"][i], st["holes_both"][i]] == holes[i].tolist()
        assert st["events_on"][i] == np.sum(mine["p"] > 0)
        assert st["events_off"][i] == np.sum(mine["p"] < 0)
        assert st["noise_events"][i] == len(mine) - n_quiet[i] > 0
        assert st["over_limit"][i] == 0
    # the high-speed scenes leave holes in both directions (Sec. 3.3 fills one from the other)
    assert np.all(st["holes_a"] > 0) and np.all(st["holes_b"] > 0)
    ctx.close()
    # without EVIS_STATS: the same events, only the always-kept counts
    sp = plain.env_stats()
    got_p = ev.sort_events(plain.read_events())
    np.testing.assert_array_equal(got_p.view(np.uint8), got.view(np.uint8))
    np.testing.assert_array_equal(sp["target_subframes"], st["target_subframes"])
    for f in ("holes_a", "holes_b", "holes_both", "events_on", "events_off", "noise_events",
              "over_limit"):
        assert np.all(sp[f] == 0), f
    plain.close()
