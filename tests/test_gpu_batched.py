"""Batched uneven form: mixed resolutions and K in one context, per-environment tile shapes,
the autotuner, and CUDA-graph replay, all against the oracle (needs a B300)."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(-1)).cuda()


def _uneven(scenes_mod, n_envs=12, scale=0.25):
    return scenes_mod.config3(n_envs=n_envs, scale=scale)


def _oracle_events(oracle_mod, envs, kfs, dt):
    o = oracle_mod.Oracle(envs, flags=oracle_mod.IN_LOG)
    for kf in kfs:
        o.step(kf.L, kf.mv, kf.Z, dt)
    return oracle_mod.sort_events(o.events()), o.state()


def _same(ev, got, want):
    got = ev.sort_events(got)
    assert len(got) == len(want) > 0
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))


def test_graph_replay_of_uneven_batch(ev, oracle_mod, scenes_mod):
    w = _uneven(scenes_mod)
    kfs = [scenes_mod.render(w.envs, k) for k in range(5)]
    want, wstate = _oracle_events(oracle_mod, w.envs, kfs, w.dt_ns)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 24, stream=stream)
        ctx.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), w.dt_ns)
        ctx.capture(w.dt_ns)
        for kf in kfs[1:]:
            ctx.write_inputs(_dev(kf.L), _dev(kf.mv), _dev(kf.Z))
            ctx.replay()
        got = ctx.read_events()
        st = ctx.state()
    _same(ev, got, want)
    np.testing.assert_array_equal(st[2], wstate[2])


def test_mixed_tile_shapes_and_autotune(ev, oracle_mod, scenes_mod):
    w = _uneven(scenes_mod, n_envs=10)
    kfs = [scenes_mod.render(w.envs, k) for k in range(4)]
    want, wstate = _oracle_events(oracle_mod, w.envs, kfs, w.dt_ns)
    shapes = ev.Context.TILE_SHAPES
    ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 24)
    ctx.set_env_tile_shapes([shapes[i % len(shapes)] for i in range(len(w.envs))])
    ctx.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), w.dt_ns)
    ctx.step(_dev(kfs[1].L), _dev(kfs[1].mv), _dev(kfs[1].Z), w.dt_ns)
    n_before = ctx.event_count()
    best = ctx.autotune(_dev(kfs[2].L), _dev(kfs[2].mv), _dev(kfs[2].Z), w.dt_ns, reps=2)
    assert best > 0
    assert ctx.event_count() == n_before           # the trials consumed nothing
    assert all(tuple(s) in shapes for s in ctx.tile_shapes())
    for kf in kfs[2:]:
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    _same(ev, ctx.read_events(), want)
    Lref, tl, clk = ctx.state()
    valid = np.zeros(Lref.size, dtype=bool)
    off, _ = scenes_mod.pixel_offsets(w.envs)
    for e, o in zip(w.envs, off):
        valid[o:o + e.H * e.W] = True
    np.testing.assert_array_equal(Lref[valid], wstate[0][valid])
    np.testing.assert_array_equal(clk, wstate[2])


def test_replay_is_discarded_by_a_plain_step(ev, scenes_mod):
    w = _uneven(scenes_mod, n_envs=4)
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 22, stream=stream)
        ctx.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), w.dt_ns)
        ctx.capture(w.dt_ns)
        ctx.step(_dev(kfs[1].L), _dev(kfs[1].mv), _dev(kfs[1].Z), w.dt_ns)
        with pytest.raises(ev.EvisError):
            ctx.replay()
    keep = ev.Context(w.envs, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=1 << 20)
    keep.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), w.dt_ns)
    with pytest.raises(ev.EvisError):
        keep.capture(w.dt_ns)                         # kept inputs cannot be baked into a graph
