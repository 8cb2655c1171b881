"""Parity of the benchmarked launches themselves (needs a B300).

The 64 x 346x260 workload is compared with the oracle on every environment (one oracle per
host thread, each on its own slice of environments).  The high-speed batch runs as the full
1024-environment launch with its autotuned tile shape: two gaps accumulate about 1.9 G event
records (indices past 2^30) in one buffer, the persistent grid works through every tile of
the list, and environments 0, 511 and 1023 (the first, middle and last pixel offsets) are
compared with the oracle bit for bit: events, reference levels and clocks."""
import ctypes
import os
from concurrent.futures import ThreadPoolExecutor

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


def _repack(envs, sample, kf, scenes_mod):
    """Keyframe arrays of the environments `sample` of envs, packed on their own."""
    off, _ = scenes_mod.pixel_offsets(envs)
    sub = [envs[i] for i in sample]
    soff, stotal = scenes_mod.pixel_offsets(sub)
    L = np.zeros(stotal, np.float32)
    mv = np.zeros((stotal, 2), np.float32)
    Z = np.ones(stotal, np.float32)
    for j, i in enumerate(sample):
        n = envs[i].H * envs[i].W
        L[soff[j]:soff[j] + n] = kf.L[off[i]:off[i] + n]
        mv[soff[j]:soff[j] + n] = kf.mv[off[i]:off[i] + n]
        Z[soff[j]:soff[j] + n] = kf.Z[off[i]:off[i] + n]
    return L, mv, Z, soff


def _oracle_slices(oracle_mod, scenes_mod, envs, kfs, dt, slices):
    """One oracle per slice of environment indices, run on the host cores at the same time;
    per slice: (events with global environment indices, Lref, t_last, clocks, offsets)."""

    def run(sample):
        sub = [envs[i] for i in sample]
        o = oracle_mod.Oracle(sub, flags=oracle_mod.IN_LOG)
        soff = None
        for kf in kfs:
            L, mv, Z, soff = _repack(envs, sample, kf, scenes_mod)
            o.step(L, mv, Z, dt)
        e = o.events()
        e["env"] = np.asarray(sample, np.uint16)[e["env"]]
        Lref, tl, clk = o.state()
        return e, Lref, tl, clk, soff

    with ThreadPoolExecutor(max_workers=min(len(slices), os.cpu_count() or 1)) as pool:
        return list(pool.map(run, slices))


def test_config2_every_environment(ev, oracle_mod, scenes_mod):
    """The benchmarked 64 x 346x260 launch (K=16, refractory 100 us, autotuned tile shape)
    over two gaps: every environment's events, reference levels, last-event times and
    clocks equal the oracle's."""
    w = scenes_mod.config2()
    kfs = [scenes_mod.render(w.envs, k) for k in range(3)]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG, capacity=1 << 28)
    ctx.step(_dev(kfs[0].L), _dev(kfs[0].mv), _dev(kfs[0].Z), w.dt_ns)
    ctx.autotune(_dev(kfs[1].L), _dev(kfs[1].mv), _dev(kfs[1].Z), w.dt_ns, reps=1)
    for kf in kfs[1:]:
        ctx.step(_dev(kf.L), _dev(kf.mv), _dev(kf.Z), w.dt_ns)
    eg = ev.sort_events(ctx.read_events())
    Lref, tl, clk = ctx.state()
    ctx.close()
    slices = [list(range(s, s + 4)) for s in range(0, 64, 4)]
    res = _oracle_slices(oracle_mod, scenes_mod, w.envs, kfs, w.dt_ns, slices)
    eo = oracle_mod.sort_events(np.concatenate([r[0] for r in res]))
    assert len(eg) == len(eo) > 50_000_000
    np.testing.assert_array_equal(eg.view(np.uint8), eo.view(np.uint8))
    off, _ = scenes_mod.pixel_offsets(w.envs)
    for sample, (_, Lo, to, co, soff) in zip(slices, res):
        for j, i in enumerate(sample):
            n = w.envs[i].H * w.envs[i].W
            np.testing.assert_array_equal(Lref[off[i]:off[i] + n], Lo[soff[j]:soff[j] + n])
            np.testing.assert_array_equal(tl[off[i]:off[i] + n], to[soff[j]:soff[j] + n])
            assert clk[i] == co[j]


def _device_events_of(ev, ctx, env_ids):
    """All buffered events copied to device memory, those of env_ids returned to the host."""
    n = ctx.event_count()
    buf = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    cnt = ctypes.c_int64()
    st = ev.lib().evis_read_events(ctx.handle, buf.data_ptr(), n, ctypes.byref(cnt))
    assert st == ev.OK, ev.status_string(st)
    env = (buf[:, 1] >> 32) & 0xFFFF
    sel = buf[torch.isin(env, torch.tensor(env_ids, device="cuda"))].cpu().numpy()
    del buf, env
    return sel.view(ev.EVENT_DTYPE).reshape(-1), cnt.value


def test_high_speed_full_launch(ev, oracle_mod, scenes_mod):
    """The full high-speed launch: 1024 environments at 640x480, K=32, autotuned tiles, two
    gaps into one buffer (about 1.9 G records), environments 0, 511 and 1023 bit for bit."""
    w = scenes_mod.config4(n_envs=1024)
    kfs = [scenes_mod.render(w.envs, k, want=("L", "mv", "Z")) for k in range(3)]
    dev = [(_dev(kf.L), _dev(kf.mv), _dev(kf.Z)) for kf in kfs]
    ctx = ev.Context(w.envs, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=int(2.6e9))
    ctx.step(*dev[0], w.dt_ns)
    ctx.autotune(*dev[1], w.dt_ns, reps=1)
    for d in dev[1:]:
        ctx.step(*d, w.dt_ns)
    sample = [0, 511, 1023]
    eg, total = _device_events_of(ev, ctx, sample)
    assert total > 2 ** 30 + 2 ** 29            # the second gap's records sit past index 2^30
    Lref, _, clk = ctx.state()
    assert np.all(ctx.env_stats()["over_limit"] == 0)
    ctx.close()
    del dev
    torch.cuda.empty_cache()
    res = _oracle_slices(oracle_mod, scenes_mod, w.envs, kfs, w.dt_ns, [[i] for i in sample])
    off, _ = scenes_mod.pixel_offsets(w.envs)
    eg = ev.sort_events(eg)
    for i, (eo, Lo, _, co, soff) in zip(sample, res):
        mine = eg[eg["env"] == i]
        theirs = oracle_mod.sort_events(eo)
        assert len(mine) == len(theirs) > 100_000
        np.testing.assert_array_equal(mine.view(np.uint8), theirs.view(np.uint8))
        n = w.envs[i].H * w.envs[i].W
        np.testing.assert_array_equal(Lref[off[i]:off[i] + n], Lo[:n])
        assert clk[i] == co[0]
