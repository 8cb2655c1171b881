"""Pipelined event read-back on the GPU (needs a B300): events copied by
evis_read_events_async while the next keyframe gaps run are the same records, gap by gap,
as a context read synchronously after every gap."""
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


def _gaps(scenes_mod, n_kf):
    w = scenes_mod.config2(n_envs=4)
    kfs = [scenes_mod.render(w.envs, k) for k in range(n_kf)]
    dev = [(torch.from_numpy(kf.L).cuda(), torch.from_numpy(kf.mv.reshape(-1)).cuda(),
            torch.from_numpy(kf.Z).cuda()) for kf in kfs]
    return w, dev


def test_pipelined_readback_matches_synchronous_reads(ev, scenes_mod):
    w, dev = _gaps(scenes_mod, 7)
    cap = 1 << 22
    a = ev.Context(w.envs, flags=ev.IN_LOG, capacity=cap)
    want = []
    for d in dev:
        a.step(*d, w.dt_ns)
        want.append(np.sort(a.read_events()))
    a.close()
    assert sum(len(x) for x in want) > 100_000
    b = ev.Context(w.envs, flags=ev.IN_LOG, capacity=cap)
    bufs = [torch.empty(cap * 16, dtype=torch.uint8).pin_memory() for _ in range(2)]
    counts = []

    def got(k):
        return np.sort(bufs[k % 2].numpy().view(ev.EVENT_DTYPE)[:counts[k]])

    for k, d in enumerate(dev[:-1]):
        b.step(*d, w.dt_ns)
        counts.append(b.read_events_async(bufs[k % 2].data_ptr(), cap))
        if k > 0:  # the previous gap's copy is complete now
            np.testing.assert_array_equal(got(k - 1), want[k - 1])
    b.read_wait()
    np.testing.assert_array_equal(got(len(dev) - 2), want[-2])
    assert counts == [len(x) for x in want[:-1]]
    # a synchronous read after the switch drains the buffer the steps now fill
    b.step(*dev[-1], w.dt_ns)
    np.testing.assert_array_equal(np.sort(b.read_events()), want[-1])
    b.close()


def test_pipelined_readback_overflow(ev, scenes_mod):
    """A gap that produces more events than the buffer holds: the asynchronous read reports
    the total with EVIS_ERR_OVERFLOW and delivers the stored ones; the next gap fills the
    other buffer from empty."""
    import ctypes
    w, dev = _gaps(scenes_mod, 3)
    cap = 1000
    c = ev.Context(w.envs, flags=ev.IN_LOG, capacity=cap)
    buf = torch.empty(cap * 16, dtype=torch.uint8).pin_memory()
    n = ctypes.c_int64()
    c.step(*dev[0], w.dt_ns)
    c.step(*dev[1], w.dt_ns)
    st = ev.lib().evis_read_events_async(c.handle, buf.data_ptr(), cap, ctypes.byref(n))
    assert st == ev.ERR_OVERFLOW and n.value > cap
    c.read_wait()
    recs = buf.numpy().view(ev.EVENT_DTYPE)[:cap]
    assert np.all(recs["env"] < len(w.envs)) and np.all(np.abs(recs["p"]) == 1)
    c.step(*dev[2], w.dt_ns)
    assert c.event_count() > cap   # counted from zero in the other buffer, beyond capacity again
    c.close()


def test_slices_on_their_own_streams_match_one_context(ev, scenes_mod):
    """Consecutive environment slices in separate contexts, each on its own stream, fed from
    host buffers; as soon as a slice's gap is done its read-back starts and its next gap is
    enqueued, while the other slices compute.  Every gap's records are those of one context
    over all environments (with the slice's environment indices)."""
    import ctypes
    w, dev = _gaps(scenes_mod, 5)
    cap = 1 << 22
    a = ev.Context(w.envs, flags=ev.IN_LOG, capacity=cap)
    want = []
    for d in dev:
        a.step(*d, w.dt_ns)
        want.append(np.sort(a.read_events()))
    a.close()
    assert sum(len(x) for x in want) > 100_000
    host = [tuple(t.cpu().pin_memory() for t in d) for d in dev]
    px = [int(v) for v in np.cumsum([0] + [e.W * e.H for e in w.envs])]
    cut = [0, 1, 3, 4]  # uneven slices: 1, 2 and 1 environments
    S = len(cut) - 1
    streams = [torch.cuda.Stream() for _ in range(S)]
    ctxs = [ev.Context(w.envs[cut[q]:cut[q + 1]], flags=ev.IN_LOG, capacity=cap, stream=streams[q])
            for q in range(S)]
    bufs = [[torch.empty(cap * 16, dtype=torch.uint8).pin_memory() for _ in range(2)]
            for _ in range(S)]
    counts = [[0] * len(dev) for _ in range(S)]
    got = [[] for _ in dev]
    n = ctypes.c_int64()

    def part(k, q):
        lo, hi = px[cut[q]], px[cut[q + 1]]
        return tuple(t[lo * (t.numel() // px[-1]):hi * (t.numel() // px[-1])] for t in host[k])

    def collect(q, k):  # slice q's copy of gap k is complete
        r = bufs[q][k % 2].numpy().view(ev.EVENT_DTYPE)[:counts[q][k]].copy()
        r["env"] += cut[q]
        got[k].append(r)

    for q, c in enumerate(ctxs):
        c.step_host(*part(0, q), w.dt_ns)
    for k in range(len(dev)):
        for q, c in enumerate(ctxs):
            assert ev.lib().evis_read_events_async(c.handle, bufs[q][k % 2].data_ptr(), cap,
                                                   ctypes.byref(n)) == ev.OK
            counts[q][k] = n.value
            if k > 0:
                collect(q, k - 1)
            if k + 1 < len(dev):
                c.step_host(*part(k + 1, q), w.dt_ns)
    for q, c in enumerate(ctxs):
        c.read_wait()
        collect(q, len(dev) - 1)
    for k in range(len(dev)):
        np.testing.assert_array_equal(np.sort(np.concatenate(got[k])), want[k])
    for c in ctxs:
        c.close()


def test_reads_do_not_wait_for_other_contexts_streams(ev, scenes_mod):
    """A context's reads copy its counter on its own stream: reading an idle context returns
    while another context's gaps still run on a blocking stream of the same device (a copy on
    the legacy default stream would wait for them)."""
    rt = pytest.importorskip("cuda.bindings.runtime")
    w = scenes_mod.config4(n_envs=16)
    kfs = [scenes_mod.render(w.envs, k, want=("L", "mv", "Z")) for k in range(6)]
    dev = [tuple(torch.from_numpy(np.ascontiguousarray(getattr(kf, a)).reshape(-1)).cuda()
                 for a in ("L", "mv", "Z")) for kf in kfs]
    handles = []
    for _ in range(2):
        err, s = rt.cudaStreamCreateWithFlags(0)   # blocking streams
        assert int(err) == 0
        handles.append(s)
    sa, sb = (torch.cuda.ExternalStream(int(s)) for s in handles)
    a = ev.Context(w.envs, flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=1 << 25, stream=sa)
    b = ev.Context(w.envs[:1], flags=ev.IN_LOG | ev.KEEP_INPUTS, capacity=1 << 20, stream=sb)
    first = tuple(t[:w.envs[0].W * w.envs[0].H * (t.numel() // sum(e.W * e.H for e in w.envs))]
                  for t in dev[0])
    b.step(*first, w.dt_ns)
    a.step(*dev[0], w.dt_ns)
    a.step(*dev[1], w.dt_ns)                     # every allocation made, nothing pending
    a.event_count()
    b.event_count()
    torch.cuda.synchronize()
    for d in dev[2:]:                            # several gaps queued on a's stream
        a.step(*d, w.dt_ns)
    assert b.event_count() == 0                  # b's own counter, read while a runs
    busy = int(rt.cudaStreamQuery(handles[0])[0]) != 0
    torch.cuda.synchronize()
    a.close()
    b.close()
    for s in handles:
        rt.cudaStreamDestroy(s)
    assert busy, "the read waited for another context's stream"
