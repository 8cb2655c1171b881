"""evis_step_noalloc, the entry point for callers that cannot allocate device memory (for
example a host engine that owns the whole GPU memory pool and only hands out buffers): it must
give exactly what the context-based evis_step gives, on two keyframe gaps in a row, while
reusing the library's static scratch array between the calls.  Kept in a file of its own that
pytest collects last."""
import ctypes

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


def _env_scene(scenes_mod, refractory_ns):
    layers = scenes_mod.config1().envs[0].layers
    return scenes_mod.EnvScene(W=160, H=100, K=6, c_on=0.2, c_off=0.25,
                               refractory_ns=refractory_ns, t0_ns=5_000, layers=layers)


@pytest.mark.parametrize("refractory_ns", [0, 150_000])
def test_noalloc_matches_evis_step_on_two_gaps(ev, scenes_mod, refractory_ns):
    es = _env_scene(scenes_mod, refractory_ns)
    n = es.W * es.H
    dt = 16_666_667
    kfs = [scenes_mod.render([es], k) for k in range(3)]
    dev = [tuple(_dev(a[:n] if a.ndim == 1 else a[:n]) for a in (kf.L, kf.mv, kf.Z)) for kf in kfs]

    # reference: the context-based path, events read after each gap
    ctx = ev.Context([es], flags=ev.IN_LOG, capacity=1 << 22)
    ref_events, ref_state = [], []
    ctx.step(*(_dev(a) for a in (kfs[0].L, kfs[0].mv, kfs[0].Z)), dt)
    for kf in kfs[1:]:
        ctx.step(*(_dev(a) for a in (kf.L, kf.mv, kf.Z)), dt)
        ref_events.append(ev.sort_events(ctx.read_events()))
        Lref, tl, _ = ctx.state()
        ref_state.append((Lref[:n].copy(), tl[:n].copy()))
    ctx.close()

    # the same two gaps through the allocation-free entry point
    desc = ev.EnvDesc(width=es.W, height=es.H, K=es.K, c_on=es.c_on, c_off=es.c_off,
                      refractory_ns=refractory_ns, t0_ns=es.t0_ns)
    Lref = dev[0][0].clone()
    t_last = torch.full((n,), np.iinfo(np.int64).min, dtype=torch.int64, device="cuda")
    cap = 1 << 21
    events = torch.empty(cap * 2, dtype=torch.int64, device="cuda")
    count = torch.zeros(2, dtype=torch.int64, device="cuda")   # events, pixels over the limit
    stream = torch.cuda.current_stream().cuda_stream
    L = ev.lib()
    for gap in range(2):
        A, B = dev[gap], dev[gap + 1]
        count.zero_()
        st = L.evis_step_noalloc(ctypes.byref(desc), 0, A[0].data_ptr(), A[1].data_ptr(),
                                 A[2].data_ptr(), B[0].data_ptr(), B[1].data_ptr(),
                                 B[2].data_ptr(), Lref.data_ptr(),
                                 t_last.data_ptr() if refractory_ns else None,
                                 es.t0_ns + gap * dt, dt, events.data_ptr(), count.data_ptr(),
                                 cap, stream)
        assert st == ev.OK, L.evis_last_error(None).decode()
        torch.cuda.synchronize()
        got_n = int(count[0].item())
        assert got_n <= cap and int(count[1].item()) == 0
        got = events[:2 * got_n].cpu().numpy().view(ev.EVENT_DTYPE)
        want = ref_events[gap]
        assert len(want) > 1000
        np.testing.assert_array_equal(ev.sort_events(got).view(np.uint8), want.view(np.uint8))
        np.testing.assert_array_equal(Lref.cpu().numpy(), ref_state[gap][0])
        if refractory_ns:
            np.testing.assert_array_equal(t_last.cpu().numpy(), ref_state[gap][1])


def test_noalloc_with_margin_matches_oracle(ev, oracle_mod, scenes_mod):
    """A 7-pixel over-render margin (Appendix B) through the allocation-free entry point."""
    rng = np.random.default_rng(4)
    es = scenes_mod.EnvScene(W=150, H=90, K=6, c_on=0.2, c_off=0.25, refractory_ns=40_000,
                             layers=scenes_mod._random_layers(rng, 150, 90, 3, 6.0, 0.08), margin=7)
    n = es.W * es.H
    kfs = [scenes_mod.render([es], k) for k in range(2)]
    o = oracle_mod.Oracle([es])
    for kf in kfs:
        o.step(kf.L, kf.mv, kf.Z, 16_666_667)
    want = oracle_mod.sort_events(o.events())
    A, B = [tuple(_dev(a[:n]) for a in (kf.L, kf.mv, kf.Z)) for kf in kfs]
    desc = ev.EnvDesc(width=es.W, height=es.H, K=es.K, c_on=es.c_on, c_off=es.c_off,
                      margin=es.margin, refractory_ns=es.refractory_ns)
    Lref = A[0].clone()
    t_last = torch.full((n,), np.iinfo(np.int64).min, dtype=torch.int64, device="cuda")
    cap = 1 << 20
    events = torch.empty(cap * 2, dtype=torch.int64, device="cuda")
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    L = ev.lib()
    st = L.evis_step_noalloc(ctypes.byref(desc), 0, A[0].data_ptr(), A[1].data_ptr(),
                             A[2].data_ptr(), B[0].data_ptr(), B[1].data_ptr(), B[2].data_ptr(),
                             Lref.data_ptr(), t_last.data_ptr(), 0, 16_666_667, events.data_ptr(),
                             count.data_ptr(), cap, torch.cuda.current_stream().cuda_stream)
    assert st == ev.OK, L.evis_last_error(None).decode()
    torch.cuda.synchronize()
    got = ev.sort_events(events[:2 * int(count[0].item())].cpu().numpy().view(ev.EVENT_DTYPE))
    assert len(got) == len(want) > 100
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    grid = np.zeros((es.H, es.W), bool)
    grid[7:es.H - 7, 7:es.W - 7] = True
    np.testing.assert_array_equal(Lref.cpu().numpy()[grid.ravel()], o.state()[0][:n][grid.ravel()])


def test_noalloc_rejects_sizes_beyond_its_scratch(ev):
    L = ev.lib()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    p = buf.data_ptr()
    for W, H in ((4097, 8), (8, 4097), (2048, 1024)):
        desc = ev.EnvDesc(width=W, height=H, K=4, c_on=0.2, c_off=0.2)
        st = L.evis_step_noalloc(ctypes.byref(desc), 0, p, p, p, p, p, p, p, None, 0, 1000,
                                 p, cnt.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
        assert st == ev.ERR_INVALID_ARG
        assert "4096" in L.evis_last_error(None).decode()
    # a margin whose double overflows 32 bits is rejected, not wrapped into a huge tile count
    for m in (1 << 30, (1 << 31) - 1):
        desc = ev.EnvDesc(width=64, height=64, K=4, c_on=0.2, c_off=0.2, margin=m)
        st = L.evis_step_noalloc(ctypes.byref(desc), 0, p, p, p, p, p, p, p, None, 0, 1000,
                                 p, cnt.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
        assert st == ev.ERR_INVALID_ARG
        assert "margin" in L.evis_last_error(None).decode()


def test_noalloc_counts_pixels_beyond_the_crossing_limit(ev, oracle_mod):
    """Pixels whose Eq. 4 count exceeds the per-sub-frame limit: none of their crossings
    is emitted, count[1] receives their number and the reference levels follow Eq. 4, as in
    the oracle."""
    W, H, C = 40, 20, 0.25
    rng = np.random.default_rng(3)
    LA = np.zeros(W * H, np.float32)
    LB = rng.normal(0, 1, W * H).astype(np.float32)
    big = rng.random(W * H) < 0.05
    # three sub-frames, each about (limit + 1.5) C beyond the last reference level
    LB[big] = np.float32((3 * (ev.MAX_CROSSINGS + 1) + 1.5) * C) * rng.choice([-1, 1], big.sum())
    mv = np.zeros((W * H, 2), np.float32)
    Z = np.ones(W * H, np.float32)

    class E:
        pass
    es = E()
    es.W, es.H, es.K, es.c_on, es.c_off, es.refractory_ns, es.t0_ns, es.margin = W, H, 3, C, C, 0, 0, 0
    o = oracle_mod.Oracle([es])
    o.step(LA, mv, Z, 1_000_000)
    o.step(LB, mv, Z, 1_000_000)
    assert o.last_over_limit
    want = oracle_mod.sort_events(o.events())
    desc = ev.EnvDesc(width=W, height=H, K=3, c_on=C, c_off=C)
    dA, dB, dmv, dZ = _dev(LA), _dev(LB), _dev(mv), _dev(Z)
    Lref = dA.clone()
    cap = 1 << 16
    events = torch.empty(cap * 2, dtype=torch.int64, device="cuda")
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    L = ev.lib()
    st = L.evis_step_noalloc(ctypes.byref(desc), 0, dA.data_ptr(), dmv.data_ptr(), dZ.data_ptr(),
                             dB.data_ptr(), dmv.data_ptr(), dZ.data_ptr(), Lref.data_ptr(), None,
                             0, 1_000_000, events.data_ptr(), count.data_ptr(), cap,
                             torch.cuda.current_stream().cuda_stream)
    assert st == ev.OK, L.evis_last_error(None).decode()
    torch.cuda.synchronize()
    assert int(count[1].item()) == int(o.over_limit()[0]) == 3 * int(big.sum())
    got = ev.sort_events(events[:2 * int(count[0].item())].cpu().numpy().view(ev.EVENT_DTYPE))
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    np.testing.assert_array_equal(Lref.cpu().numpy(), o.state()[0][:W * H])
