"""Pins of the oracle's input- and output-side stages around the warp: the over-render
margin (Appendix B).  Each is checked against a plain restatement of what the stage means,
run through the oracle's own margin-free path."""
import dataclasses

import numpy as np
import pytest

from evis_testutil import TinyEnv


def _scene(scenes_mod, W, H, K, seed, margin=0, refractory_ns=0):
    rng = np.random.default_rng(seed)
    lay = scenes_mod._random_layers(rng, W, H, 3, vmax=6.0, wmax=0.08)
    return scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.18, c_off=0.22, layers=lay, margin=margin,
                               refractory_ns=refractory_ns)


def _run(oracle_mod, envs, kfs, dt, noise=None):
    o = oracle_mod.Oracle(envs)
    if noise is not None:
        o.set_noise(noise)
    for kf in kfs:
        o.step(kf.L, kf.mv, kf.Z, dt)
    return o


@pytest.mark.parametrize("margin", [1, 4, 9])
def test_margin_is_a_crop_after_warping(oracle_mod, scenes_mod, margin):
    """Appendix B: the margin is rendered, warped with the rest, and cropped afterwards.  So
    the events of a margin run are those of the full-frame run inside the crop, shifted to
    sensor coordinates, and the per-pixel state agrees there."""
    full = _scene(scenes_mod, 61, 45, 5, seed=3, refractory_ns=20_000)
    crop = dataclasses.replace(full, margin=margin)
    kfs = [scenes_mod.render([full], k) for k in range(4)]
    a = _run(oracle_mod, [full], kfs, 16_666_667)
    b = _run(oracle_mod, [crop], kfs, 16_666_667)
    ea = oracle_mod.sort_events(a.events())
    inside = ((ea["x"] >= margin) & (ea["x"] < full.W - margin) &
              (ea["y"] >= margin) & (ea["y"] < full.H - margin))
    want = ea[inside].copy()
    want["x"] -= margin
    want["y"] -= margin
    got = oracle_mod.sort_events(b.events())
    assert len(got) == len(want) > 100 and inside.sum() < len(ea)
    np.testing.assert_array_equal(got.view(np.uint8), want.view(np.uint8))
    sa, sb = a.state(), b.state()
    grid = np.zeros((full.H, full.W), bool)
    grid[margin:full.H - margin, margin:full.W - margin] = True
    n = full.W * full.H
    np.testing.assert_array_equal(sb[0][:n][grid.ravel()], sa[0][:n][grid.ravel()])
    np.testing.assert_array_equal(sb[1][:n][grid.ravel()], sa[1][:n][grid.ravel()])
    assert np.all(got["x"] < full.W - 2 * margin) and np.all(got["y"] < full.H - 2 * margin)


def test_margin_noise_belongs_to_the_sensor(oracle_mod):
    """Noise is drawn per sensor pixel: a margin run's leak events equal those of a run on
    the bare sensor with the same seed (a constant scene has no signal events)."""
    m = 5
    big, small = TinyEnv(W=40, H=30, K=4, margin=m), TinyEnv(W=30, H=20, K=4)

    def run(env):
        n = (env.W * env.H + 3) // 4 * 4
        o = oracle_mod.Oracle([env])
        o.set_noise([dict(leak_hz=60.0, hot_hz=400.0, hot_fraction=0.05, seed=21)])
        for _ in range(3):
            o.step(np.zeros(n, np.float32), np.zeros((n, 2), np.float32), np.ones(n, np.float32),
                   10_000_000)
        return oracle_mod.sort_events(o.events())

    a, b = run(big), run(small)
    assert len(a) > 100
    np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("W,H,m", [(10, 30, 5), (30, 10, 5), (8, 8, -1)])
def test_margin_must_leave_a_sensor(oracle_mod, W, H, m):
    with pytest.raises(Exception):
        oracle_mod.Oracle([TinyEnv(W=W, H=H, K=2, margin=m)])


# ---- defocus (Sec. 3.4): separable Gaussian on the linear intensity before the log ----

ndimage = pytest.importorskip("scipy.ndimage")


def _radius(sigma):
    return int(3.0 * np.float64(np.float32(sigma)) + 0.5)


@pytest.mark.parametrize("sigma", [0.1, 0.3, 0.5, 0.7, 1.3, 2.5])
def test_defocus_weights_are_scipys_gaussian(oracle_mod, sigma):
    r = _radius(sigma)
    w = oracle_mod.defocus_weights(sigma)
    assert w.size == 2 * r + 1
    delta = np.zeros(2 * r + 1)
    delta[r] = 1.0
    ref = ndimage.gaussian_filter1d(delta, float(np.float32(sigma)), mode="constant", radius=r)
    np.testing.assert_array_equal(w, ref[::-1].astype(np.float32))   # correlation = flip


@pytest.mark.parametrize("sigma", [0.3, 0.5, 1.3, 2.5])
def test_defocus_is_scipys_separable_filter(oracle_mod, sigma):
    rng = np.random.default_rng(11)
    img = rng.uniform(0.01, 4.0, (37, 53)).astype(np.float32)
    got = oracle_mod.defocus(img, sigma)
    s64 = float(np.float32(sigma))
    r = _radius(sigma)
    ref = ndimage.gaussian_filter1d(img.astype(np.float64), s64, axis=1, mode="nearest", radius=r)
    ref = ndimage.gaussian_filter1d(ref, s64, axis=0, mode="nearest", radius=r)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=0)


def test_defocus_closed_forms(oracle_mod):
    sigma = 0.8
    w = oracle_mod.defocus_weights(sigma).astype(np.float32)
    r = w.size // 2
    # impulse response: the outer product of the weights, one binary32 product each
    img = np.zeros((31, 29), np.float32)
    img[15, 14] = 1.0
    out = oracle_mod.defocus(img, sigma)
    want = np.zeros_like(img)
    want[15 - r:15 + r + 1, 14 - r:14 + r + 1] = w[:, None] * w[None, :]
    np.testing.assert_array_equal(out, want)
    # a constant stays constant (weights sum to 1 within rounding)
    c = np.full((20, 30), 2.75, np.float32)
    np.testing.assert_allclose(oracle_mod.defocus(c, sigma), c, rtol=4 * 2.0**-23)
    # a linear ramp stays linear away from the borders (symmetric kernel)
    ramp = (0.5 + 0.01 * np.arange(40, dtype=np.float32))[None, :].repeat(12, 0)
    out = oracle_mod.defocus(ramp, sigma)
    np.testing.assert_allclose(out[:, r:-r], ramp[:, r:-r], rtol=1e-6)
    # mass is conserved for an impulse far from the borders
    assert abs(float(oracle_mod.defocus(img, 1.7).astype(np.float64).sum()) - 1.0) < 1e-6
    # sigma 0 is the identity, bit for bit
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 3, (9, 14)).astype(np.float32)
    np.testing.assert_array_equal(oracle_mod.defocus(x, 0.0), x)


@pytest.mark.parametrize("mode", [1, 2])
def test_defocus_comes_before_the_log(oracle_mod, scenes_mod, mode):
    """Events of a defocused run equal those of a plain run fed the blurred luminance:
    the blur acts on linear intensity (after Rec. 709 for RGB), before the log."""
    env = _scene(scenes_mod, 48, 36, 4, seed=8)
    envs = [env, dataclasses.replace(env)]
    sig = [0.6, 0.0]
    kfs = [scenes_mod.render(envs, k, want=("I", "rgb", "mv", "Z")) for k in range(3)]
    a = oracle_mod.Oracle(envs, flags=mode)
    a.set_defocus(sig)
    b = oracle_mod.Oracle(envs, flags=1)
    n = env.W * env.H
    per = (n + 3) // 4 * 4
    for kf in kfs:
        fr = kf.I if mode == 1 else kf.rgb.reshape(-1)
        a.step(fr, kf.mv, kf.Z, 16_666_667)
        if mode == 1:
            lum = kf.I.copy()
        else:
            lum = oracle_mod.rec709(kf.rgb.reshape(-1, 3))
        pre = lum.copy()
        pre[:n] = oracle_mod.defocus(lum[:n].reshape(env.H, env.W), sig[0]).ravel()
        assert not np.array_equal(pre[:n], lum[:n]) and np.array_equal(pre[per:per + n], lum[per:per + n])
        b.step(pre, kf.mv, kf.Z, 16_666_667)
    ea, eb = oracle_mod.sort_events(a.events()), oracle_mod.sort_events(b.events())
    assert len(ea) > 100
    np.testing.assert_array_equal(ea.view(np.uint8), eb.view(np.uint8))


def test_defocus_parameters_are_checked(oracle_mod):
    env = TinyEnv(W=8, H=8, K=2)
    with pytest.raises(ValueError):
        oracle_mod.Oracle([env], flags=0).set_defocus([0.5])       # log input: nothing to blur
    with pytest.raises(ValueError):
        oracle_mod.Oracle([env], flags=1).set_defocus([9.0])
    with pytest.raises(ValueError):
        oracle_mod.Oracle([env], flags=1).set_defocus([float("nan")])
    oracle_mod.Oracle([env], flags=0).set_defocus([0.0])


# ---- colour events (Sec. 3.2): the event model on each of R, G and B ----

def _tinted(scenes_mod, W, H, K, seed, refractory_ns=30_000):
    env = _scene(scenes_mod, W, H, K, seed, refractory_ns=refractory_ns)
    rng = np.random.default_rng(seed + 100)
    for lay in env.layers:
        lay.tint_r, lay.tint_g, lay.tint_b = rng.uniform(0.3, 1.6, 3)
    return env


def _colour_vs_mono(oracle_mod, envs, kfs, dt, noise=None, sigma=None):
    col = oracle_mod.Oracle(envs, flags=oracle_mod.IN_RGB | oracle_mod.COLOR)
    if noise is not None:
        col.set_noise(noise)
    if sigma is not None:
        col.set_defocus(sigma)
    monos = []
    for c in range(3):
        m = oracle_mod.Oracle(envs, flags=oracle_mod.IN_LUM)
        if noise is not None:
            m.set_noise(noise)
        if sigma is not None:
            m.set_defocus(sigma)
        monos.append(m)
    for kf in kfs:
        rgb = kf.rgb.reshape(-1, 3)
        col.step(rgb.reshape(-1), kf.mv, kf.Z, dt)
        for c, m in enumerate(monos):
            m.step(np.ascontiguousarray(rgb[:, c]), kf.mv, kf.Z, dt)
    return col, monos


def test_colour_is_three_independent_event_models(oracle_mod, scenes_mod):
    """Sec. 3.2: replacing I by each of R, G and B and running the event model on each gives
    colour events.  Channel c of a colour run is a luminance run fed channel c, with the
    polarity field carrying +-(1 + c); reference levels and refractory times per channel."""
    env = _tinted(scenes_mod, 52, 40, 5, seed=12)
    kfs = [scenes_mod.render([env], k, want=("rgb", "mv", "Z")) for k in range(4)]
    col, monos = _colour_vs_mono(oracle_mod, [env], kfs, 16_666_667)
    ec = oracle_mod.sort_events(col.events())
    sc = col.state()
    n = col.total
    counts = []
    for c, m in enumerate(monos):
        mine = ec[np.abs(ec["p"]) == c + 1].copy()
        mine["p"] = np.sign(mine["p"])
        want = oracle_mod.sort_events(m.events())
        counts.append(len(want))
        np.testing.assert_array_equal(mine.view(np.uint8), want.view(np.uint8))
        sm = m.state()
        np.testing.assert_array_equal(sc[0][c * n:(c + 1) * n], sm[0])
        np.testing.assert_array_equal(sc[1][c * n:(c + 1) * n], sm[1])
    assert min(counts) > 100 and len(set(counts)) == 3     # the tints make the channels differ
    assert len(ec) == sum(counts)


def test_colour_noise_defocus_and_planar_log(oracle_mod, scenes_mod):
    """Channel 0 draws the luminance run's noise; channels 1 and 2 draw their own streams.
    Defocus blurs each channel.  Planar log-intensity input equals linear RGB input."""
    env = _tinted(scenes_mod, 40, 30, 4, seed=13, refractory_ns=0)
    kfs = [scenes_mod.render([env], k, want=("rgb", "mv", "Z")) for k in range(3)]
    noise = [dict(leak_hz=40.0, hot_hz=300.0, hot_fraction=0.05, shot_hz=60.0, seed=5)]
    col, monos = _colour_vs_mono(oracle_mod, [env], kfs, 16_666_667, noise=noise, sigma=[0.7])
    ec = oracle_mod.sort_events(col.events())
    per = []
    for c, m in enumerate(monos):
        mine = ec[np.abs(ec["p"]) == c + 1].copy()
        mine["p"] = np.sign(mine["p"])
        want = oracle_mod.sort_events(m.events())
        per.append((mine, want))
    np.testing.assert_array_equal(per[0][0].view(np.uint8), per[0][1].view(np.uint8))
    for c in (1, 2):
        assert not np.array_equal(per[c][0].view(np.uint8), per[c][1].view(np.uint8))
    # planar log input: the same stream as the RGB run without noise or defocus
    a = oracle_mod.Oracle([env], flags=oracle_mod.IN_RGB | oracle_mod.COLOR)
    b = oracle_mod.Oracle([env], flags=oracle_mod.IN_LOG | oracle_mod.COLOR)
    n = (env.W * env.H + 3) // 4 * 4
    for kf in kfs:
        rgb = kf.rgb.reshape(-1, 3)
        a.step(rgb.reshape(-1), kf.mv, kf.Z, 16_666_667)
        planes = np.concatenate([oracle_mod.log_intensity(np.ascontiguousarray(rgb[:, c]), mode=1,
                                                          eps=1e-4) for c in range(3)])
        assert planes.size == 3 * n
        b.step(planes, kf.mv, kf.Z, 16_666_667)
    ea, eb = oracle_mod.sort_events(a.events()), oracle_mod.sort_events(b.events())
    assert len(ea) > 100
    np.testing.assert_array_equal(ea.view(np.uint8), eb.view(np.uint8))


def test_colour_grey_scene_gives_equal_channels(oracle_mod, scenes_mod):
    env = _scene(scenes_mod, 36, 28, 4, seed=14)
    kfs = [scenes_mod.render([env], k, want=("rgb", "mv", "Z")) for k in range(3)]
    o = oracle_mod.Oracle([env], flags=oracle_mod.IN_RGB | oracle_mod.COLOR)
    for kf in kfs:
        rgb = kf.rgb.reshape(-1, 3)
        grey = np.repeat(rgb[:, 1:2], 3, axis=1)
        o.step(grey.reshape(-1), kf.mv, kf.Z, 16_666_667)
    e = oracle_mod.sort_events(o.events())
    chans = []
    for c in range(3):
        x = e[np.abs(e["p"]) == c + 1].copy()
        x["p"] = np.sign(x["p"])
        chans.append(x)
    assert len(chans[0]) > 100
    for c in (1, 2):
        np.testing.assert_array_equal(chans[c].view(np.uint8), chans[0].view(np.uint8))
    with pytest.raises(ValueError):
        oracle_mod.Oracle([env], flags=oracle_mod.IN_LUM | oracle_mod.COLOR)
