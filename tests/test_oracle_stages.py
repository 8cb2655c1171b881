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
