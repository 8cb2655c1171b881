"""Pins of the oracle's event voxel grid (per-polarity bins, linear interpolation along time,
per-bin max normalisation: the speed-regression input of the paper's appendix)."""
import numpy as np
import pytest

EV = None


def _events(rng, n, W, H, t0, t1, env=0, margin_t=0):
    e = np.zeros(n, dtype=[("t", "<i8"), ("x", "<u2"), ("y", "<u2"), ("env", "<u2"), ("p", "<i2")])
    e["t"] = rng.integers(t0 - margin_t, t1 + 1 + margin_t, n)
    e["x"] = rng.integers(0, W, n)
    e["y"] = rng.integers(0, H, n)
    e["env"] = env
    e["p"] = rng.choice([-1, 1], n)
    return e


def _hat(ev, W, H, t0, t1, B):
    """The grid as linear interpolation written out in binary64: each event adds
    max(0, 1 - |tau - b|) to bin b, tau = (B - 1)(t - t0) / (t1 - t0)."""
    g = np.zeros((2, B, H, W))
    for r in ev:
        if not (t0 <= r["t"] <= t1):
            continue
        tau = (B - 1) * (int(r["t"]) - t0) / (t1 - t0)
        pol = 0 if r["p"] > 0 else 1
        for b in range(B):
            w = max(0.0, 1.0 - abs(tau - b))
            g[pol, b, r["y"], r["x"]] += w
    return g


@pytest.mark.parametrize("B", [1, 2, 7, 128])
def test_voxel_is_linear_interpolation_in_time(oracle_mod, B):
    rng = np.random.default_rng(B)
    W, H, t0, t1 = 9, 6, 1_000, 1_000 + 500_000_123
    ev = _events(rng, 400, W, H, t0, t1, margin_t=1000)
    acc, out = oracle_mod.voxel_grid(ev, [(W, H, t0, t1)], bins=B)
    acc = acc.reshape(2, B, H, W).astype(np.float64) / 65536.0
    want = _hat(ev, W, H, t0, t1, B)
    # each event's two weights are rounded to 2^-16 (one down, its complement up)
    inside = (ev["t"] >= t0) & (ev["t"] <= t1)
    n_at = np.zeros((2, H, W))
    for r in ev[inside]:
        n_at[0 if r["p"] > 0 else 1, r["y"], r["x"]] += 1
    assert np.all(np.abs(acc - want) <= n_at[:, None] * 2.0**-16 + 1e-12)
    # conservation: every event inside the segment adds exactly one unit over the bins
    np.testing.assert_array_equal(acc.sum(axis=1) * 65536.0, n_at * 65536.0)
    # normalisation per (polarity, bin) plane by that plane's own maximum
    a32 = (acc * 65536.0).astype(np.uint32)
    o = out.reshape(2, B, H, W)
    for pol in range(2):
        for b in range(B):
            mx = a32[pol, b].max()
            want = a32[pol, b].astype(np.float32) / np.float32(mx) if mx else np.zeros((H, W), np.float32)
            np.testing.assert_array_equal(o[pol, b], want)


def test_voxel_closed_forms_and_normalisation(oracle_mod):
    W, H, B = 4, 3, 5
    t0, t1 = 0, 400            # tau = (t - t0) / 100
    ev = np.zeros(4, dtype=oracle_mod.EVENT_DTYPE)
    ev[0] = (200, 1, 1, 0, 1)      # tau = 2: all of it in bin 2
    ev[1] = (250, 2, 0, 0, -1)     # tau = 2.5: half in bins 2 and 3 (OFF)
    ev[2] = (400, 3, 2, 0, 3)      # t = t1: bin 4; colour polarity +3 counts as ON
    ev[3] = (401, 0, 0, 0, 1)      # after the segment: skipped
    acc, out = oracle_mod.voxel_grid(ev, [(W, H, t0, t1)], bins=B)
    a = acc.reshape(2, B, H, W)
    assert a[0, 2, 1, 1] == 65536 and a[1, 2, 0, 2] == 32768 and a[1, 3, 0, 2] == 32768
    assert a[0, 4, 2, 3] == 65536 and a.sum() == 3 * 65536
    o = out.reshape(2, B, H, W)
    for pol in range(2):
        for b in range(B):
            mx = a[pol, b].max()
            if mx:
                assert o[pol, b].max() == 1.0
                np.testing.assert_array_equal(o[pol, b], (a[pol, b].astype(np.float32) / np.float32(mx)))
            else:
                assert not o[pol, b].any()


def test_voxel_multi_env_and_skips(oracle_mod):
    rng = np.random.default_rng(3)
    envs = [(6, 4, 0, 1_000_000), (3, 5, 50_000, 2_050_000)]
    e0 = _events(rng, 200, 6, 4, 0, 1_000_000, env=0)
    e1 = _events(rng, 200, 3, 5, 50_000, 2_050_000, env=1)
    junk = _events(rng, 50, 6, 4, 0, 1_000_000, env=2)              # no such environment
    far = _events(rng, 50, 3, 5, 50_000, 2_050_000, env=1)
    far["x"] = 7                                                      # outside the sensor
    allev = np.concatenate([e0, e1, junk, far])
    rng.shuffle(allev)
    acc, out = oracle_mod.voxel_grid(allev, envs, bins=16)
    a0, o0 = oracle_mod.voxel_grid(e0, envs[:1], bins=16)
    n0 = a0.size
    np.testing.assert_array_equal(acc[:n0], a0)
    np.testing.assert_array_equal(out[:n0], o0)
    e1b = e1.copy()
    e1b["env"] = 0
    a1, _ = oracle_mod.voxel_grid(e1b, envs[1:], bins=16)
    np.testing.assert_array_equal(acc[n0:], a1)
