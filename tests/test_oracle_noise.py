"""Pins of the oracle's sensor non-idealities (Sec. 3.4): leak events, shot noise and hot
pixels, drawn from a counter-based Philox4x32-10 so that the CUDA path can reproduce them.
Statistical pins: rates against the binomial expectation, placement, polarity, and that the
noise leaves the signal events and the reference levels untouched."""
from pathlib import Path

import numpy as np
import pytest

from evis_testutil import TinyEnv, packed_total


GOLDEN = Path(__file__).parent / "golden"


def test_philox_known_answers(oracle_mod):
    for line in (GOLDEN / "philox4x32_10_kat.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        v = [int(w, 16) for w in line.split()]
        got = oracle_mod.philox(1, v[1], v[2], v[3], key=(v[4], v[5]), base=v[0])[0]
        assert [int(g) for g in got] == v[6:], line


def test_philox_is_uniform_and_counter_sensitive(oracle_mod):
    out = oracle_mod.philox(50_000, c1=3, c2=7, c3=1, key=(123, 456))
    u = out.ravel().astype(np.float64) / 2**32
    hist = np.histogram(u, bins=64, range=(0, 1))[0]
    expected = u.size / 64
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 64 + 5 * np.sqrt(2 * 64)           # 63 dof, ~5 sigma
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    # changing any counter word or the key changes every output word
    a = oracle_mod.philox(1000, c1=3, c2=7, c3=1, key=(123, 456))
    for b in (oracle_mod.philox(1000, c1=4, c2=7, c3=1, key=(123, 456)),
              oracle_mod.philox(1000, c1=3, c2=8, c3=1, key=(123, 456)),
              oracle_mod.philox(1000, c1=3, c2=7, c3=2, key=(123, 456)),
              oracle_mod.philox(1000, c1=3, c2=7, c3=1, key=(124, 456))):
        assert np.mean(a == b) < 0.01
    # neighbouring counters are uncorrelated
    assert abs(np.corrcoef(u[:-4:4], u[4::4])[0, 1]) < 0.02


def _static_run(oracle_mod, env, noise, L_seq, dt):
    n = packed_total([env])
    mv = np.zeros((n, 2), np.float32)
    z = np.ones(n, np.float32)
    o = oracle_mod.Oracle([env])
    if noise is not None:
        o.set_noise([noise])
    for L in L_seq:
        o.step(L, mv, z, dt)
    return o


def test_leak_rate_times_and_isolation(oracle_mod):
    env = TinyEnv(W=64, H=40, K=8, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    rng = np.random.default_rng(0)
    L_seq = [rng.normal(0, 1, n).astype(np.float32) for _ in range(4)]
    dt = 10_000_000
    quiet = _static_run(oracle_mod, env, None, L_seq, dt)
    noisy = _static_run(oracle_mod, env, dict(leak_hz=5.0, seed=99), L_seq, dt)
    e0, e1 = oracle_mod.sort_events(quiet.events()), oracle_mod.sort_events(noisy.events())
    np.testing.assert_array_equal(quiet.state()[0], noisy.state()[0])   # L_ref untouched
    s0 = set(map(bytes, e0.view(np.dtype((np.void, 16)))))
    extra = [r for r in e1 if bytes(r.tobytes()) not in s0]
    assert len(e1) - len(e0) == len(extra) and s0 <= set(map(bytes, e1.view(np.dtype((np.void, 16)))))
    trials = env.W * env.H * env.K * (len(L_seq) - 1)
    p = 5.0 * dt / env.K * 1e-9
    mean, sd = trials * p, np.sqrt(trials * p * (1 - p))
    assert abs(len(extra) - mean) < 5 * sd, (len(extra), mean)
    assert all(r["p"] == 1 for r in extra)
    t = np.array([r["t"] for r in extra], np.int64)
    assert np.all((t >= 0) & (t < (len(L_seq) - 1) * dt))
    # uniform over each sub-frame [t_{i-1}, t_i): flat across sub-frames, phase mean 1/2
    sub = dt // env.K
    per = np.bincount((t % dt) // sub, minlength=env.K)
    assert ((per - per.mean()) ** 2 / per.mean()).sum() < env.K + 5 * np.sqrt(2 * env.K)
    phase = (t % sub) / sub
    assert abs(phase.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(t))


def test_shot_noise_follows_darkness(oracle_mod):
    env = TinyEnv(W=64, H=32, K=8, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    L = np.zeros(n, np.float32)
    L[: env.W * env.H // 2] = -5.0      # top half dark (normalised intensity 0)
    L[env.W * env.H // 2:] = 5.0        # bottom half bright (normalised intensity 1)
    o = _static_run(oracle_mod, env, dict(shot_hz=20.0, lo=-5.0, hi=5.0, seed=7), [L] * 4, 10_000_000)
    ev = o.events()
    assert len(ev) > 50
    assert np.all(ev["y"] < env.H // 2)                     # only the dark half fires
    pos = (ev["p"] > 0).mean()
    assert abs(pos - 0.5) < 5 * np.sqrt(0.25 / len(ev))      # random polarity
    trials = env.W * env.H // 2 * env.K * 3
    p = 20.0 * 10_000_000 / env.K * 1e-9
    assert abs(len(ev) - trials * p) < 5 * np.sqrt(trials * p)


def test_hot_pixels_are_a_fixed_subset(oracle_mod):
    env = TinyEnv(W=50, H=40, K=4, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    L = np.zeros(n, np.float32)
    o = _static_run(oracle_mod, env, dict(hot_hz=200.0, hot_fraction=0.05, seed=11), [L] * 7,
                    10_000_000)
    ev = o.events()
    pix = ev["y"].astype(np.int64) * env.W + ev["x"]
    counts = np.bincount(pix, minlength=env.W * env.H)
    hot = counts > 0
    frac = hot.mean()
    assert 0.02 < frac < 0.08
    # a hot pixel fires with p = 0.5 per sub-frame: over 24 sub-frames none stays silent
    assert counts[hot].min() >= 3 and np.all(ev["p"] == 1)
    o2 = _static_run(oracle_mod, env, dict(hot_hz=200.0, hot_fraction=0.05, seed=11), [L] * 3,
                     10_000_000)
    ev2 = o2.events()
    assert set(ev2["y"].astype(np.int64) * env.W + ev2["x"]) <= set(np.nonzero(hot)[0])


def test_noise_is_deterministic_per_seed(oracle_mod):
    env = TinyEnv(W=32, H=16, K=4, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    L = np.zeros(n, np.float32)
    runs = [oracle_mod.sort_events(_static_run(oracle_mod, env, dict(leak_hz=50.0, seed=s), [L] * 3,
                                               10_000_000).events()) for s in (1, 1, 2)]
    np.testing.assert_array_equal(runs[0], runs[1])
    assert not np.array_equal(runs[0], runs[2])
    with pytest.raises(ValueError):
        oracle_mod.Oracle([env]).set_noise([dict(hot_fraction=1.5)])


def test_leak_fires_in_holes_and_streams_differ_per_env(oracle_mod):
    """Leak and hot-pixel noise do not need a sample: pixels whose sources all have invalid
    depth (holes) still leak.  Two environments with the same seed draw distinct streams."""
    env = TinyEnv(W=48, H=32, K=8, c_on=0.2, c_off=0.2)
    envs = [env, env]
    n = packed_total(envs)
    mv = np.zeros((n, 2), np.float32)
    z = np.ones(n, np.float32)
    z[: env.W * env.H // 2] = 0.0              # top half of env 0: invalid depth, no sample
    L = np.zeros(n, np.float32)
    o = oracle_mod.Oracle(envs)
    o.set_noise([dict(leak_hz=50.0, seed=5)] * 2)
    for _ in range(3):
        o.step(L, mv, z, 10_000_000)
    ev = o.events()
    e0, e1 = ev[ev["env"] == 0], ev[ev["env"] == 1]
    top = e0[e0["y"] < env.H // 2]
    half = env.W * env.H // 2 * env.K * 2
    p = 50.0 * 10_000_000 / env.K * 1e-9
    assert abs(len(top) - half * p) < 5 * np.sqrt(half * p)
    k0 = set(zip(e0["x"].tolist(), e0["y"].tolist(), e0["t"].tolist()))
    k1 = set(zip(e1["x"].tolist(), e1["y"].tolist(), e1["t"].tolist()))
    assert len(k0 & k1) < 0.05 * min(len(k0), len(k1))
