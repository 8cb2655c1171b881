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
    """Only dark pixels fire, with random polarity; a pixel darker than `lo` fires at the
    same rate as one at `lo` (the normalised intensity clamps at 0)."""
    env = TinyEnv(W=64, H=48, K=8, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    L = np.zeros(n, np.float32)
    band = env.W * env.H // 3
    L[:band] = -10.0                    # top third darker than lo
    L[band:2 * band] = -5.0             # middle third at lo (normalised intensity 0)
    L[2 * band:env.W * env.H] = 5.0     # bottom third bright (normalised intensity 1)
    o = _static_run(oracle_mod, env, dict(shot_hz=20.0, lo=-5.0, hi=5.0, seed=7), [L] * 4, 10_000_000)
    ev = o.events()
    assert len(ev) > 50
    assert np.all(ev["y"] < 2 * env.H // 3)                 # only the dark two thirds fire
    pos = (ev["p"] > 0).mean()
    assert abs(pos - 0.5) < 5 * np.sqrt(0.25 / len(ev))      # random polarity
    trials = band * env.K * 3
    p = 20.0 * 10_000_000 / env.K * 1e-9
    for rows in (ev["y"] < env.H // 3, (ev["y"] >= env.H // 3) & (ev["y"] < 2 * env.H // 3)):
        assert abs(rows.sum() - trials * p) < 5 * np.sqrt(trials * p), (rows.sum(), trials * p)


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


def _subframe_of(t, dt, K):
    """Sub-frame index i (1..K) of event times inside a gap starting at a multiple of dt
    (dt divisible by K)."""
    return (t % dt) // (dt // K) + 1


def test_competing_sources_fire_at_most_once_with_the_summed_probability(oracle_mod):
    """Leak, shot and hot noise share one draw per pixel-sub-frame: at most one noise event
    per pixel and sub-frame, with probability p_leak + p_shot + p_hot, split by source; with
    the probabilities summing past 1 every pixel-sub-frame fires exactly once."""
    env = TinyEnv(W=64, H=48, K=8, c_on=0.2, c_off=0.2)
    n = packed_total([env])
    L = np.full(n, -5.0, np.float32)          # dark everywhere: normalised intensity 0
    dt = 8_000_000                             # sub-frames of 1 ms
    spec = dict(leak_hz=100.0, shot_hz=200.0, hot_hz=300.0, hot_fraction=1.0, lo=-5.0, hi=5.0, seed=3)
    o = _static_run(oracle_mod, env, spec, [L] * 5, dt)
    ev = o.events()
    i = _subframe_of(ev["t"].astype(np.int64), dt, env.K)
    key = (ev["t"].astype(np.int64) // dt) * 10**6 + (ev["y"].astype(np.int64) * env.W + ev["x"]) * 16 + i
    assert len(np.unique(key)) == len(ev)                    # one event per pixel-sub-frame
    trials = env.W * env.H * env.K * 4
    p_on, p_off = 0.1 + 0.3 + 0.1, 0.1                       # shot splits its 0.2 in halves
    for cnt, p in (((ev["p"] > 0).sum(), p_on), ((ev["p"] < 0).sum(), p_off)):
        assert abs(cnt - trials * p) < 5 * np.sqrt(trials * p * (1 - p)), (cnt, trials * p)
    sat = _static_run(oracle_mod, env, dict(spec, leak_hz=700.0), [L] * 2, dt).events()
    assert len(sat) == env.W * env.H * env.K


def test_shot_noise_follows_the_pixels_interpolated_intensity(oracle_mod):
    """Keyframe A dark, B bright, no motion: the pixel's log intensity rises linearly over the
    gap, so the shot probability of sub-frame i is shot_hz dts (1 - i / K), zero at i = K."""
    env = TinyEnv(W=64, H=64, K=8, c_on=50.0, c_off=50.0)   # thresholds no signal event reaches
    n = packed_total([env])
    dark, bright = np.full(n, -5.0, np.float32), np.full(n, 5.0, np.float32)
    dt = 8_000_000
    o = _static_run(oracle_mod, env, dict(shot_hz=400.0, lo=-5.0, hi=5.0, seed=21),
                    [dark, bright, dark, bright, dark, bright, dark], dt)
    ev = o.events()
    gap = ev["t"].astype(np.int64) // dt
    rising = (gap % 2) == 0                                  # gaps dark -> bright
    i = _subframe_of(ev["t"].astype(np.int64), dt, env.K)
    per = np.bincount(i[rising], minlength=env.K + 1)[1:]
    trials = env.W * env.H * 3                               # three rising gaps
    p = 0.4 * (1.0 - np.arange(1, env.K + 1) / env.K)
    exp = trials * p
    assert per[-1] == 0
    z = (per[:-1] - exp[:-1]) / np.sqrt(exp[:-1] * (1 - p[:-1]))
    assert np.all(np.abs(z) < 5), (per, exp)
    per_fall = np.bincount(i[~rising], minlength=env.K + 1)[1:]   # bright -> dark: rising rate
    assert per_fall[0] < per_fall[-1] and per[0] > per[-1]


def test_draw_and_time_words_follow_the_counter_layout(oracle_mod):
    """The draw of sub-frame i is word (i - 1) mod 4 of Philox4x32-10 at (pixel, gap,
    floor((i - 1) / 4), 0); a fired leak takes its time from word 0 at (pixel, gap, i, 1):
    recomputed here from the generator (pinned by its known answers) and the binary32
    threshold, event by event."""
    env = TinyEnv(W=16, H=8, K=8, c_on=50.0, c_off=50.0)
    n = packed_total([env])
    dt = 8_000_000
    seed = (5 << 32) | 77
    o = _static_run(oracle_mod, env, dict(leak_hz=500.0, seed=seed), [np.zeros(n, np.float32)] * 3, dt)
    got = oracle_mod.sort_events(o.events())
    k = (77, 5 ^ 0)                                           # (seed low, seed high ^ env)
    d = dt // env.K
    thr = np.float32(np.float32(500.0) * np.float32(np.float32(d) * np.float32(1e-9))) * np.float32(2**24)
    want = []
    for g in range(2):
        for pix in range(env.W * env.H):
            for i in range(1, env.K + 1):
                u = oracle_mod.philox(1, g, (i - 1) // 4, 0, key=k, base=pix)[0][(i - 1) % 4]
                if np.float32(int(u) >> 8) < thr:
                    v = int(oracle_mod.philox(1, g, i, 1, key=k, base=pix)[0][0])
                    t0 = g * dt + (i - 1) * d
                    want.append((t0 + (v * d >> 32), pix % env.W, pix // env.W, 0, 1))
    want = oracle_mod.sort_events(np.array(want, dtype=got.dtype))
    assert 100 < len(want)
    np.testing.assert_array_equal(got, want)
