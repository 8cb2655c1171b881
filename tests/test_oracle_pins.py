"""Pins of the oracle against things other than itself (CPU only).

Each test checks the oracle against brute force, a closed form, an invariant or a golden value
taken from the paper, chosen so that a dropped term, a flipped sign or a transposed operand in
the oracle fails at least one of them:

* splat winners   -- gather-form brute force of Eq. 6/7 over all sources (tiny images)
* warp direction  -- integer and fractional translations against the shifted image (Eq. 5)
* depth blend     -- a layer whose depth moves through another's flips at f = 1/3 (Eq. 7)
* nearer wins     -- two depth layers (Eq. 6)
* event model     -- constant image, single-pixel ramp, per-pixel linear ESIM closed form,
                     conservation of the reference level (Eq. 4 and Sec. 3.2)
* non-idealities  -- refractory filter equals a greedy filter of the unfiltered stream,
                     per-pixel ON/OFF thresholds (Eq. 8, Sec. 3.4)
* luminance / log -- Rec. 709 golden values (Eq. 3) and closed-form logarithms
"""
import os

import numpy as np
import pytest

from evis_testutil import EMPTY, TinyEnv, packed_total, split_trace

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F32 = np.float32


# ----------------------------------------------------------------------------------------
# brute force of the z-buffer splat (gather form, written from Eqs. 5-7)
# ----------------------------------------------------------------------------------------

def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)


def _valid(z):
    return (z > 0) & np.isfinite(z)


def _nn_depth(Zother, W, H, ux, uy, own):
    nx = np.floor(ux + F32(0.5))
    ny = np.floor(uy + F32(0.5))
    inside = (nx >= 0) & (nx <= W - 1) & (ny >= 0) & (ny <= H - 1)
    out = own.copy()
    ix = np.where(inside, nx, 0).astype(np.int64)
    iy = np.where(inside, ny, 0).astype(np.int64)
    z = Zother[iy * W + ix]
    take = inside & _valid(z)
    out[take] = z[take]
    return out


def brute_force_keys(W, H, K, i, mvA, ZA, mvB, ZB, tie_index=False):
    """Keys [2, H*W] for substep i: for each target, min over every covering source."""
    f = F32(i) / F32(K)
    g = F32(1) - f
    yy, xx = np.mgrid[0:H, 0:W]
    xs = xx.ravel().astype(np.float32)
    ys = yy.ravel().astype(np.float32)
    src = np.arange(H * W, dtype=np.uint64)
    # A sources: endpoints p_A = p, p_B = p - m_A(p); B sources: p_B = p, p_A = p + m_B(p)
    qAx, qAy = xs - f * mvA[:, 0], ys - f * mvA[:, 1]
    zA_t = g * ZA + f * _nn_depth(ZB, W, H, xs - mvA[:, 0], ys - mvA[:, 1], ZA)
    qBx, qBy = xs + g * mvB[:, 0], ys + g * mvB[:, 1]
    zB_t = g * _nn_depth(ZA, W, H, xs + mvB[:, 0], ys + mvB[:, 1], ZB) + f * ZB
    out = np.full((2, H * W), EMPTY, dtype=np.uint64)
    for d, (qx, qy, zt, zs) in enumerate(((qAx, qAy, zA_t, ZA), (qBx, qBy, zB_t, ZB))):
        x0, y0 = np.floor(qx), np.floor(qy)
        ax, ay = qx - x0, qy - y0
        hi = _bits(zt) << np.uint64(32)
        for t in range(H * W):
            tx, ty = t % W, t // W
            wx = np.where(x0 == tx, F32(1) - ax, np.where(x0 + 1 == tx, ax, F32(0)))
            wy = np.where(y0 == ty, F32(1) - ay, np.where(y0 + 1 == ty, ay, F32(0)))
            w = (wx * wy).astype(np.float32)
            cover = _valid(zs) & (w > 0)
            if not cover.any():
                continue
            if tie_index:
                wq = np.zeros_like(src)
            else:
                wq = np.minimum(((F32(1) - w) * F32(256)).astype(np.uint64), np.uint64(255))
            keys = hi | (wq << np.uint64(24)) | src
            out[d, t] = keys[cover].min()
    return out


def _run(oracle_mod, envs, frames, mvs, Zs, dt, flags=0, trace=False, eps=1e-4):
    o = oracle_mod.Oracle(envs, eps=eps, flags=flags)
    traces = []
    for fr, mv, z in zip(frames, mvs, Zs):
        r = o.step(fr, mv, z, dt, trace=trace)
        traces.append(r)
    return o, traces


@pytest.mark.parametrize("seed,W,H,K,tie", [(1, 7, 5, 1, False), (2, 9, 9, 3, False),
                                            (3, 8, 6, 4, True), (4, 6, 7, 2, False),
                                            (5, 10, 4, 5, False)])
def test_splat_matches_brute_force(oracle_mod, seed, W, H, K, tie):
    rng = np.random.default_rng(seed)
    n = H * W
    npk = (n + 3) // 4 * 4

    def mv_field():
        choices = np.array([0, 0.5, -0.5, 1, -1, 1.5, 2, -2.25, 0.25, 3, -7, 40, np.nan],
                           dtype=np.float32)
        mv = rng.choice(choices, size=(npk, 2)).astype(np.float32)
        rnd = rng.random((npk, 2)) < 0.4
        mv[rnd] = rng.uniform(-3, 3, size=rnd.sum()).astype(np.float32)
        return mv

    def depth():
        choices = np.array([1, 2, 2, 3, 3, 3, 2.5, np.inf, np.nan, -1, 0], dtype=np.float32)
        z = rng.choice(choices, size=npk).astype(np.float32)
        rnd = rng.random(npk) < 0.3
        z[rnd] = rng.uniform(0.5, 4, size=rnd.sum()).astype(np.float32)
        return z

    env = TinyEnv(W=W, H=H, K=K)
    L0 = rng.normal(size=npk).astype(np.float32)
    L1 = rng.normal(size=npk).astype(np.float32)
    mv0, mv1, z0, z1 = mv_field(), mv_field(), depth(), depth()
    flags = oracle_mod.TIE_INDEX if tie else 0
    _, tr = _run(oracle_mod, [env], [L0, L1], [mv0, mv1], [z0, z1], 1000, flags, trace=True)
    keys, lint = split_trace([env], *tr[1])[0]
    for i in range(1, K + 1):
        bf = brute_force_keys(W, H, K, i, mv0[:n], z0[:n], mv1[:n], z1[:n], tie_index=tie)
        np.testing.assert_array_equal(keys[i - 1].reshape(2, -1), bf, err_msg=f"substep {i}")


# ----------------------------------------------------------------------------------------
# warp direction: translations (Eq. 5) against the shifted image
# ----------------------------------------------------------------------------------------

def _plane_scene(scenes_mod, W, H, vx, vy, depth=4.0, tex=0, seed=11, bright=0.0):
    return [scenes_mod.Layer(kind=0, depth0=depth, cx0=W / 2, cy0=H / 2, vx=vx, vy=vy,
                             tex_kind=tex, seed=seed, cell=8.0, bright_rate=bright)]


def _render_env(scenes_mod, env_scene, k):
    return scenes_mod.render([env_scene], k)


@pytest.mark.parametrize("d,K", [(4, 4), (-8, 4), (2, 2), (8, 8)])
def test_integer_translation_reproduces_shifted_image(oracle_mod, scenes_mod, d, K):
    """Plane translating by d px/frame; K a power of two so f and 1-f are exact and f*d is an
    integer at every substep: L_i(x) = T(x - f d)."""
    W, H = 24, 10
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.3, c_off=0.3,
                             layers=_plane_scene(scenes_mod, W, H, float(d), 0.0))
    kf = [_render_env(scenes_mod, es, k) for k in range(2)]
    assert np.all(kf[1].mv[:W * H, 0] == -d)
    _, tr = _run(oracle_mod, [es], [k.L for k in kf], [k.mv for k in kf], [k.Z for k in kf],
                 10_000, flags=oracle_mod.MODE_B_PRIMARY, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    for i in range(1, K + 1):
        shift = d * i // K
        lay = _plane_scene(scenes_mod, W, H, float(d), 0.0)
        lay[0].cx0 += shift                      # the layer moved by f*d
        ref = scenes_mod.render([scenes_mod.EnvScene(W=W, H=H, K=K, c_on=1, c_off=1,
                                                     layers=lay)], 0).L[:W * H]
        np.testing.assert_array_equal(lint[i - 1].ravel(), ref, err_msg=f"substep {i}")


@pytest.mark.parametrize("d,K", [(3, 4), (5, 8), (-1.5, 3)])
def test_fractional_translation_takes_nearest_source(oracle_mod, scenes_mod, d, K):
    """Constant depth: every source ties on depth, so the larger bilinear weight (the nearest
    source) wins and exact half-way ties go to the lower source index.  B-primary warp:
    target x receives source round(x + (1-f) d); A alone: source round(x - f d)."""
    W, H = 20, 6
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.3, c_off=0.3,
                             layers=_plane_scene(scenes_mod, W, H, float(d), 0.0))
    kf = [_render_env(scenes_mod, es, k) for k in range(2)]
    n = W * H
    _, tr = _run(oracle_mod, [es], [k.L for k in kf], [k.mv for k in kf], [k.Z for k in kf],
                 10_000, flags=0, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    xs = np.arange(W)
    for i in range(1, K + 1):
        f = i / K
        for dirn, pos in ((1, xs + (1 - f) * d), (0, xs - f * d)):
            # nearest integer, half-way cases to the lower index
            fl = np.floor(pos)
            src = np.where(pos - fl > 0.5, fl + 1, fl).astype(np.int64)
            exact = np.abs(pos - np.round(pos)) < 1e-6
            src = np.where(exact, np.round(pos), src).astype(np.int64)
            ok = (src >= 0) & (src < W)
            got = keys[i - 1, dirn]            # [H, W]
            for y in range(H):
                for x in range(W):
                    if ok[x]:
                        assert got[y, x] != EMPTY
                        assert int(got[y, x]) & 0xFFFFFF == y * W + src[x], (i, dirn, x, y)
        # holes only where neither direction has a source
        both_missing = (keys[i - 1, 0] == EMPTY) & (keys[i - 1, 1] == EMPTY)
        assert not both_missing.any()
    del n


# ----------------------------------------------------------------------------------------
# depth: nearer wins (Eq. 6) and the depth interpolation along the correspondence (Eq. 7)
# ----------------------------------------------------------------------------------------

def test_two_layers_nearer_wins(oracle_mod, scenes_mod):
    W, H, K = 32, 24, 4
    plane = scenes_mod.Layer(kind=0, depth0=5.0, cx0=16, cy0=12, vx=1.0, tex_kind=1, mu=0.0)
    disk = scenes_mod.Layer(kind=1, radius=6.0, depth0=2.0, cx0=12, cy0=12, vx=3.0, vy=1.0,
                            tex_kind=1, mu=1.0)
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.3, c_off=0.3, layers=[plane, disk])
    kf = [scenes_mod.render([es], k) for k in range(2)]
    _, tr = _run(oracle_mod, [es], [k.L for k in kf], [k.mv for k in kf], [k.Z for k in kf],
                 10_000, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    n = W * H
    yy, xx = np.mgrid[0:H, 0:W]
    for dirn, kfr in ((0, kf[0]), (1, kf[1])):
        is_disk = kfr.Z[:n] == np.float32(2.0)
        mv = kfr.mv[:n]
        for i in range(1, K + 1):
            f = i / K
            s = -f if dirn == 0 else (1 - f)
            qx = xx.ravel() + s * mv[:, 0]
            qy = yy.ravel() + s * mv[:, 1]
            # targets covered by any disk source's footprint
            cov = np.zeros((H, W), dtype=bool)
            for q in np.nonzero(is_disk)[0]:
                x0, y0 = int(np.floor(qx[q])), int(np.floor(qy[q]))
                ax, ay = qx[q] - x0, qy[q] - y0
                for cx, wx in ((x0, 1 - ax), (x0 + 1, ax)):
                    for cy, wy in ((y0, 1 - ay), (y0 + 1, ay)):
                        if wx * wy > 1e-6 and 0 <= cx < W and 0 <= cy < H:
                            cov[cy, cx] = True
            win = keys[i - 1, dirn]
            srcs = (win & np.uint64(0xFFFFFF)).astype(np.int64)
            assert np.all(is_disk[srcs[cov]]), f"dir {dirn} substep {i}"


def test_depth_interpolation_switches_at_one_third(oracle_mod, scenes_mod):
    """A disk whose depth goes 2 -> 5 over the gap passes behind a plane at depth 3 when
    (1-f) 2 + f 5 > 3, i.e. f > 1/3 (Eq. 7)."""
    W, H, K = 24, 16, 6
    plane = scenes_mod.Layer(kind=0, depth0=3.0, cx0=12, cy0=8, tex_kind=1, mu=0.0)
    disk = scenes_mod.Layer(kind=1, radius=5.0, depth0=2.0, depth_rate=3.0, cx0=12, cy0=8,
                            tex_kind=1, mu=1.0)
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.3, c_off=0.3, layers=[plane, disk])
    kf = [scenes_mod.render([es], k) for k in range(2)]
    # keyframe A shows the disk (depth 2 < 3); keyframe B shows the plane (5 > 3)
    assert np.any(kf[0].Z == 2.0) and not np.any(kf[1].Z == 5.0)
    _, tr = _run(oracle_mod, [es], [k.L for k in kf], [k.mv for k in kf], [k.Z for k in kf],
                 10_000, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    centre = (8, 12)
    for i in range(1, K + 1):
        f = i / K
        ka = keys[i - 1, 0][centre]
        zt = np.uint32(int(ka) >> 32).view(np.float32)
        # A's disk source at the centre carries Z~ = (1-f)*2 + f*Z_B(p) with Z_B = 3 (plane)
        assert abs(zt - ((1 - f) * 2 + f * 3)) < 1e-6
        # the blended value follows the nearer layer of each direction
        if f < 1 / 3 - 1e-9:
            assert lint[i - 1][centre] == pytest.approx((1 - f) * 1.0 * np.log(10) + 0.0, abs=1e-6)


# ----------------------------------------------------------------------------------------
# event model (Eq. 4 and the reference update of Sec. 3.2)
# ----------------------------------------------------------------------------------------

def _static(n, z=1.0):
    return np.zeros((n, 2), dtype=np.float32), np.full(n, z, dtype=np.float32)


def test_constant_image_gives_no_events(oracle_mod):
    rng = np.random.default_rng(7)
    env = TinyEnv(W=13, H=11, K=6, c_on=0.1, c_off=0.1)
    n = packed_total([env])
    L = np.full(n, 0.7, dtype=np.float32)
    frames = [L] * 4
    mvs = [rng.uniform(-6, 6, size=(n, 2)).astype(np.float32) for _ in range(4)]
    zs = [rng.uniform(0.5, 9, size=n).astype(np.float32) for _ in range(4)]
    o, _ = _run(oracle_mod, [env], frames, mvs, zs, 5_000_000)
    assert len(o.events()) == 0


@pytest.mark.parametrize("n_ev,C,K,sign", [(5, 0.25, 8, 1), (3, 0.5, 4, -1), (1, 0.125, 16, 1)])
def test_single_pixel_ramp_closed_form(oracle_mod, n_ev, C, K, sign):
    """Static pixel with L going from 0 to (n + 1/2) C: exactly n events, at
    t_k = T0 + dt k C / |dL| (linear in L over the gap), polarity sgn(dL)."""
    env = TinyEnv(W=4, H=1, K=K, c_on=C, c_off=C, t0_ns=1_000)
    npx = packed_total([env])
    mv, z = _static(npx)
    L0 = np.zeros(npx, dtype=np.float32)
    L1 = np.zeros(npx, dtype=np.float32)
    dL = sign * (n_ev + 0.5) * C
    L1[2] = dL
    dt = 33_333_333
    o, _ = _run(oracle_mod, [env], [L0, L1], [mv, mv], [z, z], dt)
    ev = oracle_mod.sort_events(o.events())
    assert len(ev) == n_ev
    assert np.all(ev["x"] == 2) and np.all(ev["y"] == 0) and np.all(ev["p"] == sign)
    want = 1_000 + dt * np.arange(1, n_ev + 1) * C / abs(dL)
    assert np.all(np.abs(ev["t"] - want) <= 1.0), (ev["t"], want)


def test_emission_limit_is_reported_and_keeps_eq4_state(oracle_mod):
    """Eq. 4 sets n = floor(|dL| / C) with no bound; a pixel may emit at most MAX_CROSSINGS
    (4096) events per sub-frame.  At the limit every crossing is emitted; above it none is
    (nothing truncated), the step reports it, and the reference still moves by the whole
    p n C of Eq. 4 (closed forms with C = 1/4, K = 1 so that the sub-frame is keyframe B)."""
    C = 0.25
    env = TinyEnv(W=6, H=1, K=1, c_on=C, c_off=C, t0_ns=0)
    npx = packed_total([env])
    mv, z = _static(npx)
    L0 = np.zeros(npx, dtype=np.float32)
    L1 = np.zeros(npx, dtype=np.float32)
    lim = oracle_mod.MAX_CROSSINGS
    L1[0] = (lim + 0.5) * C          # n = 4096: all emitted
    L1[1] = (lim + 1.5) * C          # n = 4097: over the limit
    L1[2] = -(5000 + 0.5) * C        # n = 5000, OFF
    L1[3] = 2.5 * C                  # n = 2
    L1[4] = np.float32(3e38)         # |dL| / C overflows to inf: n = inf
    dt = 1_000_000
    o = oracle_mod.Oracle([env], flags=oracle_mod.IN_LOG)
    o.step(L0, mv, z, dt)
    assert not o.last_over_limit
    o.step(L1, mv, z, dt)
    assert o.last_over_limit
    assert o.over_limit().tolist() == [3]
    ev = o.events()
    per_x = np.bincount(ev["x"], minlength=6)
    assert per_x.tolist() == [lim, 0, 0, 2, 0, 0]
    assert np.all(ev["p"][ev["x"] == 0] == 1)
    Lref = o.state()[0][:env.W]
    want = np.array([lim * C, (lim + 1) * C, -5000 * C, 2 * C, np.inf, 0], dtype=np.float32)
    np.testing.assert_array_equal(Lref, want)
    # the next gap starts from the exact Eq. 4 state: 0.75 above the reference gives 3 events
    L2 = L1.copy()
    L2[1] = np.float32((lim + 1) * C + 0.75)
    o.step(L2, mv, z, dt)
    # pixel 4's infinite reference stays out of range (inf - L), and Eq. 4 makes it NaN
    assert o.last_over_limit and o.over_limit().tolist() == [4]
    assert np.isnan(o.state()[0][4])
    ev2 = o.events()
    assert np.bincount(ev2["x"], minlength=6).tolist() == [0, 3, 0, 0, 0, 0]
    # levels (lim + 2, lim + 3, lim + 4) C between L = (lim + 1.5) C at t0 + dt and
    # (lim + 4) C at t0 + 2 dt
    want_t = dt + dt * (np.array([0.5, 1.5, 2.5]) / 2.5)
    assert np.all(np.abs(np.sort(ev2["t"]) - want_t) <= 1.0)


def _linear_esim(L_seq, C, t0, dt):
    """Per-pixel textbook ESIM on a piecewise-linear log-intensity signal (fp64).

    The signal goes linearly from L_seq[s] to L_seq[s+1] over [t0 + s dt, t0 + (s+1) dt];
    the reference starts at L_seq[0] and moves by +-C at each crossing.  Returns per-pixel
    lists of (t, polarity) and the closing reference, plus a mask of pixels whose crossing
    count sits within 1e-4 C of a rounding boundary (excluded from exact comparison)."""
    L_seq = [np.asarray(x, dtype=np.float64) for x in L_seq]
    npx = L_seq[0].size
    ref = L_seq[0].copy()
    events = [[] for _ in range(npx)]
    fragile = np.zeros(npx, dtype=bool)
    for s in range(len(L_seq) - 1):
        a, b = L_seq[s], L_seq[s + 1]
        for p in range(npx):
            d = b[p] - ref[p]
            q = abs(d) / C
            if abs(q - round(q)) < 1e-4:
                fragile[p] = True
            n = int(np.floor(q))
            pol = 1 if d > 0 else -1
            for k in range(1, n + 1):
                lev = ref[p] + pol * k * C
                t = t0 + s * dt + dt * (lev - a[p]) / (b[p] - a[p])
                events[p].append((t, pol))
            ref[p] += pol * n * C
    return events, ref, fragile


def test_zero_motion_reduces_to_linear_esim(oracle_mod):
    """mv = 0, constant depth: each substep value is (1-f) L_A + f L_B and the event stream is
    the per-pixel linear-interpolation ESIM of the keyframe sequence."""
    rng = np.random.default_rng(21)
    env = TinyEnv(W=9, H=7, K=8, c_on=0.2, c_off=0.2, t0_ns=0)
    npx = packed_total([env])
    n = env.W * env.H
    mv, z = _static(npx)
    Ls = [rng.normal(0, 1.0, size=npx).astype(np.float32) for _ in range(4)]
    dt = 10_000_000
    o, tr = _run(oracle_mod, [env], Ls, [mv] * 4, [z] * 4, dt, trace=True)
    # interpolated values are the per-pixel time blend
    keys, lint = split_trace([env], *tr[1])[0]
    for i in range(1, env.K + 1):
        f = np.float32(i) / np.float32(env.K)
        g = np.float32(1) - f
        want = (g * Ls[0][:n] + f * Ls[1][:n]).reshape(env.H, env.W)
        np.testing.assert_array_equal(lint[i - 1], want)
    ev = oracle_mod.sort_events(o.events())
    exp, ref, fragile = _linear_esim([x[:n] for x in Ls], 0.2, 0, dt)
    for p in range(n):
        if fragile[p]:
            continue
        x, y = p % env.W, p // env.W
        mine = ev[(ev["x"] == x) & (ev["y"] == y)]
        want = exp[p]
        assert len(mine) == len(want), (p, len(mine), len(want))
        if want:
            wt = np.array([w[0] for w in want])
            wp = np.array([w[1] for w in want])
            assert np.all(mine["p"] == wp)
            # binary32 interpolation error of the level inside one substep
            slope = np.abs(np.diff([x[p] for x in Ls])).min()
            tol = 1.0 + 2e-6 * dt / max(slope, 1e-3)
            assert np.all(np.abs(mine["t"] - wt) <= tol), (p, mine["t"], wt)


def test_conservation_of_reference_level(oracle_mod, scenes_mod):
    """Without refractory filtering every crossing is emitted, so the reference moves by
    exactly the sum of +-theta over the pixel's events and ends within theta of L_K."""
    w = scenes_mod.config1()
    es = w.envs[0]
    es_small = scenes_mod.EnvScene(W=48, H=40, K=6, c_on=0.2, c_off=0.3, layers=es.layers)
    kfs = [scenes_mod.render([es_small], k) for k in range(4)]
    o, _ = _run(oracle_mod, [es_small], [k.L for k in kfs], [k.mv for k in kfs],
                [k.Z for k in kfs], w.dt_ns)
    Lref_end, _, _ = o.state()
    ev = o.events()
    n = es_small.W * es_small.H
    sums = np.zeros(n)
    idx = ev["y"].astype(np.int64) * es_small.W + ev["x"]
    np.add.at(sums, idx, np.where(ev["p"] > 0, 0.2, -0.3))
    L0 = kfs[0].L[:n].astype(np.float64)
    assert np.allclose(Lref_end[:n] - L0, sums, atol=2e-5)
    LK = kfs[-1].L[:n]
    assert np.all(np.abs(LK - Lref_end[:n]) < 0.3 + 1e-5)
    assert len(ev) > 100


def test_refractory_is_greedy_filter_of_unfiltered_stream(oracle_mod, scenes_mod):
    """Sec. 3.4: after firing at t_last a pixel suppresses events until t - t_last >= tau.
    The reference level moves on every crossing, so the filtered stream is the greedy
    subsequence of the unfiltered one with spacing >= tau."""
    tau = 700_000
    base = scenes_mod.config1().envs[0]
    mk = lambda r: scenes_mod.EnvScene(W=40, H=32, K=8, c_on=0.15, c_off=0.15,  # noqa: E731
                                       refractory_ns=r, layers=base.layers)
    kfs = [scenes_mod.render([mk(0)], k) for k in range(3)]
    args = ([k.L for k in kfs], [k.mv for k in kfs], [k.Z for k in kfs], 33_333_333)
    o0, _ = _run(oracle_mod, [mk(0)], *args)
    o1, _ = _run(oracle_mod, [mk(tau)], *args)
    e0 = oracle_mod.sort_events(o0.events())
    e1 = oracle_mod.sort_events(o1.events())
    assert len(e1) < len(e0)
    keep = []
    last = {}
    for r in e0:
        key = (int(r["x"]), int(r["y"]))
        if key not in last or int(r["t"]) - last[key] >= tau:
            keep.append(r)
            last[key] = int(r["t"])
    keep = oracle_mod.sort_events(np.array(keep, dtype=e0.dtype))
    np.testing.assert_array_equal(e1, keep)


def test_per_pixel_on_off_thresholds(oracle_mod):
    """Eq. 8: ON crossings use theta_ON, OFF crossings theta_OFF, per pixel."""
    env = TinyEnv(W=4, H=1, K=4, c_on=1.0, c_off=1.0)
    con = np.array([0.1, 0.25, 0.5, 0.3], dtype=np.float32)
    coff = np.array([0.4, 0.125, 0.2, 0.3], dtype=np.float32)
    env.c_on_map, env.c_off_map = con, coff
    npx = packed_total([env])
    mv, z = _static(npx)
    L0 = np.zeros(npx, dtype=np.float32)
    L1 = np.array([1.05, -1.05, 1.05, -1.05], dtype=np.float32)
    o, _ = _run(oracle_mod, [env], [L0, L1], [mv, mv], [z, z], 1_000_000)
    ev = o.events()
    counts = np.bincount(ev["x"], minlength=4)
    assert list(counts) == [10, 8, 2, 3]
    assert np.all(ev["p"][ev["x"] % 2 == 0] == 1) and np.all(ev["p"][ev["x"] % 2 == 1] == -1)


def test_first_keyframe_sets_reference_and_holes_hold_state(oracle_mod):
    env = TinyEnv(W=6, H=2, K=4, c_on=0.2, c_off=0.2)
    npx = packed_total([env])
    mv, z = _static(npx)
    L0 = np.linspace(-1, 1, npx).astype(np.float32)
    o = oracle_mod.Oracle([env])
    o.step(L0, mv, z, 1000)
    assert len(o.events()) == 0
    Lref, tl, clk = o.state()
    np.testing.assert_array_equal(Lref, L0)
    assert np.all(tl == np.iinfo(np.int64).min)
    # invalid depth everywhere in both keyframes: no source, no sample, nothing changes
    zbad = np.full(npx, np.nan, dtype=np.float32)
    o2 = oracle_mod.Oracle([env])
    o2.step(L0, mv, zbad, 1000)
    o2.step(L0 + 5, mv, zbad, 1000)
    assert len(o2.events()) == 0
    np.testing.assert_array_equal(o2.state()[0], L0)
    assert o2.state()[2][0] == 1000


def test_substep_K_equals_keyframe_B(oracle_mod, scenes_mod):
    w = scenes_mod.config1()
    es = scenes_mod.EnvScene(W=40, H=36, K=5, c_on=0.2, c_off=0.2, layers=w.envs[0].layers)
    kfs = [scenes_mod.render([es], k) for k in range(2)]
    _, tr = _run(oracle_mod, [es], [k.L for k in kfs], [k.mv for k in kfs], [k.Z for k in kfs],
                 1000, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    np.testing.assert_array_equal(lint[-1].ravel(), kfs[1].L[:es.W * es.H])


def test_b_primary_uses_b_where_present(oracle_mod, scenes_mod):
    w = scenes_mod.config1()
    es = scenes_mod.EnvScene(W=40, H=36, K=4, c_on=0.2, c_off=0.2, layers=w.envs[0].layers)
    kfs = [scenes_mod.render([es], k) for k in range(2)]
    _, tr = _run(oracle_mod, [es], [k.L for k in kfs], [k.mv for k in kfs], [k.Z for k in kfs],
                 1000, flags=oracle_mod.MODE_B_PRIMARY, trace=True)
    keys, lint = split_trace([es], *tr[1])[0]
    LA, LB = kfs[0].L, kfs[1].L
    for i in range(es.K):
        kb, ka = keys[i, 1].ravel(), keys[i, 0].ravel()
        hb = kb != EMPTY
        np.testing.assert_array_equal(lint[i].ravel()[hb], LB[(kb[hb] & np.uint64(0xFFFFFF)).astype(np.int64)])
        fill = (~hb) & (ka != EMPTY)
        np.testing.assert_array_equal(lint[i].ravel()[fill], LA[(ka[fill] & np.uint64(0xFFFFFF)).astype(np.int64)])


# ----------------------------------------------------------------------------------------
# luminance and log (Eq. 3, Sec. 3.2)
# ----------------------------------------------------------------------------------------

def test_rec709_golden(oracle_mod):
    rows = np.loadtxt(os.path.join(GOLDEN, "rec709_luminance.txt"))
    rgb = rows[:, :3].astype(np.float32)
    want = rows[:, 3]
    L = oracle_mod.log_intensity(rgb.reshape(-1), mode=oracle_mod.IN_RGB, eps=0.0)
    np.testing.assert_allclose(np.exp(L.astype(np.float64)), want, rtol=2e-7)


def test_log_closed_forms(oracle_mod):
    I = np.array([1.0, 10.0, 100.0, 1e-2, 1e3, np.e], dtype=np.float32)
    L = oracle_mod.log_intensity(I, mode=oracle_mod.IN_LUM, eps=0.0)
    want = np.array([0.0, np.log(10), 2 * np.log(10), -2 * np.log(10), 3 * np.log(10), 1.0])
    np.testing.assert_allclose(L, want, rtol=1.2e-7, atol=1e-12)
    # eps is added before the log; non-positive arguments clamp to the smallest normal float
    L2 = oracle_mod.log_intensity(np.array([0.0, -5.0], dtype=np.float32), eps=1e-4)
    assert L2[0] == np.float32(np.log(np.float32(1e-4)))
    assert L2[1] == np.float32(np.log(np.finfo(np.float32).tiny))


def test_refractory_boundary_is_inclusive(oracle_mod):
    """Sec. 3.4 suppresses events until t - t_last >= tau, so events exactly tau apart all
    fire.  L rises by exactly C per substep, so each crossing lands on a substep boundary
    t_i = T0 + i dt / K with no interpolation error."""
    K, C, dt = 4, 0.25, 8_000_000
    tau = dt // K
    env = TinyEnv(W=4, H=1, K=K, c_on=C, c_off=C, refractory_ns=tau)
    npx = packed_total([env])
    mv, z = _static(npx)
    L0 = np.zeros(npx, dtype=np.float32)
    L1 = np.zeros(npx, dtype=np.float32)
    L1[1] = K * C
    o, _ = _run(oracle_mod, [env], [L0, L1], [mv, mv], [z, z], dt)
    ev = oracle_mod.sort_events(o.events())
    assert list(ev["t"]) == [tau * i for i in range(1, K + 1)]
    # one nanosecond more of refractory suppresses every other event
    env2 = TinyEnv(W=4, H=1, K=K, c_on=C, c_off=C, refractory_ns=tau + 1)
    o2, _ = _run(oracle_mod, [env2], [L0, L1], [mv, mv], [z, z], dt)
    assert list(oracle_mod.sort_events(o2.events())["t"]) == [tau, 3 * tau]


def test_high_speed_scenes_have_disocclusion_holes(oracle_mod, scenes_mod):
    """The high-speed workload (640x480, K=32, flows up to 40 px/frame) must leave >= 10 % of
    the pixel-substeps without a source in at least one warp direction, on average."""
    w = scenes_mod.config4(n_envs=3)
    kfs = [scenes_mod.render(w.envs, k) for k in range(2)]
    o = oracle_mod.Oracle(w.envs, flags=oracle_mod.IN_LOG)
    o.step(kfs[0].L, kfs[0].mv, kfs[0].Z, w.dt_ns)
    keys, _ = o.step(kfs[1].L, kfs[1].mv, kfs[1].Z, w.dt_ns, trace=True)
    fr = []
    for k, _ in split_trace(w.envs, keys, np.zeros(sum(e.K * e.H * e.W for e in w.envs), np.float32)):
        fr.append(((k[:, 0] == EMPTY) | (k[:, 1] == EMPTY)).mean())
    assert np.mean(fr) >= 0.10, fr
    assert np.abs(kfs[1].mv).max() >= 30


def test_joint_mode_takes_the_nearer_surface(oracle_mod, scenes_mod):
    """Eq. 6 read literally: one argmin of interpolated depth over the A-forward and
    B-backward winners (equal depths go to B).  A disk passing in front of a plane: the value
    is always one of the two winners' values, the nearer one where they disagree, and it
    differs from the B-primary reading somewhere (where A's winner is the nearer one)."""
    W, H, K = 40, 24, 4
    plane = scenes_mod.Layer(kind=0, depth0=5.0, cx0=20, cy0=12, vx=1.0, tex_kind=1, mu=0.0)
    # an off-centre spinning disk: reusing m_A as a velocity is only a linear approximation of
    # the rotation, so the two directions disagree near its rim
    disk = scenes_mod.Layer(kind=1, radius=8.0, depth0=2.0, cx0=16, cy0=12, vx=2.0,
                            omega=0.6, tex_kind=1, mu=1.0)
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.3, c_off=0.3, layers=[plane, disk])
    kf = [scenes_mod.render([es], k) for k in range(2)]
    outs = {}
    for name, flags in (("joint", oracle_mod.MODE_JOINT), ("bprim", oracle_mod.MODE_B_PRIMARY)):
        o = oracle_mod.Oracle([es], flags=flags)
        o.step(kf[0].L, kf[0].mv, kf[0].Z, 1000)
        outs[name] = split_trace([es], *o.step(kf[1].L, kf[1].mv, kf[1].Z, 1000, trace=True))[0]
    keys, lint = outs["joint"]
    LA, LB = kf[0].L, kf[1].L
    differs = 0
    for i in range(K):
        kA, kB = keys[i, 0].ravel(), keys[i, 1].ravel()
        both = (kA != EMPTY) & (kB != EMPTY)
        la = LA[(kA[both] & np.uint64(0xFFFFFF)).astype(np.int64)]
        lb = LB[(kB[both] & np.uint64(0xFFFFFF)).astype(np.int64)]
        zA, zB = kA[both] >> np.uint64(32), kB[both] >> np.uint64(32)   # positive: bits order = value order
        got = lint[i].ravel()[both]
        assert np.all((got == la) | (got == lb))
        np.testing.assert_array_equal(got[la == lb], la[la == lb])
        dis = la != lb
        np.testing.assert_array_equal(got[dis], np.where(zA[dis] < zB[dis], la[dis], lb[dis]))
        differs += int((lint[i] != outs["bprim"][1][i]).sum())
    assert differs > 0
    with pytest.raises(ValueError):
        oracle_mod.Oracle([es], flags=oracle_mod.MODE_JOINT | oracle_mod.MODE_B_PRIMARY)
