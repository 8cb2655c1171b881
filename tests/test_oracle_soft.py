"""Pins of the oracle's soft event-count surrogate (CPU, binary64).

The surrogate is defined here (the paper has no backward pass): frozen discrete
decisions, a normalised bilinear splat over the winning surface, and sigmoid counts.  Its
analytic gradient is checked against central finite differences with the decisions frozen,
and the zero-motion case against its closed form."""
import numpy as np
import pytest

from evis_testutil import TinyEnv, packed_total

TAU, DELTA = 0.02, 1e-3


def _scene(scenes_mod, W=24, H=18, K=4, seed=3):
    rng = np.random.default_rng(seed)
    lay = scenes_mod._random_layers(rng, W, H, 3, vmax=3.0, wmax=0.05)
    for l in lay:
        l.sigma = 0.4  # gentle textures keep the counts away from saturation
    es = scenes_mod.EnvScene(W=W, H=H, K=K, c_on=0.2, c_off=0.2, layers=lay)
    kf = [scenes_mod.render([es], k) for k in range(2)]
    return es, kf


def _fd_safe(es, mv, sign_scale, h):
    """Sources whose target stays more than 2h|s| away from an integer at every sub-frame."""
    n = es.W * es.H
    ok = np.ones(n, dtype=bool)
    yy, xx = np.mgrid[0:es.H, 0:es.W]
    for i in range(1, es.K + 1):
        s = sign_scale(i / es.K)
        if s == 0:
            continue  # q does not move with m at this sub-frame
        for c, base in ((0, xx.ravel()), (1, yy.ravel())):
            q = base + s * mv[:n, c].astype(np.float64)
            fr = q - np.floor(q)
            ok &= (fr > 2 * h * abs(s) + 1e-6) & (fr < 1 - 2 * h * abs(s) - 1e-6)
    return ok


def test_soft_gradient_matches_central_differences(oracle_mod, scenes_mod):
    es, kf = _scene(scenes_mod)
    envs = [es]
    n = es.W * es.H
    LA, LB, mvA, mvB, ZA, ZB = kf[0].L, kf[1].L, kf[0].mv, kf[1].mv, kf[0].Z, kf[1].Z
    Lref0 = LA.copy()
    C = np.array([0.2])
    gc = np.random.default_rng(0).normal(size=2 * packed_total(envs))
    args = (envs, TAU, DELTA, LA, LB, mvA, mvB, ZA, ZB, Lref0, C)
    counts, g = oracle_mod.soft_counts(*args, gcounts=gc)
    assert counts.sum() > 1.0
    base = {"LA": LA.astype(np.float64), "LB": LB.astype(np.float64),
            "mvA": mvA.astype(np.float64).reshape(-1), "mvB": mvB.astype(np.float64).reshape(-1),
            "C": C.astype(np.float64)}

    def loss(sm):
        return float(gc @ oracle_mod.soft_counts(*args, smooth=sm))

    rng2 = np.random.default_rng(1)
    n_nonzero = 0
    for h, stencil, rtol in ((1e-5, 2, 1e-4), (1e-3, 4, 1e-3)):
        safeA = _fd_safe(es, mvA, lambda f: -f, 2 * h)
        safeB = _fd_safe(es, mvB, lambda f: 1 - f, 2 * h)
        checks = [("LA", i) for i in rng2.choice(n, 10, replace=False)] + \
                 [("LB", i) for i in rng2.choice(n, 10, replace=False)] + \
                 [("mvA", 2 * i + c) for i in rng2.choice(np.nonzero(safeA)[0], 8, replace=False) for c in (0, 1)] + \
                 [("mvB", 2 * i + c) for i in rng2.choice(np.nonzero(safeB)[0], 8, replace=False) for c in (0, 1)] + \
                 [("C", 0)]
        for key, idx in checks:
            def at(step):
                sm = {k: v.copy() for k, v in base.items()}
                sm[key][idx] += step
                return loss(sm)
            if stencil == 2:
                fd = (at(h) - at(-h)) / (2 * h)
            else:  # fourth-order central difference
                fd = (-at(2 * h) + 8 * at(h) - 8 * at(-h) + at(-2 * h)) / (12 * h)
            an = g[key][idx]
            assert abs(fd - an) <= rtol * max(abs(fd), abs(an)) + 1e-7, (h, key, idx, fd, an)
            n_nonzero += abs(an) > 1e-6
    assert n_nonzero > 20


def test_zero_motion_closed_form(oracle_mod):
    """Static scene, one depth: every target's winner surface is its own source, so
    L_i = (1-f) L_A + f L_B, the counts are sums of sigmoids and dN/dL_A is their slope."""
    rng = np.random.default_rng(4)
    env = TinyEnv(W=7, H=5, K=5)
    n = packed_total([env])
    LA = rng.normal(0, 0.3, n).astype(np.float32)
    LB = (LA + rng.normal(0, 0.3, n)).astype(np.float32)
    mv = np.zeros((n, 2), np.float32)
    Z = np.ones(n, np.float32)
    C = float(np.float32(0.2))  # the smooth part sees the binary32 threshold
    gc = rng.normal(size=2 * n)
    counts, g = oracle_mod.soft_counts([env], TAU, DELTA, LA, LB, mv, mv, Z, Z, LA, [C], gcounts=gc)
    m = env.W * env.H
    lref = LA[:m].astype(np.float32).copy()
    want = np.zeros((2, m))
    dLA = np.zeros(m)
    sig = lambda u: 1 / (1 + np.exp(-u))  # noqa: E731
    for i in range(1, env.K + 1):
        f = np.float32(i) / np.float32(env.K)
        g32 = np.float32(1) - f
        fd, gd = i / env.K, 1 - i / env.K
        Ls = gd * LA[:m].astype(np.float64) + fd * LB[:m].astype(np.float64)
        lr = lref.astype(np.float64)
        on, off = sig((Ls - lr - C) / TAU), sig((lr - Ls - C) / TAU)
        want[0] += on
        want[1] += off
        dLA += gd * (gc[:m] * on * (1 - on) / TAU - gc[m:2 * m] * off * (1 - off) / TAU)
        Lh = (g32 * LA[:m] + f * LB[:m]).astype(np.float32)       # frozen discrete trajectory
        d = Lh - lref
        q = np.abs(d) / np.float32(C)
        k = np.where(q >= 1, np.floor(q), 0).astype(np.float32)
        lref = np.where(k > 0, lref + (np.sign(d) * k).astype(np.float32) * np.float32(C), lref).astype(np.float32)
    np.testing.assert_allclose(counts[:m], want[0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(counts[m:2 * m], want[1], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(g["LA"][:m], dLA, rtol=1e-8, atol=1e-10)
