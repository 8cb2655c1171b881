"""Small helpers shared by the tests (no method arithmetic here)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@dataclass
class TinyEnv:
    W: int
    H: int
    K: int
    c_on: float = 0.2
    c_off: float = 0.2
    refractory_ns: int = 0
    t0_ns: int = 0
    c_on_map: np.ndarray | None = None
    c_off_map: np.ndarray | None = None
    margin: int = 0


def packed_total(envs):
    return sum((e.H * e.W + 3) // 4 * 4 for e in envs)


def offsets(envs):
    out, acc = [], 0
    for e in envs:
        out.append(acc)
        acc += (e.H * e.W + 3) // 4 * 4
    return out


def split_trace(envs, keys, lint):
    """Per env: keys [K, 2, H, W] and interpolated L [K, H, W]."""
    res, ko, lo = [], 0, 0
    for e in envs:
        hw = e.H * e.W
        k = keys[ko:ko + e.K * 2 * hw].reshape(e.K, 2, e.H, e.W)
        l = lint[lo:lo + e.K * hw].reshape(e.K, e.H, e.W)
        res.append((k, l))
        ko += e.K * 2 * hw
        lo += e.K * hw
    return res
