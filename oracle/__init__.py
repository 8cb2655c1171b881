"""Oracle for the EVIS event-synthesis path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product (``paper_2607_08098_b300``) never imports it and fails
loudly when its CUDA library is missing.

The arithmetic lives in ``evis_oracle.cpp`` (single-threaded C++17, ``-O2 -ffp-contract=off``);
this file only compiles it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evis_oracle.cpp")
_SO = os.path.join(_HERE, "libevis_oracle.so")
_lib = None

IN_LOG, IN_LUM, IN_RGB = 0, 1, 2
MODE_B_PRIMARY = 0x10
TIE_INDEX = 0x20
MODE_JOINT = 0x40
COLOR = 0x200          # Sec. 3.2: events of the R, G and B channels (polarity field +-(1 + c))
MAX_CROSSINGS = 4096   # events one pixel may emit in one sub-frame (per channel)

EVENT_DTYPE = np.dtype([("t", "<i8"), ("x", "<u2"), ("y", "<u2"), ("env", "<u2"), ("p", "<i2")])


class _Env(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("K", ctypes.c_int32),
                ("c_on", ctypes.c_float), ("c_off", ctypes.c_float), ("margin", ctypes.c_int32),
                ("c_on_map", ctypes.c_void_p), ("c_off_map", ctypes.c_void_p),
                ("refractory_ns", ctypes.c_int64), ("t0_ns", ctypes.c_int64)]


class _Noise(ctypes.Structure):
    _fields_ = [("leak_hz", ctypes.c_float), ("shot_hz", ctypes.c_float),
                ("hot_hz", ctypes.c_float), ("hot_fraction", ctypes.c_float),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float), ("seed", ctypes.c_uint64)]


class _VoxelEnv(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("t0_ns", ctypes.c_int64), ("t1_ns", ctypes.c_int64)]


def voxel_grid(events, envs, bins: int = 128):
    """Event voxel grid of each environment's segment: envs is a list of (width, height,
    t0_ns, t1_ns); returns (acc uint32, grid float32), each the concatenation over
    environments of [2][bins][H][W] (polarity 0 = ON)."""
    lib = _load()
    lib.orc_voxel_grid.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    arr = (_VoxelEnv * len(envs))()
    total = 0
    for i, (W, H, t0, t1) in enumerate(envs):
        arr[i] = _VoxelEnv(int(W), int(H), int(t0), int(t1))
        total += 2 * bins * int(W) * int(H)
    acc = np.empty(total, dtype=np.uint32)
    out = np.empty(total, dtype=np.float32)
    lib.orc_voxel_grid(ev.ctypes.data, ev.size, ctypes.addressof(arr), len(envs), int(bins),
                       acc.ctypes.data, out.ctypes.data)
    return acc, out


def rec709(rgb) -> np.ndarray:
    """Rec. 709 luminance (Eq. 3) of [n, 3] linear RGB, binary32."""
    lib = _load()
    lib.orc_rec709.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    a = np.ascontiguousarray(rgb, dtype=np.float32).reshape(-1, 3)
    out = np.empty(a.shape[0], dtype=np.float32)
    lib.orc_rec709(a.ctypes.data, a.shape[0], out.ctypes.data)
    return out


def defocus(plane, sigma: float) -> np.ndarray:
    """Separable Gaussian blur of one linear plane [H, W] (Sec. 3.4), binary32."""
    lib = _load()
    lib.orc_defocus.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                ctypes.c_void_p]
    a = np.ascontiguousarray(plane, dtype=np.float32)
    out = np.empty_like(a)
    lib.orc_defocus(a.ctypes.data, a.shape[1], a.shape[0], float(sigma), out.ctypes.data)
    return out


def defocus_weights(sigma: float) -> np.ndarray:
    lib = _load()
    lib.orc_defocus_weights.restype = ctypes.c_int32
    lib.orc_defocus_weights.argtypes = [ctypes.c_float, ctypes.c_void_p]
    buf = np.empty(128, dtype=np.float32)
    r = lib.orc_defocus_weights(float(sigma), buf.ctypes.data)
    return buf[:2 * r + 1].copy()


def philox(n, c1=0, c2=0, c3=0, key=(0, 0), base=0) -> np.ndarray:
    """n outputs [n, 4] of the oracle's Philox4x32-10 at counters (base + j, c1, c2, c3)."""
    lib = _load()
    lib.orc_philox.argtypes = [ctypes.c_uint32] * 6 + [ctypes.c_int64, ctypes.c_void_p]
    out = np.empty((n, 4), dtype=np.uint32)
    lib.orc_philox(base, c1, c2, c3, key[0], key[1], n, out.ctypes.data)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (g++, host only, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", _SRC, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_uint32]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_step.restype = ctypes.c_int32
        lib.orc_step.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64] + [ctypes.c_void_p] * 2
        lib.orc_num_events.restype = ctypes.c_int64
        lib.orc_num_events.argtypes = [ctypes.c_void_p]
        lib.orc_take_events.restype = ctypes.c_int64
        lib.orc_take_events.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        lib.orc_get_state.restype = ctypes.c_int32
        lib.orc_get_state.argtypes = [ctypes.c_void_p] * 4
        lib.orc_log_intensity.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_float, ctypes.c_void_p]
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """One oracle context over a list of ``scenes.EnvScene``-like environments."""

    def __init__(self, envs, eps: float = 1e-4, flags: int = 0):
        lib = _load()
        self._keep = []
        arr = (_Env * len(envs))()
        for i, e in enumerate(envs):
            con = coff = None
            if getattr(e, "c_on_map", None) is not None:
                con = np.ascontiguousarray(e.c_on_map, dtype=np.float32)
                coff = np.ascontiguousarray(e.c_off_map, dtype=np.float32)
                self._keep += [con, coff]
            arr[i] = _Env(e.W, e.H, e.K, e.c_on, e.c_off, int(getattr(e, "margin", 0)), _ptr(con), _ptr(coff),
                          int(e.refractory_ns), int(e.t0_ns))
        self._h = lib.orc_create(ctypes.addressof(arr), len(envs), float(eps), int(flags))
        if not self._h:
            raise ValueError("oracle rejected the environment table")
        self.envs = list(envs)
        self.last_over_limit = False
        self.nc = 3 if flags & COLOR else 1   # planes of L, Lref and t_last
        self.total = 0
        self.offsets = []
        for e in envs:
            self.offsets.append(self.total)
            self.total += (e.H * e.W + 3) // 4 * 4

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.orc_destroy(self._h)
            self._h = None

    def trace_sizes(self):
        nk = sum(e.K * 2 * e.H * e.W for e in self.envs)
        nl = sum(e.K * self.nc * e.H * e.W for e in self.envs)
        return nk, nl

    def step(self, frames, mv, depth, dt_ns: int, trace: bool = False):
        frames = np.ascontiguousarray(frames, dtype=np.float32)
        mv = np.ascontiguousarray(mv, dtype=np.float32)
        depth = np.ascontiguousarray(depth, dtype=np.float32)
        keys = lint = None
        if trace:
            nk, nl = self.trace_sizes()
            keys = np.empty(nk, dtype=np.uint64)
            lint = np.empty(nl, dtype=np.float32)
        rc = _lib.orc_step(self._h, _ptr(frames), _ptr(mv), _ptr(depth), int(dt_ns), _ptr(keys),
                           _ptr(lint))
        if rc == 1:
            raise ValueError("oracle step rejected its arguments")
        # 2: some pixel-sub-frame of this gap had more crossings than a pixel may emit
        self.last_over_limit = rc == 2
        return (keys, lint) if trace else None

    def over_limit(self) -> np.ndarray:
        """Per environment: pixel-sub-frames (per channel) since creation whose crossing
        count n of Eq. 4 exceeded the emission limit (none of their crossings was emitted)."""
        lib = _load()
        lib.orc_over_limit.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        out = np.zeros(len(self.envs), dtype=np.uint64)
        lib.orc_over_limit(self._h, out.ctypes.data)
        return out

    def events(self) -> np.ndarray:
        n = _lib.orc_num_events(self._h)
        out = np.empty(n, dtype=EVENT_DTYPE)
        got = _lib.orc_take_events(self._h, _ptr(out), n)
        return out[:got]

    def set_noise(self, specs):
        """Per-environment sensor noise (Sec. 3.4): dicts with leak_hz, shot_hz, hot_hz,
        hot_fraction, lo, hi, seed (missing keys: off / defaults)."""
        lib = _load()
        if not hasattr(lib, "_noise_sig"):
            lib.orc_set_noise.restype = ctypes.c_int32
            lib.orc_set_noise.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            lib._noise_sig = True
        arr = (_Noise * len(self.envs))()
        for i, sp in enumerate(specs):
            arr[i] = _Noise(sp.get("leak_hz", 0.0), sp.get("shot_hz", 0.0), sp.get("hot_hz", 0.0),
                            sp.get("hot_fraction", 0.0), sp.get("lo", -5.0), sp.get("hi", 5.0),
                            int(sp.get("seed", 0)))
        if lib.orc_set_noise(self._h, ctypes.addressof(arr)) != 0:
            raise ValueError("oracle rejected the noise parameters")

    def set_defocus(self, sigmas):
        """Per-environment defocus sigma in pixels (Sec. 3.4); linear inputs only."""
        lib = _load()
        lib.orc_set_defocus.restype = ctypes.c_int32
        lib.orc_set_defocus.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        sg = np.ascontiguousarray(sigmas, dtype=np.float32)
        if sg.size != len(self.envs) or lib.orc_set_defocus(self._h, sg.ctypes.data) != 0:
            raise ValueError("oracle rejected the defocus parameters")

    def state(self):
        Lref = np.empty(self.nc * self.total, dtype=np.float32)
        tl = np.empty(self.nc * self.total, dtype=np.int64)
        clk = np.empty(len(self.envs), dtype=np.int64)
        _lib.orc_get_state(self._h, _ptr(Lref), _ptr(tl), _ptr(clk))
        return Lref, tl, clk


def log_intensity(x, mode: int = IN_LUM, eps: float = 1e-4) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.size // 3 if mode == IN_RGB else x.size
    out = np.empty(n, dtype=np.float32)
    lib.orc_log_intensity(_ptr(x), n, mode, float(eps), _ptr(out))
    return out


def sort_events(ev: np.ndarray) -> np.ndarray:
    """Canonical order used by every parity comparison: (env, t, y, x, p)."""
    idx = np.lexsort((ev["p"], ev["x"], ev["y"], ev["t"], ev["env"]))
    return ev[idx]


def soft_counts(envs, tau, delta, LA, LB, mvA, mvB, ZA, ZB, Lref0, C, smooth=None, gcounts=None):
    """Soft event-count surrogate of one keyframe gap (binary64).

    Decisions come from the binary32 inputs and each env's c_on / c_off (the frozen reference
    trajectory); ``C`` is the smooth threshold of the sigmoids.  ``smooth`` optionally overrides
    the values the
    smooth part uses (dict with keys LA, LB, mvA, mvB, C as float64), which is how finite
    differences keep the decisions frozen.  Returns counts (packed [2][H][W] per env) and,
    with ``gcounts``, the gradients dict (LA, LB, mvA, mvB, C)."""
    lib = _load()
    if not hasattr(lib, "_soft_sig"):
        lib.orc_soft.restype = ctypes.c_int32
        lib.orc_soft.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_float] + \
            [ctypes.c_void_p] * 19
        lib._soft_sig = True
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32).reshape(-1)  # noqa: E731
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)  # noqa: E731
    dec = [f32(a) for a in (LA, LB, mvA, mvB, ZA, ZB, Lref0)]
    sm = smooth or {}
    sLA, sLB = f64(sm.get("LA", dec[0])), f64(sm.get("LB", dec[1]))
    smA, smB = f64(sm.get("mvA", dec[2])), f64(sm.get("mvB", dec[3]))
    sC = f64(sm.get("C", f32(C)))
    arr = (_Env * len(envs))()
    for i, e in enumerate(envs):
        arr[i] = _Env(e.W, e.H, e.K, e.c_on, e.c_off, int(getattr(e, "margin", 0)), None, None, 0, 0)
    n = dec[0].size
    counts = np.zeros(2 * n, dtype=np.float64)
    grads = None
    gp = [None] * 5
    if gcounts is not None:
        gcounts = f64(gcounts)
        grads = {"LA": np.zeros(n), "LB": np.zeros(n), "mvA": np.zeros(2 * n),
                 "mvB": np.zeros(2 * n), "C": np.zeros(len(envs))}
        gp = [grads[k].ctypes.data for k in ("LA", "LB", "mvA", "mvB", "C")]
    lib.orc_soft(ctypes.addressof(arr), len(envs), float(tau), float(delta),
                 *[a.ctypes.data for a in dec], sLA.ctypes.data, sLB.ctypes.data,
                 smA.ctypes.data, smB.ctypes.data, sC.ctypes.data, counts.ctypes.data,
                 None if gcounts is None else gcounts.ctypes.data, *gp)
    return (counts, grads) if gcounts is not None else counts
